"""Pins of the oracle's Dirichlet walls (C = 0 on the wall faces, the
Rayleigh-Benard setting of Sec. 4.3): antisymmetric ghost cells, the wall rows
of the pentadiagonal operator (symmetric, positive definite, with the sine
modes of the odd extension as eigenvectors), and one RK3/CN/AF step of a
linearised sine mode against the closed-form gain."""
import numpy as np
import pytest

from oracle import ch_oracle as co
from oracle.ch_oracle import DIRICHLET, PERIODIC, Params


def test_ghosts_are_the_negated_mirror():
    f = np.arange(1.0, 1.0 + 5 * 4 * 3).reshape(5, 4, 3)
    g = co.pad(f, (PERIODIC, PERIODIC, DIRICHLET), 2)
    inner = g[:, 2:-2, 2:-2]
    np.testing.assert_array_equal(inner[0], -f[1])
    np.testing.assert_array_equal(inner[1], -f[0])
    np.testing.assert_array_equal(inner[-1], -f[-2])
    np.testing.assert_array_equal(inner[-2], -f[-1])
    # the wall-face value (mean of the two cells across the face) is zero
    np.testing.assert_array_equal(0.5 * (inner[1] + inner[2]), 0.0)


@pytest.mark.parametrize("n", [5, 8, 13])
def test_wall_operator_has_the_sine_modes_as_eigenvectors(n):
    kappa = 2.5
    A = co.line_operator(n, DIRICHLET, kappa)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12)
    i = np.arange(n) + 0.5
    for m in range(1, n + 1):
        v = np.sin(np.pi * m * i / n)
        lam = kappa * (4.0 * np.sin(np.pi * m / (2 * n)) ** 2) ** 2
        np.testing.assert_allclose(A @ v, lam * v, rtol=0, atol=1e-10 * max(1.0, lam))
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("mx,mz", [(1, 1), (2, 3), (0, 5)])
def test_linear_sine_mode_matches_closed_form(mx, mz):
    nx, ny, nz = 12, 6, 10
    h = 1.0 / 12
    p = Params(nx, ny, nz, h, cn=0.75 * h, pe=40.0, dt=4e-3, bc=(PERIODIC, PERIODIC, DIRICHLET))
    psi2 = 0.5
    x = (np.arange(nx) + 0.5) * h
    kz = np.arange(nz) + 0.5
    mode = np.cos(2 * np.pi * mx * x)[None, None, :] * np.sin(np.pi * mz * kz / nz)[:, None, None]
    mode = np.broadcast_to(mode, p.shape).copy()
    out = co.step(0.05 * mode, None, p, 2, psi_p=lambda c: psi2 * c)
    s = [4 * np.sin(np.pi * mx / nx) ** 2 / h ** 2, 0.0, 4 * np.sin(np.pi * mz / (2 * nz)) ** 2 / h ** 2]
    lam = -p.mobility * psi2 * sum(s)
    a = [p.w * p.cn ** 2 * sd ** 2 for sd in s]
    q, hp = 1.0, 0.0
    for g, r in zip((8 / 15, 5 / 12, 3 / 4), (0.0, -17 / 60, -5 / 12)):
        al = g + r
        den = np.prod([1 + al * p.dt * p.mobility * ad / 2 for ad in a])
        dq = (p.dt * (g * lam * q + r * hp) - al * p.dt * p.mobility * sum(a) * q) / den
        hp = lam * q
        q = q + dq
    np.testing.assert_allclose(out, 0.05 * q ** 2 * mode, rtol=0, atol=1e-13)


def test_flow_walls_are_walls():
    """A Dirichlet direction is a wall for the flow: n + 1 face planes and zero
    advective flux through the wall faces."""
    p = Params(6, 5, 7, 0.1, cn=0.075, pe=10.0, dt=1e-3, bc=(PERIODIC, PERIODIC, DIRICHLET))
    assert p.nfaces(2) == 8
    rng = np.random.default_rng(0)
    C = rng.random(p.shape)
    w = rng.standard_normal((8, 5, 6))
    F = co.face_fluxes(C, w, p, 2)
    assert np.all(F[0] == 0) and np.all(F[-1] == 0)
