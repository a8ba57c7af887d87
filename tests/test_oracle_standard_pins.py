"""Pins of the oracle's standard explicit scheme (Sec. 3.1, Eq. eq-disbi), the
discretisation the paper's split operator replaces: the printed 2D stencil,
the 25-point 3D stencil, its Fourier symbol, wall symmetry and conservation,
and one RK3 step of a linearised Fourier mode against the closed-form
amplification."""
import json
import os

import numpy as np
import pytest

from oracle import ch_oracle as co
from oracle.ch_oracle import NOFLUX, PERIODIC, Params
from paper_2105_01865_gb300 import stability

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_stencils.json")


def delta_response(shape, h, centre):
    nz, ny, nx = shape
    p = Params(nx, ny, nz, h, cn=0.75 * h, pe=10.0, dt=1e-3)
    d = np.zeros(shape)
    d[centre] = 1.0
    return co.biharmonic_h(d, p) * h ** 4


def test_2d_biharmonic_is_the_printed_eq_disbi_stencil():
    """A field constant along z sees exactly the 13 points printed in Eq.
    (eq-disbi) (coefficients times 1/h^4), and nothing else."""
    pts = json.load(open(GOLDEN))["disbi_2d"]["points"]
    shape, c = (1, 11, 11), (0, 5, 5)
    got = delta_response(shape, 0.1, c)
    want = np.zeros(shape)
    for dx, dy, v in pts:
        want[0, 5 + dy, 5 + dx] += v   # the stencil is symmetric: response = coefficient
    assert np.allclose(got, want, rtol=0, atol=1e-9)


def test_3d_biharmonic_is_the_25_point_stencil():
    shape, c = (9, 9, 9), (4, 4, 4)
    got = delta_response(shape, 0.05, c)
    want = np.zeros(shape)
    want[c] = 42.0
    for ax in range(3):
        for off, v in ((1, -12.0), (2, 1.0)):
            for sgn in (-1, 1):
                idx = list(c)
                idx[ax] += sgn * off
                want[tuple(idx)] = v
    for a in range(3):
        for b in range(a + 1, 3):
            for sa in (-1, 1):
                for sb in (-1, 1):
                    idx = list(c)
                    idx[a] += sa
                    idx[b] += sb
                    want[tuple(idx)] = 2.0
    assert np.allclose(got, want, rtol=0, atol=1e-8)
    assert np.count_nonzero(np.abs(want) > 0) == 25


def test_biharmonic_symbol_on_fourier_modes():
    nz, ny, nx = 10, 6, 8
    h = 0.125
    p = Params(nx, ny, nz, h, cn=0.75 * h, pe=10.0, dt=1e-3)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for k in [(1, 2, 3), (4, 3, 5), (0, 1, 0)]:
        th = [2 * np.pi * k[0] / nx, 2 * np.pi * k[1] / ny, 2 * np.pi * k[2] / nz]
        f = np.cos(th[0] * x + th[1] * y + th[2] * z)
        S = sum(4 * np.sin(t / 2) ** 2 / h ** 2 for t in th)
        assert np.allclose(co.biharmonic_h(f, p), S * S * f, rtol=0, atol=1e-9 * S * S)


def test_biharmonic_with_walls_is_symmetric_and_conservative():
    nz, ny, nx = 5, 4, 6
    h = 0.2
    p = Params(nx, ny, nz, h, cn=0.75 * h, pe=10.0, dt=1e-3, bc=(NOFLUX, PERIODIC, NOFLUX))
    N = nx * ny * nz
    B = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        B[:, i] = co.biharmonic_h(e.reshape(p.shape), p).ravel()
    assert np.allclose(B, B.T, rtol=0, atol=1e-9 * np.abs(B).max())
    assert np.allclose(B.sum(axis=0), 0.0, atol=1e-9 * np.abs(B).max())
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() >= -1e-9 * np.abs(B).max()


@pytest.mark.parametrize("psi2", [0.5, -0.25])
def test_rk3_step_of_a_linear_mode_matches_closed_form(psi2):
    """psi' linearised as psi'' C: a cosine mode is multiplied by the closed-form
    explicit RK3 gain per step."""
    nz, ny, nx = 6, 8, 10
    h = 1.0 / 10
    cn, pe = 0.75 * h, 50.0
    k = (3, 2, 1)
    th = [2 * np.pi * k[0] / nx, 2 * np.pi * k[1] / ny, 2 * np.pi * k[2] / nz]
    s = [4 * np.sin(t / 2) ** 2 / h ** 2 for t in th]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = 1e-3 * np.cos(th[0] * x + th[1] * y + th[2] * z)
    dt = 0.5 * stability.stable_dt_standard((nz, ny, nx), h, (0, 0, 0), cn, pe, psi2=max(psi2, 0.0))
    p = Params(nx, ny, nz, h, cn=cn, pe=pe, dt=dt)
    nsteps = 4
    got = co.step_standard(f, None, p, nsteps, psi_p=lambda C: psi2 * C)
    # closed form, written as the recurrence on (q, H^{l-1}) of one step
    S = sum(s)
    lam = -(1.0 / pe) * (psi2 * S + cn * cn * S * S)
    q, hp = 1.0, 0.0
    for g, r in zip((8 / 15, 5 / 12, 3 / 4), (0.0, -17 / 60, -5 / 12)):
        hl = lam * q
        q, hp = q + dt * (g * hl + r * hp), hl
    assert np.allclose(got, q ** nsteps * f, rtol=0, atol=1e-12 * np.abs(f).max())


def test_stability_bound_separates_decay_from_growth():
    """At 0.98 dt_stab the highest grid mode does not grow over 20 steps of the
    oracle; at 1.05 dt_stab it grows."""
    n = 8
    h = 1.0 / n
    cn, pe = 0.75 * h, 20.0
    dts = stability.stable_dt_standard((n, n, n), h, (0, 0, 0), cn, pe, psi2=0.5)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    f = 1e-6 * np.cos(np.pi * (x + y + z))     # the checkerboard, S = 12 / h^2
    amp = []
    for fac in (0.98, 1.05):
        p = Params(n, n, n, h, cn=cn, pe=pe, dt=fac * dts)
        amp.append(np.abs(co.step_standard(f, None, p, 20, psi_p=lambda C: 0.5 * C)).max() / 1e-6)
    assert amp[0] <= 1.0 and amp[1] > 1.5


def test_standard_step_conserves_mass_with_walls_and_shear():
    from paper_2105_01865_gb300 import inputs
    nz, ny, nx = 12, 10, 14
    h = 1.0 / 12
    cn = 0.75 * h
    pe = 0.9 / cn
    bc = (PERIODIC, PERIODIC, NOFLUX)
    C0 = inputs.drops_field((nz, ny, nx), h, bc, [(0.6, 0.4, 0.5)], [0.25], cn)
    vel = inputs.shear_velocity((nz, ny, nx), h, 1.0, bc)
    dt = 0.9 * min(stability.stable_dt_standard((nz, ny, nx), h, bc, cn, pe), 0.5 * h)
    p = Params(nx, ny, nz, h, cn=cn, pe=pe, dt=dt, bc=bc)
    C = co.step_standard(C0, vel, p, 30)
    assert abs(co.mass(C, p) - co.mass(C0, p)) <= 1e-13 * co.mass(C0, p)
    assert np.all(np.isfinite(C))
