"""Pins of the oracle's down-sampling (Sec. 3.4 back-coupling) and of the
coarse quantities it feeds (Eqs. eq-rho, eq-mu, eq-fst): identity for
coincident meshes, exactness for linear fields on stretched meshes and for
quadratics away from clamped ends, the density/viscosity definitions, and
second-order convergence of the discrete surface-tension force to its
continuum value."""
import numpy as np
import pytest

from oracle import ch_oracle as co
from oracle import mr_oracle as mo
from paper_2105_01865_gb300 import inputs

PER, WALL = co.PERIODIC, co.NOFLUX


def fine_params(n, h, bc):
    nx, ny, nz = n
    return co.Params(nx, ny, nz, h, cn=0.75 * h, pe=10.0, dt=1e-3, bc=bc)


@pytest.mark.parametrize("bc", [(PER, PER, WALL), (WALL, WALL, WALL), (PER,) * 3])
def test_coincident_meshes_give_the_identity(bc):
    n, h = (12, 10, 8), 0.125
    p = fine_params(n, h, bc)
    rng = np.random.default_rng(1)
    C = rng.random((n[2], n[1], n[0]))
    faces = [inputs.uniform_faces(m, m * h) for m in n]
    Cc, rho, mu, F = mo.restrict_to_coarse(C, p, *faces, 0.1, 0.01)
    np.testing.assert_allclose(Cc, C, rtol=0, atol=1e-13)
    for fc, ff in zip(F, co.surface_tension(C, p)):
        np.testing.assert_allclose(fc, ff, rtol=0, atol=1e-12 * np.abs(ff).max())


def test_linear_fields_are_exact_on_stretched_meshes():
    n, h = (16, 12, 20), 1.0 / 20
    bc = (WALL, WALL, WALL)
    faces = (inputs.stretched_faces(5, n[0] * h, 1.5), inputs.stretched_faces(4, n[1] * h, 2.0),
             inputs.stretched_faces(6, n[2] * h, 2.0))
    tabs = mo.restriction_tables(*faces, n, h, bc)
    x, y, z = ((np.arange(m) + 0.5) * h for m in n)
    f = 0.3 + 1.7 * x[None, None, :] - 0.4 * y[None, :, None] + 2.2 * z[:, None, None]
    xc, yc, zc = (mo.centres(fc) for fc in faces)
    want = 0.3 + 1.7 * xc[None, None, :] - 0.4 * yc[None, :, None] + 2.2 * zc[:, None, None]
    np.testing.assert_allclose(mo.interp_3d(f, tabs), want, rtol=0, atol=1e-12)


def test_quadratics_are_exact_away_from_clamped_ends():
    """Catmull-Rom slopes on the uniform fine nodes are exact for quadratics, so
    coarse centres whose stencil is not clamped reproduce them."""
    n, h = (24, 8, 8), 1.0 / 24
    bc = (WALL, PER, PER)
    faces = (inputs.stretched_faces(7, n[0] * h, 2.0), inputs.uniform_faces(2, n[1] * h),
             inputs.uniform_faces(2, n[2] * h))
    tabs = mo.restriction_tables(*faces, n, h, bc)
    x = (np.arange(n[0]) + 0.5) * h
    f = np.broadcast_to((1.0 + x - 3.0 * x * x)[None, None, :], (n[2], n[1], n[0]))
    got = mo.interp_3d(np.array(f), tabs)[0, 0]
    xc = mo.centres(faces[0])
    inner = (xc > 1.5 * h) & (xc < (n[0] - 1.5) * h)
    np.testing.assert_allclose(got[inner], (1.0 + xc - 3.0 * xc * xc)[inner], rtol=0, atol=1e-12)


def test_density_and_viscosity_definitions():
    C = np.array([0.0, 1.0, 0.5, 0.25])
    np.testing.assert_allclose(co.density(C, 0.1), [0.1, 1.0, 0.55, 0.325], rtol=1e-15)
    np.testing.assert_allclose(co.viscosity(C, 2.0), [2.0, 1.0, 1.5, 1.75], rtol=1e-15)


def test_surface_tension_converges_to_the_continuum_force():
    """C = 0.5 + a sin(kx) on a periodic box (Cn fixed): the discrete F_x tends
    to 6 sqrt(2)/Cn [psi'(C) - Cn^2 C''] C' at second order; F_y = F_z = 0."""
    L, a, cn = 1.0, 0.3, 0.05
    k = 2 * np.pi / L
    errs = []
    for nx in (32, 64, 128):
        h = L / nx
        p = co.Params(nx, 5, 5, h, cn=cn, pe=10.0, dt=1e-3)
        x = (np.arange(nx) + 0.5) * h
        C = np.broadcast_to(0.5 + a * np.sin(k * x)[None, None, :], p.shape).copy()
        F = co.surface_tension(C, p)
        c1 = 0.5 + a * np.sin(k * x)
        phi = co.psi_prime(c1) + cn ** 2 * a * k ** 2 * np.sin(k * x)
        want = 6 * np.sqrt(2) / cn * phi * a * k * np.cos(k * x)
        errs.append(np.abs(F[0][0, 0] - want).max() / np.abs(want).max())
        assert np.abs(F[1]).max() < 1e-12 and np.abs(F[2]).max() < 1e-12
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
