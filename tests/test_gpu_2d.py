"""GPU parity of the 2D scheme (a single periodic z-plane: A_x + A_y, Eq.
eq-a2d with w = 2; no z-solve) against the oracle, with and without a
discretely divergence-free 2D flow."""
import numpy as np
import pytest

from oracle import ch_oracle as co
from paper_2105_01865_gb300 import inputs

from _parity import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2105_01865_gb300 import build, capi
    build.build()
    capi.load()


def flow_2d(nx, ny, h, bc, seed):
    """u = d(psi)/dy, v = -d(psi)/dx from a random corner stream function: zero
    discrete divergence; psi = 0 on walls keeps the normal velocity zero there;
    w = 0 on the single z-face plane."""
    rng = np.random.default_rng(seed)
    ncx = nx + (1 if bc[0] == co.NOFLUX else 0)
    ncy = ny + (1 if bc[1] == co.NOFLUX else 0)
    X, Y = np.meshgrid(np.arange(ncx) * h, np.arange(ncy) * h)
    psi = np.zeros((ncy, ncx))
    for _ in range(4):
        kx, ky = rng.integers(1, 3, size=2)
        psi += rng.standard_normal() * np.sin(2 * np.pi * kx * X / (nx * h) + rng.random()) * \
            np.sin(2 * np.pi * ky * Y / (ny * h) + rng.random())
    if bc[0] == co.NOFLUX:
        psi[:, 0] = psi[:, -1] = 0.0
    if bc[1] == co.NOFLUX:
        psi[0, :] = psi[-1, :] = 0.0
    psi *= 0.02 / (np.abs(psi).max() + 1e-30)
    pc = lambda i, j: psi[j % ncy, i % ncx]
    nfx = nx + (1 if bc[0] == co.NOFLUX else 0)
    nfy = ny + (1 if bc[1] == co.NOFLUX else 0)
    u = np.array([[(pc(i, j + 1) - pc(i, j)) / h for i in range(nfx)] for j in range(ny)])[None]
    v = np.array([[-(pc(i + 1, j) - pc(i, j)) / h for i in range(nx)] for j in range(nfy)])[None]
    if bc[0] == co.NOFLUX:
        u[..., 0] = u[..., -1] = 0.0
    if bc[1] == co.NOFLUX:
        v[:, 0, :] = v[:, -1, :] = 0.0
    w = np.zeros((1, ny, nx))
    return u, v, w


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("shape,bc,advect", [
    ((1, 40, 36), (co.PERIODIC, co.PERIODIC, co.PERIODIC), False),
    ((1, 33, 50), (co.NOFLUX, co.PERIODIC, co.PERIODIC), True),      # even nx: paired kernels
    ((1, 24, 37), (co.PERIODIC, co.NOFLUX, co.PERIODIC), True),      # odd nx: one-column forms
])
def test_2d_box_matches_oracle(prec, tol, shape, bc, advect):
    from paper_2105_01865_gb300.solver import Solver
    _, ny, nx = shape
    h = 1.0 / 32
    cn = 0.75 * h
    pe = 0.9 / cn
    rng = np.random.default_rng(5)
    C0 = inputs.drops_field(shape, h, bc, [(nx * h / 2, ny * h / 2, 0.5 * h)], [0.3], cn)
    C0 = C0 + 0.02 * rng.standard_normal(shape)
    vel = flow_2d(nx, ny, h, bc, 3) if advect else None
    dt = 2e-3
    s = Solver(shape, h, bc, cn, pe, dt, C0, precision=prec, w=2.0, advect=advect)
    if advect:
        s.set_velocity_fine(*vel)
    m0 = s.mass()
    s.step(10)
    p = co.Params(nx, ny, 1, h, cn=cn, pe=pe, dt=dt, bc=bc, w=2.0)
    C0r = C0.astype(np.float32).astype(np.float64) if prec == "f32" else C0
    ref = co.step(C0r, vel, p, 10)
    assert_parity(s.field(), ref, tol, f"2D {prec} {shape} {bc} advect={advect}")
    assert abs(s.mass() - m0) <= (1e-13 if prec == "f64" else 1e-6) * abs(m0)
