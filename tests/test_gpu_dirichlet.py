"""GPU parity of Dirichlet z-walls (C = 0 on the wall faces, Sec. 4.3's
Rayleigh-Benard setting) against the oracle: the split step in FP64 to 1e-12
and FP32 to 1e-5, the free energy with the antisymmetric ghost, and the
velocity transfer, which treats a Dirichlet direction as a wall exactly as a
no-flux one."""
import numpy as np
import pytest

from oracle import ch_oracle as co
from paper_2105_01865_gb300 import inputs, stability

from _parity import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P, N, D = co.PERIODIC, co.NOFLUX, co.DIRICHLET


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2105_01865_gb300 import build, capi
    build.build()
    capi.load()


def case(shape, bc, seed, advect):
    h = 1.0 / 16
    cn = 0.75 * h
    pe = 0.9 / cn
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    centres, radii = inputs.random_drops(rng, 3, (nx * h, ny * h, nz * h), 0.05, 0.15, 2 * cn,
                                         tuple(b != P for b in bc))
    C0 = inputs.drops_field(shape, h, (bc[0], bc[1], N), centres, radii, cn) + 0.05 * rng.standard_normal(shape)
    vel = None
    if advect:
        vel = inputs.curl_velocity(inputs.uniform_faces(nx, nx * h), inputs.uniform_faces(ny, ny * h),
                                   inputs.uniform_faces(nz, nz * h), bc, seed, kmax=3)
    dt = min(0.9 * stability.stable_dt(shape, h, bc, cn, pe), 0.4 * h)
    return h, cn, pe, dt, C0, vel


def make(shape, h, bc, cn, pe, dt, C0, prec, vel=None):
    from paper_2105_01865_gb300.solver import Solver
    s = Solver(shape, h, bc, cn, pe, dt, C0, precision=prec, advect=vel is not None)
    if vel is not None:
        s.set_velocity_fine(*vel)
    return s


@pytest.mark.parametrize("shape,bc,advect", [
    ((12, 10, 16), (P, P, D), False),
    ((20, 17, 34), (N, P, D), True),     # even nx: paired kernels, two-column z solve
    ((9, 11, 33), (P, N, D), True),      # odd nx: scalar kernel, one-column z solve
    ((5, 6, 5), (N, N, D), False),       # minimum size
])
def test_fp64_step_matches_oracle(shape, bc, advect):
    h, cn, pe, dt, C0, vel = case(shape, bc, 3, advect)
    s = make(shape, h, bc, cn, pe, dt, C0, "f64", vel)
    s.step(6)
    nz, ny, nx = shape
    p = co.Params(nx, ny, nz, h, cn=cn, pe=pe, dt=dt, bc=bc)
    ref = co.step(C0, vel, p, 6)
    assert_parity(s.field(), ref, 1e-12, f"FP64 Dirichlet z {shape} {bc}, 6 steps")
    assert abs(s.free_energy() - co.free_energy(ref, p)) <= 1e-12 * abs(co.free_energy(ref, p))


def test_fp32_step_matches_oracle():
    shape, bc = (24, 20, 32), (P, P, D)
    h, cn, pe, dt, C0, vel = case(shape, bc, 7, True)
    s = make(shape, h, bc, cn, pe, dt, C0, "f32", vel)
    s.step(20)
    nz, ny, nx = shape
    ref = co.step(C0.astype(np.float32).astype(np.float64), vel, co.Params(nx, ny, nz, h, cn=cn, pe=pe, dt=dt,
                                                                          bc=bc), 20)
    assert_parity(s.field(), ref, 1e-5, "FP32 Dirichlet z, 32x20x24, 20 steps")


def test_transfer_treats_dirichlet_as_a_wall():
    from paper_2105_01865_gb300.solver import Solver
    fine_n, h = (40, 36, 20), 1.0 / 20
    box = (2.0, 1.8, 1.0)
    faces = (inputs.uniform_faces(10, box[0]), inputs.uniform_faces(9, box[1]), inputs.stretched_faces(7, box[2], 2.0))
    uc, vc, wc = inputs.curl_velocity(*faces, (P, P, N), 3, kmax=4)
    out = []
    for bcz in (N, D):
        nx, ny, nz = fine_n
        s = Solver((nz, ny, nx), h, (P, P, bcz), 0.75 * h, 100.0, 1e-3, np.zeros((nz, ny, nx)), precision="f64",
                   coarse_faces=faces)
        s.set_velocity_coarse(uc, vc, wc)
        s.interp_to_fine()
        out.append([t.cpu().numpy() for t in s.velocity_fine()])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
