"""GPU parity of the standard explicit comparison scheme (Sec. 3.1, Eq.
eq-disbi: the 25-point biharmonic, every term explicit in the same RK3)
against the oracle's step_standard on the same seeded inputs.

Bars as for the split scheme: FP64 <= 1e-12 relative L2 on C, FP32 <= 1e-5,
mass conserved to rounding."""
import numpy as np
import pytest

from oracle import ch_oracle as co
from paper_2105_01865_gb300 import inputs, stability

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


def make(shape, h, bc, cn, pe, dt, C0, prec, vel=None):
    from paper_2105_01865_gb300.solver import Solver
    s = Solver(shape, h, bc, cn, pe, dt, C0, precision=prec, advect=vel is not None, scheme="standard")
    if vel is not None:
        s.set_velocity_fine(*vel)
    return s


def params(shape, h, bc, cn, pe, dt):
    nz, ny, nx = shape
    return co.Params(nx, ny, nz, h, cn=cn, pe=pe, dt=dt, bc=bc)


def case(shape, bc, seed, advect):
    h = 1.0 / 16
    cn = 0.75 * h
    pe = 0.9 / cn
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    centres, radii = inputs.random_drops(rng, 3, (nx * h, ny * h, nz * h), 0.05, 0.15, 2 * cn,
                                         tuple(b == co.NOFLUX for b in bc))
    C0 = inputs.drops_field(shape, h, bc, centres, radii, cn) + 0.05 * rng.standard_normal(shape)
    vel = None
    if advect:
        vel = inputs.curl_velocity(inputs.uniform_faces(nx, nx * h), inputs.uniform_faces(ny, ny * h),
                                   inputs.uniform_faces(nz, nz * h), bc, seed, kmax=3)
    dt = 0.9 * min(stability.stable_dt_standard(shape, h, bc, cn, pe), 0.4 * h)
    return h, cn, pe, dt, C0, vel


@pytest.mark.parametrize("shape,bc,advect", [
    ((9, 17, 33), (co.NOFLUX, co.PERIODIC, co.NOFLUX), True),     # odd nx: scalar advection kernel
    ((20, 10, 70), (co.PERIODIC, co.PERIODIC, co.NOFLUX), True),  # even nx: paired advection kernel
    ((6, 5, 6), (co.PERIODIC, co.NOFLUX, co.PERIODIC), True),     # minimum even size
    ((5, 6, 5), (co.NOFLUX, co.NOFLUX, co.NOFLUX), False),        # minimum size, all walls, u = 0
    ((12, 40, 36), (co.PERIODIC,) * 3, False),                    # several tiles, ragged y
])
def test_fp64_matches_oracle(shape, bc, advect):
    h, cn, pe, dt, C0, vel = case(shape, bc, 3, advect)
    s = make(shape, h, bc, cn, pe, dt, C0, "f64", vel)
    s.step(8)
    ref = co.step_standard(C0, vel, params(shape, h, bc, cn, pe, dt), 8)
    assert_parity(s.field(), ref, 1e-12, f"FP64 standard scheme {shape} {bc}, 8 steps")


def test_fp32_matches_oracle_and_conserves_mass():
    shape, bc = (24, 20, 32), (co.PERIODIC, co.PERIODIC, co.NOFLUX)
    h, cn, pe, dt, C0, vel = case(shape, bc, 7, True)
    s = make(shape, h, bc, cn, pe, dt, C0, "f32", vel)
    m0 = s.mass()
    s.step(40)
    ref = co.step_standard(C0.astype(np.float32).astype(np.float64), vel, params(shape, h, bc, cn, pe, dt), 40)
    assert_parity(s.field(), ref, 1e-5, "FP32 standard scheme 32x20x24, 40 steps")
    assert abs(s.mass() - m0) <= 1e-6 * abs(m0)


def test_fp64_mass_conserved_with_walls_and_shear():
    f = inputs.shear_drop_box(48, 32, 24)
    h = f["h"]
    dt = 0.9 * min(stability.stable_dt_standard(f["shape"], h, f["bc"], f["cn"], f["pe"]), 0.5 * h / 0.5)
    s = make(f["shape"], h, f["bc"], f["cn"], f["pe"], dt, f["C"], "f64", f["vel"])
    m0 = s.mass()
    s.step(60)
    assert abs(s.mass() - m0) <= 1e-13 * abs(m0)


def test_launch_count_and_adjoint_refused():
    from paper_2105_01865_gb300 import capi
    shape, bc = (8, 8, 8), (co.PERIODIC,) * 3
    h, cn, pe, dt, C0, vel = case(shape, bc, 1, True)
    assert make(shape, h, bc, cn, pe, dt, C0, "f32", vel).launches_per_step() == 9
    s = make(shape, h, bc, cn, pe, dt, C0, "f32")
    assert s.launches_per_step() == 6
    with pytest.raises(capi.CHError):
        s.adjoint(C0, 2, np.ones(shape), 1)


def test_full_size_shear_drop_one_step():
    """The bench's comparison box (256 x 256 x 128 shear drop, FP32) at the
    standard scheme's stable dt: one step against the oracle."""
    f = inputs.shear_drop_box(256, 256, 128)
    h = f["h"]
    dt = min(0.9 * stability.stable_dt_standard(f["shape"], h, f["bc"], f["cn"], f["pe"]), 0.5 * h / 0.5)
    s = make(f["shape"], h, f["bc"], f["cn"], f["pe"], dt, f["C"], "f32", f["vel"])
    s.step(1)
    ref = co.step_standard(f["C"].astype(np.float32).astype(np.float64), f["vel"],
                           params(f["shape"], h, f["bc"], f["cn"], f["pe"], dt), 1)
    assert_parity(s.field(), ref, 1e-6, "FP32 standard scheme 256x256x128, 1 step")
