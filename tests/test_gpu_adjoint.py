"""GPU tests of the differentiation form (u = 0): the library's adjoint
against the oracle's adjoint, against central finite differences of the
library's own forward (step 1e-4, relative for M), and through
torch.autograd."""
import numpy as np
import pytest

from oracle import ch_adjoint as ca
from oracle import ch_oracle as co
from paper_2105_01865_gb300 import inputs, stability

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2105_01865_gb300 import build, capi
    build.build()
    capi.load()


def small_case(bc, seed):
    rng = np.random.default_rng(seed)
    shape = (10, 12, 14)
    h = 1.0 / 14
    cn = 0.75 * h
    C0 = inputs.drops_field(shape, h, bc, [(0.5, 0.4, 0.35)], [0.25], cn) + 0.05 * rng.standard_normal(shape)
    pe = 30.0
    dt = 0.5 * stability.stable_dt(shape, h, bc, cn, pe)
    lamT = rng.standard_normal(shape)
    return shape, h, cn, pe, dt, C0, lamT


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("bc", [(co.PERIODIC,) * 3, (co.PERIODIC, co.NOFLUX, co.NOFLUX), (co.NOFLUX,) * 3])
@pytest.mark.parametrize("ckpt", [1, 2, 5])
def test_fp64_adjoint_matches_oracle(bc, ckpt):
    from paper_2105_01865_gb300.solver import Solver
    shape, h, cn, pe, dt, C0, lamT = small_case(bc, 3)
    nsteps = 5
    s = Solver(shape, h, bc, cn, pe, dt, C0, precision="f64")
    lam0, dM = s.adjoint(C0, nsteps, lamT, ckpt)
    nz, ny, nx = shape
    p = co.Params(nx, ny, nz, h, cn=cn, pe=pe, dt=dt, bc=bc)
    ref0, refM = ca.rollout_adjoint(C0, nsteps, lamT, p)
    assert rel(lam0.cpu().numpy(), ref0) <= 1e-11
    assert abs(dM - refM) <= 1e-11 * abs(refM)


def test_fp32_adjoint_matches_oracle():
    from paper_2105_01865_gb300.solver import Solver
    bc = (co.PERIODIC, co.PERIODIC, co.NOFLUX)
    shape, h, cn, pe, dt, C0, lamT = small_case(bc, 4)
    nsteps = 6
    s = Solver(shape, h, bc, cn, pe, dt, C0, precision="f32")
    lam0, dM = s.adjoint(C0, nsteps, lamT, 3)
    nz, ny, nx = shape
    p = co.Params(nx, ny, nz, h, cn=cn, pe=pe, dt=dt, bc=bc)
    ref0, refM = ca.rollout_adjoint(C0.astype(np.float32).astype(np.float64), nsteps, lamT.astype(np.float32), p)
    err0 = rel(lam0.cpu().numpy().astype(np.float64), ref0)
    errM = abs(dM - refM) / abs(refM)
    print(f"FP32 adjoint vs oracle: lam0 rel L2 {err0:.2e}, dL/dM rel {errM:.2e}")
    assert err0 <= 1e-5 and errM <= 1e-4


def eight_drop_box(n=128, seed=5):
    """Periodic unit box n^3, 8 drops R ~ U[0.08, 0.15], Cn = 0.75 h, Pe = 1e3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    cn = 0.75 * h
    bc = (co.PERIODIC,) * 3
    centres, radii = inputs.random_drops(rng, 8, (1.0, 1.0, 1.0), 0.08, 0.15, 4 * cn, (False,) * 3)
    C0 = inputs.drops_field((n, n, n), h, bc, centres, radii, cn)
    return (n, n, n), h, bc, cn, C0


def test_gradients_match_central_differences_128cubed():
    """L = h^3 sum (C_T - C_target)^2 after 50 steps (checkpoints every 10):
    dL/dC0 along a seeded direction and dL/dM against central differences
    of the FP64 forward (step 1e-4, relative for M), and the FP32 adjoint
    against the FP64 one."""
    from paper_2105_01865_gb300.solver import Solver
    shape, h, bc, cn, C0 = eight_drop_box()
    pe = 1e3
    dt = 0.9 * stability.stable_dt(shape, h, bc, cn, pe)
    nsteps, ckpt = 50, 10
    # target: a run with mobility x 1.1 from drops shifted by 2h
    tgt0 = np.roll(C0, 2, axis=2)
    t = Solver(shape, h, bc, cn, pe / 1.1, dt, tgt0, precision="f64")
    t.step(nsteps)
    target = t.field()

    def run(C, pe_, prec="f64"):
        s = Solver(shape, h, bc, cn, pe_, dt, C, precision=prec)
        s.step(nsteps)
        return s.field()

    def loss(CT):
        return h ** 3 * float(np.sum((CT - target) ** 2))

    CT = run(C0, pe)
    lamT = 2 * h ** 3 * (CT - target)
    s = Solver(shape, h, bc, cn, pe, dt, C0, precision="f64")
    lam0, dM = s.adjoint(C0, nsteps, lamT, ckpt)
    lam0 = lam0.cpu().numpy()
    v = np.random.default_rng(55).standard_normal(shape)
    M = 1.0 / pe

    def fd_c(eps):
        return (loss(run(C0 + eps * v, pe)) - loss(run(C0 - eps * v, pe))) / (2 * eps)

    def fd_m(eps):
        return (loss(run(C0, 1.0 / (M * (1 + eps)))) - loss(run(C0, 1.0 / (M * (1 - eps))))) / (2 * eps * M)

    # central differences with step 1e-4 carry an O(eps^2) truncation error;
    # Richardson extrapolation with eps/2 removes it
    ad = float(np.sum(lam0 * v))
    f1, f2 = fd_c(1e-4), fd_c(5e-5)
    print(f"dL/dC0.v: adjoint {ad:.10e}  FD(1e-4) {f1:.10e}  Richardson {(4 * f2 - f1) / 3:.10e}")
    assert abs(f1 - ad) <= 1e-4 * abs(ad)
    assert abs((4 * f2 - f1) / 3 - ad) <= 1e-6 * abs(ad)
    g1, g2 = fd_m(1e-4), fd_m(5e-5)
    print(f"dL/dM:    adjoint {dM:.10e}  FD(1e-4) {g1:.10e}  Richardson {(4 * g2 - g1) / 3:.10e}")
    assert abs(g1 - dM) <= 1e-4 * abs(dM)
    assert abs((4 * g2 - g1) / 3 - dM) <= 1e-6 * abs(dM)
    # FP32 forward + adjoint on the same problem
    CT32 = run(C0, pe, "f32")
    s32 = Solver(shape, h, bc, cn, pe, dt, C0, precision="f32")
    lam32, dM32 = s32.adjoint(C0, nsteps, 2 * h ** 3 * (CT32 - target), ckpt)
    e0 = rel(lam32.cpu().numpy().astype(np.float64), lam0)
    eM = abs(dM32 - dM) / abs(dM)
    print(f"FP32 vs FP64 adjoint, 128^3, 50 steps: dL/dC0 rel L2 {e0:.2e}, dL/dM rel {eM:.2e}")
    assert e0 <= 1e-3 and eM <= 1e-3


def test_autograd_function():
    from paper_2105_01865_gb300 import autograd as cag
    from paper_2105_01865_gb300.solver import Solver
    bc = (co.PERIODIC, co.PERIODIC, co.NOFLUX)
    shape, h, cn, pe, dt, C0, _ = small_case(bc, 9)
    target = torch.as_tensor(np.roll(C0, 1, axis=1), dtype=torch.float64, device="cuda")
    C0t = torch.as_tensor(C0, dtype=torch.float64, device="cuda").requires_grad_(True)
    M = torch.tensor(1.0 / pe, dtype=torch.float64, requires_grad=True)
    CT = cag.rollout(C0t, M, shape, h, bc, cn, dt, 7, ckpt_every=3, precision="f64")
    L = h ** 3 * ((CT - target) ** 2).sum()
    L.backward()
    s = Solver(shape, h, bc, cn, pe, dt, C0, precision="f64")
    lam0, dM = s.adjoint(C0, 7, (2 * h ** 3 * (CT.detach() - target)).cpu().numpy(), 3)
    assert torch.allclose(C0t.grad, lam0, rtol=0, atol=1e-14 * float(lam0.abs().max()))
    assert abs(float(M.grad) - dM) <= 1e-12 * abs(dM)
