"""GPU parity of the down-sampling back-coupling (Sec. 3.4) and the coarse
density, viscosity and surface tension (Eqs. eq-rho, eq-mu, eq-fst) against
the oracle's restrict_to_coarse: FP64 to 1e-12 and FP32 within its rounding
(relative to each field's largest magnitude)."""
import numpy as np
import pytest

from oracle import ch_oracle as co
from oracle import mr_oracle as mo
from paper_2105_01865_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PER, WALL = co.PERIODIC, co.NOFLUX


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2105_01865_gb300 import build, capi
    build.build()
    capi.load()


def case(fine_n, h, nc, bc, seed):
    nx, ny, nz = fine_n
    box = (nx * h, ny * h, nz * h)
    faces = tuple(inputs.stretched_faces(m, L, 2.0) if b == WALL else inputs.uniform_faces(m, L)
                  for m, L, b in zip(nc, box, bc))
    rng = np.random.default_rng(seed)
    cn = 0.75 * h
    centres, radii = inputs.random_drops(rng, 3, box, 0.1, 0.25, 2 * cn, tuple(b == WALL for b in bc))
    shape = (nz, ny, nx)
    C = inputs.drops_field(shape, h, bc, centres, radii, cn) + 0.02 * rng.standard_normal(shape)
    return faces, C, cn


@pytest.mark.parametrize("prec,tol,ftol", [("f64", 1e-12, 1e-12), ("f32", 2e-6, 2e-5)])
@pytest.mark.parametrize("bc,nc", [((PER, PER, WALL), (10, 9, 7)), ((WALL, PER, PER), (13, 6, 5)),
                                   ((PER, PER, PER), (12, 9, 5))])
def test_restriction_matches_oracle(prec, tol, ftol, bc, nc):
    from paper_2105_01865_gb300.solver import Solver
    fine_n, h = (40, 36, 20), 1.0 / 20
    faces, C, cn = case(fine_n, h, nc, bc, 4)
    nx, ny, nz = fine_n
    s = Solver((nz, ny, nx), h, bc, cn, 0.9 / cn, 1e-3, C, precision=prec, coarse_faces=faces)
    lam_rho, lam_mu = 0.05, 0.3
    for _ in range(2):  # twice in a row: the workspace is reused
        got = {k: v.cpu().numpy().astype(np.float64) for k, v in s.restrict_to_coarse(lam_rho, lam_mu).items()}
        s.sync()
    p = co.Params(nx, ny, nz, h, cn=cn, pe=0.9 / cn, dt=1e-3, bc=bc)
    Cin = C.astype(np.float32).astype(np.float64) if prec == "f32" else C
    Cc, rho, mu, F = mo.restrict_to_coarse(Cin, p, *faces, lam_rho, lam_mu)
    ref = dict(C=Cc, rho=rho, mu=mu, Fx=F[0], Fy=F[1], Fz=F[2])
    for k, r in ref.items():
        assert got[k].shape == r.shape == (nc[2], nc[1], nc[0])
        t = ftol if k.startswith("F") else tol
        err = np.abs(got[k] - r).max() / np.abs(r).max()
        assert err <= t, (k, err)
