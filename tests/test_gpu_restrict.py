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


def _bc_index(i, n, bc):
    """Ghost rule of the step: wrap, or the mirror about a wall face."""
    i = np.asarray(i)
    if bc == PER:
        return i % n
    return np.where(i < 0, -1 - i, np.where(i >= n, 2 * n - 1 - i, i))


def test_full_size_restriction_sampled_cells():
    """Fine 1024 x 1024 x 512 (h = 1/512) down-sampled to the tanh-stretched
    256 x 256 x 128 mesh in FP32, as the bench times it: sampled coarse cells
    against the oracle evaluated on the 6 x 6 x 6 block of fine cells that
    their stencil and its neighbours touch."""
    from paper_2105_01865_gb300.solver import Solver
    bc = (PER, PER, WALL)
    fine_n, h = (1024, 1024, 512), 1.0 / 512
    nx, ny, nz = fine_n
    faces = (inputs.uniform_faces(256, 2.0), inputs.uniform_faces(256, 2.0), inputs.stretched_faces(128, 1.0, 2.0))
    cn = 0.75 * h
    rng = np.random.Generator(np.random.PCG64(8))
    centres, radii = inputs.random_drops(rng, 60, (2.0, 2.0, 1.0), 0.02, 0.05, 4 * cn, (True, True, True))
    C = inputs.drops_field_local((nz, ny, nx), h, centres, radii, cn, 8 * cn)
    s = Solver((nz, ny, nx), h, bc, cn, 0.9 / cn, 1e-4, C, precision="f32", coarse_faces=faces)
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in s.restrict_to_coarse(0.05, 0.3).items()}
    s.close()
    scale = {k: np.abs(v).max() for k, v in out.items()}
    assert scale["Fx"] > 0 and scale["Fz"] > 0
    tabs = mo.restriction_tables(*faces, fine_n, h, bc)
    # sampled cells: near drops (large F_st), at both walls, and random
    big = np.argwhere(np.abs(out["Fz"]) > 0.3 * scale["Fz"])
    pick = [tuple(big[q]) for q in rng.choice(len(big), size=8, replace=False)]
    pick += [(0, 17, 40), (127, 200, 3), (1, 255, 255), (126, 0, 128)]
    pick += [tuple(int(rng.integers(n)) for n in (128, 256, 256)) for _ in range(6)]
    Cf = C.astype(np.float64)
    for kc, jc, ic in pick:
        (sx, wx), (sy, wy), (sz, wz) = tabs[0], tabs[1], tabs[2]
        ix = _bc_index(sx[ic] - 1 + np.arange(6), nx, bc[0])
        jy = _bc_index(sy[jc] - 1 + np.arange(6), ny, bc[1])
        kz = _bc_index(sz[kc] - 1 + np.arange(6), nz, bc[2])
        block = Cf[np.ix_(kz, jy, ix)]
        pb = co.Params(6, 6, 6, h, cn=cn, pe=0.9 / cn, dt=1e-4)   # the block carries its own ghosts
        F = co.surface_tension(block, pb)
        wt = wz[kc][:, None, None] * wy[jc][None, :, None] * wx[ic][None, None, :]
        ref = dict(C=float(np.sum(wt * block[1:5, 1:5, 1:5])))
        for name, f in zip(("Fx", "Fy", "Fz"), F):
            ref[name] = float(np.sum(wt * f[1:5, 1:5, 1:5]))
        ref["rho"] = ref["C"] + 0.05 * (1 - ref["C"])
        ref["mu"] = ref["C"] + 0.3 * (1 - ref["C"])
        for name, r in ref.items():
            tol = 2e-5 if name.startswith("F") else 2e-6
            assert abs(out[name][kc, jc, ic] - r) <= tol * scale[name], (name, (kc, jc, ic), out[name][kc, jc, ic], r)
