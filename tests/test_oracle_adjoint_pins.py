"""Pins of the oracle adjoint: transposition identities against the exact
complex-step derivative of the oracle's forward step, and the loss gradient
against central finite differences (step 1e-4, relative for M)."""
import numpy as np
import pytest

from oracle import ch_adjoint as ca
from oracle import ch_oracle as co
from oracle.ch_oracle import NOFLUX, PERIODIC, Params

EPS = 1e-30


def setup(bc, seed=0):
    shape = (6, 7, 8)
    h = 1.0 / 8
    rng = np.random.default_rng(seed)
    C0 = 0.5 + 0.35 * rng.standard_normal(shape)
    p = Params(8, 7, 6, h, cn=0.75 * h, pe=20.0, dt=0.01, bc=bc)
    return C0, p, rng


def with_mobility(p, M):
    return Params(p.nx, p.ny, p.nz, p.h, cn=p.cn, pe=1.0 / M, dt=p.dt, bc=p.bc, w=p.w, eps=p.eps)


@pytest.mark.parametrize("bc", [(PERIODIC, PERIODIC, PERIODIC), (PERIODIC, NOFLUX, NOFLUX), (NOFLUX,) * 3])
def test_adjoint_transposes_complex_step_jvp(bc):
    C0, p, rng = setup(bc, 1)
    nsteps = 3
    v = rng.standard_normal(C0.shape)
    w = rng.standard_normal(C0.shape)
    # exact forward-mode derivatives by the complex step (no cancellation)
    Jv = np.imag(co.step(C0 + 1j * EPS * v, None, p, nsteps)) / EPS
    M = p.mobility
    JM = np.imag(co.step(C0, None, with_mobility(p, M + 1j * EPS), nsteps)) / EPS
    lam0, dM = ca.rollout_adjoint(C0, nsteps, w, p)
    lhs = float(np.sum(Jv * w))
    assert abs(lhs - float(np.sum(v * lam0))) <= 1e-12 * abs(lhs)
    lhsM = float(np.sum(JM * w))
    assert abs(lhsM - dM) <= 1e-12 * abs(lhsM)


def test_loss_gradient_matches_central_differences():
    C0, p, rng = setup((PERIODIC, PERIODIC, NOFLUX), 2)
    target = co.step(C0 + 0.1 * rng.standard_normal(C0.shape), None, p, 2)
    nsteps = 4
    L, g0, gM = ca.loss_gradient(C0, target, nsteps, p)
    v = rng.standard_normal(C0.shape)
    hstep = 1e-4
    Lp = ca.loss(co.step(C0 + hstep * v, None, p, nsteps), target, p)
    Lm = ca.loss(co.step(C0 - hstep * v, None, p, nsteps), target, p)
    fd = (Lp - Lm) / (2 * hstep)
    assert abs(fd - np.sum(g0 * v)) <= 1e-6 * abs(fd)
    M = p.mobility
    LpM = ca.loss(co.step(C0, None, with_mobility(p, M * (1 + hstep)), nsteps), target, p)
    LmM = ca.loss(co.step(C0, None, with_mobility(p, M * (1 - hstep)), nsteps), target, p)
    fdM = (LpM - LmM) / (2 * hstep * M)
    assert abs(fdM - gM) <= 1e-6 * abs(fdM)
