"""Plain FP64 CPU oracle of the adjoint (reverse-mode derivative) of the
Cahn-Hilliard step without advection (u = 0).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this module.

The forward substep l is the one of ``ch_oracle.substep`` (Sec. 3, Eqs.
eq-re .. eq-fac-3 of arXiv 2105.01865) with u = 0:
    H  = M lap(psi'(C))
    r  = dt (gamma_l H + rho_l Hp) - alpha_l dt M A C,     A = A_x + A_y + A_z
    dq = P^-1 r,  P = P_x P_y P_z,  P_d = I + c A_d,  c = alpha_l dt M / 2
    C' = C + dq,  and H is the next substep's Hp.
Every operator is symmetric (wrapped or mirrored stencils) and the P_d act
on different axes, so they commute.  Its transpose, for adjoints lam_C' of C'
and lam_H' of H (as next substep's Hp), is:
    lam_r  = P^-1 lam_C'
    lam_H  = dt gamma_l lam_r + lam_H'
    lam_Hp = dt rho_l lam_r
    lam_C  = lam_C' - alpha_l dt M A lam_r + psi''(C) M lap(lam_H)
    dL/dM += <lam_H, lap psi'(C)> - alpha_l dt <lam_r, A C>
             - (alpha_l dt / 2) sum_d <A_d lam_r, P_d^-1 r>
The last term is d(P^-1)/dM: -P^-1 (dP/dM) P^-1 r with dP/dM =
(alpha_l dt / 2) sum_d A_d prod_{e != d} P_e, and prod_{e != d} P_e P^-1 = P_d^-1.
"""
from __future__ import annotations

import numpy as np

from oracle import ch_oracle as co


def psi_pp(C):
    """psi''(C) = 3 C^2 - 3 C + 1/2."""
    return 3.0 * C ** 2 - 3.0 * C + 0.5


def apply_A_all(f, p):
    return co.apply_A(f, p, 0) + co.apply_A(f, p, 1) + co.apply_A(f, p, 2)


def substep_parts(C, Hp, p, l):
    """Forward pieces of substep l (u = 0): H, r and dq."""
    g, rho, a = co.RK3_GAMMA[l], co.RK3_RHO[l], co.RK3_ALPHA[l]
    M = p.mobility
    H = M * co.lap_h(co.psi_prime(C), p)
    r = p.dt * (g * H + rho * Hp) - a * p.dt * M * apply_A_all(C, p)
    c = a * p.dt * M / 2.0
    dq = co.line_solve(co.line_solve(co.line_solve(r, p, 0, c), p, 1, c), p, 2, c)
    return H, r, dq


def substep_adjoint(C, Hp, lamC_next, lamH_next, p, l):
    """Reverse substep l: returns (lam_C, lam_Hp, dL/dM contribution)."""
    g, rho, a = co.RK3_GAMMA[l], co.RK3_RHO[l], co.RK3_ALPHA[l]
    M = p.mobility
    c = a * p.dt * M / 2.0
    _, r, _ = substep_parts(C, Hp, p, l)
    lam_r = co.line_solve(co.line_solve(co.line_solve(lamC_next, p, 0, c), p, 1, c), p, 2, c)
    lam_H = p.dt * g * lam_r + lamH_next
    lam_Hp = p.dt * rho * lam_r
    lam_C = lamC_next - a * p.dt * M * apply_A_all(lam_r, p) + psi_pp(C) * (M * co.lap_h(lam_H, p))
    dM = np.sum(lam_H * co.lap_h(co.psi_prime(C), p))
    dM -= a * p.dt * np.sum(lam_r * apply_A_all(C, p))
    for d in range(3):
        dM -= 0.5 * a * p.dt * np.sum(co.apply_A(lam_r, p, d) * co.line_solve(r, p, d, c))
    return lam_C, lam_Hp, float(dM)


def step_adjoint(C_start, lam_end, p):
    """Reverse one full RK3 step from its start state; returns (lam_start, dL/dM)."""
    Cs, Hps = [], []
    C = np.array(C_start, dtype=np.float64)
    Hp = np.zeros(p.shape)
    for l in range(3):
        Cs.append(C)
        Hps.append(Hp)
        H, _, dq = substep_parts(C, Hp, p, l)
        C = C + dq
        Hp = H
    lamC, lamH, dM = lam_end, np.zeros(p.shape), 0.0
    for l in (2, 1, 0):
        lamC, lamH, d = substep_adjoint(Cs[l], Hps[l], lamC, lamH, p, l)
        dM += d
    return lamC, dM


def rollout_adjoint(C0, nsteps, lam_T, p):
    """Reverse nsteps steps from C0 (all step states recomputed and kept)."""
    states = [np.array(C0, dtype=np.float64)]
    for _ in range(nsteps - 1):
        states.append(co.step(states[-1], None, p, 1))
    lam, dM = np.array(lam_T, dtype=np.float64), 0.0
    for s in range(nsteps - 1, -1, -1):
        lam, d = step_adjoint(states[s], lam, p)
        dM += d
    return lam, dM


def loss(CT, target, p):
    """L = h^3 sum (C_T - C_target)^2."""
    return p.h ** 3 * float(np.sum((CT - target) ** 2))


def loss_gradient(C0, target, nsteps, p):
    """L, dL/dC0 and dL/dM of the nsteps rollout."""
    CT = co.step(C0, None, p, nsteps)
    lam_T = 2.0 * p.h ** 3 * (CT - target)
    lam0, dM = rollout_adjoint(C0, nsteps, lam_T, p)
    return loss(CT, target, p), lam0, dM
