"""Plain FP64 CPU oracle of the Cahn-Hilliard fine-grid time step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this module.  The CUDA
library never calls it, and this module never imports the CUDA side.

It follows "An efficient phase-field method for turbulent multiphase flows"
(Liu, Ng, Chong, Lohse, Verzicco; arXiv 2105.01865) step by step:

* Sec. 2.1, Eq. (eq-ch): dC/dt + div(uC) = (1/Pe)[-Cn^2 lap^2 C + lap(C^3 - 1.5C^2 + 0.5C)].
* Sec. 3: staggered mesh, C at cell centres of a uniform mesh of spacing h,
  low-storage RK3 for all terms, Crank-Nicolson for the biharmonic term,
  second-order central differences for lap(psi'), fifth-order WENO for div(uC).
* Sec. 3.1, Eq. (eq-a3d): the biharmonic term is replaced by a sum of three
  one-dimensional pentadiagonal operators A_x + A_y + A_z.
* Sec. 3.1, Eqs. (eq-re), (eq-fac), (eq-fac-1..3): Crank-Nicolson in delta
  form, approximately factorised into an x-, a y- and a z-line solve.

Readings where the paper is silent:
* RK3 coefficients (gamma, rho) = (8/15, 0), (5/12, -17/60), (3/4, -5/12) and
  the per-substep Crank-Nicolson step alpha_l*dt, alpha_l = gamma_l + rho_l
  (the low-storage scheme the paper cites for Sec. 3).
* A_d = (w Cn^2 / h^4) [1, -4, 6, -4, 1]; the printed 3D operator is w = 4,
  a re-derivation from Eq. (eq-trans1) gives w = 3; w is a parameter.
* No-flux walls mirror the field about the wall face (ghost C_{-1-m} = C_m);
  periodic directions wrap.  Wall faces carry zero advective flux.
* WENO5 is the Jiang-Shu variant (eps = 1e-6, power 2) applied to C with the
  upwind side chosen by the sign of the face velocity.
* The mass correction the paper cites (Sec. 2.1) is not applied.

Everything is written with whole-array numpy operations in float64 and a
dense LU solve per line direction (scipy), with no blocking or fusion, so
that each function can be read against the equation it cites.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

PERIODIC = 0
NOFLUX = 1
DIRICHLET = 2   # C = 0 on the wall faces (the Rayleigh-Benard walls of Sec. 4.3); walls for the flow

# Low-storage RK3 of Sec. 3 (coefficients not printed in the paper; the
# published three-substep scheme of the cited RK reference).
RK3_GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RK3_RHO = (0.0, -17.0 / 60.0, -5.0 / 12.0)
RK3_ALPHA = tuple(g + r for g, r in zip(RK3_GAMMA, RK3_RHO))


@dataclass
class Params:
    """Problem definition on the fine uniform mesh (Sec. 3, uniform h).

    Arrays are indexed [z][y][x] (x fastest).  ``bc`` is (bc_x, bc_y, bc_z).
    M = 1/Pe (Eq. eq-ch).  ``w`` is the biharmonic weight of Eq. (eq-a3d)
    (4 as printed).  ``eps`` is the WENO regulariser.
    """

    nx: int
    ny: int
    nz: int
    h: float
    cn: float
    pe: float
    dt: float
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)
    w: float = 4.0
    eps: float = 1e-6

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def mobility(self):
        return 1.0 / self.pe

    @property
    def kappa(self):
        """Prefactor of A_d: w Cn^2 / h^4 (Eq. eq-a3d with Cn = 0.75 h / L, L = 1)."""
        return self.w * self.cn ** 2 / self.h ** 4

    def n(self, d):
        return (self.nx, self.ny, self.nz)[d]

    def nfaces(self, d):
        """Number of face-velocity planes normal to direction d (staggered mesh)."""
        return self.n(d) + (1 if self.bc[d] != PERIODIC else 0)


# ---------------------------------------------------------------------------
# Double-well potential, Sec. 1 and Eq. (eq-ch)
# ---------------------------------------------------------------------------

def psi(C):
    """Bulk free energy density psi = C^2 (C - 1)^2 / 4 (Sec. 1)."""
    return 0.25 * C ** 2 * (C - 1.0) ** 2


def psi_prime(C):
    """psi'(C) = C^3 - 1.5 C^2 + 0.5 C, the bracket of Eq. (eq-ch)."""
    return C ** 3 - 1.5 * C ** 2 + 0.5 * C


# ---------------------------------------------------------------------------
# Ghost cells and shifts
# ---------------------------------------------------------------------------

def _axis(d):
    return 2 - d  # direction x=0,y=1,z=2 -> numpy axis of a [z][y][x] array


def pad(f, bc, g):
    """Add g ghost layers per side: wrap (periodic), mirror about the wall face
    (no-flux), or mirror with the sign flipped (Dirichlet C = 0 on the wall
    face: the ghost C_{-1-m} = -C_m)."""
    for d in range(3):
        width = [(0, 0)] * 3
        a = _axis(d)
        width[a] = (g, g)
        f = np.pad(f, width, mode="wrap" if bc[d] == PERIODIC else "symmetric")
        if bc[d] == DIRICHLET:
            f = f.copy()
            lo = [slice(None)] * 3
            lo[a] = slice(0, g)
            hi = [slice(None)] * 3
            hi[a] = slice(f.shape[a] - g, f.shape[a])
            f[tuple(lo)] *= -1.0
            f[tuple(hi)] *= -1.0
    return f


def shifted(fp, g, d, s, shape):
    """Interior-shaped view of a g-padded array, shifted by s cells along d."""
    sl = [slice(g, g + n) for n in shape]
    a = _axis(d)
    sl[a] = slice(g + s, g + s + shape[a])
    return fp[tuple(sl)]


# ---------------------------------------------------------------------------
# Explicit terms of Sec. 3
# ---------------------------------------------------------------------------

def lap_h(f, p: Params):
    """Second-order central 7-point Laplacian (Sec. 3, 'central second-order')."""
    fp = pad(f, p.bc, 1)
    out = np.zeros(p.shape, dtype=np.result_type(f, 1.0))
    for d in range(3):
        out = out + (shifted(fp, 1, d, 1, p.shape) - 2.0 * f + shifted(fp, 1, d, -1, p.shape)) / p.h ** 2
    return out


def apply_A(C, p: Params, d):
    """(A_d C)_i = kappa (C_{i-2} - 4C_{i-1} + 6C_i - 4C_{i+1} + C_{i+2}) along d (Eq. eq-a3d)."""
    Cp = pad(C, p.bc, 2)
    s = lambda k: shifted(Cp, 2, d, k, p.shape)
    return p.kappa * (s(-2) - 4.0 * s(-1) + 6.0 * C - 4.0 * s(1) + s(2))


def weno5_reconstruct(v1, v2, v3, v4, v5, eps):
    """Fifth-order WENO (Jiang-Shu) value at the face between v3 and v4,
    biased towards v1..v3 (the upwind side).  Sec. 3: 'fifth-order WENO'."""
    q0 = (2.0 * v1 - 7.0 * v2 + 11.0 * v3) / 6.0
    q1 = (-v2 + 5.0 * v3 + 2.0 * v4) / 6.0
    q2 = (2.0 * v3 + 5.0 * v4 - v5) / 6.0
    b0 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) ** 2 + 0.25 * (v1 - 4.0 * v2 + 3.0 * v3) ** 2
    b1 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
    b2 = 13.0 / 12.0 * (v3 - 2.0 * v4 + v5) ** 2 + 0.25 * (3.0 * v3 - 4.0 * v4 + v5) ** 2
    a0 = 0.1 / (eps + b0) ** 2
    a1 = 0.6 / (eps + b1) ** 2
    a2 = 0.3 / (eps + b2) ** 2
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2)


def face_fluxes(C, vel, p: Params, d):
    """Advective flux u_f * C_f through the lower face of every cell along d.

    ``vel`` holds the face-normal velocity on the nfaces(d) face planes of the
    staggered mesh; face f lies between cells f-1 and f.  Returns an array of
    nfaces(d) planes along d.  Wall faces (no-flux) carry zero flux.
    """
    g = 3
    Cp = pad(C, p.bc, g)
    s = lambda k: shifted(Cp, g, d, k, p.shape)
    n = p.n(d)
    a = _axis(d)
    # Upwind for u >= 0: cells f-3..f+1 ; for u < 0: cells f+2..f-2 (mirrored).
    left = weno5_reconstruct(s(-3), s(-2), s(-1), s(0), s(1), p.eps)
    right = weno5_reconstruct(s(2), s(1), s(0), s(-1), s(-2), p.eps)
    vlow = np.take(vel, np.arange(n), axis=a)          # velocity at face f = lower face of cell f
    Cf = np.where(vlow >= 0.0, left, right)
    F = vlow * Cf
    if p.bc[d] != PERIODIC:
        F = F.copy()
        idx = [slice(None)] * 3
        idx[a] = 0
        F[tuple(idx)] = 0.0                              # wall at the lower boundary
        zero = np.zeros_like(np.take(F, [0], axis=a))
        F = np.concatenate([F, zero], axis=a)            # wall at the upper boundary
    return F


def advection(C, vel, p: Params):
    """-div(u C) = -sum_d (F_{f+1} - F_f) / h, conservative (Sec. 3)."""
    out = np.zeros(p.shape, dtype=np.result_type(C, 1.0))
    for d in range(3):
        F = face_fluxes(C, vel[d], p, d)
        a = _axis(d)
        n = p.n(d)
        lower = np.take(F, np.arange(n), axis=a)
        upper = np.take(F, (np.arange(n) + 1) % F.shape[a], axis=a)
        out = out - (upper - lower) / p.h
    return out


# ---------------------------------------------------------------------------
# Implicit biharmonic: the line operators and the factorised solve
# ---------------------------------------------------------------------------

def line_operator(n, bc, kappa):
    """Dense n x n matrix of the 1D pentadiagonal operator A_d of Eq. (eq-a3d).

    Each row applies kappa*[1, -4, 6, -4, 1]; neighbours beyond the boundary
    are the wrapped (periodic) or mirrored (no-flux wall) cells, the mirrored
    ones with a sign flip for a Dirichlet wall, which fixes the 'first and last
    rows determined by boundary conditions' of Eq. (eq-a2d).
    """
    A = np.zeros((n, n))
    for i in range(n):
        for s, c in zip((-2, -1, 0, 1, 2), (1.0, -4.0, 6.0, -4.0, 1.0)):
            j = i + s
            sign = 1.0
            if bc == PERIODIC:
                j %= n
            elif j < 0:
                j = -1 - j
                sign = -1.0 if bc == DIRICHLET else 1.0
            elif j >= n:
                j = 2 * n - 1 - j
                sign = -1.0 if bc == DIRICHLET else 1.0
            A[i, j] += sign * kappa * c
    return A


def line_solve(rhs, p: Params, d, c):
    """Solve (I + c A_d) x = rhs along every line of direction d (Eq. eq-fac-1..3)."""
    n = p.n(d)
    Mat = np.eye(n) + c * line_operator(n, p.bc[d], p.kappa)
    a = _axis(d)
    R = np.moveaxis(rhs, a, 0)
    shp = R.shape
    X = scipy.linalg.solve(Mat, R.reshape(n, -1))
    return np.moveaxis(X.reshape(shp), 0, a)


# ---------------------------------------------------------------------------
# One full RK3 step (Sec. 3 and Eqs. eq-example .. eq-fac-3)
# ---------------------------------------------------------------------------

def explicit_H(C, vel, p: Params, psi_p=psi_prime):
    """Explicit right-hand side H = -div(uC) + M lap(psi'(C))  (Eq. eq-ch)."""
    H = p.mobility * lap_h(psi_p(C), p)
    if vel is not None:
        H = H + advection(C, vel, p)
    return H


def substep(C, Hprev, vel, p: Params, l, psi_p=psi_prime):
    """One RK3 substep l (0-based).  Returns (C_new, H_l).

    In the paper's delta form (Eq. eq-re) with delta-t = alpha_l dt,
    beta = -M and delta-t*E = dt (gamma_l H^l + rho_l H^{l-1}):
      [1 + (alpha_l dt M / 2) sum_d A_d] dq = dt(gamma_l H^l + rho_l H^{l-1})
                                              - alpha_l dt M sum_d A_d C,
    with the left operator factorised as (Eq. eq-fac) and solved by an x-, a y-
    and a z-line solve (Eqs. eq-fac-1, eq-fac-2, eq-fac-3).
    """
    g, r, a = RK3_GAMMA[l], RK3_RHO[l], RK3_ALPHA[l]
    H = explicit_H(C, vel, p, psi_p)
    AC = apply_A(C, p, 0) + apply_A(C, p, 1) + apply_A(C, p, 2)
    rhs = p.dt * (g * H + r * Hprev) - a * p.dt * p.mobility * AC
    c = a * p.dt * p.mobility / 2.0
    dq_star = line_solve(rhs, p, 0, c)          # Eq. (eq-fac-1)
    dq_2star = line_solve(dq_star, p, 1, c)     # Eq. (eq-fac-2)
    dq = line_solve(dq_2star, p, 2, c)          # Eq. (eq-fac-3)
    return C + dq, H


def step(C, vel, p: Params, nsteps=1, psi_p=psi_prime):
    """Advance C by nsteps full RK3 steps (three substeps each).

    ``vel`` is None (u = 0) or a tuple (u, v, w) of face velocities with
    shapes (nz, ny, nfx), (nz, nfy, nx), (nfz, ny, nx).
    """
    C = np.array(C, dtype=np.result_type(C, np.float64), copy=True)
    for _ in range(nsteps):
        Hprev = np.zeros(p.shape, dtype=C.dtype)
        for l in range(3):
            C, Hprev = substep(C, Hprev, vel, p, l, psi_p)
    return C


# ---------------------------------------------------------------------------
# The standard scheme the paper replaces (Sec. 3.1, Eq. eq-disbi): the full
# discrete biharmonic with its mixed derivatives, advanced explicitly
# ---------------------------------------------------------------------------

def biharmonic_h(C, p: Params):
    """Standard discrete biharmonic: the 7-point Laplacian applied twice.

    Written out, this is Eq. (eq-disbi)'s 13-point stencil in 2D (axis
    20, -8, 1 and diagonals 2, times 1/h^4) and its 25-point extension in 3D
    (centre 42, axis neighbours -12 and 1, the 12 edge diagonals 2).  Each
    Laplacian takes the same ghost cells as lap_h, so at a no-flux wall the
    operator is the mirrored (conservative) stencil.
    """
    return lap_h(lap_h(C, p), p)


def explicit_H_standard(C, vel, p: Params, psi_p=psi_prime):
    """H = -div(uC) + M [lap(psi'(C)) - Cn^2 lap^2 C], every term explicit
    (Eq. eq-ch with the biharmonic of Eq. eq-disbi)."""
    H = p.mobility * (lap_h(psi_p(C), p) - p.cn ** 2 * biharmonic_h(C, p))
    if vel is not None:
        H = H + advection(C, vel, p)
    return H


def step_standard(C, vel, p: Params, nsteps=1, psi_p=psi_prime):
    """nsteps of the same low-storage RK3 with all terms explicit:
    C <- C + dt (gamma_l H^l + rho_l H^{l-1}) for l = 1, 2, 3.  This is the
    comparison scheme whose time step the paper reports as limited to 5e-5
    against 2e-3 for the split implicit scheme (Sec. 4.1)."""
    C = np.array(C, dtype=np.result_type(C, np.float64), copy=True)
    for _ in range(nsteps):
        Hprev = np.zeros(p.shape, dtype=C.dtype)
        for l in range(3):
            H = explicit_H_standard(C, vel, p, psi_p)
            C = C + p.dt * (RK3_GAMMA[l] * H + RK3_RHO[l] * Hprev)
            Hprev = H
    return C


# ---------------------------------------------------------------------------
# Back-coupling quantities of Sec. 2.2 (Eqs. eq-rho, eq-mu, eq-fst)
# ---------------------------------------------------------------------------

def chemical_potential(C, p: Params):
    """phi = psi'(C) - Cn^2 lap_h C, the bracket of Eq. (eq-ch)."""
    return psi_prime(C) - p.cn ** 2 * lap_h(C, p)


def grad_c(C, p: Params, d):
    """Central difference (C_{+d} - C_{-d}) / (2h) along d, with the ghost
    cells of lap_h (wrap, or the mirror about a wall face)."""
    Cp = pad(C, p.bc, 1)
    return (shifted(Cp, 1, d, 1, p.shape) - shifted(Cp, 1, d, -1, p.shape)) / (2.0 * p.h)


def surface_tension(C, p: Params):
    """F_st = 6 sqrt(2) phi grad C / Cn at the fine cell centres (Eq. eq-fst,
    with phi the chemical potential); returns the (x, y, z) components."""
    phi = chemical_potential(C, p)
    k = 6.0 * np.sqrt(2.0) / p.cn
    return tuple(k * phi * grad_c(C, p, d) for d in range(3))


def density(C, lam_rho):
    """rho = C + lambda_rho (1 - C), Eq. (eq-rho)."""
    return C + lam_rho * (1.0 - C)


def viscosity(C, lam_mu):
    """mu = C + lambda_mu (1 - C), Eq. (eq-mu)."""
    return C + lam_mu * (1.0 - C)


# ---------------------------------------------------------------------------
# Diagnostics: mass (Sec. 4.3, l_loss) and free energy (Sec. 1)
# ---------------------------------------------------------------------------

def mass(C, p: Params):
    """m = h^3 sum C, the drop mass whose relative change is l_loss (Sec. 4.3)."""
    return p.h ** 3 * float(np.sum(C))


def free_energy(C, p: Params):
    """F = h^3 sum [psi(C) + (Cn^2/2) sum_d ((C_{+e_d} - C)/h)^2].

    The paper names the free energy (Sec. 1) but does not write it out; this
    is the Ginzburg-Landau functional whose variation gives the chemical
    potential of Eq. (eq-ch), with forward differences; a wall face
    contributes zero gradient (mirror ghost).
    """
    Cp = pad(C, p.bc, 1)
    grad2 = np.zeros(p.shape)
    for d in range(3):
        grad2 += ((shifted(Cp, 1, d, 1, p.shape) - C) / p.h) ** 2
    return p.h ** 3 * float(np.sum(psi(C) + 0.5 * p.cn ** 2 * grad2))
