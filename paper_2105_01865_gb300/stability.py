"""Linear stability bound of the time step (host-side helper for choosing dt).

The paper runs its new scheme at a time step far above the explicit limit
(Sec. 4.1: 2e-3 against 5e-5) but gives no formula for the bound.  This helper
takes the largest dt for which one RK3 step of the linearised scheme does not
amplify any grid mode.  With psi' linearised about a state of slope psi'' the
discrete operators are diagonal in the grid's Fourier (periodic) or cosine
(mirror-wall) modes: lap_h -> -sum_d s_d, A_d -> w Cn^2 s_d^2 with
s_d = 4 sin^2(theta_d / 2) / h^2, theta_d = 2 pi m / n (periodic) or
pi m / n (walls; m = 1 .. n for Dirichlet walls, whose modes are sines).  Each substep l then maps (q, H^{l-1}) linearly, and the
step's amplification is the product of the three substep maps.

stable_dt_standard does the same for the explicit comparison scheme of
Sec. 3.1, Eq. (eq-disbi), whose biharmonic lap_h^2 has the symbol
(sum_d s_d)^2 and is advanced explicitly by the same RK3.
"""
from __future__ import annotations

import numpy as np

GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RHO = (0.0, -17.0 / 60.0, -5.0 / 12.0)


def _thetas(n, bc, max_modes):
    # periodic: Fourier modes 2 pi m / n; no-flux walls: cosine modes pi m / n,
    # m = 0 .. n-1; Dirichlet walls: sine modes pi m / n, m = 1 .. n
    m = np.arange(1, n + 1, dtype=np.float64) if bc == 2 else np.arange(n, dtype=np.float64)
    th = (2.0 if bc == 0 else 1.0) * np.pi * m / n
    if n > max_modes:
        th = np.unique(np.concatenate([th[:: max(1, n // max_modes)], th[-1:]]))
    return th


def gain(dt, s, mobility, psi2, wcn2):
    """Amplification of one RK3 step for modes with symbols s = (s_x, s_y, s_z)
    (arrays broadcasting together)."""
    lam = -mobility * psi2 * (s[0] + s[1] + s[2])
    a = [wcn2 * sd * sd for sd in s]
    asum = a[0] + a[1] + a[2]
    q = np.ones(np.broadcast(*s).shape)
    hp = np.zeros_like(q)
    for g, r in zip(GAMMA, RHO):
        al = g + r
        den = (1 + al * dt * mobility * a[0] / 2) * (1 + al * dt * mobility * a[1] / 2) * (1 + al * dt * mobility * a[2] / 2)
        dq = (dt * (g * lam * q + r * hp) - al * dt * mobility * asum * q) / den
        hp = lam * q
        q = q + dq
    return q


def stable_dt(shape, h, bc, cn, pe, w=4.0, psi2=0.5, dt_max=1.0, max_modes=64):
    """Largest dt (bisection, relative tolerance 1e-6) with |gain| <= 1 for all
    sampled grid modes.  shape = (nz, ny, nx); bc = (bc_x, bc_y, bc_z)."""
    nz, ny, nx = shape
    th = [_thetas(n, b, max_modes) for n, b in zip((nx, ny, nz), bc)]
    s = [4.0 * np.sin(t / 2.0) ** 2 / h ** 2 for t in th]
    S = np.meshgrid(*s, indexing="ij")
    mob = 1.0 / pe
    wcn2 = w * cn * cn

    def ok(dt):
        return np.abs(gain(dt, S, mob, psi2, wcn2)).max() <= 1.0 + 1e-12

    if ok(dt_max):
        return dt_max
    lo, hi = 0.0, dt_max
    while hi - lo > 1e-6 * hi:
        mid = 0.5 * (lo + hi)
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo


def gain_standard(dt, s, mobility, psi2, cn2):
    """Amplification of one all-explicit RK3 step of dq/dt = lam q with
    lam = -M (psi'' S + Cn^2 S^2), S = s_x + s_y + s_z."""
    S = s[0] + s[1] + s[2]
    lam = -mobility * (psi2 * S + cn2 * S * S)
    q = np.ones(np.broadcast(*s).shape)
    hp = np.zeros_like(q)
    for g, r in zip(GAMMA, RHO):
        hl = lam * q
        q = q + dt * (g * hl + r * hp)
        hp = hl
    return q


def stable_dt_standard(shape, h, bc, cn, pe, psi2=0.5, dt_max=1.0, max_modes=64):
    """Largest dt (bisection, relative tolerance 1e-6) for which the explicit
    comparison scheme amplifies no sampled grid mode."""
    nz, ny, nx = shape
    th = [_thetas(n, b, max_modes) for n, b in zip((nx, ny, nz), bc)]
    s = [4.0 * np.sin(t / 2.0) ** 2 / h ** 2 for t in th]
    S = np.meshgrid(*s, indexing="ij")
    mob = 1.0 / pe

    def ok(dt):
        return np.abs(gain_standard(dt, S, mob, psi2, cn * cn)).max() <= 1.0 + 1e-12

    if ok(dt_max):
        return dt_max
    lo, hi = 0.0, dt_max
    while hi - lo > 1e-6 * hi:
        mid = 0.5 * (lo + hi)
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo
