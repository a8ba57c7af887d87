"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: the coefficients the
paper prints (tests/golden/paper_stencils.json), closed-form Fourier
amplification factors, dense Kronecker-product solves, conservation
invariants, polynomial exactness and convergence order.
"""
import json
import os

import numpy as np
import pytest

from oracle import ch_oracle as co
from oracle.ch_oracle import NOFLUX, PERIODIC, Params

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_stencils.json")))


# ---------------------------------------------------------------------------
# Printed stencils (Sec. 3.1)
# ---------------------------------------------------------------------------

def _delta_response(p, d):
    C = np.zeros(p.shape)
    c = tuple(n // 2 for n in p.shape)
    C[c] = 1.0
    out = co.apply_A(C, p, d)
    a = 2 - d
    line = [slice(c[0], c[0] + 1), slice(c[1], c[1] + 1), slice(c[2], c[2] + 1)]
    line[a] = slice(c[a] - 2, c[a] + 3)
    return out[tuple(line)].ravel(), out


@pytest.mark.parametrize("d", [0, 1, 2])
def test_A_matches_printed_eq_a3d(d):
    """A_d with w = 4 and Cn = 0.75h equals (0.75/h)^2 [4,-16,24,-16,4] (Eq. eq-a3d)."""
    h = 1.0 / 16
    p = Params(12, 11, 10, h, cn=0.75 * h, pe=1.0, dt=1.0, w=4.0)
    row, full = _delta_response(p, d)
    printed = np.array(GOLD["a3d"]["row"], float) * (0.75 / h) ** 2
    np.testing.assert_allclose(row, printed, rtol=1e-14)
    assert np.count_nonzero(full) == 5          # only on the axis of d


def _replace_diagonals(st, ndim):
    """Apply Eq. (eq-trans1) in every coordinate plane (d, e): the four
    diagonal points of equal coefficient c are replaced by
    c [0.5 (2C + C_{+2d} + C_{-2d}) + 0.5 (2C + C_{+2e} + C_{-2e})]."""
    zero = (0,) * ndim
    new = {k: v for k, v in st.items() if sum(1 for x in k if x) <= 1}
    for d in range(ndim):
        for e in range(d + 1, ndim):
            diag = [k for k in st if k[d] and k[e] and sum(1 for x in k if x) == 2]
            coefs = {st[k] for k in diag}
            assert len(diag) == 4 and len(coefs) == 1
            c = coefs.pop()
            new[zero] += 2.0 * c
            for ax in (d, e):
                for s in (-2, 2):
                    kk = [0] * ndim
                    kk[ax] = s
                    new[tuple(kk)] += 0.5 * c
    return new


def _lap_squared(ndim):
    lap = {(0,) * ndim: -2 * ndim}
    for d in range(ndim):
        for s in (-1, 1):
            e = [0] * ndim
            e[d] = s
            lap[tuple(e)] = 1
    sq = {}
    for a, u in lap.items():
        for b, v in lap.items():
            k = tuple(x + y for x, y in zip(a, b))
            sq[k] = sq.get(k, 0) + u * v
    return {k: v for k, v in sq.items() if v}


def test_2d_replacement_gives_printed_eq_a2d():
    """Eq. (eq-trans1) applied to the printed Eq. (eq-disbi) stencil gives the
    printed Eq. (eq-a2d) rows; the printed centre 10 of Eq. (eq-new) does not
    have a zero row sum (typo), 12 does."""
    pts = {(a, b): c for a, b, c in GOLD["disbi_2d"]["points"]}
    assert _lap_squared(2) == pts          # (eq-disbi) is the squared 5-point Laplacian
    new = _replace_diagonals(pts, 2)
    row_x = [new[(-2, 0)], new[(-1, 0)], new[(0, 0)] / 2, new[(1, 0)], new[(2, 0)]]
    assert row_x == GOLD["a2d"]["row"]
    assert sum(GOLD["a2d"]["row"]) == 0
    assert sum(GOLD["new_2d_printed"]["row"]) != 0


def test_eq_trans1_is_fourth_order():
    """The diagonal-sum identity of Eq. (eq-trans1) has an O(h^4) residual."""
    f = lambda x, y: np.sin(1.3 * x + 0.4) * np.cos(0.7 * y - 0.2) + x ** 2 * y
    x0, y0 = 0.31, -0.12
    res = []
    for hh in (0.02, 0.01):
        diag = sum(f(x0 + a * hh, y0 + b * hh) for a in (-1, 1) for b in (-1, 1))
        rhs = 0.5 * (2 * f(x0, y0) + f(x0 + 2 * hh, y0) + f(x0 - 2 * hh, y0)) \
            + 0.5 * (2 * f(x0, y0) + f(x0, y0 + 2 * hh) + f(x0, y0 - 2 * hh))
        res.append(abs(diag - rhs))
    assert 12 < res[0] / res[1] < 20


def test_3d_replacement_gives_w3():
    """The same replacement applied to the 3D 25-point stencil (square of the
    7-point Laplacian) yields w = 3, i.e. [3,-12,18,-12,3] per direction, not
    the printed w = 4 of Eq. (eq-a3d) (reading R1: w is a parameter)."""
    sq = _lap_squared(3)
    assert len(sq) == 25 and sq[(0, 0, 0)] == 42
    new = _replace_diagonals(sq, 3)
    row = [new[(-2, 0, 0)], new[(-1, 0, 0)], new[(0, 0, 0)] / 3, new[(1, 0, 0)], new[(2, 0, 0)]]
    assert row == [3, -12, 18, -12, 3]
    assert [4 * r for r in (1, -4, 6, -4, 1)] == GOLD["a3d"]["row"]


def test_psi_prime_is_derivative_of_psi():
    """psi' of Eq. (eq-ch) is d/dC of psi = C^2 (C-1)^2 / 4 (complex-step derivative)."""
    C = np.linspace(-0.5, 1.5, 41)
    hstep = 1e-30
    dpsi = np.imag(co.psi(C + 1j * hstep)) / hstep
    np.testing.assert_allclose(co.psi_prime(C), dpsi, rtol=1e-14, atol=1e-15)
    for m in GOLD["psi"]["minima"]:
        assert co.psi(np.float64(m)) == 0.0 and co.psi_prime(np.float64(m)) == 0.0


# ---------------------------------------------------------------------------
# Linear step against the closed-form Fourier amplification factor
# ---------------------------------------------------------------------------

def closed_form_gain(k, p, psi2):
    """Amplification of one RK3 step for the Fourier mode k (periodic box),
    psi' linearised about C0 with slope psi2.  Symbols: lap_h -> -sum s_d,
    A_d -> w Cn^2 s_d^2 with s_d = 4 sin^2(k_d h / 2) / h^2."""
    s = [4.0 * np.sin(kd * p.h / 2) ** 2 / p.h ** 2 for kd in k]
    lam = -p.mobility * psi2 * sum(s)
    a = [p.w * p.cn ** 2 * sd ** 2 for sd in s]
    q, hp = 1.0, 0.0
    for g, r in zip((8 / 15, 5 / 12, 3 / 4), (0.0, -17 / 60, -5 / 12)):
        al = g + r
        denom = np.prod([1.0 + al * p.dt * p.mobility * ad / 2 for ad in a])
        dq = (p.dt * (g * lam * q + r * hp) - al * p.dt * p.mobility * sum(a) * q) / denom
        hp = lam * q
        q = q + dq
    return q


@pytest.mark.parametrize("C0", [0.5, 0.1, 0.0])
@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 1), (3, 2, 4), (8, 6, 5)])
def test_linear_mode_matches_closed_form(C0, m):
    nx, ny, nz = 16, 12, 10
    h = 1.0 / 16
    p = Params(nx, ny, nz, h, cn=0.75 * h, pe=50.0, dt=3e-3, w=4.0)
    psi2 = 3 * C0 ** 2 - 3 * C0 + 0.5
    k = [2 * np.pi * md / (n * h) for md, n in zip(m, (nx, ny, nz))]
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    z = (np.arange(nz) + 0.5) * h
    mode = np.cos(k[2] * z[:, None, None] + k[1] * y[None, :, None] + k[0] * x[None, None, :])
    eps = 0.1                     # the linearised step is linear: amplitude is arbitrary
    C = C0 + eps * mode
    nsteps = 5
    out = co.step(C, None, p, nsteps, psi_p=lambda c: psi2 * (c - C0))
    g = closed_form_gain(k, p, psi2)
    np.testing.assert_allclose(out - C0, eps * g ** nsteps * mode, rtol=0, atol=1e-13 * eps * max(1, abs(g) ** nsteps))


# ---------------------------------------------------------------------------
# Line solves against dense Kronecker-product systems
# ---------------------------------------------------------------------------

def test_line_solves_match_dense_kronecker():
    nx, ny, nz = 7, 6, 5
    h = 0.1
    p = Params(nx, ny, nz, h, cn=0.09, pe=1.0, dt=1.0, bc=(PERIODIC, NOFLUX, NOFLUX))
    N = nx * ny * nz
    # dense 3D operator of each A_d, column by column through the stencil path
    dense = []
    for d in range(3):
        A = np.zeros((N, N))
        for col in range(N):
            e = np.zeros(N)
            e[col] = 1.0
            A[:, col] = co.apply_A(e.reshape(p.shape), p, d).ravel()
        dense.append(A)
        assert np.allclose(A, A.T)                       # symmetric boundary rows
        np.testing.assert_allclose(A.sum(axis=0), 0, atol=1e-9 * p.kappa)   # conservative
    rng = np.random.default_rng(0)
    r = rng.standard_normal(p.shape)
    c = 0.37
    for d in range(3):
        x = co.line_solve(r, p, d, c)
        ref = np.linalg.solve(np.eye(N) + c * dense[d], r.ravel()).reshape(p.shape)
        np.testing.assert_allclose(x, ref, rtol=1e-12, atol=1e-12)
    # the factorised product differs from the unfactorised operator by the cross terms only (Eq. eq-fac)
    I = np.eye(N)
    prod = (I + c * dense[0]) @ (I + c * dense[1]) @ (I + c * dense[2])
    cross = c ** 2 * (dense[0] @ dense[1] + dense[0] @ dense[2] + dense[1] @ dense[2]) + c ** 3 * dense[0] @ dense[1] @ dense[2]
    np.testing.assert_allclose(prod, I + c * sum(dense) + cross, rtol=0, atol=1e-9 * np.abs(prod).max())


# ---------------------------------------------------------------------------
# Conservation and invariants
# ---------------------------------------------------------------------------

def _curl_vel(shape, h, bc, seed):
    from paper_2105_01865_gb300 import inputs
    nz, ny, nx = shape
    return inputs.curl_velocity(inputs.uniform_faces(nx, nx * h), inputs.uniform_faces(ny, ny * h),
                                inputs.uniform_faces(nz, nz * h), bc, seed, kmax=3)


@pytest.mark.parametrize("bc", [(PERIODIC, PERIODIC, PERIODIC), (PERIODIC, PERIODIC, NOFLUX), (NOFLUX, NOFLUX, NOFLUX)])
def test_mass_conserved_to_roundoff(bc):
    from paper_2105_01865_gb300 import inputs
    shape = (10, 12, 14)
    h = 1.0 / 12
    cn = 0.75 * h
    C = inputs.drops_field(shape, h, bc, [(0.6, 0.5, 0.4)], [0.25], cn)
    vel = _curl_vel(shape, h, bc, 1)
    p = Params(14, 12, 10, h, cn=cn, pe=0.9 / cn, dt=0.2 * h, bc=bc)
    m0 = co.mass(C, p)
    C1 = co.step(C, vel, p, 20)
    assert abs(co.mass(C1, p) - m0) / m0 < 1e-13
    assert np.abs(C1 - C).max() > 1e-3          # it did move


def test_free_stream_preserved():
    shape = (8, 9, 10)
    h = 0.1
    bc = (PERIODIC, PERIODIC, NOFLUX)
    vel = _curl_vel(shape, h, bc, 2)
    p = Params(10, 9, 8, h, cn=0.07, pe=10.0, dt=0.02, bc=bc)
    C = np.full(shape, 0.3)
    C1 = co.step(C, vel, p, 5)
    np.testing.assert_allclose(C1, 0.3, rtol=0, atol=1e-13)


def test_free_energy_decays_without_flow():
    from paper_2105_01865_gb300 import inputs
    n = 24
    f = inputs.single_drop_box(n)
    h = f["h"]
    cn = 0.75 * h
    p = Params(n, n, n, h, cn=cn, pe=1e2, dt=2e-3)
    C = inputs.drops_field(f["shape"], h, f["bc"], [(0.5, 0.45, 0.55)], [0.3], cn)
    C = C + 0.02 * np.random.default_rng(3).standard_normal(C.shape)
    E = [co.free_energy(C, p)]
    for _ in range(15):
        C = co.step(C, None, p, 1)
        E.append(co.free_energy(C, p))
    assert np.all(np.diff(E) <= 1e-12 * abs(E[0]))


# ---------------------------------------------------------------------------
# WENO5
# ---------------------------------------------------------------------------

def test_weno_candidates_exact_for_quadratic_cell_averages():
    """Every candidate, hence any convex weighting, reproduces a quadratic
    from its cell averages at the face (fifth-order WENO construction)."""
    a, b, c = 0.3, -1.7, 2.9
    P = lambda x: a * x + b * x ** 2 / 2 + c * x ** 3 / 3      # antiderivative of a + b x + c x^2
    hh = 0.13
    xf = np.arange(-3, 3) * hh                                  # faces -3h .. 2h ; target face at 0
    avg = (P(xf[1:]) - P(xf[:-1])) / hh                         # cells -3..1 (5 cells)
    for eps in (1e-6, 1e3):
        v = co.weno5_reconstruct(*[np.float64(t) for t in avg], eps)
        assert abs(v - a) < 1e-12


def _advect_1d_error(n, sign):
    h = 1.0 / n
    p = Params(n, 5, 5, h, cn=1e-3, pe=1e30, dt=0.25 * h)
    x = (np.arange(n) + 0.5) * h
    f = lambda xx: 0.5 + 0.25 * np.sin(2 * np.pi * xx)
    C = np.broadcast_to(f(x)[None, None, :], p.shape).copy()
    u = np.full((5, 5, n), sign * 1.0)
    vel = (u, np.zeros((5, 5, n)), np.zeros((5, 5, n)))
    T = 0.25
    steps = int(round(T / p.dt))
    C1 = co.step(C, vel, p, steps)
    # finite-difference WENO advects point values: exact = translate of f
    exact = f(x - sign * T)
    return np.abs(C1[0, 0] - exact).max()


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_weno_advection_upwind_and_converges(sign):
    e1 = _advect_1d_error(32, sign)
    e2 = _advect_1d_error(64, sign)
    assert e1 < 2e-4
    assert e2 < e1 / 7.0        # at least third order (RK3 time error included)


def test_weno_step_no_new_extrema():
    n = 40
    h = 1.0 / n
    p = Params(n, 5, 5, h, cn=1e-3, pe=1e30, dt=0.4 * h)
    C = np.zeros(p.shape)
    C[:, :, 10:20] = 1.0
    u = np.full((5, 5, n), 1.0)
    vel = (u, np.zeros((5, 5, n)), np.zeros((5, 5, n)))
    C1 = co.step(C, vel, p, 10)
    assert C1.min() > -0.05 and C1.max() < 1.05


def test_weno_linear_weights_exact_for_quartic():
    """With smoothness indicators negligible against eps, the weights reduce to
    the linear weights (1/10, 6/10, 3/10), the unique combination of the three
    candidates that reproduces a quartic from its five cell averages."""
    cf = [0.3, -1.7, 2.9, 0.8, -1.1]                            # p(x) = sum cf[m] x^m
    P = lambda x: sum(c * x ** (m + 1) / (m + 1) for m, c in enumerate(cf))
    hh = 0.05
    xf = np.arange(-3, 3) * hh
    avg = (P(xf[1:]) - P(xf[:-1])) / hh
    v = co.weno5_reconstruct(*[np.float64(t) for t in avg], 1e6)
    assert abs(v - cf[0]) < 1e-12
    # and the reconstruction is fifth order at the default eps on smooth data
    errs = []
    for hh in (0.02, 0.01):
        xf = 0.3 + np.arange(-3, 3) * hh
        f = lambda x: -np.cos(3 * x) / 3                         # antiderivative of sin(3x)
        avg = (f(xf[1:]) - f(xf[:-1])) / hh
        errs.append(abs(co.weno5_reconstruct(*avg, 1e-6) - np.sin(3 * 0.3)))
    assert errs[0] / errs[1] > 24


# ---------------------------------------------------------------------------
# Temporal order of the whole step (RK3 with Crank-Nicolson and approximate
# factorisation, Sec. 3 and Eqs. eq-fac-1..3): second order in dt
# ---------------------------------------------------------------------------

def _time_self_convergence(ns, T=0.5):
    """Differences between solutions at time T with dt = T/n for successive
    n, and the observed orders log2(e_i / e_{i+1}), on a smooth nonlinear
    field of an 8^3 periodic box (psi'' > 0 everywhere, so the explicit term
    is stable at every dt used)."""
    n = 8
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    C0 = 0.2 + 0.1 * np.cos(2 * np.pi * X) + 0.05 * np.sin(2 * np.pi * Y) * np.cos(2 * np.pi * Z)
    sols = [co.step(C0, None, Params(n, n, n, h, cn=0.75 * h, pe=50.0, dt=T / m), m) for m in ns]
    e = [np.linalg.norm(sols[i] - sols[i + 1]) for i in range(len(ns) - 1)]
    return [np.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]


def test_step_is_second_order_in_time():
    orders = _time_self_convergence([4, 8, 16, 32, 64])
    assert all(1.9 <= q <= 2.1 for q in orders[-2:]), orders


def test_time_order_pin_detects_wrong_rk_coefficients(monkeypatch):
    """Planted mistakes in the oracle's RK3 coefficient set fail the pin above:
    a first-order set with the same sums, and an implicit weight alpha_3 off
    by 2 % (the CN part then no longer sums to dt)."""
    monkeypatch.setattr(co, "RK3_GAMMA", (1 / 3, 1 / 3, 1 / 3))
    monkeypatch.setattr(co, "RK3_RHO", (0.0, 0.0, 0.0))
    monkeypatch.setattr(co, "RK3_ALPHA", (1 / 3, 1 / 3, 1 / 3))
    assert max(_time_self_convergence([4, 8, 16, 32, 64])[-2:]) < 1.2
    monkeypatch.setattr(co, "RK3_GAMMA", (8 / 15, 5 / 12, 3 / 4))
    monkeypatch.setattr(co, "RK3_RHO", (0.0, -17 / 60, -5 / 12))
    monkeypatch.setattr(co, "RK3_ALPHA", (8 / 15, 2 / 15, 0.34))
    assert _time_self_convergence([4, 8, 16, 32, 64])[-1] < 1.85


# ---------------------------------------------------------------------------
# Spatial order of the whole step (Sec. 3: second-order central differences,
# the pentadiagonal A_d, WENO5 advection): second order in h at fixed Cn
# ---------------------------------------------------------------------------

def test_step_is_second_order_in_space():
    """Self-convergence of a smooth x-dependent field advected at u = 0.5 to
    T = 0.02 on 32, 64 and 128 cells (Cn = 0.05 fixed, dt = 1e-4 so the time
    error is negligible): the coarse solution against the mean of the two fine
    cells that share its centre."""
    def solve(n, T=0.02, dt=1e-4):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        prof = 0.3 + 0.2 * np.sin(2 * np.pi * x) + 0.1 * np.cos(4 * np.pi * x)
        C0 = np.broadcast_to(prof[None, None, :], (4, 4, n)).copy()
        vel = (np.full((4, 4, n), 0.5), np.zeros((4, 4, n)), np.zeros((4, 4, n)))
        return co.step(C0, vel, Params(n, 4, 4, h, cn=0.05, pe=10.0, dt=dt), int(round(T / dt)))[0, 0]
    s = [solve(n) for n in (32, 64, 128)]
    e = [np.abs(s[i] - 0.5 * (s[i + 1][0::2] + s[i + 1][1::2])).max() for i in range(2)]
    order = np.log2(e[0] / e[1])
    assert 1.9 <= order <= 2.1, (e, order)


def test_weno_matches_the_integral_definition_of_smoothness():
    """WENO5-JS from its definition (Jiang and Shu 1996): the three quadratics
    with the stencils' cell averages, evaluated at the face; smoothness
    indicators beta_k = sum_{l=1,2} h^{2l-1} int_cell (d^l p_k/dx^l)^2 over the
    upwind cell; weights d_k / (eps + beta_k)^2 with d = (1/10, 6/10, 3/10).
    Random (non-smooth) data, so the nonlinear weights matter."""
    def from_definition(v, eps):
        vals, betas = [], []
        for cells in ([-2, -1, 0], [-1, 0, 1], [0, 1, 2]):      # cell 0 holds v3; the face is at x = 1/2 (h = 1)
            A = np.array([[1.0, j, j * j + 1.0 / 12.0] for j in cells])   # averages of 1, x, x^2 over cell j
            c0, c1, c2 = np.linalg.solve(A, np.array([v[j + 2] for j in cells]))
            vals.append(c0 + c1 / 2 + c2 / 4)
            betas.append(c1 ** 2 + c2 ** 2 / 3 + 4 * c2 ** 2)   # int_{-1/2}^{1/2} p'^2 + p''^2
        a = [dk / (eps + b) ** 2 for dk, b in zip((0.1, 0.6, 0.3), betas)]
        return sum(ai * q for ai, q in zip(a, vals)) / sum(a)
    rng = np.random.default_rng(5)
    for _ in range(200):
        v = rng.standard_normal(5)
        got = co.weno5_reconstruct(*[np.float64(t) for t in v], 1e-6)
        assert abs(got - from_definition(v, 1e-6)) <= 1e-13 * max(1.0, abs(got))


# ---------------------------------------------------------------------------
# Free energy of a planar interface: 2 sigma A with sigma = sqrt(2) Cn / 12,
# the surface energy of the equilibrium profile C = (1 + tanh(x / (2 sqrt(2) Cn))) / 2
# of psi = C^2 (C - 1)^2 / 4 with gradient coefficient Cn^2
# ---------------------------------------------------------------------------

def test_free_energy_of_a_planar_interface():
    cn = 0.02
    sigma = np.sqrt(2.0) * cn / 12.0
    errs = []
    for n in (64, 128):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        w = 2.0 * np.sqrt(2.0) * cn
        prof = 0.5 * (np.tanh((x - 0.25) / w) - np.tanh((x - 0.75) / w))   # two interfaces, periodic
        C = np.broadcast_to(prof[None, None, :], (4, 4, n)).copy()
        F = co.free_energy(C, Params(n, 4, 4, h, cn=cn, pe=1.0, dt=1.0))
        errs.append(F / (2.0 * sigma * (4 * h) ** 2) - 1.0)
    assert abs(errs[1]) < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5        # second order in h
