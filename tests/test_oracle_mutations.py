"""Planted mistakes in the oracle, each caught by a pin.

Every case below plants one plausible mistake in the CPU oracle (a wrong
sign, coefficient, index, boundary rule or a dropped term), by patching the
oracle module for the duration of the case only, then runs the pins named for
it and requires at least one of them to fail.  This is the evidence that the
pins of tests/test_oracle_*_pins.py fix the oracle, not merely agree with it.
Nothing here touches a GPU.
"""
import importlib.util
import os

import numpy as np
import pytest

from oracle import ch_adjoint as ca
from oracle import ch_oracle as co
from oracle import mr_oracle as mo
from oracle.ch_oracle import DIRICHLET, NOFLUX, PERIODIC

HERE = os.path.dirname(os.path.abspath(__file__))


def _load(name):
    spec = importlib.util.spec_from_file_location(f"pins_{name}", os.path.join(HERE, f"{name}.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PINS = _load("test_oracle_pins")
DIRI = _load("test_oracle_dirichlet_pins")
STD = _load("test_oracle_standard_pins")
MR = _load("test_oracle_mr_pins")
RS = _load("test_oracle_restrict_pins")
ADJ = _load("test_oracle_adjoint_pins")

# ---------------------------------------------------------------------------
# the mistakes (each patches the oracle through monkeypatch)
# ---------------------------------------------------------------------------

_orig = dict(apply_A=co.apply_A, line_solve=co.line_solve, lap_h=co.lap_h, face_fluxes=co.face_fluxes,
             pad=co.pad, hermite_segment=mo.hermite_segment, biharmonic_h=co.biharmonic_h,
             density=co.density, free_energy=co.free_energy, coarse_gradients=mo.coarse_gradients,
             interp_plane=mo.interp_plane, surface_tension=co.surface_tension,
             restriction_tables=mo.restriction_tables)


def rk3_rho_sign(mp):
    mp.setattr(co, "RK3_RHO", (0.0, 17.0 / 60.0, -5.0 / 12.0))
    mp.setattr(co, "RK3_ALPHA", (8.0 / 15.0, 5.0 / 12.0 + 17.0 / 60.0, 1.0 / 3.0))


def rk3_gamma_order(mp):
    mp.setattr(co, "RK3_GAMMA", (5.0 / 12.0, 8.0 / 15.0, 3.0 / 4.0))


def dropped_h_prev(mp):
    mp.setattr(co, "RK3_RHO", (0.0, 0.0, 0.0))


def cn_half_dropped(mp):
    mp.setattr(co, "line_solve", lambda rhs, p, d, c: _orig["line_solve"](rhs, p, d, 2.0 * c))


def solve_axis(mp):
    mp.setattr(co, "line_solve", lambda rhs, p, d, c: _orig["line_solve"](rhs, p, (d + 1) % 3, c))


def a_centre_coefficient(mp):
    mp.setattr(co, "apply_A", lambda C, p, d: _orig["apply_A"](C, p, d) + 0.5 * p.kappa * C)


def laplacian_centre_coefficient(mp):
    mp.setattr(co, "lap_h", lambda f, p: _orig["lap_h"](f, p) + 0.1 * f / p.h ** 2)


def psi_prime_sign(mp):
    mp.setattr(co, "psi_prime", lambda C: C ** 3 + 1.5 * C ** 2 + 0.5 * C)


def weno_downwind(mp):
    mp.setattr(co, "face_fluxes", lambda C, vel, p, d: -_orig["face_fluxes"](C, -vel, p, d))


def weno_linear_weight(mp):
    def weno(v1, v2, v3, v4, v5, eps):
        q0 = (2.0 * v1 - 7.0 * v2 + 11.0 * v3) / 6.0
        q1 = (-v2 + 5.0 * v3 + 2.0 * v4) / 6.0
        q2 = (2.0 * v3 + 5.0 * v4 - v5) / 6.0
        b0 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) ** 2 + 0.25 * (v1 - 4.0 * v2 + 3.0 * v3) ** 2
        b1 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
        b2 = 13.0 / 12.0 * (v3 - 2.0 * v4 + v5) ** 2 + 0.25 * (3.0 * v3 - 4.0 * v4 + v5) ** 2
        a = [w / (eps + b) ** 2 for w, b in zip((0.1, 0.5, 0.4), (b0, b1, b2))]   # 0.6, 0.3 -> 0.5, 0.4
        return (a[0] * q0 + a[1] * q1 + a[2] * q2) / (a[0] + a[1] + a[2])
    mp.setattr(co, "weno5_reconstruct", weno)


def weno_smoothness_coefficient(mp):
    def weno(v1, v2, v3, v4, v5, eps):
        q0 = (2.0 * v1 - 7.0 * v2 + 11.0 * v3) / 6.0
        q1 = (-v2 + 5.0 * v3 + 2.0 * v4) / 6.0
        q2 = (2.0 * v3 + 5.0 * v4 - v5) / 6.0
        b0 = (v1 - 2.0 * v2 + v3) ** 2 + 0.25 * (v1 - 4.0 * v2 + 3.0 * v3) ** 2          # 13/12 -> 1
        b1 = (v2 - 2.0 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
        b2 = (v3 - 2.0 * v4 + v5) ** 2 + 0.25 * (3.0 * v3 - 4.0 * v4 + v5) ** 2
        a = [w / (eps + b) ** 2 for w, b in zip((0.1, 0.6, 0.3), (b0, b1, b2))]
        return (a[0] * q0 + a[1] * q1 + a[2] * q2) / (a[0] + a[1] + a[2])
    mp.setattr(co, "weno5_reconstruct", weno)


def wall_mirror_rule(mp):
    def pad(f, bc, g):   # 'reflect' (ghost C_{-1-m} = C_{m+1}) instead of the mirror about the wall face
        for d in range(3):
            width = [(0, 0)] * 3
            width[2 - d] = (g, g)
            f = np.pad(f, width, mode="wrap" if bc[d] == PERIODIC else "reflect")
        return f
    mp.setattr(co, "pad", pad)


def line_operator_wall_rule(mp):
    def line_operator(n, bc, kappa):
        A = np.zeros((n, n))
        for i in range(n):
            for s, c in zip((-2, -1, 0, 1, 2), (1.0, -4.0, 6.0, -4.0, 1.0)):
                j = i + s
                if bc == PERIODIC:
                    j %= n
                elif j < 0:
                    j = -j                   # reflect instead of the mirror about the wall face
                elif j >= n:
                    j = 2 * n - 2 - j
                A[i, j] += kappa * c
        return A
    mp.setattr(co, "line_operator", line_operator)


def dirichlet_ghost_sign(mp):
    mp.setattr(co, "pad", lambda f, bc, g: _orig["pad"](f, tuple(NOFLUX if b == DIRICHLET else b for b in bc), g))


def standard_biharmonic_scale(mp):
    mp.setattr(co, "biharmonic_h", lambda C, p: 1.01 * _orig["biharmonic_h"](C, p))


def hermite_basis(mp):
    def seg(f0, f1, m0, m1, x0, x1, x):
        dx = x1 - x0
        t = (x - x0) / dx
        h00 = 2 * t ** 3 - 3 * t ** 2 + 1
        h10 = t ** 3 - 2 * t ** 2 + 1.1 * t                  # t -> 1.1 t
        h01 = -2 * t ** 3 + 3 * t ** 2
        h11 = t ** 3 - t ** 2
        return h00 * f0 + h10 * dx * m0 + h01 * f1 + h11 * dx * m1
    mp.setattr(mo, "hermite_segment", seg)


def density_phases_swapped(mp):
    mp.setattr(co, "density", lambda C, lam: _orig["density"](1.0 - C, lam))


def adjoint_psi_pp(mp):
    mp.setattr(ca, "psi_pp", lambda C: 3.0 * C ** 2 - 3.0 * C + 0.4)


def energy_gradient_weight(mp):
    mp.setattr(co, "free_energy", lambda C, p: _orig["free_energy"](C, p) + 0.5 * (
        _orig["free_energy"](C, p) - p.h ** 3 * float(np.sum(co.psi(C)))))


def transfer_gradient_scale(mp):
    def grads(*a):
        gx, gy, gz = _orig["coarse_gradients"](*a)
        return 1.01 * gx, gy, gz
    mp.setattr(mo, "coarse_gradients", grads)


def transfer_reference_plane(mp):
    mp.setattr(mo, "interp_plane", lambda P, r, c: 0.9 * _orig["interp_plane"](P, r, c))


def surface_tension_coefficient(mp):
    mp.setattr(co, "surface_tension", lambda C, p: tuple(1.05 * f for f in _orig["surface_tension"](C, p)))


def restriction_weights(mp):
    mp.setattr(mo, "restriction_tables",
               lambda *a: [(s, 1.01 * w) for s, w in _orig["restriction_tables"](*a)])


# mistake -> the pins that must catch it (at least one fails)
CASES = {
    "rk3_rho_sign": (rk3_rho_sign, [lambda: PINS.test_linear_mode_matches_closed_form(0.5, (1, 0, 0)),
                                    PINS.test_step_is_second_order_in_time]),
    "rk3_gamma_order": (rk3_gamma_order, [lambda: PINS.test_linear_mode_matches_closed_form(0.5, (1, 0, 0))]),
    "dropped_h_prev": (dropped_h_prev, [lambda: PINS.test_linear_mode_matches_closed_form(0.5, (1, 0, 0))]),
    "cn_half_dropped": (cn_half_dropped, [lambda: PINS.test_linear_mode_matches_closed_form(0.5, (1, 0, 0))]),
    "solve_axis": (solve_axis, [PINS.test_line_solves_match_dense_kronecker]),
    "a_centre_coefficient": (a_centre_coefficient, [lambda: PINS.test_A_matches_printed_eq_a3d(0)]),
    "laplacian_centre_coefficient": (laplacian_centre_coefficient,
                                     [lambda: PINS.test_linear_mode_matches_closed_form(0.5, (1, 0, 0))]),
    "psi_prime_sign": (psi_prime_sign, [PINS.test_psi_prime_is_derivative_of_psi]),
    "weno_downwind": (weno_downwind, [lambda: PINS.test_weno_advection_upwind_and_converges(1.0)]),
    "weno_linear_weight": (weno_linear_weight, [PINS.test_weno_linear_weights_exact_for_quartic]),
    "weno_smoothness_coefficient": (weno_smoothness_coefficient,
                                    [PINS.test_weno_matches_the_integral_definition_of_smoothness]),
    "wall_mirror_rule": (wall_mirror_rule, [lambda: PINS.test_mass_conserved_to_roundoff((PERIODIC, PERIODIC,
                                                                                          NOFLUX)),
                                            PINS.test_line_solves_match_dense_kronecker]),
    "line_operator_wall_rule": (line_operator_wall_rule, [PINS.test_line_solves_match_dense_kronecker]),
    "dirichlet_ghost_sign": (dirichlet_ghost_sign, [DIRI.test_ghosts_are_the_negated_mirror]),
    "standard_biharmonic_scale": (standard_biharmonic_scale, [STD.test_3d_biharmonic_is_the_25_point_stencil]),
    "hermite_basis": (hermite_basis, [MR.test_hermite_basis_matches_scipy,
                                      MR.test_linear_exact_on_stretched_walled_grid_incl_ends]),
    "density_phases_swapped": (density_phases_swapped, [RS.test_density_and_viscosity_definitions]),
    "adjoint_psi_pp": (adjoint_psi_pp, [lambda: ADJ.test_adjoint_transposes_complex_step_jvp((PERIODIC,) * 3)]),
    "energy_gradient_weight": (energy_gradient_weight, [PINS.test_free_energy_of_a_planar_interface]),
    "standard_rk3_rho_dropped": (dropped_h_prev, [lambda: STD.test_rk3_step_of_a_linear_mode_matches_closed_form(0.5)]),
    "transfer_gradient_scale": (transfer_gradient_scale,
                                [lambda: MR.test_fine_field_solenoidal((PERIODIC, PERIODIC, NOFLUX))]),
    "transfer_reference_plane": (transfer_reference_plane, [MR.test_linear_shear_transfers_exactly]),
    "surface_tension_coefficient": (surface_tension_coefficient,
                                    [RS.test_surface_tension_converges_to_the_continuum_force]),
    "restriction_weights": (restriction_weights,
                            [lambda: RS.test_coincident_meshes_give_the_identity((PERIODIC, PERIODIC, NOFLUX))]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_planted_mistake_is_caught(name, monkeypatch):
    plant, pins = CASES[name]
    for pin in pins:                      # the pins pass on the oracle as it stands
        pin()
    plant(monkeypatch)
    caught = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError):
            caught.append(pin)
    assert caught, f"no pin caught the planted mistake {name}"
