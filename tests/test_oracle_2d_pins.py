"""Pins of the 2D scheme (Sec. 3.1, Eq. eq-a2d): a box of one periodic z-plane
runs A_x + A_y only.  The split operator with w = 2 is the printed 2D row, and
one RK3/CN/AF step of a linearised 2D Fourier mode matches the closed form."""
import json
import os

import numpy as np
import pytest

from oracle import ch_oracle as co
from oracle.ch_oracle import Params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_stencils.json")


def test_a2d_row_is_the_printed_one():
    """A_x of Eq. (eq-a2d) is (0.75 L / h)^2 [2, -8, 12, -8, 2]; with Cn = 0.75 h
    (L = 1) that is w = 2 in (w Cn^2 / h^4)[1, -4, 6, -4, 1].  A_z vanishes on a
    single periodic plane."""
    row = json.load(open(GOLDEN))["a2d"]["row"]
    nx, ny, h = 11, 9, 0.1
    p = Params(nx, ny, 1, h, cn=0.75 * h, pe=10.0, dt=1e-3, w=2.0)
    d = np.zeros((1, ny, nx))
    d[0, 4, 5] = 1.0
    pref = (0.75 / h) ** 2
    ax = co.apply_A(d, p, 0)
    want = np.zeros_like(d)
    for off, v in zip(range(-2, 3), row):
        want[0, 4, 5 + off] = pref * v
    np.testing.assert_allclose(ax, want, rtol=0, atol=1e-9 * pref)
    ay = co.apply_A(d, p, 1)
    want = np.zeros_like(d)
    for off, v in zip(range(-2, 3), row):
        want[0, 4 + off, 5] = pref * v
    np.testing.assert_allclose(ay, want, rtol=0, atol=1e-9 * pref)
    assert np.abs(co.apply_A(d, p, 2)).max() == 0.0


@pytest.mark.parametrize("m", [(1, 0), (2, 3), (5, 4)])
def test_2d_linear_mode_matches_closed_form(m):
    """Closed form of one step with the z-symbol absent: lap_h -> -(s_x + s_y),
    A_d -> w Cn^2 s_d^2, and the factorised operator (1 + c A_x)(1 + c A_y)."""
    nx, ny, h = 16, 12, 1.0 / 16
    p = Params(nx, ny, 1, h, cn=0.75 * h, pe=50.0, dt=3e-3, w=2.0)
    psi2 = 0.5
    k = [2 * np.pi * md / (n * h) for md, n in zip(m, (nx, ny))]
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    mode = np.cos(k[1] * y[None, :, None] + k[0] * x[None, None, :])
    out = co.step(0.1 * mode, None, p, 3, psi_p=lambda c: psi2 * c)
    s = [4.0 * np.sin(kd * h / 2) ** 2 / h ** 2 for kd in k]
    lam = -p.mobility * psi2 * sum(s)
    a = [p.w * p.cn ** 2 * sd ** 2 for sd in s]
    q, hp = 1.0, 0.0
    for g, r in zip((8 / 15, 5 / 12, 3 / 4), (0.0, -17 / 60, -5 / 12)):
        al = g + r
        den = (1 + al * p.dt * p.mobility * a[0] / 2) * (1 + al * p.dt * p.mobility * a[1] / 2)
        dq = (p.dt * (g * lam * q + r * hp) - al * p.dt * p.mobility * (a[0] + a[1]) * q) / den
        hp = lam * q
        q = q + dq
    np.testing.assert_allclose(out, 0.1 * q ** 3 * mode, rtol=0, atol=1e-13)
