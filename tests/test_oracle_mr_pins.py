"""Pins of the multiple-resolution oracle (Sec. 3.4) against library routines,
polynomial exactness and the divergence identity."""
import numpy as np
import pytest
from scipy.interpolate import CubicHermiteSpline

from oracle import mr_oracle as mo
from oracle.mr_oracle import NOFLUX, PERIODIC
from paper_2105_01865_gb300 import inputs


def _stretched_nodes(n=12):
    return mo.centres(inputs.stretched_faces(n, 1.0, 2.0))


def test_hermite_basis_matches_scipy():
    """Interior segments equal scipy's cubic Hermite spline given the same
    node slopes (central differences over neighbouring nodes)."""
    nodes = _stretched_nodes()
    vals = np.sin(3 * nodes) + nodes ** 2
    slopes = np.empty_like(vals)
    slopes[1:-1] = (vals[2:] - vals[:-2]) / (nodes[2:] - nodes[:-2])
    slopes[0] = (vals[1] - vals[0]) / (nodes[1] - nodes[0])
    slopes[-1] = (vals[-1] - vals[-2]) / (nodes[-1] - nodes[-2])
    spl = CubicHermiteSpline(nodes, vals, slopes)
    xq = np.linspace(nodes[0], nodes[-1], 97)
    got = np.array([mo.interp_1d(vals, nodes, x, NOFLUX, 1.0) for x in xq])
    np.testing.assert_allclose(got, spl(xq), rtol=0, atol=1e-13)


def test_linear_exact_on_stretched_walled_grid_incl_ends():
    nodes = _stretched_nodes()
    vals = 2.5 * nodes - 0.7
    xq = np.linspace(0.0, 1.0, 53)                   # includes extrapolated end segments
    got = np.array([mo.interp_1d(vals, nodes, x, NOFLUX, 1.0) for x in xq])
    np.testing.assert_allclose(got, 2.5 * xq - 0.7, rtol=0, atol=1e-13)


def test_quadratic_exact_on_uniform_interior():
    nodes = (np.arange(10) + 0.5) / 10
    vals = 3 * nodes ** 2 - nodes + 0.2
    xq = np.linspace(nodes[1], nodes[-2], 31)
    got = np.array([mo.interp_1d(vals, nodes, x, NOFLUX, 1.0) for x in xq])
    np.testing.assert_allclose(got, 3 * xq ** 2 - xq + 0.2, rtol=0, atol=1e-13)


def test_periodic_wrap_and_order():
    errs = []
    for n in (16, 32):
        nodes = (np.arange(n) + 0.5) * (2.0 / n)
        f = lambda x: np.sin(np.pi * x + 0.3)
        xq = np.linspace(0, 2, 77, endpoint=False)
        got = np.array([mo.interp_1d(f(nodes), nodes, x, PERIODIC, 2.0) for x in xq])
        errs.append(np.abs(got - f(xq)).max())
    assert errs[0] < 1e-2 and errs[0] / errs[1] > 7        # third order (FD slopes)


@pytest.mark.parametrize("bc", [PERIODIC, NOFLUX])
def test_tables_identity_and_partition_of_unity(bc):
    n = 12
    faces = inputs.uniform_faces(n, 1.0)
    starts, w = mo.tables(faces, faces, faces, (n, n, n), 1.0 / n, (bc, bc, bc))[0]
    np.testing.assert_allclose(w.sum(1), 1.0, rtol=0, atol=1e-14)
    # fine centres coincide with coarse centres -> each weight row is a unit vector on the node itself
    for i in range(n):
        pos = [(starts[i] + m) % n for m in range(4)]
        assert abs(w[i, pos.index(i)] - 1.0) < 1e-14
        assert np.abs(np.delete(w[i], pos.index(i))).max() < 1e-14


def test_index_map_left_closed_base():
    nodes = np.array([0.1, 0.3, 0.35, 0.6, 0.9])
    starts, _ = mo.weight_table(nodes, np.array([0.0, 0.1, 0.2, 0.3, 0.34, 0.35, 0.5, 0.6, 0.95]), NOFLUX, 1.0)
    # base j = max{j: node_j <= x}; start = clamp(clamp(j, 0, n-2) - 1, 0, n-4)
    assert starts.tolist() == [0, 0, 0, 0, 0, 1, 1, 1, 1]


def _coarse_case(ncx, ncy, ncz, bc, seed):
    xf = inputs.uniform_faces(ncx, 2.0)
    yf = inputs.uniform_faces(ncy, 2.0)
    zf = inputs.stretched_faces(ncz, 1.0, 2.0) if bc[2] == NOFLUX else inputs.uniform_faces(ncz, 1.0)
    uc, vc, wc = inputs.curl_velocity(xf, yf, zf, bc, seed, kmax=3)
    return xf, yf, zf, uc, vc, wc


@pytest.mark.parametrize("bc", [(PERIODIC, PERIODIC, NOFLUX), (PERIODIC, PERIODIC, PERIODIC)])
def test_fine_field_solenoidal(bc):
    xf, yf, zf, uc, vc, wc = _coarse_case(8, 6, 6, bc, 7)
    gx, gy, gz = mo.coarse_gradients(uc, vc, wc, xf, yf, zf, bc)
    assert np.abs(gx + gy + gz).max() < 1e-11 * np.abs(gx).max()
    fine_n = (16, 16, 8)
    h = 1.0 / 8
    (u, v, w), tabs = mo.transfer(uc, vc, wc, xf, yf, zf, fine_n, h, bc)
    Gs = [mo.interp_3d(g, tabs) for g in (gx, gy, gz)]
    scale = np.abs(Gs[0]).max()
    assert np.abs(sum(Gs)).max() < 1e-11 * scale
    div = mo.fine_divergence(u, v, w, h, fine_n)
    # every cell but the last of each periodic line (where the wrap residual sits)
    inner = div[:, :-1, :-1] if bc[2] == NOFLUX else div[:-1, :-1, :-1]
    assert np.abs(inner).max() < 1e-11 * scale
    if bc[2] == NOFLUX:
        assert np.all(w[0] == 0.0)


def test_linear_shear_transfers_exactly():
    bc = (PERIODIC, PERIODIC, NOFLUX)
    xf = inputs.uniform_faces(4, 2.0)
    yf = inputs.uniform_faces(4, 2.0)
    zf = inputs.stretched_faces(8, 1.0, 2.0)
    zc = mo.centres(zf)
    uc = np.broadcast_to((zc - 0.5)[:, None, None], (8, 4, 4)).copy()
    vc = np.zeros((8, 4, 4))
    wc = np.zeros((9, 4, 4))
    fine_n = (16, 16, 8)
    h = 1.0 / 8
    (u, v, w), _ = mo.transfer(uc, vc, wc, xf, yf, zf, fine_n, h, bc)
    zfine = (np.arange(8) + 0.5) * h
    np.testing.assert_allclose(u, np.broadcast_to((zfine - 0.5)[:, None, None], u.shape), rtol=0, atol=1e-14)
    assert np.abs(v).max() < 1e-14 and np.abs(w).max() < 1e-14
