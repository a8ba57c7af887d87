"""Plain FP64 CPU oracle of the multiple-resolution velocity transfer.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this module.

Sec. 3.4 of arXiv 2105.01865: the face velocity of a stretched coarse mesh is
transferred to the uniform fine mesh of C by
  (1) computing the face-normal velocity gradients du/dx, dv/dy, dw/dz on the
      coarse mesh (at coarse cell centres, one per cell);
  (2) interpolating them to the fine cell centres with a tri-cubic Hermite
      spline of four points per direction (a 64-point stencil), whose indices
      and weights are built once and reused;
  (3) interpolating a 2D velocity plane at a reference location in each
      direction, and integrating the interpolated gradients from it along
      every fine line.
Because the three gradients share the same tensor-product weights, the fine
discrete divergence equals the interpolated coarse divergence.

The back-coupling of C (Sec. 3.4, last step) projects the fine field directly
to the stretched mesh; ``restrict_to_coarse`` takes that projection to be the
same 4-point-per-direction Hermite stencil with the roles swapped (nodes at
the fine cell centres, queries at the coarse cell centres), applied to C and
to the fine surface-tension force, from which the coarse density and
viscosity follow (Eqs. eq-rho, eq-mu, eq-fst).

Readings where the paper is silent: the cubic Hermite segment on [x_j, x_{j+1}]
takes node slopes from central differences over the neighbouring nodes
(non-uniform Catmull-Rom); the base node is the last node at or left of the
query point; walled directions clamp the stencil into the node range and use
a one-sided slope at the two end nodes; periodic directions wrap.  Reference
planes are the lower face plane of each direction (x = 0 for u, y = 0 for v,
z = 0 for w, where w = 0 at a wall).
"""
from __future__ import annotations

import numpy as np

PERIODIC = 0
NOFLUX = 1


def centres(faces):
    """Cell-centre coordinates from face coordinates."""
    faces = np.asarray(faces, dtype=np.float64)
    return 0.5 * (faces[:-1] + faces[1:])


def hermite_segment(f0, f1, m0, m1, x0, x1, x):
    """Cubic Hermite interpolant on [x0, x1] with end values f and slopes m."""
    dx = x1 - x0
    t = (x - x0) / dx
    h00 = 2 * t ** 3 - 3 * t ** 2 + 1
    h10 = t ** 3 - 2 * t ** 2 + t
    h01 = -2 * t ** 3 + 3 * t ** 2
    h11 = t ** 3 - t ** 2
    return h00 * f0 + h10 * dx * m0 + h01 * f1 + h11 * dx * m1


def stencil(nodes, x, bc, period):
    """Return (start, xs) for one query point: the first of the four stencil
    nodes (wrapped index for periodic) and the four node coordinates (unwrapped)
    plus the segment index within the four (1 for interior use).

    Base node j = max{j : nodes[j] <= x} (-1 if none).
    """
    n = len(nodes)
    j = int(np.searchsorted(nodes, x, side="right")) - 1
    if bc == PERIODIC:
        start = (j - 1) % n
        xs = []
        for m in range(4):
            k = j - 1 + m
            xs.append(nodes[k % n] + period * (k // n))
        return start, np.array(xs), 1
    seg = min(max(j, 0), n - 2)             # segment [x_seg, x_seg+1]
    start = min(max(seg - 1, 0), n - 4)
    return start, np.asarray(nodes[start:start + 4], dtype=np.float64), seg - start


def interp_1d(values, nodes, x, bc, period):
    """Evaluate the 1D Hermite interpolant of node values at x (Sec. 3.4).

    Interior slopes are (f_{k+1} - f_{k-1}) / (x_{k+1} - x_{k-1}); at the end
    nodes of a walled direction the slope is the one-sided difference.
    """
    n = len(nodes)
    start, xs, seg = stencil(nodes, x, bc, period)
    if bc == PERIODIC:
        f = np.array([values[(start + m) % n] for m in range(4)])
        m0 = (f[2] - f[0]) / (xs[2] - xs[0])
        m1 = (f[3] - f[1]) / (xs[3] - xs[1])
        return hermite_segment(f[1], f[2], m0, m1, xs[1], xs[2], x)
    f = np.asarray(values[start:start + 4], dtype=np.float64)
    gk = start + seg                          # global index of the segment's left node

    def slope(k):                              # k global node index
        lo, hi = max(k - 1, 0), min(k + 1, n - 1)
        return (values[hi] - values[lo]) / (nodes[hi] - nodes[lo])

    return hermite_segment(f[seg], f[seg + 1], slope(gk), slope(gk + 1), xs[seg], xs[seg + 1], x)


def weight_table(nodes, xq, bc, period):
    """Index map and weights of the 1D interpolant: for every query point,
    the stencil start (int) and the 4 weights, obtained by interpolating the
    four unit vectors (so the table is exactly the interpolant above)."""
    n = len(nodes)
    starts = np.zeros(len(xq), dtype=np.int32)
    wts = np.zeros((len(xq), 4))
    for q, x in enumerate(xq):
        start, _, _ = stencil(nodes, x, bc, period)
        starts[q] = start
        for m in range(4):
            e = np.zeros(n)
            e[(start + m) % n] = 1.0
            wts[q, m] = interp_1d(e, nodes, x, bc, period)
    return starts, wts


def coarse_gradients(uc, vc, wc, xf, yf, zf, bc):
    """Step (1): face-normal gradients at coarse cell centres.

    uc: (ncz, ncy, nfx) x-face velocity, vc: (ncz, nfy, ncx), wc: (nfz, ncy, ncx),
    where nf = nc for a periodic direction and nc + 1 with walls.
    """
    gx = (np.roll(uc, -1, axis=2)[:, :, :len(xf) - 1] - uc[:, :, :len(xf) - 1]) / np.diff(xf)[None, None, :]
    gy = (np.roll(vc, -1, axis=1)[:, :len(yf) - 1, :] - vc[:, :len(yf) - 1, :]) / np.diff(yf)[None, :, None]
    gz = (np.roll(wc, -1, axis=0)[:len(zf) - 1] - wc[:len(zf) - 1]) / np.diff(zf)[:, None, None]
    return gx, gy, gz


def tables(xf, yf, zf, fine_n, h, bc):
    """Index maps and weights from coarse cell centres to fine cell centres."""
    out = []
    for d, faces in enumerate((xf, yf, zf)):
        faces = np.asarray(faces, dtype=np.float64)
        nodes = centres(faces)
        xq = (np.arange(fine_n[d]) + 0.5) * h
        out.append(weight_table(nodes, xq, bc[d], faces[-1] - faces[0]))
    return out


def interp_3d(G, tabs):
    """Step (2): Sec. 3.4's 64-point tri-cubic Hermite stencil at every fine
    cell centre: sum_{a,b,c} wx[a] wy[b] wz[c] G[kz+c, ky+b, kx+a] (wrapped)."""
    (sx, wx), (sy, wy), (sz, wz) = tabs
    ncz, ncy, ncx = G.shape
    nz, ny, nx = len(sz), len(sy), len(sx)
    out = np.zeros((nz, ny, nx))
    for c in range(4):
        iz = (sz + c) % ncz
        for b in range(4):
            iy = (sy + b) % ncy
            for a in range(4):
                ix = (sx + a) % ncx
                out += (wz[:, c][:, None, None] * wy[:, b][None, :, None] * wx[:, a][None, None, :]
                        * G[iz[:, None, None], iy[None, :, None], ix[None, None, :]])
    return out


def interp_plane(P, tab_row, tab_col):
    """2D Hermite of a plane P[row][col] (16-point stencil)."""
    (sr, wr), (sc, wc) = tab_row, tab_col
    nr, nc = P.shape
    out = np.zeros((len(sr), len(sc)))
    for b in range(4):
        ir = (sr + b) % nr
        for a in range(4):
            ic = (sc + a) % nc
            out += wr[:, b][:, None] * wc[:, a][None, :] * P[ir[:, None], ic[None, :]]
    return out


def transfer(uc, vc, wc, xf, yf, zf, fine_n, h, bc):
    """Steps (1)-(3): fine face velocities (u, v, w) on the staggered fine mesh.

    Returns u (nz, ny, nfx), v (nz, nfy, nx), w (nfz, ny, nx) and the tables.
    Along each direction the fine face velocity is the reference-plane value
    plus h times the running sum of the interpolated normal gradient.
    """
    nx, ny, nz = fine_n
    tabs = tables(xf, yf, zf, fine_n, h, bc)
    gx, gy, gz = coarse_gradients(uc, vc, wc, xf, yf, zf, bc)
    Gx, Gy, Gz = interp_3d(gx, tabs), interp_3d(gy, tabs), interp_3d(gz, tabs)
    tx, ty, tz = tabs

    def integrate(G, ref, axis, walled):
        csum = np.cumsum(G, axis=axis) * h
        n = G.shape[axis]
        zero = np.zeros_like(np.take(G, [0], axis=axis))
        run = np.concatenate([zero, csum], axis=axis)           # n + 1 planes
        if not walled:
            run = np.take(run, np.arange(n), axis=axis)
        return np.expand_dims(ref, axis) + run

    # reference planes: u at x-face 0 interpolated in (z, y); v at y-face 0 in (z, x); w at z-face 0 in (y, x)
    u_ref = np.zeros((nz, ny)) if bc[0] != PERIODIC else interp_plane(uc[:, :, 0], tz, ty)
    v_ref = np.zeros((nz, nx)) if bc[1] != PERIODIC else interp_plane(vc[:, 0, :], tz, tx)
    w_ref = np.zeros((ny, nx)) if bc[2] != PERIODIC else interp_plane(wc[0, :, :], ty, tx)
    u = integrate(Gx, u_ref, 2, bc[0] != PERIODIC)
    v = integrate(Gy, v_ref, 1, bc[1] != PERIODIC)
    w = integrate(Gz, w_ref, 0, bc[2] != PERIODIC)
    return (u, v, w), tabs


def fine_divergence(u, v, w, h, fine_n):
    """Discrete divergence of a staggered fine face field at cell centres."""
    nx, ny, nz = fine_n
    du = np.roll(u, -1, axis=2)[:, :, :nx] - u[:, :, :nx] if u.shape[2] == nx else u[:, :, 1:] - u[:, :, :-1]
    dv = np.roll(v, -1, axis=1)[:, :ny, :] - v[:, :ny, :] if v.shape[1] == ny else v[:, 1:, :] - v[:, :-1, :]
    dw = np.roll(w, -1, axis=0)[:nz] - w[:nz] if w.shape[0] == nz else w[1:] - w[:-1]
    return (du + dv + dw) / h


def restriction_tables(xf, yf, zf, fine_n, h, bc):
    """Index maps and weights from fine cell centres to coarse cell centres."""
    out = []
    for d, faces in enumerate((xf, yf, zf)):
        faces = np.asarray(faces, dtype=np.float64)
        nodes = (np.arange(fine_n[d]) + 0.5) * h
        out.append(weight_table(nodes, centres(faces), bc[d], fine_n[d] * h))
    return out


def restrict_to_coarse(C, p, xf, yf, zf, lam_rho, lam_mu):
    """Down-sampling of Sec. 3.4: C and the fine surface-tension force F_st
    (Eq. eq-fst) interpolated to the coarse cell centres by the 64-point
    Hermite stencil, then rho and mu from the coarse C (Eqs. eq-rho, eq-mu).
    ``p`` is the fine-mesh ch_oracle.Params.  Returns (C_c, rho_c, mu_c,
    (Fx_c, Fy_c, Fz_c)), each [ncz][ncy][ncx]."""
    from oracle import ch_oracle as co
    tabs = restriction_tables(xf, yf, zf, (p.nx, p.ny, p.nz), p.h, p.bc)
    Cc = interp_3d(np.asarray(C, dtype=np.float64), tabs)
    F = co.surface_tension(np.asarray(C, dtype=np.float64), p)
    Fc = tuple(interp_3d(f, tabs) for f in F)
    return Cc, co.density(Cc, lam_rho), co.viscosity(Cc, lam_mu), Fc
