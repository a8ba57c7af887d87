"""Seeded synthetic inputs for the Cahn-Hilliard step and the velocity transfer.

This module builds initial fields, face velocities and coarse grids only; it
holds none of the method's arithmetic and imports nothing else from this
package, so the tests can feed the same arrays to the CUDA library and to the
CPU oracle.  All randomness comes from numpy's PCG64 with fixed seeds.

Workload shapes follow the paper's cases (arXiv 2105.01865, Sec. 4): a drop
in shear (Sec. 4.1) and O(10^3) drops in a 2H x 2H x H wall-bounded box on a
uniform fine mesh above a wall-stretched coarse mesh (Secs. 3.4, 4.3, 4.4).
"""
from __future__ import annotations

import numpy as np

PERIODIC = 0
NOFLUX = 1


def cell_centres(n, h):
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def drop_profile(r, R, cn):
    """Equilibrium tanh profile C = (1 + tanh((R - r) / (2 sqrt(2) Cn))) / 2."""
    return 0.5 * (1.0 + np.tanh((R - r) / (2.0 * np.sqrt(2.0) * cn)))


def drops_field(shape, h, bc, centres, radii, cn):
    """C = max over drops of the tanh profile, with minimum-image distances in
    periodic directions.  shape = (nz, ny, nx); centres are (x, y, z)."""
    nz, ny, nx = shape
    L = (nx * h, ny * h, nz * h)
    x, y, z = cell_centres(nx, h), cell_centres(ny, h), cell_centres(nz, h)
    C = np.zeros(shape)
    for (cx, cy, cz), R in zip(centres, radii):
        dist = []
        for d, (coord, c) in enumerate(zip((x, y, z), (cx, cy, cz))):
            dd = coord - c
            if bc[d] == PERIODIC:
                dd = dd - L[d] * np.round(dd / L[d])
            dist.append(dd)
        r = np.sqrt(dist[2][:, None, None] ** 2 + dist[1][None, :, None] ** 2 + dist[0][None, None, :] ** 2)
        C = np.maximum(C, drop_profile(r, R, cn))
    return C


def drops_field_local(shape, h, centres, radii, cn, reach):
    """Same as drops_field for walled/periodic-free boxes, but each drop only
    touches cells within R + reach of its centre (for 10^8-cell grids)."""
    nz, ny, nx = shape
    C = np.zeros(shape, dtype=np.float32)
    for (cx, cy, cz), R in zip(centres, radii):
        lo = [max(int((c - R - reach) / h), 0) for c in (cx, cy, cz)]
        hi = [min(int((c + R + reach) / h) + 2, n) for c, n in zip((cx, cy, cz), (nx, ny, nz))]
        x = cell_centres(nx, h)[lo[0]:hi[0]] - cx
        y = cell_centres(ny, h)[lo[1]:hi[1]] - cy
        z = cell_centres(nz, h)[lo[2]:hi[2]] - cz
        r = np.sqrt(z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2)
        blk = C[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        np.maximum(blk, drop_profile(r, R, cn).astype(np.float32), out=blk)
    return C


def shear_velocity(shape, h, gamma_dot, bc):
    """Imposed shear u = gamma_dot (z - 1/2), v = w = 0 on the staggered mesh.

    u lives on x-faces at the cell-centre height; walls at z = 0, 1 when
    bc_z is a wall (then w has nz + 1 planes, all zero)."""
    nz, ny, nx = shape
    nfx = nx + (1 if bc[0] != PERIODIC else 0)
    nfy = ny + (1 if bc[1] != PERIODIC else 0)
    nfz = nz + (1 if bc[2] != PERIODIC else 0)
    z = cell_centres(nz, h)
    u = np.broadcast_to((gamma_dot * (z - 0.5))[:, None, None], (nz, ny, nfx)).copy()
    if bc[0] != PERIODIC:
        u[:, :, 0] = 0.0
        u[:, :, -1] = 0.0
    v = np.zeros((nz, nfy, nx))
    w = np.zeros((nfz, ny, nx))
    return u, v, w


def stretched_faces(n, length, s):
    """Wall-clustered face coordinates z_k = L/2 [1 + tanh(s(2k/n - 1)) / tanh(s)]."""
    k = np.arange(n + 1, dtype=np.float64)
    return 0.5 * length * (1.0 + np.tanh(s * (2.0 * k / n - 1.0)) / np.tanh(s))


def uniform_faces(n, length):
    return np.arange(n + 1, dtype=np.float64) * (length / n)


def curl_velocity(xf, yf, zf, bc, seed, kmax=8, slope=-11.0 / 6.0, umax=1.0):
    """Divergence-free staggered velocity as the discrete curl of a seeded
    random-Fourier vector potential (A_x, A_y, A_z) on cell edges.

    Because it is a discrete curl, the discrete face-flux divergence of every
    cell vanishes up to rounding on any (stretched) mesh.  Mode amplitudes
    follow |k|^slope for 1 <= |k| <= kmax (units of 2 pi / L in periodic
    directions, pi / L across walls).  Tangential potential components vanish
    on walls, so the normal velocity is zero there.  Scaled to max |u| = umax.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    faces = [np.asarray(a, dtype=np.float64) for a in (xf, yf, zf)]
    Ls = [f[-1] - f[0] for f in faces]
    ncs = [len(f) - 1 for f in faces]
    cents = [0.5 * (f[:-1] + f[1:]) for f in faces]

    def basis(d, coords, wall_zero):
        """Real 1D mode functions along d evaluated at coords: (nmodes, len)."""
        if bc[d] == PERIODIC:
            ks = np.arange(-kmax, kmax + 1)
            ph = 2.0 * np.pi * np.outer(ks, coords) / Ls[d]
            return ks.astype(np.float64), np.cos(ph), np.sin(ph)
        ks = np.arange(0, kmax + 1)
        ph = np.pi * np.outer(ks, coords - faces[d][0]) / Ls[d]
        f = np.sin(ph) if wall_zero else np.cos(ph)
        return ks.astype(np.float64), f, f

    # positions of each potential component: A_x at (xc, yf, zf), A_y at (xf, yc, zf), A_z at (xf, yf, zc)
    def component(pos, wall_zero_dirs):
        out = None
        bx = basis(0, pos[0], 0 in wall_zero_dirs)
        by = basis(1, pos[1], 1 in wall_zero_dirs)
        bz = basis(2, pos[2], 2 in wall_zero_dirs)
        KX, KY, KZ = np.meshgrid(bx[0], by[0], bz[0], indexing="ij")
        kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
        mask = (kk >= 1.0) & (kk <= kmax)
        amp = np.where(mask, np.maximum(kk, 1.0) ** slope, 0.0)
        a = amp * rng.standard_normal(amp.shape)
        b = amp * rng.standard_normal(amp.shape)
        # field = sum a*cx*cy*cz + b*sx*sy*sz  (separable contractions)
        for coef, fx, fy, fz in ((a, bx[1], by[1], bz[1]), (b, bx[2], by[2], bz[2])):
            t = np.einsum("xyz,zk->xyk", coef, fz)
            t = np.einsum("xyk,yj->xjk", t, fy)
            t = np.einsum("xjk,xi->kji", t, fx)
            out = t if out is None else out + t
        return out

    walled = {d for d in range(3) if bc[d] != PERIODIC}
    # a tangential component must vanish on walls normal to another direction
    Ax = component((cents[0], faces[1], faces[2]), walled - {0})
    Ay = component((faces[0], cents[1], faces[2]), walled - {1})
    Az = component((faces[0], faces[1], cents[2]), walled - {2})
    dx, dy, dz = (np.diff(f) for f in faces)

    def diff(a, axis, periodic_n):
        """Forward difference along axis; for a periodic direction the edge array
        carries n+1 points (the last duplicates the first), difference gives n."""
        return np.diff(a, axis=axis)

    # u at (xf, yc, zc): dAz/dy - dAy/dz
    u = diff(Az, 1, None) / dy[None, :, None] - diff(Ay, 0, None) / dz[:, None, None]
    # v at (xc, yf, zc): dAx/dz - dAz/dx
    v = diff(Ax, 0, None) / dz[:, None, None] - diff(Az, 2, None) / dx[None, None, :]
    # w at (xc, yc, zf): dAy/dx - dAx/dy
    w = diff(Ay, 2, None) / dx[None, None, :] - diff(Ax, 1, None) / dy[None, :, None]
    # drop the duplicated periodic face plane
    if bc[0] == PERIODIC:
        u = u[:, :, :ncs[0]]
    if bc[1] == PERIODIC:
        v = v[:, :ncs[1], :]
    if bc[2] == PERIODIC:
        w = w[:ncs[2]]
    scale = umax / max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max(), 1e-300)
    return (np.ascontiguousarray(u * scale), np.ascontiguousarray(v * scale),
            np.ascontiguousarray(w * scale))


def random_drops(rng, n, box, rmin, rmax, gap, walls, max_tries=200000):
    """Rejection-sample n non-overlapping drops: pairwise distance >= R1 + R2
    + gap, and >= R + gap from walls (walls: tuple of bools per direction)."""
    centres, radii = [], []
    tries = 0
    while len(centres) < n and tries < max_tries:
        tries += 1
        R = rng.uniform(rmin, rmax)
        c = np.array([rng.uniform(0, L) for L in box])
        ok = all(not walls[d] or (c[d] >= R + gap and c[d] <= box[d] - R - gap) for d in range(3))
        if ok and centres:
            P = np.array(centres)
            dd = np.abs(P - c)
            for d in range(3):
                if not walls[d]:
                    dd[:, d] = np.minimum(dd[:, d], box[d] - dd[:, d])
            ok = bool(np.all(np.sqrt((dd ** 2).sum(1)) >= np.array(radii) + R + gap))
        if ok:
            centres.append(c)
            radii.append(R)
    return centres, radii


# ---------------------------------------------------------------------------
# Workloads (fields only; the caller chooses the time step and the physical
# constants)
# ---------------------------------------------------------------------------

def single_drop_box(n=64):
    """Periodic unit box n^3, h = 1/n, one drop R = 0.25 at the centre, Cn = 1/64."""
    h = 1.0 / n
    bc = (PERIODIC, PERIODIC, PERIODIC)
    cn = 1.0 / 64.0
    C = drops_field((n, n, n), h, bc, [(0.5, 0.5, 0.5)], [0.25], cn)
    return dict(shape=(n, n, n), h=h, bc=bc, cn=cn, pe=1e3, C=C, vel=None)


def shear_drop_box(nx=256, ny=256, nz=128):
    """Drop R = 0.2 in the shear u = z - 1/2 between no-flux walls z = 0, 1;
    x, y periodic on [0, 2]; h = 1/nz; Cn = 0.75 h; Pe = 0.9 / Cn."""
    h = 1.0 / nz
    bc = (PERIODIC, PERIODIC, NOFLUX)
    cn = 0.75 * h
    shape = (nz, ny, nx)
    C = drops_field(shape, h, bc, [(nx * h / 2, ny * h / 2, 0.5)], [0.2], cn)
    vel = shear_velocity(shape, h, 1.0, bc)
    return dict(shape=shape, h=h, bc=bc, cn=cn, pe=0.9 / cn, C=C, vel=vel)


def batch_boxes(nbox=64, seed=4, sizes=(32, 48, 64, 96, 128), only=None):
    """Independent periodic unit boxes of uneven size and parameters: n^3 with
    n ~ U{sizes}, h = 1/n, Cn ~ U[0.5 h, h], Pe log-uniform on [1e2, 1e4],
    1..8 drops with R ~ U[0.08, 0.25] (non-overlapping, rejection sampled).
    With only = i the random draws are the same but only box i's field is
    built (the others carry C = None)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    boxes = []
    bc = (PERIODIC, PERIODIC, PERIODIC)
    for _ in range(nbox):
        n = int(rng.choice(sizes))
        h = 1.0 / n
        cn = float(rng.uniform(0.5 * h, 1.0 * h))
        pe = float(10.0 ** rng.uniform(2.0, 4.0))
        ndrop = int(rng.integers(1, 9))
        centres, radii = random_drops(rng, ndrop, (1.0, 1.0, 1.0), 0.08, 0.25, 4 * cn, (False, False, False),
                                      max_tries=2000)
        C = drops_field((n, n, n), h, bc, centres, radii, cn) if only is None or only == len(boxes) else None
        boxes.append(dict(shape=(n, n, n), h=h, bc=bc, cn=cn, pe=pe, C=C, vel=None))
    return boxes


def multires_box(fine=(1024, 1024, 512), coarse=(256, 256, 128), ndrops=1000, seed=3, stretch=2.0, kmax=8,
                 rmin=0.01, rmax=0.03):
    """Multiple-resolution workload (Secs. 3.4, 4.4): a wall-bounded box
    [0, 2] x [0, 2] x [0, 1] (x, y periodic, no-flux walls at z = 0, 1), a
    coarse mesh tanh-stretched in z carrying a seeded divergence-free
    random-Fourier face velocity (max |u| = 1), and a uniform fine mesh of
    spacing h = 1 / nz_fine holding up to ndrops drops of radius U[rmin, rmax]
    at seeded positions (pairwise gap and wall gap >= 4 Cn), Cn = 0.75 h,
    Pe = 0.9 / Cn.  fine and coarse are (nx, ny, nz)."""
    nx, ny, nz = fine
    h = 1.0 / nz
    bc = (PERIODIC, PERIODIC, NOFLUX)
    cn = 0.75 * h
    xf = uniform_faces(coarse[0], nx * h)
    yf = uniform_faces(coarse[1], ny * h)
    zf = stretched_faces(coarse[2], nz * h, stretch)
    uc, vc, wc = curl_velocity(xf, yf, zf, bc, seed, kmax=kmax)
    rng = np.random.Generator(np.random.PCG64(seed))
    centres, radii = random_drops(rng, ndrops, (nx * h, ny * h, nz * h), rmin, rmax, 4 * cn, (True, True, True))
    C = drops_field_local((nz, ny, nx), h, centres, radii, cn, 8 * cn)
    return dict(shape=(nz, ny, nx), h=h, bc=bc, cn=cn, pe=0.9 / cn, faces=(xf, yf, zf), vel_coarse=(uc, vc, wc),
                C=C, ndrops=len(radii))
