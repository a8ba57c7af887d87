"""The algebra of a z-slab partition of the line solve (I + c A_z) x = r
(Eqs. eq-fac-3 and eq-a3d), checked among gloo ranks on the CPU against the
oracle's dense solve.

This is the exchange a box sharded into z-slabs over several GPUs would need
for its z-solve: each rank holds rows [a_r, b_r) of every z-line.  The banded
factors L U of the non-cyclic part B are known to every rank (they depend on
the coefficients only).  Per solve:

* forward elimination: each rank runs its rows from a zero state; the end
  states (2 values per line) are all-gathered, and each rank composes those of
  the ranks before it with their 2x2 transfer matrices to get its incoming
  state, then reruns its rows;
* back substitution: the same from the last rank down;
* periodic lines: the corner rows 0, 1, n-2, n-1 of the banded solution
  (4 values per line, on the first and last rank) are summed over ranks and
  give the rank-4 Woodbury correction x = y - Z K y_c, Z's rows local.

So a slab boundary costs 2 + 2 values per line per solve, plus 4 per line for
periodic lines, whatever the slab height.
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import ch_oracle as co


def band_lu(Bm):
    """LU without pivoting of a pentadiagonal matrix: multipliers l1, l2
    (sub-diagonals of the unit L), and U's diagonal and two super-diagonals."""
    n = Bm.shape[0]
    U = Bm.astype(float).copy()
    l1 = np.zeros(n)
    l2 = np.zeros(n)
    for k in range(n):
        for i, lo in ((k + 1, l1), (k + 2, l2)):
            if i < n:
                f = U[i, k] / U[k, k]
                lo[i] = f
                U[i, k:min(n, k + 3)] -= f * U[k, k:min(n, k + 3)]
    d = np.diag(U).copy()
    u1 = np.array([U[i, i + 1] if i + 1 < n else 0.0 for i in range(n)])
    u2 = np.array([U[i, i + 2] if i + 2 < n else 0.0 for i in range(n)])
    return l1, l2, d, u1, u2


def rows_of(n, world, rank):
    """Slab rows [a, b) of rank (uneven heights allowed)."""
    return n * rank // world, n * (rank + 1) // world


def fwd_map(l1, l2, a, b):
    """2x2 map of the state (z_i, z_{i-1}) across rows [a, b) of
    z_i = r_i - l1_i z_{i-1} - l2_i z_{i-2}, homogeneous part."""
    T = np.eye(2)
    for i in range(a, b):
        T = np.array([[-l1[i], -l2[i]], [1.0, 0.0]]) @ T
    return T


def bwd_map(d, u1, u2, a, b):
    """2x2 map of the state (y_i, y_{i+1}) across rows [a, b), from b - 1 down
    to a, of y_i = (z_i - u1_i y_{i+1} - u2_i y_{i+2}) / d_i, homogeneous part."""
    T = np.eye(2)
    for i in range(b - 1, a - 1, -1):
        T = np.array([[-u1[i] / d[i], -u2[i] / d[i]], [1.0, 0.0]]) @ T
    return T


def slab_solve(r_loc, n, bc, c, kappa, world, rank):
    """Distributed solve of (I + c A) x = r for the lines r_loc[rows, lines]
    held by this rank; returns this rank's rows of x."""
    a, b = rows_of(n, world, rank)
    A = co.line_operator(n, bc, kappa)
    M = np.eye(n) + c * A
    corner = [0, 1, n - 2, n - 1]
    Bm = M.copy()
    if bc == co.PERIODIC:          # B: the band without the wrapped corner entries
        for i in corner:
            for j in corner:
                if abs(i - j) > 2:
                    Bm[i, j] = 0.0
    l1, l2, d, u1, u2 = band_lu(Bm)
    nl = r_loc.shape[1]

    # forward elimination: zero-start pass, exchange end states, rerun
    def fwd(incoming):
        z = np.zeros_like(r_loc)
        zm1, zm2 = incoming
        for i in range(a, b):
            zi = r_loc[i - a] - l1[i] * zm1 - l2[i] * zm2
            z[i - a] = zi
            zm2, zm1 = zm1, zi
        return z, np.stack([zm1, zm2])
    _, end0 = fwd((np.zeros(nl), np.zeros(nl)))
    ends = [torch.zeros(2, nl, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(ends, torch.from_numpy(end0))
    s = np.zeros((2, nl))
    for q in range(rank):
        qa, qb = rows_of(n, world, q)
        s = fwd_map(l1, l2, qa, qb) @ s + ends[q].numpy()
    z, _ = fwd((s[0], s[1]))

    # back substitution: zero-start pass, exchange, rerun (from the last rank)
    def bwd(incoming):
        y = np.zeros_like(z)
        yp1, yp2 = incoming
        for i in range(b - 1, a - 1, -1):
            yi = (z[i - a] - u1[i] * yp1 - u2[i] * yp2) / d[i]
            y[i - a] = yi
            yp2, yp1 = yp1, yi
        return y, np.stack([yp1, yp2])
    _, bend0 = bwd((np.zeros(nl), np.zeros(nl)))
    bends = [torch.zeros(2, nl, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(bends, torch.from_numpy(bend0))
    t = np.zeros((2, nl))
    for q in range(world - 1, rank, -1):
        qa, qb = rows_of(n, world, q)
        t = bwd_map(d, u1, u2, qa, qb) @ t + bends[q].numpy()
    y, _ = bwd((t[0], t[1]))
    if bc != co.PERIODIC:
        return y

    # periodic: Woodbury from the corner rows of the banded solution
    yc = torch.zeros(4, nl, dtype=torch.float64)
    for k, i in enumerate(corner):
        if a <= i < b:
            yc[k] = torch.from_numpy(y[i - a])
    dist.all_reduce(yc)  # the corner rows live on the first and last rank
    P = np.zeros((n, 4))
    P[corner, range(4)] = 1.0
    Z = np.linalg.solve(Bm, P)                 # B^-1 P_c (line-independent)
    G = (M - Bm)[np.ix_(corner, corner)]       # the wrapped corner couplings
    K = np.linalg.solve(np.eye(4) + G @ Z[corner], G)
    return y - Z[a:b] @ (K @ yc.numpy())


def _worker(rank, world, port, cases, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = []
        for n, bc, c, kappa, R in cases:
            a, b = rows_of(n, world, rank)
            res.append(slab_solve(R[a:b], n, bc, c, kappa, world, rank))
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_z_slab_solve_matches_oracle(world):
    rng = np.random.default_rng(21)
    cases = []
    for n, bc in ((24, co.PERIODIC), (25, co.NOFLUX), (23, co.DIRICHLET), (31, co.PERIODIC)):
        h = 1.0 / n
        kappa = 4.0 * (0.75 * h) ** 2 / h ** 4
        for c in (1.5e-4, 4e-3):  # c kappa from about 0.2 to 5: weak and strong coupling across slabs
            cases.append((n, bc, c, kappa, rng.standard_normal((n, 7))))
    port = 29600 + (os.getpid() % 1000) + 10 * world
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, cases, out), nprocs=world, join=True)
        res = dict(out)
    for k, (n, bc, c, kappa, R) in enumerate(cases):
        x = np.concatenate([res[r][k] for r in range(world)], axis=0)
        ref = np.linalg.solve(np.eye(n) + c * co.line_operator(n, bc, kappa), R)
        assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref), (n, bc)
