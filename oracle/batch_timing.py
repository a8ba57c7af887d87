"""CPU timing of the oracle on the bench's workloads (test infrastructure).

Only bench.py's CPU-baseline legs use this module.  It runs the unmodified
oracle (oracle/ch_oracle.py, oracle/mr_oracle.py) in the processes of a pool
(one single-threaded process per core):

* the 64 independent boxes of the batched workload, one RK3 step per box, one
  box at a time in each process, so the wall time is the all-cores time of the
  plain method on that workload and the sum of the per-box times is its
  single-core time;
* one hot-path step of the multiple-resolution workload on a sample mesh
  (velocity transfer, RK3 step, mass and free energy), the same sample in
  every process, so the pool's cells over its wall time is the all-cores rate.
"""
from __future__ import annotations

import time

from paper_2105_01865_gb300 import inputs

from . import ch_oracle as co
from . import mr_oracle as mo


def ready(delay: float) -> bool:
    """Warm-up task: holds a pool worker for delay seconds, so that every
    worker is started and has imported this module before the timing."""
    time.sleep(delay)
    return True


def box_step(i: int, dt: float, nbox: int = 64, seed: int = 4):
    """One oracle step of size dt of box i of the batched workload (the
    seeded generator's boxes).  Returns (cells, seconds of the step alone)."""
    box = inputs.batch_boxes(nbox, seed, only=i)[i]
    nz, ny, nx = box["shape"]
    p = co.Params(nx, ny, nz, box["h"], cn=box["cn"], pe=box["pe"], dt=dt, bc=box["bc"])
    t0 = time.perf_counter()
    co.step(box["C"], None, p, 1)
    return nx * ny * nz, time.perf_counter() - t0


_MR_CACHE = {}


def multires_step(fine, coarse, ndrops, dt):
    """One oracle step of the whole hot path on the multiple-resolution
    workload of the given sizes (inputs.multires_box): the Sec. 3.4 velocity
    transfer, one RK3 step of Sec. 3, then mass and free energy.  The inputs
    are built (and cached per process) outside the timed region.  Returns
    (cells, seconds)."""
    key = (tuple(fine), tuple(coarse), ndrops)
    if key not in _MR_CACHE:
        _MR_CACHE[key] = inputs.multires_box(tuple(fine), tuple(coarse), ndrops)
    f = _MR_CACHE[key]
    nz, ny, nx = f["shape"]
    p = co.Params(nx, ny, nz, f["h"], cn=f["cn"], pe=f["pe"], dt=dt, bc=f["bc"])
    C0 = f["C"].astype("float64")
    t0 = time.perf_counter()
    vel, _ = mo.transfer(*f["vel_coarse"], *f["faces"], (nx, ny, nz), f["h"], f["bc"])
    C = co.step(C0, vel, p, 1)
    co.mass(C, p)
    co.free_energy(C, p)
    return nx * ny * nz, time.perf_counter() - t0
