"""CPU timing of the oracle on the batched workload (test infrastructure).

Only bench.py's CPU-baseline leg uses this module.  It runs the unmodified
oracle (oracle/ch_oracle.py) on the 64 independent boxes of the batched
workload, one RK3 step per box, one box at a time in each process of a pool
(one process per core), so the wall time is the all-cores time of the plain
method on that workload and the sum of the per-box times is its single-core
time.
"""
from __future__ import annotations

import time

from paper_2105_01865_gb300 import inputs

from . import ch_oracle as co


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
