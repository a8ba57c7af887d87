"""Small, self-contained runs of the library's kernels for profilers.

``python -m paper_2105_01865_gb300.profile_case step NX NY NZ`` builds the
multiple-resolution recipe (uniform fine mesh NX x NY x NZ, x/y periodic,
no-flux z-walls, a tanh-stretched coarse mesh of a quarter of the cells per
direction with a seeded divergence-free velocity, 20 drops), then runs the
velocity transfer, two FP32 RK3 steps, and the mass and free energy in one
pass (ch_diagnostics): every
kernel of the hot path launches a few times, on inputs a few hundred MB in
size, so a one-kernel ncu capture (``-k <name> -c 1``) ends quickly.

``python -m paper_2105_01865_gb300.profile_case restrict NX NY NZ`` runs the
down-sampling of the fine fields to the coarse mesh of the same recipe twice.

``python -m paper_2105_01865_gb300.profile_case batch NBOX MODE`` runs two
steps of the first NBOX boxes of the batched workload (64 uneven periodic
boxes, u = 0) with the persistent (MODE = persistent) or per-phase
(MODE = phased) schedule.

Each prints one JSON line with its CUDA-event times.
"""
from __future__ import annotations

import json
import sys


def step_case(nx, ny, nz):
    import torch

    from . import build, capi, inputs, stability
    from .solver import Solver
    build.build()
    capi.load()
    f = inputs.multires_box((nx, ny, nz), (max(nx // 4, 4), max(ny // 4, 4), max(nz // 4, 4)), 20)
    h = f["h"]
    dt = min(0.9 * stability.stable_dt(f["shape"], h, f["bc"], f["cn"], f["pe"]), 0.5 * h)
    s = Solver(f["shape"], h, f["bc"], f["cn"], f["pe"], dt, f["C"], precision="f32", coarse_faces=f["faces"])
    s.set_velocity_coarse(*f["vel_coarse"])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s.stream):
        a.record(s.stream)
        s.interp_to_fine()
        s.step(2)
        b.record(s.stream)
    m, e = s.diagnostics()
    out = dict(case="step", fine=[nx, ny, nz], ms=a.elapsed_time(b), mass=m, free_energy=e)
    s.close()
    return out


def restrict_case(nx, ny, nz):
    """The down-sampling of the fine C to the coarse mesh (C, rho, mu, F_st) on
    the step case's recipe, twice."""
    import torch

    from . import build, capi, inputs
    from .solver import Solver
    build.build()
    capi.load()
    f = inputs.multires_box((nx, ny, nz), (max(nx // 4, 4), max(ny // 4, 4), max(nz // 4, 4)), 20)
    s = Solver(f["shape"], f["h"], f["bc"], f["cn"], f["pe"], 1e-4, f["C"], precision="f32", coarse_faces=f["faces"])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.restrict_to_coarse(0.05, 1.0)
    with torch.cuda.stream(s.stream):
        a.record(s.stream)
        s.restrict_to_coarse(0.05, 1.0)
        b.record(s.stream)
    s.sync()
    out = dict(case="restrict", fine=[nx, ny, nz], ms=a.elapsed_time(b))
    s.close()
    return out


def batch_case(nbox, mode):
    import numpy as np
    import torch

    from . import build, capi, inputs, stability
    from .solver import Batch
    build.build()
    capi.load()
    boxes = inputs.batch_boxes(64, seed=4)[:nbox]
    for b in boxes:
        b["dt"] = 0.9 * stability.stable_dt(b["shape"], b["h"], b["bc"], b["cn"], b["pe"])
    B = Batch(boxes)
    B.set_schedule(0 if mode == "persistent" else 1, 3, 16, 1)
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(B.stream):
        a.record(B.stream)
        B.step(2)
        c.record(B.stream)
    B.sync()
    out = dict(case="batch", boxes=nbox, mode=mode, cells=int(sum(np.prod(b["shape"]) for b in boxes)),
               ms_per_step=a.elapsed_time(c) / 2)
    B.close()
    return out


def main(argv):
    if len(argv) >= 4 and argv[0] == "step":
        print(json.dumps(step_case(int(argv[1]), int(argv[2]), int(argv[3]))))
    elif len(argv) >= 4 and argv[0] == "restrict":
        print(json.dumps(restrict_case(int(argv[1]), int(argv[2]), int(argv[3]))))
    elif len(argv) >= 3 and argv[0] == "batch":
        print(json.dumps(batch_case(int(argv[1]), argv[2])))
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
