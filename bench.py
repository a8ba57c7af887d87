"""Throughput of the Cahn-Hilliard fine-grid step on GB300.

Workload (default): drop in imposed shear on a 256 x 256 x 128 uniform mesh,
x/y periodic on [0, 2], no-flux walls at z = 0, 1, u = (z - 1/2, 0, 0),
Cn = 0.75 h, Pe = 0.9 / Cn, FP32 fields (the precision form), dt =
min(0.9 dt_stab, CFL 0.5).  One step = one full RK3 step (three substeps of
explicit RHS + x, y, z line solves) over every cell.  Metric: fine-grid
cell-updates/s.  The working set (C, two H, rhs, three face velocities,
~235 MB) exceeds the 129 MB L2, and L2 is also flushed between timed steps.

``python bench.py [--gpus N --steps K --warmup W]`` prints one JSON line.
``--impl reference`` times the CPU FP64 oracle instead (the slow baseline).
Under torchrun every rank runs an independent replica of the workload
(one box does not shard: replicas only); value = all ranks' cell updates
divided by the max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="shear_drop_256x256x128", nx=256, ny=256, nz=128)
# CPU sample for the oracle legs: the same workload recipe on a 128 x 128 x 64 mesh
SAMPLE = dict(nx=128, ny=128, nz=64)
METRIC = "fine-grid CH cell-updates/s"
L2_FLUSH_BYTES = 256 << 20


def _rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def workload_inputs(nx, ny, nz):
    from paper_2105_01865_gb300 import inputs, stability
    f = inputs.shear_drop_box(nx, ny, nz)
    h = f["h"]
    dt = min(0.9 * stability.stable_dt(f["shape"], h, f["bc"], f["cn"], f["pe"]), 0.5 * h / 0.5)
    f["dt"] = dt
    return f


# ---------------------------------------------------------------------------
# oracle (CPU) legs, run in a fresh single-threaded interpreter
# ---------------------------------------------------------------------------

_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import ch_oracle as co
import bench
f = bench.workload_inputs({nx}, {ny}, {nz})
nz, ny, nx = f["shape"]
p = co.Params(nx, ny, nz, f["h"], cn=f["cn"], pe=f["pe"], dt=f["dt"], bc=f["bc"])
C = f["C"]
times = []
for s in range({total}):
    t0 = time.perf_counter()
    C = co.step(C, f["vel"], p, 1)
    times.append(time.perf_counter() - t0)
print(json.dumps(dict(times=times, cells=nx * ny * nz)))
"""


def run_oracle(steps, warmup, sample=SAMPLE):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = _ORACLE_SNIPPET.format(root=ROOT, total=steps + warmup, **sample)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if out.returncode != 0:
        raise RuntimeError("oracle leg failed:\n" + out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    t = r["times"][warmup:]
    return r["cells"], t


_ORACLE_BATCH_SNIPPET = """
import json, os, sys, time
sys.path.insert(0, {root!r})
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor
import numpy as np
from oracle import batch_timing as bt
from paper_2105_01865_gb300 import inputs
if __name__ == "__main__":
    boxes = inputs.batch_boxes(64, 4, only=-1)
    dts = json.loads(sys.stdin.read())
    order = sorted(range(len(boxes)), key=lambda i: -int(np.prod(boxes[i]["shape"])))
    n = len(os.sched_getaffinity(0))
    with ProcessPoolExecutor(n, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(bt.ready, [0.5] * n))
        t0 = time.perf_counter()
        res = list(ex.map(bt.box_step, order, [dts[i] for i in order]))
        wall = time.perf_counter() - t0
    print(json.dumps(dict(cells=sum(c for c, _ in res), wall=wall, cpu=sum(t for _, t in res), workers=n)))
"""


def run_oracle_batch(dts):
    """The oracle on all 64 boxes of the batched workload (box i with step
    dts[i]), one step each, over a spawn pool of one single-threaded oracle
    process per available core."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = _ORACLE_BATCH_SNIPPET.format(root=ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                         input=json.dumps(list(dts)))
    if out.returncode != 0:
        raise RuntimeError("batched oracle leg failed:\n" + out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    return dict(value=r["cells"] / r["wall"], unit="cell-updates/s", cores=r["workers"], kind="oracle",
                single_core_value=r["cells"] / r["cpu"],
                sample="all 64 boxes of the batched workload, one RK3 step each (FP64 numpy oracle), largest "
                       "first over a spawn pool of one single-threaded oracle process per available core; "
                       f"host CPU {cpu_model()}")


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def reference_arm(args):
    rank, world, _ = _rank()
    if rank != 0:
        return
    cells, times = run_oracle(args.steps, args.warmup)
    sec = sum(times)
    value = cells * len(times) / sec
    line = dict(metric=METRIC, value=value, unit="cell-updates/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * sec / len(times), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD["name"], global_batch=1, seq_len=0, parallelism="replicas"),
                cpu_baseline=dict(value=value, unit="cell-updates/s", cores=1, kind="oracle",
                                  sample=f"FP64 numpy oracle, one RK3 step per timed step of the same shear-drop "
                                         f"recipe on a {SAMPLE['nx']}x{SAMPLE['ny']}x{SAMPLE['nz']} mesh, "
                                         f"single thread, host CPU {cpu_model()}"),
                e2e=dict(value=value, unit="cell-updates/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                gpu_launches=0)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, out_dir=None):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: --clocks-dir if given, else a temporary directory
        base = out_dir or os.path.join(tempfile.gettempdir(), "ch_bench_clocks")
        self.path = os.path.join(base, f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (data sheet); the measured copy peak is the roofline's denominator


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        for k in ("hbm_gbs", "hbm_GBps", "hbm"):
            if k in d:
                v = d[k]
                return float(v["value"] if isinstance(v, dict) else v), "measured"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6800.0, "fallback"


def kernel_source_sha():
    import hashlib
    csrc = os.path.join(ROOT, "paper_2105_01865_gb300", "csrc")
    hsh = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as fh:
            hsh.update(name.encode() + fh.read())
    return hsh.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch (ncu dram__bytes_read + write) recorded in
    profiles/ncu_traffic.json, only if it was taken on the current kernels."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except (OSError, ValueError):
        return {}
    if rec.get("source_sha") != kernel_source_sha():
        return {}
    return rec.get("bytes_per_launch", {})


def batched_leg(args, dev, flush, rank=0, world=1):
    """The batched form on 64 uneven periodic boxes (32^3 .. 128^3), u = 0.
    With several ranks the boxes are placed by LPT on cell counts (no
    collective on the data path); the time is the max over ranks."""
    import torch
    from paper_2105_01865_gb300 import inputs, stability
    from paper_2105_01865_gb300.sharding import lpt_assign, max_over_ranks
    from paper_2105_01865_gb300.solver import Batch
    all_boxes = inputs.batch_boxes(64, seed=4)
    cells_all = [int(np.prod(b["shape"])) for b in all_boxes]
    mine = lpt_assign(cells_all, world)[rank]
    boxes = [all_boxes[i] for i in mine]
    for box in boxes:
        box["dt"] = 0.9 * stability.stable_dt(box["shape"], box["h"], box["bc"], box["cn"], box["pe"])
    cells = sum(cells_all)
    b = Batch(boxes, device=dev)
    report = b.autotune(2)
    st = b.stream
    for _ in range(args.warmup):
        b.step(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(st):
        for a, c in ev:
            flush.fill_(1)
            a.record(st)
            b.step(1)
            c.record(st)
    torch.cuda.synchronize(dev)
    b.sync()
    sec = max_over_ranks(sum(a.elapsed_time(c) for a, c in ev) / 1e3)
    sched = b.schedule()
    out = dict(value=cells * args.steps / sec, unit="cell-updates/s", ms_per_step=1e3 * sec / args.steps,
               boxes=len(all_boxes), cells=cells, dtype="f32", placement="LPT on cell counts, no collective",
               schedule=dict(mode="persistent" if sched[0] == 0 else "phased", blocks_per_sm=sched[1],
                             zchunk=sched[2], lpt=sched[3]),
               launches_per_step=b.launches_per_step(), autotune_candidates=report.count("\n") - 1)
    b.close()
    # per-box steps for the CPU baseline of this workload (popped before printing)
    out["_dts"] = {i: box["dt"] for i, box in zip(mine, boxes)}
    return out


def multires_leg(args, dev, flush):
    """Multiple-resolution workload: seeded divergence-free coarse velocity on
    a 256 x 256 x 128 mesh (tanh-stretched z, walls at z = 0, 1) transferred
    to the 1024 x 1024 x 512 uniform FP32 fine mesh holding ~1000 drops of
    radius U[0.01, 0.03]; times the transfer, the down-sampling of C (with
    rho, mu, F_st on the coarse mesh) and the fine CH step."""
    import torch
    from paper_2105_01865_gb300 import inputs, stability
    from paper_2105_01865_gb300.solver import Solver
    nx, ny, nz = 1024, 1024, 512
    h = 1.0 / nz
    bc = (0, 0, 1)
    cn = 0.75 * h
    pe = 0.9 / cn
    xf, yf = inputs.uniform_faces(256, 2.0), inputs.uniform_faces(256, 2.0)
    zf = inputs.stretched_faces(128, 1.0, 2.0)
    uc, vc, wc = inputs.curl_velocity(xf, yf, zf, bc, 3, kmax=8)
    rng = np.random.Generator(np.random.PCG64(3))
    centres, radii = inputs.random_drops(rng, 1000, (2.0, 2.0, 1.0), 0.01, 0.03, 4 * cn, (True, True, True))
    C0 = inputs.drops_field_local((nz, ny, nx), h, centres, radii, cn, 8 * cn)
    dt = min(0.9 * stability.stable_dt((nz, ny, nx), h, bc, cn, pe), 0.5 * h / 1.0)
    s = Solver((nz, ny, nx), h, bc, cn, pe, dt, C0, precision="f32", coarse_faces=(xf, yf, zf), device=dev)
    s.set_velocity_coarse(uc, vc, wc)
    st = s.stream

    def timed(fn, reps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(st):
            for a, c in ev:
                flush.fill_(1)
                a.record(st)
                fn()
                c.record(st)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(c) for a, c in ev) / reps

    s.interp_to_fine()
    interp_ms = timed(s.interp_to_fine, 3)
    # down-sampling back-coupling: coarse C, rho, mu and F_st (Sec. 3.4)
    s.restrict_to_coarse(0.05, 1.0)
    restrict_ms = timed(lambda: s.restrict_to_coarse(0.05, 1.0), 3)
    for _ in range(3):
        s.step(1)
    k = max(3, min(args.steps, 20))
    step_ms = timed(lambda: s.step(1), k)
    s.sync()
    cells = nx * ny * nz
    out = dict(value=cells / (step_ms * 1e-3), unit="cell-updates/s", step_ms=step_ms, interp_ms=interp_ms,
               cells=cells, coarse_cells=256 * 256 * 128, drops=len(radii), steps=k, dtype="f32",
               interp_fine_faces_gbs=3 * cells * 4 / (interp_ms * 1e-3) / 1e9,
               restrict_ms=restrict_ms,
               restrict_fine_read_gbs=cells * 4 / (restrict_ms * 1e-3) / 1e9)
    s.close()
    return out


def scheme_leg(args, dev, W):
    """Time to solution of the paper's split scheme against the standard
    explicit 25-point scheme (Eq. eq-disbi) it replaces (Sec. 4.1 reports
    dt = 2e-3 against 5e-5 for its shear drop): both FP32, on the bench's
    shear-drop box, from the same C0 to the same time T = 10 steps of the
    split scheme, each at its largest stable dt (linear bound x 0.9, CFL
    0.5 h / max|u|).  Per-kernel times of the standard scheme come from
    ch_profile_step (chemical potential, advection, update)."""
    import math

    import torch
    from paper_2105_01865_gb300 import capi, inputs, stability
    from paper_2105_01865_gb300.solver import Solver
    f = inputs.shear_drop_box(W["nx"], W["ny"], W["nz"])
    h, bc, cn, pe = f["h"], f["bc"], f["cn"], f["pe"]
    ncell = W["nx"] * W["ny"] * W["nz"]
    cfl = 0.5 * h / 0.5
    dt_split = min(0.9 * stability.stable_dt(f["shape"], h, bc, cn, pe), cfl)
    dt_std_max = min(0.9 * stability.stable_dt_standard(f["shape"], h, bc, cn, pe), cfl)
    n_split = 10
    T = n_split * dt_split
    n_std = int(math.ceil(T / dt_std_max))
    dt_std = T / n_std
    C0 = torch.as_tensor(f["C"], dtype=torch.float32)
    out = {}
    fields = {}
    for name, scheme, dt, n in (("split", "split", dt_split, n_split), ("standard", "standard", dt_std, n_std)):
        s = Solver(f["shape"], h, bc, cn, pe, dt, f["C"], precision="f32", advect=True, device=dev, scheme=scheme)
        s.set_velocity_fine(*f["vel"])
        s.step(1)                     # captures the step graph
        s.C.copy_(C0.to(dev))         # restart from C0
        s._order()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s.stream):
            a.record(s.stream)
            s.step(n)
            b.record(s.stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b)
        fields[name] = s.field()
        out[name] = dict(dt=dt, steps=n, ms=ms, ms_per_step=ms / n)
        if name == "standard":
            kms = [0.0] * 4
            for _ in range(3):
                kms = [x + y for x, y in zip(kms, capi.ch_profile_step(s.handle, 1))]
            names = ("ch_std_mu", "advection", "ch_std_update")
            kbytes = (8.0, 80.0 / 3.0 - 8.0, 24.0)  # algorithmic B/cell: mu, advection (C, u, v, w; H), update
            out[name]["kernels"] = {nm: dict(ms=k / 3, gbs=b * ncell / (k / 3 * 1e-3) / 1e9)
                                    for nm, k, b in zip(names, kms[:3], kbytes)}
        s.close()
    ref = fields["split"]
    out.update(T=T, dt_ratio=dt_split / dt_std_max,
               time_to_solution_speedup=out["standard"]["ms"] / out["split"]["ms"],
               rel_l2_standard_vs_split=float(np.linalg.norm(fields["standard"] - ref) / np.linalg.norm(ref)),
               paper_dt_ratio=2e-3 / 5e-5)
    return out


def dirichlet_leg(args, dev, flush, W):
    """The bench's shear-drop box with Dirichlet walls (C = 0 on z = 0, 1, the
    Rayleigh-Benard setting of Sec. 4.3) instead of no-flux ones: FP32 step
    time, L2 flushed between steps."""
    import torch
    from paper_2105_01865_gb300 import capi, inputs, stability
    from paper_2105_01865_gb300.solver import Solver
    f = inputs.shear_drop_box(W["nx"], W["ny"], W["nz"])
    h, cn, pe = f["h"], f["cn"], f["pe"]
    bc = (capi.CH_PERIODIC, capi.CH_PERIODIC, capi.CH_DIRICHLET)
    dt = min(0.9 * stability.stable_dt(f["shape"], h, bc, cn, pe), 0.5 * h / 0.5)
    s = Solver(f["shape"], h, bc, cn, pe, dt, f["C"], precision="f32", advect=True, device=dev)
    s.set_velocity_fine(*f["vel"])
    st = s.stream
    for _ in range(3):
        s.step(1)
    k = max(3, min(args.steps, 20))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(st):
        for a, b in ev:
            flush.fill_(1)
            a.record(st)
            s.step(1)
            b.record(st)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in ev) / k
    cells = W["nx"] * W["ny"] * W["nz"]
    s.close()
    return dict(value=cells / (ms * 1e-3), unit="cell-updates/s", ms_per_step=ms, steps=k, dtype="f32",
                bc="x, y periodic; z Dirichlet walls (C = 0)")


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    from paper_2105_01865_gb300 import build
    from paper_2105_01865_gb300.solver import Solver
    from paper_2105_01865_gb300 import capi

    rank, world, local = _rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    capi.load()

    W = WORKLOAD
    f = workload_inputs(W["nx"], W["ny"], W["nz"])
    ncell = W["nx"] * W["ny"] * W["nz"]

    def make(prec):
        s = Solver(f["shape"], f["h"], f["bc"], f["cn"], f["pe"], f["dt"], f["C"], precision=prec, advect=True,
                   device=dev)
        s.set_velocity_fine(*f["vel"])
        return s

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(s, steps, warmup, per_step=None):
        """Sum of per-step CUDA-event durations on the solver's stream; L2
        flushed between steps, outside the events."""
        st = s.stream
        for _ in range(warmup):
            s.step(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        with torch.cuda.stream(st):
            for a, b in ev:
                flush.fill_(1)
                a.record(st)
                (per_step or s.step)(1)
                b.record(st)
        barrier()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    # main FP32 line; nvidia-smi samples the clocks from here through the
    # batched and multi-resolution legs (all timed regions of this run)
    s32 = make("f32")
    clk = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local,
                       args.clocks_dir)
    clk.__enter__()
    sec = timed(s32, args.steps, args.warmup)
    s32.sync()
    sec_t = torch.tensor([sec], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(sec_t, op=dist.ReduceOp.MAX)
    sec = float(sec_t)
    value = ncell * args.steps * world / sec

    # per-kernel durations (events around every launch), same L2 flush between steps
    ksum = [0.0] * 4
    kreps = max(3, min(args.steps, 10))
    for _ in range(kreps):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        ms = capi.ch_profile_step(s32.handle, 1)
        ksum = [a + b for a, b in zip(ksum, ms)]
    kms = [x / kreps for x in ksum]
    names = ["ch_explicit_rhs", "ch_solve_x", "ch_solve_y", "ch_solve_z_update"]
    # algorithmic bytes per cell of one launch (FP32): the explicit kernel
    # averages its three substeps (24, 28, 28 B), x/y solves 8 B, z solve +
    # update 12 B; algorithmic FP32 flops per cell of the explicit kernel
    # (3 WENO5 face reconstructions of ~75 flops, 7 psi', Laplacian, A_d
    # fourth differences, divergence and the RK/CN combination)
    kbytes = [80.0 / 3.0, 8.0, 8.0, 12.0]
    explicit_flops = 300.0
    peak_hbm, peak_src = measured_peak_hbm()
    sm_mhz = 2070.0  # the maximum SM clock; the sampled median is reported in "clocks"
    peak_fp32 = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12     # TFLOP/s: SMs x FP32 lanes x 2 flops x clock
    traffic = recorded_traffic()
    achieved = explicit_flops * ncell / (kms[0] * 1e-3) / 1e12
    roofline = dict(bound="alu", kernel=names[0], achieved=achieved, peak=peak_fp32, unit="TFLOP/s",
                    frac=achieved / peak_fp32, traffic=traffic.get(names[0]),
                    peak_source=f"derived: 152 SMs x 128 FP32 lanes x 2 flops x {sm_mhz:.0f} MHz",
                    kernels={n: dict(ms=m, algo_bytes_per_cell=b, gbs=b * ncell / (m * 1e-3) / 1e9,
                                     hbm_frac=b * ncell / (m * 1e-3) / 1e9 / peak_hbm,
                                     hbm_frac_nominal=b * ncell / (m * 1e-3) / 1e9 / NOMINAL_HBM_GBS,
                                     traffic=traffic.get(n))
                             for n, m, b in zip(names, kms, kbytes)},
                    hbm_peak=dict(value=peak_hbm, unit="GB/s", source=peak_src, nominal=NOMINAL_HBM_GBS))

    # end to end through the public API with host buffers: pinned H2D of C,
    # one step, D2H of C, every step
    hostC = torch.from_numpy(f["C"].astype("float32")).pin_memory()
    outC = torch.empty_like(hostC).pin_memory()
    s_e2e = make("f32")

    def e2e_step(_n):
        s_e2e.C.copy_(hostC, non_blocking=True)
        s_e2e.step(1)
        outC.copy_(s_e2e.C, non_blocking=True)

    for _ in range(args.warmup):
        with torch.cuda.stream(s_e2e.stream):
            e2e_step(1)
    sec_e2e = timed(s_e2e, args.steps, 0, per_step=e2e_step)
    t = torch.tensor([sec_e2e], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e = dict(value=ncell * args.steps * world / float(t), unit="cell-updates/s",
               h2d_bytes_per_step=ncell * 4, d2h_bytes_per_step=ncell * 4)

    batched = batched_leg(args, dev, flush, rank, world)
    batch_dts = batched.pop("_dts")
    multires = multires_leg(args, dev, flush) if not args.no_multires else None
    schemes = scheme_leg(args, dev, W) if not args.no_scheme else None
    dirichlet = dirichlet_leg(args, dev, flush, W) if not args.no_scheme else None
    clk.__exit__(None, None, None)
    clocks = clk.summary()

    # the plain FP64 GPU step on the same workload, for the precision speedup
    s64 = make("f64")
    k64 = max(3, args.steps // 4)
    sec64 = timed(s64, k64, min(args.warmup, 3))
    fp64 = dict(ms_per_step=1e3 * sec64 / k64, value=ncell * k64 / sec64, unit="cell-updates/s",
                fp32_speedup=(ncell * k64 / sec64) and (value / world) / (ncell * k64 / sec64))

    line = dict(metric=METRIC, value=value, unit="cell-updates/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * sec / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=W["name"], global_batch=world, seq_len=0,
                            parallelism=f"replicas{world}", cells=ncell, precision="f32 fields, f64 reductions",
                            l2="flushed between timed steps (256 MB write); working set 235 MB > L2"),
                roofline=roofline, e2e=e2e, fp64_plain=fp64, batched=batched, multires=multires,
                scheme_comparison=schemes, dirichlet_walls=dirichlet, clocks=clocks,
                gpu_launches=args.steps * s32.launches_per_step())
    if rank == 0 and not args.no_cpu_baseline:
        if world == 1:
            batched["cpu_baseline"] = run_oracle_batch([batch_dts[i] for i in range(len(batch_dts))])
        cells, times = run_oracle(1, 0)
        cpu_v = cells * len(times) / sum(times)
        line["cpu_baseline"] = dict(value=cpu_v, unit="cell-updates/s", cores=1, kind="oracle",
                                    sample=f"FP64 numpy oracle, one RK3 step of the same shear-drop recipe on a "
                                           f"{SAMPLE['nx']}x{SAMPLE['ny']}x{SAMPLE['nz']} mesh, single thread, "
                                           f"host CPU {cpu_model()}")
    if rank == 0:
        print(json.dumps(line), flush=True)
    for s in (s32, s_e2e, s64):
        s.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=None, help="directory for the raw nvidia-smi clock samples")
    ap.add_argument("--no-multires", action="store_true", help="skip the 1024x1024x512 transfer + step leg")
    ap.add_argument("--no-scheme", action="store_true",
                    help="skip the split vs standard scheme comparison and the Dirichlet-wall leg")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
