"""Throughput of the Cahn-Hilliard hot path on GB300.

Headline workload: the multiple-resolution case, the largest configuration
that fits one GPU.  A coarse 256 x 256 x 128 mesh, tanh-stretched in z
(walls at z = 0, 1; x, y periodic on [0, 2]), carries a seeded
divergence-free random-Fourier face velocity; it is transferred to the
uniform 1024 x 1024 x 512 fine mesh (h = 1/512, 5.37e8 cells) of the volume
fraction C, which holds ~1000 drops of radius U[0.01, 0.03]; Cn = 0.75 h,
Pe = 0.9 / Cn, FP32 fields with FP64 reductions, dt = min(0.9 dt_stab, CFL
0.5).  One step is one pass of the whole hot path: the coarse velocity handed
in, the velocity transfer (normal gradients, Hermite interpolation,
integration), one full RK3 step (three substeps of explicit right-hand side
and x, y, z line solves), and the FP64 mass and free energy.  Metric:
fine-grid cell-updates/s.  The working set (~15 GB) exceeds the 129 MB L2,
which is also flushed between timed steps.

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

HEADLINE = dict(name="multires_1024x1024x512_from_256x256x128", fine=(1024, 1024, 512), coarse=(256, 256, 128),
                ndrops=1000)
# CPU sample of the headline workload for the oracle legs: the same recipe on
# a 128 x 128 x 64 fine mesh over a 32 x 32 x 16 coarse one (50 drops)
SAMPLE = dict(fine=(128, 128, 64), coarse=(32, 32, 16), ndrops=50)
SHEAR = dict(name="shear_drop_256x256x128", nx=256, ny=256, nz=128)
METRIC = "fine-grid CH cell-updates/s"
L2_FLUSH_BYTES = 256 << 20
# kernel launches of one hot-path step besides ch_step's own: 7 transfer
# kernels (gradients; plane + line per direction) and 3 for the one-pass mass
# and free-energy reduction (block partials of both, then one finish each)
LAUNCHES_AROUND_STEP = 7 + 3


def _rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def multires_inputs(fine, coarse, ndrops):
    from paper_2105_01865_gb300 import inputs, stability
    f = inputs.multires_box(tuple(fine), tuple(coarse), ndrops)
    h = f["h"]
    f["dt"] = min(0.9 * stability.stable_dt(f["shape"], h, f["bc"], f["cn"], f["pe"]), 0.5 * h / 1.0)
    return f


def shear_inputs(nx, ny, nz):
    from paper_2105_01865_gb300 import inputs, stability
    f = inputs.shear_drop_box(nx, ny, nz)
    h = f["h"]
    f["dt"] = min(0.9 * stability.stable_dt(f["shape"], h, f["bc"], f["cn"], f["pe"]), 0.5 * h / 0.5)
    return f


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ---------------------------------------------------------------------------
# oracle (CPU) legs, run in fresh single-threaded interpreters
# ---------------------------------------------------------------------------

_ENV1 = dict(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")

_ORACLE_MR_SNIPPET = """
import json, os, sys, time
sys.path.insert(0, {root!r})
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor
from oracle import batch_timing as bt
if __name__ == "__main__":
    a = json.loads(sys.stdin.read())
    fine, coarse, ndrops, dt = a["fine"], a["coarse"], a["ndrops"], a["dt"]
    out = dict()
    if a["single"]:
        # single thread, this process: warm-up steps, then the timed steps
        times = [bt.multires_step(fine, coarse, ndrops, dt)[1] for _ in range(a["warmup"] + a["steps"])]
        cells = fine[0] * fine[1] * fine[2]
        out["single"] = dict(cells=cells, times=times[a["warmup"]:])
    if a["pool"]:
        # all cores: one single-threaded oracle process per available core, each
        # running one step of the same sample after a warm-up step of its own
        n = len(os.sched_getaffinity(0))
        with ProcessPoolExecutor(n, mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(bt.multires_step, [fine] * n, [coarse] * n, [ndrops] * n, [dt] * n))
            t0 = time.perf_counter()
            res = list(ex.map(bt.multires_step, [fine] * n, [coarse] * n, [ndrops] * n, [dt] * n))
            wall = time.perf_counter() - t0
        out["pool"] = dict(cells=sum(c for c, _ in res), wall=wall, workers=n)
    print(json.dumps(out))
"""


def run_oracle_multires(steps, warmup, single=True, pool=True, sample=SAMPLE):
    """The oracle's hot-path step (transfer, RK3 step, mass, free energy) on the
    CPU sample of the headline workload: `steps` timed single-threaded steps
    after `warmup`, and/or one step in every process of an all-cores pool."""
    f = multires_inputs(sample["fine"], sample["coarse"], sample["ndrops"])
    env = dict(os.environ, **_ENV1)
    arg = dict(fine=list(sample["fine"]), coarse=list(sample["coarse"]), ndrops=sample["ndrops"], dt=f["dt"],
               steps=steps, warmup=warmup, single=single, pool=pool)
    out = subprocess.run([sys.executable, "-c", _ORACLE_MR_SNIPPET.format(root=ROOT)], capture_output=True,
                         text=True, env=env, cwd=ROOT, input=json.dumps(arg))
    if out.returncode != 0:
        raise RuntimeError("oracle leg failed:\n" + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def sample_text(extra=""):
    fx, fy, fz = SAMPLE["fine"]
    cx, cy, cz = SAMPLE["coarse"]
    return (f"FP64 numpy oracle, one hot-path step (velocity transfer, RK3 step, mass, free energy) of the "
            f"multiple-resolution recipe on a {fx}x{fy}x{fz} fine mesh over a {cx}x{cy}x{cz} stretched coarse "
            f"mesh ({SAMPLE['ndrops']} drops){extra}; host CPU {cpu_model()}")


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
    env = dict(os.environ, **_ENV1)
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


def reference_arm(args):
    rank, world, _ = _rank()
    if rank != 0:
        return
    r = run_oracle_multires(args.steps, args.warmup, single=True, pool=False)["single"]
    sec = sum(r["times"])
    value = r["cells"] * len(r["times"]) / sec
    line = dict(metric=METRIC, value=value, unit="cell-updates/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * sec / len(r["times"]), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=HEADLINE["name"], global_batch=1, seq_len=0, parallelism="replicas"),
                cpu_baseline=dict(value=value, unit="cell-updates/s", cores=1, kind="oracle",
                                  sample=sample_text(", one step per timed step, single thread")),
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
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
PEAK_FP32_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12  # FFMA per lane per clock, 2 flops
# Algorithmic FP32 flops per cell of one explicit right-hand-side launch with
# advection (every +, -, x, / of the formulas counted once):
# 3 WENO5 faces x 68 (candidates 13, second differences 9, first-moment
# combinations 9, smoothness indicators 18, squares 3, weights 6, normalised
# combination 9, flux 1) = 204; divergence 6; psi'(C) 4; 7-point Laplacian of
# psi' 12; H = M lap psi' - div 2; the three fourth differences A_d C and
# their sum 32; RK/CN combination 5 (3 without H^{l-1} in substep 1).  Mean
# over the three substeps: 264.
EXPLICIT_FLOPS_PER_CELL = 264.0
# Algorithmic bytes per cell of one launch (FP32): explicit = C + u + v + w
# read, H + r written (24 B), + H^{l-1} read on substeps 2 and 3 (28 B), mean
# 80/3; x and y solves 8 B; z solve + update 12 B.
STEP_KERNELS = ["ch_explicit_rhs", "ch_solve_x", "ch_solve_y", "ch_solve_z_update"]
STEP_BYTES = [80.0 / 3.0, 8.0, 8.0, 12.0]
# the transfer per direction: interpolation across the lines at the coarse nodes along
# them, then the integration along the fine lines
INTERP_KERNELS = ["mr_gradients", "mr_transfer_x", "mr_transfer_y", "mr_transfer_z"]


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


# the sources the step kernels (explicit right-hand side, x, y, z solves) are
# built from: a change to any of them voids the recorded DRAM traffic
STEP_SOURCES = ["ch_step.cu", "ch_kernels.cuh", "ch_explicit2.cuh", "ch_cols2.cuh", "line_tables.h", "ch_internal.h"]


def kernel_source_sha():
    import hashlib
    csrc = os.path.join(ROOT, "paper_2105_01865_gb300", "csrc")
    hsh = hashlib.sha256()
    for name in STEP_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            hsh.update(name.encode() + fh.read())
    with open(os.path.join(ROOT, "include", "ch.h"), "rb") as fh:
        hsh.update(b"ch.h" + fh.read())
    return hsh.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per cell of one launch (ncu dram__bytes_read + write divided
    by the cells of the captured case) recorded in profiles/ncu_traffic.json,
    only if it was taken on the current kernels."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except (OSError, ValueError):
        return {}
    if rec.get("source_sha") != kernel_source_sha():
        return {}
    return rec.get("bytes_per_cell", {})


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
    k = max(3, min(args.steps, 20))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
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
    peak_hbm, _ = measured_peak_hbm()
    out = dict(value=cells * k / sec, unit="cell-updates/s", ms_per_step=1e3 * sec / k, steps=k,
               boxes=len(all_boxes), cells=cells, dtype="f32", placement="LPT on cell counts, no collective",
               schedule=dict(mode="persistent" if sched[0] == 0 else "phased", blocks_per_sm=sched[1],
                             zchunk=sched[2], lpt=sched[3]),
               launches_per_step=b.launches_per_step(), autotune_candidates=report.count("\n") - 1,
               hbm_frac=128.0 * cells / (sec / k) / 1e9 / peak_hbm)
    b.close()
    # per-box steps for the CPU baseline of this workload (popped before printing)
    out["_dts"] = {i: box["dt"] for i, box in zip(mine, boxes)}
    return out


def shear_leg(args, dev, flush):
    """The drop in imposed shear, 256 x 256 x 128 (x, y periodic on [0, 2],
    no-flux walls at z = 0, 1, u = (z - 1/2, 0, 0)), FP32: the step alone
    (u is prescribed, no transfer), L2 flushed between steps, with per-kernel
    durations and HBM fractions; the plain FP64 step on the same box."""
    import torch
    from paper_2105_01865_gb300 import capi
    from paper_2105_01865_gb300.solver import Solver
    W = SHEAR
    f = shear_inputs(W["nx"], W["ny"], W["nz"])
    ncell = W["nx"] * W["ny"] * W["nz"]
    out = {}
    for prec in ("f32", "f64"):
        s = Solver(f["shape"], f["h"], f["bc"], f["cn"], f["pe"], f["dt"], f["C"], precision=prec, advect=True,
                   device=dev)
        s.set_velocity_fine(*f["vel"])
        k = max(3, min(args.steps, 20)) if prec == "f32" else 5
        for _ in range(3):
            s.step(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(s.stream):
            for a, b in ev:
                flush.fill_(1)
                a.record(s.stream)
                s.step(1)
                b.record(s.stream)
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in ev) / k
        out[prec] = dict(ms_per_step=ms, value=ncell / (ms * 1e-3), steps=k)
        if prec == "f32":
            kms = kernel_means(s, flush, dev, 10)
            peak_hbm, _ = measured_peak_hbm()
            out["kernels"] = {n: dict(ms=m, gbs=b * ncell / (m * 1e-3) / 1e9,
                                      hbm_frac=b * ncell / (m * 1e-3) / 1e9 / peak_hbm)
                              for n, m, b in zip(STEP_KERNELS, kms, STEP_BYTES)}
            out["explicit_tflops"] = EXPLICIT_FLOPS_PER_CELL * ncell / (kms[0] * 1e-3) / 1e12
            out["step_hbm_frac"] = 164.0 * ncell / (ms * 1e-3) / 1e9 / peak_hbm
        s.close()
    return dict(workload=W["name"], cells=ncell, unit="cell-updates/s", dtype="f32", value=out["f32"]["value"],
                ms_per_step=out["f32"]["ms_per_step"], fp64_ms_per_step=out["f64"]["ms_per_step"],
                fp32_speedup_over_fp64=out["f64"]["ms_per_step"] / out["f32"]["ms_per_step"],
                step_hbm_frac=out["step_hbm_frac"], explicit_tflops=out["explicit_tflops"], kernels=out["kernels"])


def kernel_means(s, flush, dev, reps):
    """Mean ms per launch of each step-kernel class (ch_profile_step: events
    around every launch, same kernels launched directly), L2 flushed between
    steps."""
    import torch
    from paper_2105_01865_gb300 import capi
    ksum = [0.0] * 4
    for _ in range(reps):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        ms = capi.ch_profile_step(s.handle, 1)
        ksum = [a + b for a, b in zip(ksum, ms)]
    return [x / reps for x in ksum]


def scheme_leg(args, dev):
    """Time to solution of the paper's split scheme against the standard
    explicit 25-point scheme (Eq. eq-disbi) it replaces (Sec. 4.1 reports
    dt = 2e-3 against 5e-5 for its shear drop): both FP32, on the
    256 x 256 x 128 shear-drop box, from the same C0 to the same time T = 10
    steps of the split scheme, each at its largest stable dt (linear bound x
    0.9, CFL 0.5 h / max|u|).  Per-kernel times of the standard scheme come
    from ch_profile_step (chemical potential, advection, update)."""
    import math

    import torch
    from paper_2105_01865_gb300 import capi, inputs, stability
    from paper_2105_01865_gb300.solver import Solver
    W = SHEAR
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


def dirichlet_leg(args, dev, flush):
    """The shear-drop box with Dirichlet walls (C = 0 on z = 0, 1, the
    Rayleigh-Benard setting of Sec. 4.3) instead of no-flux ones: FP32 step
    time, L2 flushed between steps."""
    import torch
    from paper_2105_01865_gb300 import capi, inputs, stability
    from paper_2105_01865_gb300.solver import Solver
    W = SHEAR
    f = inputs.shear_drop_box(W["nx"], W["ny"], W["nz"])
    h, cn, pe = f["h"], f["cn"], f["pe"]
    bc = (capi.CH_PERIODIC, capi.CH_PERIODIC, capi.CH_DIRICHLET)
    dt = min(0.9 * stability.stable_dt(f["shape"], h, bc, cn, pe), 0.5 * h / 0.5)
    s = Solver(f["shape"], h, bc, cn, pe, dt, f["C"], precision="f32", advect=True, device=dev)
    s.set_velocity_fine(*f["vel"])
    st = s.stream
    m0 = s.mass()
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
    m1 = s.mass()
    s.close()
    # the walls hold C = 0, so mass leaves through the diffusive wall flux (no
    # correction is applied: the paper does not specify one)
    return dict(value=cells / (ms * 1e-3), unit="cell-updates/s", ms_per_step=ms, steps=k, dtype="f32",
                bc="x, y periodic; z Dirichlet walls (C = 0)", mass_change=(m1 - m0) / m0, mass_change_steps=k + 3)


class HotPath:
    """One solver of the headline workload and its hot-path step, every stage a
    call into libch.so: the coarse velocity handed in (ch_set_velocity_coarse),
    the transfer (ch_interp_to_fine), one RK3 step (ch_step), mass and free
    energy from one pass over C (ch_diagnostics)."""

    def __init__(self, f, prec, dev):
        import torch
        from paper_2105_01865_gb300.solver import Solver
        self.s = Solver(f["shape"], f["h"], f["bc"], f["cn"], f["pe"], f["dt"], f["C"], precision=prec,
                        coarse_faces=f["faces"], device=dev)
        self.velc = [self.s._dev(a) for a in f["vel_coarse"]]
        self.velc_host = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32 if prec == "f32" else np.float64))
                          .pin_memory() for a in f["vel_coarse"]]
        self.s._order()
        self.mass = self.energy = None

    def step(self, _n=1):
        from paper_2105_01865_gb300 import capi
        h = self.s.handle
        capi.ch_set_velocity_coarse(h, *self.velc)
        capi.ch_interp_to_fine(h)
        capi.ch_step(h, 1)
        self.mass, self.energy = capi.ch_diagnostics(h)

    def launches_per_step(self):
        return self.s.launches_per_step() + LAUNCHES_AROUND_STEP


def e2e_pipelined(hps, hostC, outC, steps, dev):
    """`steps` hot-path steps through the public API with host buffers, with
    the copies overlapped with compute on k = len(hps) solver instances of the
    same workload: step n runs on instance n % k, whose C and coarse velocity
    were copied from pinned host memory (one copy stream) while step n - 1
    ran; step n's result C is copied back to pinned host memory (a second copy
    stream) while step n + 1 runs.  An instance takes new inputs only once its
    last result is back on the host, so with k = 3 the two copy directions
    never wait for each other.  Compute stays one step at a time: each step
    waits for the end of the previous one.  Returns the seconds from the first
    host-to-device copy to the end of the last device-to-host copy."""
    import torch
    h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    k = len(hps)
    free = [None] * k           # the instance's last result is back on the host
    ready = [None] * steps      # step n's inputs are on the device
    done = [None] * steps       # step n has finished
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)

    def upload(n):
        hp = hps[n % k]
        with torch.cuda.stream(h2d):
            if free[n % k] is not None:
                h2d.wait_event(free[n % k])
            hp.s.C.copy_(hostC, non_blocking=True)
            for d, s in zip(hp.velc, hp.velc_host):
                d.copy_(s, non_blocking=True)
            ready[n] = torch.cuda.Event()
            ready[n].record(h2d)

    t0.record(h2d)
    upload(0)
    for n in range(steps):
        hp = hps[n % k]
        st = hp.s.stream
        if n + 1 < steps:
            upload(n + 1)
        st.wait_event(ready[n])
        if n > 0:
            st.wait_event(done[n - 1])
        hp.step(1)
        done[n] = torch.cuda.Event()
        done[n].record(st)
        d2h.wait_event(done[n])
        with torch.cuda.stream(d2h):
            outC.copy_(hp.s.C, non_blocking=True)
            free[n % k] = torch.cuda.Event()
            free[n % k].record(d2h)
    t1.record(d2h)
    torch.cuda.synchronize(dev)
    return t0.elapsed_time(t1) / 1e3


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    from paper_2105_01865_gb300 import build
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

    W = HEADLINE
    f = multires_inputs(W["fine"], W["coarse"], W["ndrops"])
    nx, ny, nz = W["fine"]
    ncell = nx * ny * nz
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(hp, steps, warmup, per_step=None):
        """Sum of per-step CUDA-event durations on the solver's stream; L2
        flushed between steps, outside the events."""
        st = hp.s.stream
        for _ in range(warmup):
            (per_step or hp.step)(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        with torch.cuda.stream(st):
            for a, b in ev:
                flush.fill_(1)
                a.record(st)
                (per_step or hp.step)(1)
                b.record(st)
        barrier()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    def max_ranks(sec):
        t = torch.tensor([sec], device=dev, dtype=torch.float64)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t)

    # headline: the FP32 hot path on the 1024 x 1024 x 512 workload; nvidia-smi
    # samples the clocks from here through the last timed leg
    hp = HotPath(f, "f32", dev)
    clk = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local,
                       args.clocks_dir)
    clk.__enter__()
    sec = max_ranks(timed(hp, args.steps, args.warmup))
    hp.s.sync()
    value = ncell * args.steps * world / sec
    ms_step = 1e3 * sec / args.steps

    # per-launch durations: the step's kernel classes (ch_profile_step), the
    # transfer's four kernels (ch_profile_interp), the diagnostics
    kms = kernel_means(hp.s, flush, dev, 5)
    ims = [0.0] * 4
    for _ in range(3):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        ims = [a + b for a, b in zip(ims, capi.ch_profile_interp(hp.s.handle))]
    ims = [x / 3 for x in ims]
    red = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        a.record(hp.s.stream)
        capi.ch_diagnostics(hp.s.handle)
        b.record(hp.s.stream)
        torch.cuda.synchronize(dev)
        red.append(a.elapsed_time(b))
    red = [sum(red) / len(red)]
    # the down-sampling back-coupling (coarse C, rho, mu, F_st; Sec. 3.4) on the
    # same solver: not part of the step above, timed on its own
    hp.s.restrict_to_coarse(0.05, 1.0)
    rms = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        a.record(hp.s.stream)
        hp.s.restrict_to_coarse(0.05, 1.0)
        b.record(hp.s.stream)
        torch.cuda.synchronize(dev)
        rms.append(a.elapsed_time(b))
    restrict = dict(ms=sum(rms) / len(rms), fine_cells=ncell, coarse_cells=int(np.prod(W["coarse"])),
                    fine_read_gbs=ncell * 4 / (sum(rms) / len(rms) * 1e-3) / 1e9,
                    outputs="coarse C, rho, mu and the three F_st components")
    per_step_sum = 3 * sum(kms) + sum(ims) + sum(red)
    peak_hbm, peak_src = measured_peak_hbm()
    traffic = recorded_traffic()
    achieved = EXPLICIT_FLOPS_PER_CELL * ncell / (kms[0] * 1e-3) / 1e12
    fine_faces = 3 * ncell * 4  # bytes of fine face velocity written per transfer (FP32)
    kernels = {n: dict(ms=m, launches_per_step=3, algo_bytes_per_cell=b, gbs=b * ncell / (m * 1e-3) / 1e9,
                       hbm_frac=b * ncell / (m * 1e-3) / 1e9 / peak_hbm,
                       hbm_frac_nominal=b * ncell / (m * 1e-3) / 1e9 / NOMINAL_HBM_GBS,
                       traffic=(traffic[n] * ncell if n in traffic else None))
               for n, m, b in zip(STEP_KERNELS, kms, STEP_BYTES)}
    for n, m in zip(INTERP_KERNELS, ims):
        kernels[n] = dict(ms=m, launches_per_step=1)
    for n, b in zip(INTERP_KERNELS[1:], (4.0, 4.0, 4.0)):
        kernels[n].update(algo_bytes_per_cell=b, gbs=b * ncell / (kernels[n]["ms"] * 1e-3) / 1e9,
                          hbm_frac=b * ncell / (kernels[n]["ms"] * 1e-3) / 1e9 / peak_hbm)
    kernels["ch_diagnostics"] = dict(ms=red[0], launches_per_step=1, algo_bytes_per_cell=4.0,
                                     hbm_frac=4.0 * ncell / (red[0] * 1e-3) / 1e9 / peak_hbm)
    share = {n: k["ms"] * k["launches_per_step"] / per_step_sum for n, k in kernels.items()}
    roofline = dict(bound="alu", kernel=STEP_KERNELS[0], achieved=achieved, peak=PEAK_FP32_TFLOPS, unit="TFLOP/s",
                    frac=achieved / PEAK_FP32_TFLOPS,
                    traffic=(traffic[STEP_KERNELS[0]] * ncell if STEP_KERNELS[0] in traffic else None),
                    flops_per_cell=EXPLICIT_FLOPS_PER_CELL,
                    peak_source=f"derived: {SM_COUNT} SMs x {FP32_LANES} FP32 lanes x 2 flops x {SM_MAX_MHZ:.0f} MHz",
                    kernels=kernels, share_of_kernel_time=share,
                    kernel_sum_ms=per_step_sum, step_ms=ms_step, kernel_sum_over_step=per_step_sum / ms_step,
                    step_hbm_frac=(164.0 + 12.0 + 4.0) * ncell / (ms_step * 1e-3) / 1e9 / peak_hbm,
                    transfer_ms=sum(ims), transfer_fine_faces_gbs=fine_faces / (sum(ims) * 1e-3) / 1e9,
                    hbm_peak=dict(value=peak_hbm, unit="GB/s", source=peak_src, nominal=NOMINAL_HBM_GBS))

    # end to end through the public API with host buffers, every step: pinned
    # H2D of C and of the coarse velocity, the hot-path step, D2H of C
    hostC = torch.from_numpy(np.ascontiguousarray(f["C"], dtype=np.float32)).pin_memory()
    outC = torch.empty_like(hostC).pin_memory()
    velc_dev = hp.velc

    def e2e_step(_n):
        st = hp.s.stream
        with torch.cuda.stream(st):
            hp.s.C.copy_(hostC, non_blocking=True)
            for d, hsrc in zip(velc_dev, hp.velc_host):
                d.copy_(hsrc, non_blocking=True)
        hp.step(1)
        with torch.cuda.stream(st):
            outC.copy_(hp.s.C, non_blocking=True)

    k_e2e = max(3, min(args.steps, 10))
    h2d_bytes = ncell * 4 + sum(t.numel() * 4 for t in hp.velc_host)
    sec_serial = max_ranks(timed(hp, k_e2e, 2, per_step=e2e_step))
    # the host link on its own: one C each way (the overlapped form below is
    # bound by these when they exceed a step)
    link = {}
    for name, fn in (("h2d_gbs", lambda: hp.s.C.copy_(hostC, non_blocking=True)),
                     ("d2h_gbs", lambda: outC.copy_(hp.s.C, non_blocking=True))):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(hp.s.stream):
            a.record(hp.s.stream)
            fn()
            b.record(hp.s.stream)
        torch.cuda.synchronize(dev)
        link[name] = ncell * 4 / (a.elapsed_time(b) * 1e-3) / 1e9
    extra_hp = [HotPath(f, "f32", dev) for _ in range(2)]  # instances 2 and 3 of the overlapped form
    sec_e2e = max_ranks(e2e_pipelined([hp] + extra_hp, hostC, outC, k_e2e, dev))
    for x in extra_hp:
        x.s.close()
    del extra_hp
    e2e = dict(value=ncell * k_e2e * world / sec_e2e, unit="cell-updates/s", steps=k_e2e,
               h2d_bytes_per_step=h2d_bytes, d2h_bytes_per_step=ncell * 4,
               pipelined=("every step copies its inputs (C and the coarse velocity) from pinned host memory and "
                          "its result C back; three solver instances take turns, so step n+1's inputs are copied "
                          "in and step n-1's result is copied out while step n runs (compute one step at a time)"),
               host_link=link,
               serial_value=ncell * k_e2e * world / sec_serial,
               serial="the same copies, not overlapped: H2D, step, D2H in order on one stream")
    launches = hp.launches_per_step()
    mass_last = hp.mass
    hp.s.close()
    del hp

    def leg(fn, *a):
        """A secondary leg; its failure is recorded in the line instead of
        ending the run (the headline above is already measured)."""
        try:
            return fn(*a)
        except Exception as e:  # noqa: BLE001
            torch.cuda.synchronize(dev)
            return dict(error=f"{type(e).__name__}: {e}"[:500])

    def fp64_leg():
        hp64 = HotPath(f, "f64", dev)
        k64 = 3
        sec64 = max_ranks(timed(hp64, k64, 1))
        hp64.s.close()
        return dict(ms_per_step=1e3 * sec64 / k64, value=ncell * k64 * world / sec64, unit="cell-updates/s",
                    steps=k64, fp32_speedup=(1e3 * sec64 / k64) / ms_step)

    extra = not (args.no_extra or args.headline_only)
    batched, batch_dts = None, None
    if not args.headline_only:
        batched = leg(batched_leg, args, dev, flush, rank, world)
        batch_dts = batched.pop("_dts", None)
    shear = leg(shear_leg, args, dev, flush) if extra else None
    schemes = leg(scheme_leg, args, dev) if extra else None
    dirichlet = leg(dirichlet_leg, args, dev, flush) if extra else None
    # the plain FP64 GPU hot path on the headline workload: the precision speedup
    fp64 = leg(fp64_leg) if not args.headline_only else None
    clk.__exit__(None, None, None)
    clocks = clk.summary()

    line = dict(metric=METRIC, value=value, unit="cell-updates/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms_step, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=W["name"], global_batch=world, seq_len=0, parallelism=f"replicas{world}",
                            cells=ncell, coarse_cells=int(np.prod(W["coarse"])), drops=f["ndrops"],
                            precision="f32 fields, f64 reductions",
                            step="coarse velocity in, transfer to the fine mesh, one RK3 step, mass and free energy",
                            l2="flushed between timed steps (256 MB write); working set ~15 GB > L2"),
                roofline=roofline, e2e=e2e, fp64_plain=fp64, mass_after=mass_last, restrict_to_coarse=restrict, batched=batched,
                shear_drop=shear, scheme_comparison=schemes, dirichlet_walls=dirichlet, clocks=clocks,
                gpu_launches=args.steps * launches)
    if rank == 0 and not (args.no_cpu_baseline or args.headline_only):
        if world == 1 and batch_dts:
            batched["cpu_baseline"] = run_oracle_batch([batch_dts[i] for i in range(len(batch_dts))])
        r = run_oracle_multires(1, 1, single=True, pool=(world == 1))
        single = r["single"]["cells"] * len(r["single"]["times"]) / sum(r["single"]["times"])
        if "pool" in r:
            p = r["pool"]
            line["cpu_baseline"] = dict(value=p["cells"] / p["wall"], unit="cell-updates/s", cores=p["workers"],
                                        kind="oracle", single_core_value=single,
                                        sample=sample_text(f", one step in each of {p['workers']} single-threaded "
                                                           "processes (all cores); single_core_value: one step in "
                                                           "one process"))
        else:
            line["cpu_baseline"] = dict(value=single, unit="cell-updates/s", cores=1, kind="oracle",
                                        sample=sample_text(", single thread"))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=None, help="directory for the raw nvidia-smi clock samples")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the shear-drop, scheme-comparison and Dirichlet-wall legs")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the headline workload only (no other legs, no FP64 or CPU baseline), for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
