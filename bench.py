#!/usr/bin/env python
"""Benchmark: narrow-band first-order upwind level-set throughput on one B300.

Workload (the standard sphere-union case): 512^3 FP32 grid, h = 1/512,
phi^0 = signed distance to the union of 20 seeded spheres (centres
U[0.15,0.85]^3, radii U[0.05,0.15]), F = 1 + 0.5 sin(2 pi x) sin(2 pi y)
sin(2 pi z), band half-width 6h on 8^3 tiles, band rebuilt every 5 steps,
500 steps at CFL 0.5.  One bench step = one whole run of that workload
through the C ABI: ls_restore(phi^0, a device snapshot made after the
library's own Step 0 kernels generated it) -> ls_band_rebuild(6) ->
ls_step(500, CFL 0.5, rebuild every 5).  The metric is grid-point updates
per second over the band (GLUPS: sum over steps of the points of the active
tiles, divided by the device time).

Timing: W untimed warm-up steps, then K steps between CUDA events on the
stream the library launches on, with a barrier and a synchronize on both
sides; max over ranks.  The inputs (phi, F: 1.5 GB) and the active working
set of a step (~0.2 GB) are larger than the 126 MB L2, so no L2 flush is
needed between steps.

Extra keys: roofline of the dominant kernel (the upwind step) from CUDA
events around every step launch, e2e (the same run with host buffers and the
host<->device copies inside the timed region), cpu_baseline (the FP64 CPU
oracle on a bounded sample of the same workload), clocks sampled with
nvidia-smi during the timed region.

--impl reference times the FP64 CPU oracle on the same workload (each step a
bounded sample: one rebuild period of 5 level-set steps), on rank 0 only.
With --gpus N > 1 (torchrun) every rank runs an independent replica of the
workload ("replicas only": the single-grid path has no sharded variant here);
value = all ranks' updates / max time, scaling "weak".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "narrow-band upwind GLUPS"
UNIT = "GLUPS"
BYTES_PER_UPDATE = 12  # FP32: read phi (4) + read F (4) + write phi (4)
# FP64 operations of one update of Eq. 3-5 as defined (one upwind branch):
# 6 differences and 6 divisions by h, 6 squares + 3 per-axis sums + 2 sums
# + 1 square root (Eq. 4 or 5), F * G, dt * (.), phi - (.)
FLOPS_PER_UPDATE_F64 = 27
WORKLOAD = "sphere-union 512^3 FP32, band 6h on 8^3 tiles, rebuild/5, 500 steps CFL 0.5"
WORKLOAD_LOCAL = ("sphere-union 512^3 FP32, local scheme (cut-off advance beta 3h, gamma 6h; %d "
                  "reinitialisation iterations dtau h/2; clamp), 8^3 tiles, rebuild/5, 500 steps CFL 0.5")
METRIC_LOCAL = "local-scheme GLUPS (advance point updates per second, reinitialisation included)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["mine", "reference"], default="mine")
    p.add_argument("--grid", type=int, default=512, help="grid edge (512 = the standard workload)")
    p.add_argument("--e2e-steps", type=int, default=-1,
                   help="problems in the end-to-end measurement (-1: as many as --steps; 0: skip)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", choices=["sphere-union", "batch", "learned", "perturbed", "sphere64", "local"],
                   default="sphere-union",
                   help="sphere-union: the standard 512^3 run (the default line); "
                        "batch: 256 independent grids in one batched context; "
                        "learned: corrector training + learned-coarse vs plain at equal error; "
                        "local: the 512^3 run with the paper's local scheme (cut-off advance, "
                        "reinitialisation on N, clamp)")
    p.add_argument("--output-every", type=int, default=0,
                   help="sphere-union / local: write phi every N steps during the timed runs with the "
                        "library's overlapped output (host writer thread) into a temporary directory")
    p.add_argument("--output-format", choices=["vts", "vti"], default="vts")
    p.add_argument("--steps-per-pass", type=int, choices=[1, 2], default=None,
                   help="sphere-union: force one or two upwind steps per stencil pass instead of "
                        "the autotuner's choice")
    p.add_argument("--perturbed-n", type=int, default=1024,
                   help="perturbed workload: grid edge (1024 = the standard workload)")
    p.add_argument("--reinit-iters", type=int, default=-1,
                   help="local workload: reinitialisation iterations per step (-1: ceil(halfwidth/dtau))")
    p.add_argument("--batch-count", type=int, default=256,
                   help="batch workload: the first N of its 256 instances (smaller cases for profiling)")
    p.add_argument("--pairs", type=int, default=2000)
    p.add_argument("--train-iters", type=int, default=2000)
    p.add_argument("--parallelism", choices=["replicas", "slab"], default="replicas",
                   help="sphere-union with --gpus N: independent replicas (default) or one grid split "
                        "into z-slabs, one per GPU, balanced by Eq. 14 (NCCL exchanges)")
    p.add_argument("--slabs", type=int, default=1,
                   help="--parallelism slab on one GPU: number of slabs in this process (device "
                        "copies instead of NCCL)")
    p.add_argument("--slab-graphs", type=int, choices=[0, 1], default=0,
                   help="--parallelism slab with every slab in this process: replay the rebuild "
                        "periods from CUDA graphs (1) or issue them eagerly (0)")
    p.add_argument("--rebalance-gain", type=float, default=0.1,
                   help="--parallelism slab: move rows to the Eq. 14 partition after a rebuild only "
                        "when that lowers the largest slab's active tiles by more than this fraction")
    p.add_argument("--step-config", default=None, metavar="STAGES,GRID_PCT,PPT",
                   help="fix the stencil launch configuration instead of autotuning it "
                        "(so that a profiler run times the same kernel as the plain run)")
    a = p.parse_args()
    if a.e2e_steps < 0:
        a.e2e_steps = a.steps  # the end-to-end run covers as many problems as the timed one
    return a


def tune(obj, args):
    """Autotune the stencil launch configuration, or apply --step-config."""
    if args.step_config:
        st, pct, ppt = (int(v) for v in args.step_config.split(","))
        obj.set_step_config(st, pct, ppt)
        return st, pct, ppt
    return obj.autotune(reps=5)


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local, pg


def aggregate(pg, t_s, updates, device="cpu"):
    """Whole-job time and work over the ranks: the slowest rank's time and the
    sum of all ranks' updates (replicas: every rank did its own work)."""
    if pg is None:
        return t_s, updates
    import torch
    t = torch.tensor([t_s], dtype=torch.float64, device=device)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    pg.all_reduce(u, op=pg.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def measured_bf16():
    """Dense bf16 tensor-core peak (TFLOP/s): the measured burst figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    return 1800.0, "fallback"


PROFILE_EVERY = 5  # plain scheme: one run of stencil launches in 5 timed with CUDA events


def kernel_source_hash():
    """Hash of the one-step FP32 stencils' source (the kernel files of the 4/8
    and 16 points-per-thread decompositions, the shared per-point
    arithmetic they include, and the band kernels, which mark the frozen
    x-faces the one-warp kernel reads from their copies)."""
    h = hashlib.sha256()
    for name in ("ls_step.cu", "ls_step_z4.cu", "ls_stencil.cuh", "ls_band.cu"):
        with open(os.path.join(ROOT, "paper_1612_04040_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


STENCIL_KERNELS = {4: "k_step_f32 (128 threads per 8^3 tile, 4 points per thread)",
                   8: "k_step_f32_z2 (64 threads per 8^3 tile, 8 points per thread)",
                   16: "k_step_f32_z4 (one warp per 8^3 tile, 16 points per thread)"}


def recorded_traffic(ppt, workload="sphere-union", field="dram_bytes_per_update"):
    """DRAM bytes per grid-point update (or another recorded `field`) of the
    step kernel with `ppt` points per thread on `workload` from the last ncu
    capture of that decomposition, if it was taken on the current kernel
    source (else None).  The records in profiles/stencil_traffic.txt are
    separated by blank lines; a record without a workload line is the
    sphere union's."""
    path = os.path.join(ROOT, "profiles", "stencil_traffic.txt")
    if not os.path.exists(path):
        return None
    recs, d = [], {}
    with open(path) as f:
        for line in f:
            if not line.strip():
                if d:
                    recs.append(d)
                d = {}
            elif ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                d[k.strip()] = v.strip()
    if d:
        recs.append(d)
    for d in recs:
        if (d.get("stencil_source_sha256_16") == kernel_source_hash()
                and int(d.get("points_per_thread", "0")) == int(ppt)
                and d.get("workload", "sphere-union") == workload and field in d):
            return float(d[field])
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) != 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, v in zip(names[1:], r[3][1:]):
                if v.lower() == "active":
                    reasons.add(name)
        loaded = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def cpu_baseline(phi0_f32, F_f32, w, steps=40):
    """The FP64 CPU oracle, as it stands, on the first `steps` level-set steps
    of the same workload (inputs: the same FP32 arrays, widened)."""
    import numpy as np
    import oracle
    phi = phi0_f32.astype(np.float64)
    F = F_f32.astype(np.float64)
    o = oracle.Oracle(phi.shape, w.h)
    o.set_phi(phi)
    o.set_speed(F)
    t0 = time.perf_counter()
    o.band_rebuild(w.halfwidth)
    updates = 0
    for _ in range(steps):
        o.step(1, w.cfl, oracle.DT_CFL, w.rebuild_every)
        updates += int(o.active.sum()) * 512
    t = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    out = {"value": updates / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "first %d level-set steps (%d band rebuilds) of the %d^3 workload, FP64 C oracle "
                     "with OpenMP on %d host threads, %.1f s" % (steps, (steps + w.rebuild_every - 1)
                                                                   // w.rebuild_every, w.n, cores, t)}
    return out, o


def oracle_one_thread(o, w, steps=2):
    """The same oracle continued for `steps` further level-set steps on one
    host thread (OpenMP's thread count of the calling thread set through
    libgomp, then restored), beside the all-threads figure; None where
    libgomp cannot be loaded."""
    import ctypes
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
    except OSError:
        return None
    import oracle
    nmax = gomp.omp_get_max_threads()
    gomp.omp_set_num_threads(1)
    try:
        t0 = time.perf_counter()
        updates = 0
        for _ in range(steps):
            o.step(1, w.cfl, oracle.DT_CFL, w.rebuild_every)
            updates += int(o.active.sum()) * 512
        t = time.perf_counter() - t0
    finally:
        gomp.omp_set_num_threads(nmax)
    return {"value": updates / t / 1e9, "unit": UNIT, "cores": 1,
            "sample": "%d further level-set steps of the same run on one host thread, %.1f s" % (steps, t)}


def parity_vs_oracle(g, o, w, steps):
    """The GPU's state after the same first `steps` steps, against the
    oracle's: max |phi_gpu - phi_oracle| over the points of the oracle's
    active tiles (bar 1e-5 h steps) and whether the active-tile sets agree."""
    import numpy as np
    from paper_1612_04040_b300 import native as ls
    g.restore()
    g.band_rebuild(w.halfwidth, want_count=False)
    g.step(steps, w.cfl, ls.LS_DT_CFL, w.rebuild_every)
    got = g.get_phi().astype(np.float64)
    act = o.active.astype(bool)
    m = np.repeat(np.repeat(np.repeat(act, 8, 0), 8, 1), 8, 2)
    err = float(np.max(np.abs(got[m] - o.phi[m]))) if m.any() else 0.0
    bar = 1e-5 * w.h * steps
    same = bool(np.array_equal(np.sort(g.active_tiles()), np.flatnonzero(act.ravel())))
    return {"steps": steps, "max_abs_err_on_band": err, "bar": bar, "within_bar": err <= bar,
            "active_tiles_equal": same, "active_tiles": int(act.sum())}


def cpu_baseline_local(phi0_f32, F_f32, w, beta_h, iters, dtau_h, steps=2):
    """The FP64 CPU oracle's local scheme, as it stands (pointwise over the
    whole grid), on the first `steps` steps of the local workload; counted
    like the library: points of the oracle's own active tiles per step."""
    import numpy as np
    import oracle
    o = oracle.Oracle(phi0_f32.shape, w.h)
    o.set_phi(phi0_f32.astype(np.float64))
    o.set_speed(F_f32.astype(np.float64))
    o.set_scheme(oracle.SCHEME_LOCAL, beta_h, iters, dtau_h)
    t0 = time.perf_counter()
    o.band_rebuild(w.halfwidth)
    updates = 0
    for _ in range(steps):
        o.step(1, w.cfl, oracle.DT_CFL, w.rebuild_every)
        updates += int(o.active.sum()) * 512
    t = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    return {"value": updates / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d local-scheme steps (advance + %d reinitialisation iterations + clamp, "
                      "pointwise over the whole grid) of the %d^3 workload, FP64 C oracle with OpenMP "
                      "on %d host threads, %.1f s" % (steps, iters, w.n, cores, t)}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the same workload and metric.
    Each step = one rebuild period (5 level-set steps) of the 512^3 run."""
    import numpy as np
    import oracle
    from paper_1612_04040_b300 import inputs
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = inputs.SphereUnion(n=args.grid)
    phi = w.phi(out_dtype=inputs.torch.float32).numpy().astype(np.float64)
    F = w.speed(out_dtype=inputs.torch.float32).numpy().astype(np.float64)
    o = oracle.Oracle(phi.shape, w.h)
    o.set_phi(phi)
    o.set_speed(F)
    o.band_rebuild(w.halfwidth)

    def one_step():
        u = 0
        for _ in range(w.rebuild_every):
            o.step(1, w.cfl, oracle.DT_CFL, w.rebuild_every)
            u += int(o.active.sum()) * 512
        return u

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    updates = 0
    for _ in range(args.steps):
        updates += one_step()
    t = time.perf_counter() - t0
    value = updates / t / 1e9
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "grid": args.grid, "reference_step": "5 level-set steps (one rebuild period)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d x 5 level-set steps of the %d^3 workload after %d warm-up periods"
                                   % (args.steps, args.grid, args.warmup)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_batch(insts, budget_s=12.0, steps=10):
    """The FP64 CPU oracle, as it stands, on the batch's instances in order
    (each: band 4h, `steps` steps at CFL 0.5, rebuild every 5) until about
    `budget_s` seconds of CPU work have been spent."""
    import numpy as np
    import oracle
    t_all = 0.0
    updates = 0
    done = 0
    for it in insts:
        phi = it.phi().numpy().astype(np.float64)
        o = oracle.Oracle(phi.shape, it.h)
        o.set_phi(phi)
        o.set_speed_const(it.speed)
        t0 = time.perf_counter()
        o.band_rebuild(4.0)
        for _ in range(steps):
            o.step(1, 0.5, oracle.DT_CFL, 5)
            updates += int(o.active.sum()) * 512
        t_all += time.perf_counter() - t0
        done += 1
        if t_all >= budget_s:
            break
    cores = len(os.sched_getaffinity(0))
    return {"value": updates / t_all / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d of the batch's instances, %d level-set steps each (band 4h, CFL 0.5, "
                      "rebuild every 5), FP64 C oracle with OpenMP on %d host threads, %.1f s"
                      % (done, steps, cores, t_all)}


def run_batch(args):
    """256 independent grids (edges 32..192, sphere or torus, constant F in
    [-1, 1]), band 4h, rebuild every 5, 200 steps at CFL 0.5, FP32, one
    batched context: one stencil launch per step for all instances, launch
    configuration from the autotuner.  One bench step = restore phi^0
    (device snapshot) -> ls_band_rebuild(4) -> ls_step(200).  The stencil's
    roofline comes from CUDA events around one run of back-to-back stencil
    launches in PROFILE_EVERY inside the timed region (eager launches: the
    200-step call replayed as a CUDA graph measured no faster, 38.6 against
    38.5 ms, and a graph cannot carry the event records)."""
    import torch
    from paper_1612_04040_b300 import inputs
    from paper_1612_04040_b300 import native as ls
    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    insts = inputs.batch_instances()[:max(1, min(args.batch_count, 256))]
    b = ls.Batch([i.edge for i in insts], [i.h for i in insts], stream=stream.cuda_stream)
    for k, it in enumerate(insts):
        b.set_phi_i(k, it.phi(device=dev).to(torch.float32).contiguous())
        b.set_speed_const_i(k, it.speed)
    total_pts = sum(i.edge ** 3 for i in insts)
    b.snapshot()
    b.band_rebuild(4.0)
    b.step(5, 0.5, ls.LS_DT_CFL, 5)
    stages, pct, ppt = tune(b, args)

    def run_once():
        b.restore()
        b.band_rebuild(4.0, want_count=False)
        b.step(200, 0.5, ls.LS_DT_CFL, 5)

    for _ in range(max(args.warmup, 0)):
        run_once()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    b.reset_profile()
    b.profile_enable(PROFILE_EVERY)
    u0 = b.updates()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run_once()
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    b.profile_enable(False)
    prof = b.profile()
    updates = b.updates() - u0
    t_s, total_updates = aggregate(pg, ms / 1e3, float(updates), dev)
    value = total_updates / t_s / 1e9
    peak, peak_kind = measured_peaks()
    st_s = prof["stencil_ms"] / 1e3
    n_launch = max(prof["stencil_timed"], 1)
    achieved = prof["stencil_updates"] * 8 / 1e9 / st_s if st_s > 0 else None
    tpu_b = recorded_traffic(ppt, "batch")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_batch(insts)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": "batch of %d grids (edges 32..192, sphere/torus, constant F in "
                                   "[-1,1]), band 4h, rebuild/5, 200 steps CFL 0.5" % len(insts),
                       "total_points": total_pts, "graphs": False,
                       "autotuned": {"stages": stages, "grid_pct": pct, "points_per_thread": ppt},
                       "l2": "inputs larger than L2 (phi 2 x 2.3 GB)"},
            "updates_per_step": updates / max(args.steps, 1),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None,
                         "traffic": (tpu_b * prof["stencil_updates"] / n_launch)
                                    if tpu_b is not None else None,
                         "peak_kind": peak_kind, "bytes_per_update": 8,
                         "kernel": STENCIL_KERNELS.get(ppt, "k_step_f32") + ", batched",
                         "avg_launch_us": 1e6 * st_s / n_launch,
                         "launches": prof["stencil_launches"], "launches_timed": prof["stencil_timed"],
                         "timed_runs": "one run of back-to-back stencil launches in %d" % PROFILE_EVERY,
                         "share_of_step_time": (st_s / n_launch * prof["stencil_launches"] / t_s)
                                               if t_s > 0 else None},
            "e2e": None, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": prof["kernel_launches"],
        }), flush=True)
    b.close()
    if pg:
        pg.destroy_process_group()


def restrict_to(a, factor):
    """Mean of the 2^3 points around each coarse cell centre (evaluation only)."""
    import torch
    if factor == 1:
        return a
    lo = factor // 2 - 1
    nz, ny, nx = a.shape
    v = a.view(nz // factor, factor, ny // factor, factor, nx // factor, factor)
    return v[:, lo:lo + 2, :, lo:lo + 2, :, lo:lo + 2].mean(dim=(1, 3, 5))


def run_learned(args):
    """Learned corrector on the 128^3 coarse grid, trained on pairs from
    512^3 plain runs (random sphere unions, 8-mode Fourier F), measured against
    the 512^3 plain run; plain runs at 128^3, 256^3 and 512^3 give the
    error/wall-time curve the learned run is placed on."""
    import numpy as np
    import torch
    from paper_1612_04040_b300 import corrector
    from paper_1612_04040_b300 import native as ls
    torch.cuda.set_device(0)
    n_c = 128
    h_c = 1.0 / n_c
    cs = (n_c, n_c, n_c)
    t0 = time.perf_counter()
    gen = corrector.PairGenerator(cs, h_c)
    ctx = ls.LevelSet(n_c, n_c, n_c, h_c, ls.LS_FP32)
    ctx.learned_init(seed=1)
    rng = np.random.default_rng(1004)
    per_run = 50
    runs = max(1, args.pairs // per_run)
    for _ in range(runs):
        c, r, m = corrector.random_problem(rng, gen.box())
        for a, b, F in gen.run(c, r, m, per_run):
            ctx.learned_add_pair(a, b, F)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    t0 = time.perf_counter()
    final = ctx.learned_train(args.train_iters, 1e-3, gen.dt_c, 6.0, seed=7)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    nsteps = 64
    results = []
    for k in range(2):
        c, r, m = corrector.random_problem(np.random.default_rng(5000 + k), gen.box())
        phi_f, F_f = gen.fields(c, r, m)
        # reference: the 512^3 plain run (band as wide as the pair runs)
        runs_out = {}
        for n in (512, 256, 128):
            f = n // n_c
            h = 1.0 / n
            g = ls.LevelSet(n, n, n, h, ls.LS_FP32)
            phi = restrict_to(phi_f, 4 // f) if n < 512 else phi_f
            F = restrict_to(F_f, 4 // f) if n < 512 else F_f
            g.set_phi(phi.contiguous())
            g.set_speed(F.contiguous())
            hw = 6.0 * f
            g.band_rebuild(hw)
            g.step(4, 0.5 * h, ls.LS_DT_FIXED, 4)  # warm-up (first-call costs)
            g.set_phi(phi.contiguous())
            g.band_rebuild(hw)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.step(nsteps * f, 0.5 * h, ls.LS_DT_FIXED, 4)
            e1.record()
            torch.cuda.synchronize()
            out = torch.empty_like(phi)
            g.get_phi(out)
            runs_out[n] = (restrict_to(out, f), e0.elapsed_time(e1))
            g.close()
        ref = runs_out[512][0]
        phi0_c = restrict_to(phi_f, 4).contiguous()
        F_c = restrict_to(F_f, 4).contiguous()
        ctx.set_phi(phi0_c)
        ctx.set_speed(F_c)
        ctx.set_step_mode(ls.LS_LEARNED)
        ctx.band_rebuild(6.0)
        ctx.step(4, gen.dt_c, ls.LS_DT_FIXED, 4)  # warm-up
        ctx.set_phi(phi0_c)
        ctx.band_rebuild(6.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.step(nsteps, gen.dt_c, ls.LS_DT_FIXED, 4)
        e1.record()
        torch.cuda.synchronize()
        out = torch.empty_like(phi0_c)
        ctx.get_phi(out)
        ctx.set_step_mode(ls.LS_PLAIN)
        res = {"learned_128": {"err_h": corrector.front_error(out, ref, h_c), "ms": e0.elapsed_time(e1)}}
        for n in (128, 256):
            res["plain_%d" % n] = {"err_h": corrector.front_error(runs_out[n][0], ref, h_c),
                                   "ms": runs_out[n][1]}
        res["plain_512_ms"] = runs_out[512][1]
        results.append(res)
    # equal-error comparison: the coarsest plain resolution whose mean error is
    # at most the learned mean error (512 = the reference itself otherwise)
    cmp = []
    for res in results:
        le = res["learned_128"]["err_h"][1]
        match = next((n for n in (128, 256) if res["plain_%d" % n]["err_h"][1] <= le), 512)
        plain_ms = res["plain_512_ms"] if match == 512 else res["plain_%d" % match]["ms"]
        cmp.append({"plain_resolution_at_equal_error": match,
                    "speedup_learned_vs_plain": plain_ms / res["learned_128"]["ms"]})
    # the convolution's roofline: one 16 -> 16 layer on the whole 128^3 grid
    # (forward, input gradient, weight gradient), CUDA events over 20 calls of
    # the layer primitives (each forward / input-gradient call also packs its
    # weights: a 3 us launch, counted)
    g0 = torch.Generator(device="cuda").manual_seed(0)
    xa = torch.randn(cs + (16,), device="cuda", generator=g0).to(torch.bfloat16)
    ga = torch.randn(cs + (16,), device="cuda", generator=g0).to(torch.bfloat16)
    Wl = torch.randn(27, 16, 16, device="cuda", generator=g0) * 0.1
    bl = torch.zeros(16, device="cuda")
    mk = torch.relu(torch.randn(cs + (16,), device="cuda", generator=g0)).to(torch.bfloat16)
    ol = torch.empty(cs + (16,), dtype=torch.bfloat16, device="cuda")
    flop = 2 * 27 * 16 * 16 * n_c ** 3
    bf16_peak, bf16_kind = measured_bf16()

    def conv_rate(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        for _ in range(20):
            fn()
        c1.record()
        torch.cuda.synchronize()
        us = c0.elapsed_time(c1) / 20 * 1e3
        return {"us": us, "achieved": flop / us / 1e6, "frac": flop / us / 1e6 / bf16_peak}

    conv = {"bound": "tensor", "unit": "TFLOP/s", "peak": bf16_peak, "peak_kind": bf16_kind,
            "flop_per_layer": flop,
            "forward (k_conv3_tc)": conv_rate(lambda: ls.conv3_bf16(xa, Wl, bl, 0, out=ol)),
            "input_gradient (k_conv3_tc, mode 2)": conv_rate(lambda: ls.conv3_bf16(ga, Wl, None, 2, mask=mk,
                                                                                    out=ol)),
            "weight_gradient (k_conv3_wgrad_tc)": conv_rate(lambda: ls.conv3_wgrad(xa, ga, 16, 16))}
    print(json.dumps({
        "metric": "learned-coarse vs plain at equal error", "workload": "learned corrector 128^3 / 512^3",
        "unit": "wall-time ratio (plain at equal error / learned)", "value": float(np.mean(
            [c["speedup_learned_vs_plain"] for c in cmp])), "higher_is_better": True,
        "pairs": runs * per_run, "train_iters": args.train_iters, "final_loss": final,
        "pair_generation_s": t_pairs, "training_s": t_train, "coarse_steps": nsteps,
        "error_unit": "coarse cells h_c (max, mean of |phi - ref| within 1.5 h_c of the reference front)",
        "problems": results, "comparison": cmp, "fallbacks": ctx.learned_fallbacks(),
        "conv_roofline": conv, "data": "synthetic (seeded)"}), flush=True)
    ctx.close()


def run_perturbed(args):
    """1024^3 perturbed sphere, F = cos 4 pi x cos 4 pi y, band 6h: GLUPS of
    FP32 and FP64, narrow band and full domain (one line per combination;
    steps = level-set steps timed after 5 warm-up steps)."""
    import torch
    from paper_1612_04040_b300 import inputs
    from paper_1612_04040_b300 import native as ls
    torch.cuda.set_device(0)
    dev = torch.device("cuda")
    w = inputs.PerturbedSphere(n=args.perturbed_n)
    phi64 = w.phi(device=dev).contiguous()
    F64 = w.speed(device=dev).contiguous()
    nsteps = max(args.steps, 1) * 10
    dfma = ls.probe_dfma()
    for prec, name, bpu in ((ls.LS_FP32, "f32", 12), (ls.LS_FP64, "f64", 24)):
        dt_t = torch.float32 if prec == ls.LS_FP32 else torch.float64
        for full in (False, True):
            g = ls.LevelSet(w.n, w.n, w.n, w.h, prec)
            g.set_speed(F64.to(dt_t).contiguous())
            g.set_phi(phi64.to(dt_t).contiguous())
            if full:
                g.set_full_domain(True)
            else:
                g.band_rebuild(w.halfwidth)
            g.step(5, 0.5, ls.LS_DT_CFL, 5)
            tuned = g.autotune(reps=3) if prec == ls.LS_FP32 else None
            torch.cuda.synchronize()
            u0 = g.updates()
            g.reset_profile()
            g.profile_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.step(nsteps, 0.5, ls.LS_DT_CFL, 5)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            prof = g.profile()
            u = g.updates() - u0
            st = prof["stencil_ms"] / 1e3
            line = {
                "metric": "upwind GLUPS", "workload": "perturbed sphere %d^3 %s %s" % (
                    w.n, name, "full domain" if full else "band 6h"),
                "value": u / (ms / 1e3) / 1e9, "unit": "GLUPS", "dtype": name, "steps": nsteps,
                "ms_per_level_set_step": ms / nsteps, "updates_per_step": u / nsteps,
                "stencil_GBps_algorithmic": u * bpu / 1e9 / st if st > 0 else None,
                "stencil_share": st / (ms / 1e3)}
            if tuned is not None:
                line["autotuned"] = {"stages": tuned[0], "grid_pct": tuned[1], "points_per_thread": tuned[2],
                                     "steps_per_pass": g.steps_per_pass()}
            if prec == ls.LS_FP32 and st > 0:
                peak, peak_kind = measured_peaks()
                gbps = u * bpu / 1e9 / st
                line["roofline"] = {"bound": "hbm", "achieved": gbps, "peak": peak, "unit": "GB/s",
                                    "frac": gbps / peak, "traffic": None, "peak_kind": peak_kind,
                                    "kernel": STENCIL_KERNELS.get(tuned[2], "k_step_f32") if tuned
                                              else "k_step_f32", "bytes_per_update": bpu}
            if prec == ls.LS_FP64 and st > 0:
                ach = u * FLOPS_PER_UPDATE_F64 / st / 1e12
                line["roofline"] = {"bound": "fp64", "achieved": ach, "peak": dfma, "unit": "TFLOP/s",
                                    "frac": ach / dfma if dfma else None,
                                    "peak_kind": "measured (DFMA probe, this run; FMA = 2)",
                                    "flops_per_update": FLOPS_PER_UPDATE_F64}
            print(json.dumps(line), flush=True)
            g.close()


def run_sphere64(args):
    """64^3 single sphere, F = 1, dt = h/2, 100 full-domain steps, FP64."""
    import torch
    from paper_1612_04040_b300 import inputs
    from paper_1612_04040_b300 import native as ls
    torch.cuda.set_device(0)
    w = inputs.SingleSphere()
    g = ls.LevelSet(w.n, w.n, w.n, w.h, ls.LS_FP64)
    phi = w.phi(device="cuda").contiguous()
    g.set_speed_const(w.speed)
    g.set_full_domain(True)
    g.set_graphs(True)
    for _ in range(max(args.warmup, 1)):
        g.set_phi(phi)
        g.step(w.steps, w.h / 2, ls.LS_DT_FIXED)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 1)
    u0 = g.updates()
    t_ms = 0.0
    for _ in range(reps):
        g.set_phi(phi)
        e0.record()
        g.step(w.steps, w.h / 2, ls.LS_DT_FIXED)
        e1.record()
        torch.cuda.synchronize()
        t_ms += e0.elapsed_time(e1)
    u = g.updates() - u0
    dfma = ls.probe_dfma()
    ach = u * FLOPS_PER_UPDATE_F64 / (t_ms / 1e3) / 1e12
    print(json.dumps({"metric": "upwind GLUPS", "workload": "single sphere 64^3 FP64, 100 full-domain steps",
                      "value": u / (t_ms / 1e3) / 1e9, "unit": "GLUPS", "dtype": "f64",
                      "ms_per_run": t_ms / reps, "graphs": True,
                      "roofline": {"bound": "fp64", "achieved": ach, "peak": dfma, "unit": "TFLOP/s",
                                   "frac": ach / dfma if dfma else None,
                                   "peak_kind": "measured (DFMA probe, this run; FMA = 2)",
                                   "flops_per_update": FLOPS_PER_UPDATE_F64, "time": "whole run"},
                      "note": "whole state (4 MiB) sits in L2: launch/latency-bound, no HBM claim"}),
          flush=True)


def run_slab(args):
    """The standard 512^3 run split into z-slabs (section 2 of the paper):
    one slab per rank (NCCL exchanges) or --slabs slabs on one GPU (device
    copies), rows shared out by Eq. 14 (checked every 10 rebuild periods).
    The common dt is made on the device from the max-reduced bounds, so no
    rebuild period waits on the host (--slab-graphs 1 replays two periods
    at a time from a CUDA graph instead: measured slower).  One bench step = one whole 500-step run from phi^0
    (slab contexts, the initial rebuild and partition set up before the
    timed region); value = all slabs' updates (the library's device
    counters) / max time over ranks.  The total work is fixed as N grows
    (one grid): scaling "strong"."""
    import torch
    from paper_1612_04040_b300 import inputs
    from paper_1612_04040_b300 import native as ls
    from paper_1612_04040_b300 import slab
    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    w = inputs.SphereUnion(n=args.grid)
    # phi^0 and F by the library's Step 0 kernels on every rank (the same
    # seeded parameters), kept as device tensors to slice the slabs from
    g = ls.LevelSet(w.n, w.n, w.n, w.h, ls.LS_FP32, stream=stream.cuda_stream)
    g.init_speed(ls.LS_SPEED_SINUSOID)
    g.init_phi(ls.LS_SHAPE_SPHERES, inputs.spheres_params(w.centres, w.radii))
    phi0 = torch.empty((w.n,) * 3, dtype=torch.float32, device=dev)
    F0 = torch.empty_like(phi0)
    g.get_phi(phi0)
    g.get_speed(F0)
    # the stencil launch configuration the autotuner picks on the unsplit
    # grid (a band from the middle of the run), used by every slab
    g.band_rebuild(w.halfwidth, want_count=False)
    g.step(w.steps // 2, w.cfl, ls.LS_DT_CFL, w.rebuild_every)
    tuned = tune(g, args)
    g.close()
    comm = slab.DistComm(pg, dev) if world > 1 else slab.LocalComm(max(args.slabs, 1))
    # a stream of its own (the rebuild periods can be captured in CUDA graphs on it)
    run_stream = torch.cuda.Stream()

    def make(nx, ny, rows, h, lo, hi):
        return slab.GpuSlab(nx, ny, rows, h, lo, hi, ls.LS_FP32, run_stream.cuda_stream, tuned)

    def new_run():
        return slab.DeviceSlabRun(comm, make, (w.n,) * 3, w.h, w.halfwidth,
                                  lambda z0, z1: (phi0[z0:z1], F0[z0:z1]), rebalance=True,
                                  rebalance_gain=args.rebalance_gain, rebalance_every=10,
                                  graphs=bool(args.slab_graphs), stream=run_stream)

    for _ in range(max(args.warmup, 0)):
        r = new_run()
        r.step(w.steps, w.cfl, w.rebuild_every)
        r.close()
    torch.cuda.synchronize()
    total_ms, updates, migrations, bounds = 0.0, 0, 0, None
    for _ in range(args.steps):
        r = new_run()
        r.prepare(w.cfl, w.rebuild_every)   # the graph of the first two periods, recorded untimed
        u0 = r.updates_done
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(run_stream)
        r.step(w.steps, w.cfl, w.rebuild_every)
        e1.record(run_stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        total_ms += e0.elapsed_time(e1)
        updates += r.updates_done - u0
        migrations += r.migrations
        bounds = list(r.bounds)
        r.close()
    t_s, all_updates = aggregate(pg, total_ms / 1e3, float(updates), device=dev)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": all_updates / t_s / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_s / max(args.steps, 1),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "grid": args.grid, "parallelism": "slab",
                       "stencil_config": {"stages": tuned[0], "grid_pct": tuned[1],
                                          "points_per_thread": tuned[2]},
                       "slabs": comm.nparts, "transport": "nccl" if world > 1 else "device copies",
                       "final_bounds_tile_rows": bounds, "migrations_per_run": migrations / max(args.steps, 1),
                       "l2": "inputs larger than L2 (phi + F 1.5 GB)"},
            "updates_per_step": all_updates / max(args.steps, 1),
        }), flush=True)


def main():
    args = parse()
    if args.parallelism == "slab" and args.impl == "mine":
        run_slab(args)
        return
    if args.workload == "perturbed":
        run_perturbed(args)
        return
    if args.workload == "sphere64":
        run_sphere64(args)
        return
    if args.workload == "learned":
        run_learned(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    import numpy as np
    import torch
    from paper_1612_04040_b300 import inputs
    from paper_1612_04040_b300 import native as ls

    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    w = inputs.SphereUnion(n=args.grid)
    g = ls.LevelSet(w.n, w.n, w.n, w.h, ls.LS_FP32, stream=stream.cuda_stream)
    local_scheme = args.workload == "local"
    if local_scheme:
        # beta = gamma/2, dtau = h/2; iterations default to ceil(halfwidth / dtau)
        beta_h, dtau_h = w.halfwidth / 2, 0.5
        iters = args.reinit_iters if args.reinit_iters >= 0 else int(np.ceil(w.halfwidth / dtau_h))
        g.set_scheme(ls.LS_SCHEME_LOCAL, beta_h, iters, dtau_h)
    # Step 0 on the device: the library's own SDF / speed generators (FP64
    # evaluation, stored FP32); phi^0 kept as a device snapshot for the runs
    g.init_speed(ls.LS_SPEED_SINUSOID)
    g.init_phi(ls.LS_SHAPE_SPHERES, inputs.spheres_params(w.centres, w.radii))
    g.snapshot()
    phi0 = torch.empty((w.n,) * 3, dtype=torch.float32, device=dev)
    g.get_phi(phi0)
    torch.cuda.synchronize()

    def run_once():
        g.restore()
        g.band_rebuild(w.halfwidth, want_count=False)
        g.step(w.steps, w.cfl, ls.LS_DT_CFL, w.rebuild_every)

    # autotune the stencil launch configuration on a band from the middle of
    # the run (setup, before the timed region)
    g.restore()
    g.band_rebuild(w.halfwidth, want_count=False)
    g.step(w.steps // 2, w.cfl, ls.LS_DT_CFL, w.rebuild_every)
    tuned = tune(g, args)
    if args.steps_per_pass is not None:
        g.set_steps_per_pass(args.steps_per_pass)
    spp = g.steps_per_pass()
    for _ in range(max(args.warmup, 0)):
        run_once()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    time.sleep(0.3)

    out_dir = None
    if args.output_every > 0:
        import tempfile
        out_dir = tempfile.mkdtemp(prefix="ls_out_")
        g.output_open(os.path.join(out_dir, "phi_"), args.output_every,
                      ls.LS_OUTPUT_VTS if args.output_format == "vts" else ls.LS_OUTPUT_VTI, slots=2)
    u0 = g.updates()
    g.reset_profile()
    r0 = g.profile()["reinit_updates"]
    tsp0 = g.profile()["two_step_points"]
    # the plain scheme's runs of stencil launches (the up to 5 steps between
    # two rebuilds) are timed one in PROFILE_EVERY: an event record between
    # two launches costs the next one its overlap with the previous one
    # (measured: 2 % of the step with every run timed); the local scheme and
    # two steps per pass time every run
    prof_every = PROFILE_EVERY if (not local_scheme and spp == 1) else 1
    g.profile_enable(prof_every)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run_once()
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    g.profile_enable(False)
    prof = g.profile()
    updates = g.updates() - u0
    output = None
    if out_dir is not None:
        import shutil
        rep_ = g.output_stats()
        fin = g.output_close()
        shutil.rmtree(out_dir, ignore_errors=True)
        output = {"every": args.output_every, "format": args.output_format,
                  "files_in_timed_region": rep_["files"], "files": fin["files"], "bytes": fin["bytes"],
                  "writer_seconds": fin["write_seconds"], "step_wait_seconds": fin["wait_seconds"],
                  "status": fin["status"]}

    t_s, total_updates = aggregate(pg, ms / 1e3, float(updates), dev)
    value = total_updates / t_s / 1e9

    # dominant kernel: the upwind step, timed by events around every launch
    peak, peak_kind = measured_peaks()
    roofline_advance = None
    if not local_scheme:
        stencil_s = prof["stencil_ms"] / 1e3
        n_launch = max(prof["stencil_timed"], 1)
        upd_timed = prof["stencil_updates"]
        # a two-step pass reads phi and F and writes phi once for two updates
        # (with two steps per pass every run is timed)
        tsp = prof["two_step_points"] - tsp0
        point_passes = upd_timed - tsp if prof_every == 1 else upd_timed
        achieved = (point_passes * BYTES_PER_UPDATE / 1e9) / stencil_s if stencil_s > 0 else None
        tpu = recorded_traffic(tuned[2]) if tsp == 0 else None
        traffic = tpu * upd_timed / n_launch if tpu is not None else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                    "peak_kind": peak_kind,
                    "kernel": STENCIL_KERNELS.get(tuned[2], "k_step_f32") if tsp == 0 else
                              "k_step2_f32 / k_step_f32 (two / one upwind steps per pass)",
                    "bytes_per_update": BYTES_PER_UPDATE * point_passes / max(upd_timed, 1),
                    "avg_launch_us": 1e6 * stencil_s / n_launch,
                    "launches": prof["stencil_launches"], "launches_timed": prof["stencil_timed"],
                    "timed_runs": "one run of back-to-back stencil launches in %d" % prof_every,
                    "share_of_step_time": (stencil_s / n_launch * prof["stencil_launches"] / t_s)
                                          if t_s > 0 else None}
    else:
        # the advance covers the active tiles: read phi and F, write phi and the
        # N mask (64 B per tile); the reinitialisation passes (K per step)
        # cover the tiles holding N points: read d + write d + the mask
        rein_s = prof["reinit_ms"] / 1e3
        adv_s = (prof["stencil_ms"] - prof["reinit_ms"]) / 1e3
        n_rein = max(prof["reinit_timed"], 1)
        n_adv = max(prof["stencil_timed"] - prof["reinit_timed"], 1)
        b_rein, b_adv = 8 + 64 / 512, 12 + 64 / 512
        rupd = prof["reinit_updates"] - r0   # point-iterations over the tiles holding N points
        a_rein = (rupd * b_rein / 1e9) / rein_s if rein_s > 0 else None
        a_adv = (updates * b_adv / 1e9) / adv_s if adv_s > 0 else None
        roofline = {"bound": "hbm", "achieved": a_rein, "peak": peak, "unit": "GB/s",
                    "frac": (a_rein / peak) if a_rein else None, "traffic": None,
                    "peak_kind": peak_kind,
                    "kernel": "k_step_f32_z2<..., OP_REINIT> (Eq. 12 iteration on N over the tiles holding N points, 8 points per thread)",
                    "bytes_per_update": b_rein, "avg_launch_us": 1e6 * rein_s / n_rein,
                    # thread instructions per point-iteration of the pass (ncu
                    # record of the current source; the pass is issue-bound)
                    "instructions_per_point_iteration":
                        recorded_traffic(8, "local", "instructions_per_point_iteration"),
                    "launches": prof["reinit_timed"], "point_iterations": rupd,
                    "share_of_step_time": rein_s / t_s if t_s > 0 else None}
        roofline_advance = {"bound": "hbm", "achieved": a_adv, "peak": peak, "unit": "GB/s",
                            "frac": (a_adv / peak) if a_adv else None,
                            "kernel": ("k_local_z4<..., OP_CUT> (Eq. 8 advance + N mask, one warp per tile)"
                                       if tuned[2] == 16 else
                                       "k_step_f32<..., OP_CUT> (Eq. 8 advance + N mask, 4 points per thread)"),
                            "bytes_per_update": b_adv, "avg_launch_us": 1e6 * adv_s / n_adv,
                            "launches": n_adv, "share_of_step_time": adv_s / t_s if t_s > 0 else None}

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        phi_h = phi0.cpu().pin_memory()
        F_h = w.speed(out_dtype=torch.float32).contiguous().pin_memory()
        out_h = torch.empty_like(phi_h).pin_memory()
        u1 = g.updates()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # a sequence of problems through the stream-ordered host I/O: the
        # next problem's phi and F travel to the device and the previous
        # result back while the current one computes; every copy is inside
        # the timed region (the first upload and the last read-back too)
        g.stage_inputs(phi_h, F_h)
        for i in range(args.e2e_steps):
            g.load_staged()
            if i + 1 < args.e2e_steps:
                g.stage_inputs(phi_h, F_h)
            g.band_rebuild(w.halfwidth, want_count=False)
            g.step(w.steps, w.cfl, ls.LS_DT_CFL, w.rebuild_every)
            g.get_phi_async(out_h)
        g.wait_host()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        ue = g.updates() - u1
        nb = phi_h.numel() * 4
        e2e = {"value": ue / te / 1e9 * world, "unit": UNIT, "h2d_bytes_per_step": 2 * nb,
               "d2h_bytes_per_step": nb,
               "note": "per step: phi and F from pinned host memory (ls_stage_inputs, "
                       "ls_load_staged), rebuild, 500 steps, phi to pinned host memory "
                       "(ls_get_phi_async); transfers of neighbouring steps overlap the "
                       "computation on copy streams; host wall clock over %d steps" % args.e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        F_np = F_h.numpy() if args.e2e_steps > 0 else w.speed(out_dtype=torch.float32).numpy()
        if local_scheme:
            cpu = cpu_baseline_local(phi0.cpu().numpy(), F_np, w, beta_h, iters, dtau_h)
        else:
            cpu, orc = cpu_baseline(phi0.cpu().numpy(), F_np, w)
            cpu["parity"] = parity_vs_oracle(g, orc, w, 40)
            cpu["single_thread"] = oracle_one_thread(orc, w)
            del orc

    # band points (|phi| < gamma) of the final state of the last run
    fin = torch.empty((w.n,) * 3, dtype=torch.float32, device=dev)
    g.get_phi(fin)
    band_points = int((fin.abs().double() < w.halfwidth * w.h).sum().item())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD if not local_scheme else WORKLOAD_LOCAL % iters,
                       "grid": w.n, "halfwidth_h": w.halfwidth,
                       "autotuned": {"stages": tuned[0], "grid_pct": tuned[1], "points_per_thread": tuned[2],
                                     "steps_per_pass": spp},
                       "rebuild_every": w.rebuild_every, "level_set_steps_per_bench_step": w.steps,
                       "cfl": w.cfl, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (phi + F 1.5 GB; active set per step ~0.2 GB)"},
            "updates_per_step": updates / max(args.steps, 1),
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": prof["kernel_launches"], "band_points_final": band_points,
        }
        if output is not None:
            line["output"] = output
        if local_scheme:
            line["metric"] = METRIC_LOCAL
            line["config"]["local_scheme"] = {"beta_h": beta_h, "reinit_iters": iters, "dtau_h": dtau_h}
            line["roofline_advance"] = roofline_advance
            line["band_breaches"] = g.band_breaches()
        print(json.dumps(line), flush=True)
    g.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
