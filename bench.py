"""Benchmark of the fused phase-field LB step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload bubble1024x2048|droplets8192] [--precision fp32|fp64|bf16|fp16]

One step = one pass of the whole hot path over the grid: pull-streaming of
f, g, h1, h2, zeroth moments, stencils, flow macros, collision of the four
lattices and the store (one launch of the fused kernel).  The default workload
is the 1024 x 2048 wall-bounded rising bubble (density ratio 1000, viscosity
ratio 100, mu = mu0 exp(-beta T)), FP32.  Its state (0.5 GB) is larger than
L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  Metric: MLUPS (million lattice-node updates per
second), whole job.  Multi-GPU: one process per GPU (torchrun), each runs an
independent replica of the workload (the path is data parallel per case; there
is no exchange step), scaling "weak".
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

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_FILE = os.path.join(ROOT, "profiles", "fused_step_fp32_bubble1024x2048.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2402_15752_gb300", "csrc", f)
                  for f in ("lbm_kernels.cuh", "lbm_internal.h")]
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bubble1024x2048",
                    choices=["bubble1024x2048", "droplets8192", "batched256"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16", "fp16"],
                    help="population storage (bf16/fp16: 16-bit storage, FP32 arithmetic)")
    ap.add_argument("--cases", type=int, default=256, help="batched256: number of lattices (a smaller "
                    "sample of the same generator, for profiling)")
    ap.add_argument("--tiling", default=None, help="batched256: tile WxH instead of the autotuner's choice")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the short measurements of the other workloads that the default run "
                    "adds to its line (N = 1 only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank number over all ranks (identity when world == 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, cells: int, steps: int, ms_max: float) -> float:
    """Units processed by all ranks (each runs its own replica) over the slowest rank's time."""
    return world * cells * steps / (ms_max * 1e-3) / 1e6


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def read_profile_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    only if it was taken on the current kernel source."""
    if not os.path.exists(PROFILE_FILE):
        return None
    rec = {}
    for line in open(PROFILE_FILE):
        if ":" in line:
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("kernel_source_sha256_16") != kernel_hash():
        return None
    try:
        return float(rec["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def hbm_peak():
    try:
        return float(json.load(open(PEAKS_FILE))["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(name, cells_cap=None):
    from paper_2402_15752_gb300 import workloads as wl
    if name == "batched256":
        # one case of the batch stands for it on the CPU: the largest that fits
        cases = wl.batched()
        fit = [w for w in cases if cells_cap is None or w.cells <= cells_cap]
        return max(fit or [min(cases, key=lambda w: w.cells)], key=lambda w: w.cells)
    if cells_cap is None:
        return wl.get(name)
    # bounded sample: the same workload with both sides scaled down
    w = wl.get(name)
    nx, ny = int(w.params["nx"]), int(w.params["ny"])
    s = 1.0
    while (nx * s) * (ny * s) > cells_cap and s > 1 / 64:
        s /= 2
    if s == 1.0:
        return w
    if name == "bubble1024x2048":
        return wl.bubble1024x2048(nx=int(nx * s), ny=int(ny * s))
    return wl.droplets8192(nx=int(nx * s), ny=int(ny * s))


def oracle_mlups(name, steps_budget_s, cells_cap, min_steps=2, threads=1):
    """Time the FP64 CPU oracle on a bounded sample of the workload with
    `threads` host threads (its per-node loops; results do not depend on it)."""
    import oracle
    oracle.set_threads(threads)
    w = make_workload(name, cells_cap)
    s = oracle.OracleSim(w.params)
    s.init(w.sdf, w.c1_tilde, w.c2_tilde)
    t = time.perf_counter()
    s.step(1)
    one = time.perf_counter() - t
    steps = max(min_steps, int(steps_budget_s / max(one, 1e-6)))
    t = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t
    oracle.set_threads(1)
    return w.cells * steps / dt / 1e6, w, steps, dt


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baseline(name, cells_cap, what):
    """The oracle on all host cores (the baseline value) and on one thread."""
    cores = host_cores()
    mlups, sw, steps, dt = oracle_mlups(name, 10.0, cells_cap, threads=cores)
    one, _, steps1, dt1 = oracle_mlups(name, 10.0, cells_cap, threads=1)
    return {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "single_thread_value": one,
            "sample": "%s %dx%d, FP64: %d steps in %.1f s on %d threads; %d steps in %.1f s on one" % (
                what, sw.params["nx"], sw.params["ny"], steps, dt, cores, steps1, dt1)}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    if world > 1 and rank != 0:
        return
    import oracle
    cores = host_cores()
    oracle.set_threads(cores)
    full = make_workload(args.workload)
    # each step a bounded sample so that warmup + steps end within ~2-3 minutes
    per_step_cells = int(max(4096, min(full.cells, 0.6e6 * 150.0 / max(1, args.steps + args.warmup))))
    w = make_workload(args.workload, per_step_cells)
    s = oracle.OracleSim(w.params)
    s.init(w.sdf, w.c1_tilde, w.c2_tilde)
    s.step(args.warmup)
    t = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t
    value = w.cells * args.steps / dt / 1e6
    sample = "%s scaled to %dx%d (%d nodes), %d steps" % (args.workload, w.params["nx"],
                                                         w.params["ny"], w.cells, args.steps)
    line = {
        "impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "nx": full.params["nx"], "ny": full.params["ny"],
                   "sample_nx": w.params["nx"], "sample_ny": w.params["ny"]},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2402_15752_gb300 import LBMError, Simulation

    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the GPU path has no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    w = make_workload(args.workload)
    sim = Simulation(w.params, precision=args.precision, device=dev)
    sim.init(w.sdf, w.c1_tilde, w.c2_tilde)
    stream = sim.stream
    sim.step(max(3, args.warmup))
    try:
        sim.sync()
    except LBMError as e:  # a reduced storage precision that cannot carry this flow
        if rank == 0:
            print(json.dumps({"metric": "MLUPS", "value": None, "unit": "MLUPS", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup,
                              "config": {"workload": args.workload, "precision": args.precision},
                              "failed": "non-finite state during warm-up: %s" % e}))
        return

    # ---- device-timed region: K fused steps, inputs resident in HBM ----
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if \
        os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    sampler = ClockSampler(int(phys) if phys.isdigit() else local)
    sampler.start()
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    state_ok = True
    try:
        sim.sync()
    except LBMError:
        state_ok = False  # timed, but the state went non-finite: flagged in the line
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    cells = w.cells
    value = whole_job_mlups(world, cells, args.steps, ms)

    # ---- roofline of the fused kernel (the only kernel in the timed region) ----
    q = int(w.params.get("scalar_q", 5))
    elem = {"fp64": 8, "fp32": 4}.get(args.precision, 2)  # bytes of a stored population
    relem = 8 if args.precision == "fp64" else 4          # bytes of a previous-step macro
    bytes_per_cell = 2 * (18 + 2 * q) * elem + 2 * 5 * relem
    if elem == 2:
        # 16-bit storage: the writer's bases, (p, phi) in FP32 and (c1, c2) in
        # halves, written beside its populations and read once for the
        # populations pulled from it
        bytes_per_cell += 2 * 12
    launch_s = ms * 1e-3 / args.steps
    achieved = bytes_per_cell * cells / launch_s / 1e9
    peak, peak_kind = hbm_peak()
    traffic = read_profile_traffic() if (args.workload == "bubble1024x2048" and args.precision == "fp32") else None

    # ---- end to end through the public API, host buffers, copies timed ----
    e2e = None
    if not args.no_e2e and state_ok:
        sdf_host = torch.from_numpy(np.ascontiguousarray(w.sdf, dtype=np.float64)).pin_memory()
        out_host = torch.empty((6, w.params["ny"], w.params["nx"]), dtype=torch.float32).pin_memory()
        names = ("phi", "ux", "uy", "p", "c1", "c2")
        # one untimed pass through the same buffers first: the device's first
        # touches of newly page-locked host memory are a one-time cost, as the
        # warm-up steps are for the device-timed loop
        sim.init(sdf_host, w.c1_tilde, w.c2_tilde)
        sim.step(max(3, args.warmup))
        sim.fields(names=names, dtype="f32", out=out_host.numpy())
        barrier()
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        sim.init(sdf_host, w.c1_tilde, w.c2_tilde)
        sim.step(args.steps)
        sim.fields(names=names, dtype="f32", out=out_host.numpy())
        t1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ems = max_over_ranks(t0.elapsed_time(t1), world, dev)
        e2e = {"value": whole_job_mlups(world, cells, args.steps, ems), "unit": "MLUPS",
               "h2d_bytes_per_step": cells * 8 / args.steps,
               "d2h_bytes_per_step": 6 * cells * 4 / args.steps}
        sim.sync()

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, 256 * 512, args.workload + " scaled to")
    others = None
    if (world == 1 and not args.no_secondary and args.workload == "bubble1024x2048"
            and args.precision == "fp32"):
        others = secondary(dev)

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "nx": w.params["nx"], "ny": w.params["ny"],
                       "bc": "walls" if w.params["wall_x"] else "periodic", "scalar_q": q,
                       "precision": args.precision, "l2": "state larger than L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_kind, "bytes_per_cell": bytes_per_cell},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
        if others is not None:
            line["secondary"] = others
        if not state_ok:
            line["failed"] = "the state went non-finite during the timed steps"
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        dist.destroy_process_group()


def timed_steps(step, stream, steps, warmup):
    """CUDA-event milliseconds of `steps` calls' worth of step(n), after warm-up."""
    import torch
    step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def secondary(dev):
    """Short measurements of the other workloads, outside the timed region of the
    line's own number: the 8192 x 8192 droplets (FP32), the bubble in bfloat16
    storage, and the 256 batched droplets (autotuned tiles).  Each: node updates
    per second over a fixed number of steps after 5 warm-up steps, and the
    fraction of the measured copy bandwidth at its algorithmic bytes per node."""
    from paper_2402_15752_gb300 import Batch, Simulation
    from paper_2402_15752_gb300 import workloads as wl

    peak, _ = hbm_peak()
    out = {}

    def entry(cells, steps, ms, bpc, **extra):
        mlups = cells * steps / (ms * 1e-3) / 1e6
        return dict(value=mlups, unit="MLUPS", steps=steps, ms_per_step=ms / steps, bytes_per_cell=bpc,
                    frac=bpc * mlups * 1e6 / 1e9 / peak, **extra)

    for name, prec, steps, bpc in (("droplets8192", "fp32", 100, 264), ("bubble1024x2048", "bf16", 2000, 176)):
        key = "%s_%s" % (name, prec)
        sim = None
        try:
            w = wl.get(name)
            sim = Simulation(w.params, precision=prec, device=dev)
            sim.init(w.sdf, w.c1_tilde, w.c2_tilde)
            ms = timed_steps(sim.step, sim.stream, steps, 5)
            sim.sync()
            out[key] = entry(w.cells, steps, ms, bpc)
        except Exception as e:  # reported in the line; the line's own number stands
            out[key] = {"failed": str(e)[:200]}
        finally:
            if sim is not None:
                sim.close()
    sims, b = [], None
    try:
        cases = wl.batched()
        sims = [Simulation(w.params, precision="fp32", device=dev) for w in cases]
        for sm, w in zip(sims, cases):
            sm.init(w.sdf, w.c1_tilde, w.c2_tilde)
        b = Batch(sims)
        tune = b.autotune(steps_per_trial=10)
        ms = timed_steps(b.step, sims[0].stream, 200, 5)
        b.sync()
        out["batched256_fp32"] = entry(sum(w.cells for w in cases), 200, ms, 264, cases=len(cases),
                                       tiling={k: tune[k] for k in ("tile_w", "tile_h")})
    except Exception as e:
        out["batched256_fp32"] = {"failed": str(e)[:200]}
    finally:
        if b is not None:
            b.close()
        for sm in sims:
            sm.close()
    return out


def run_batched(args, rank, world, local):
    """256 independent droplets of uneven sizes in the persistent batched kernel,
    tile shape picked by the autotuner; compared with stepping every case with its
    own launches (graph-replayed lbm_step), one case after another."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2402_15752_gb300 import Batch, Simulation
    from paper_2402_15752_gb300 import workloads as wl

    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the GPU path has no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    cases = wl.batched(n=args.cases)
    cells = sum(w.cells for w in cases)
    sims = [Simulation(w.params, precision="fp32", device=dev) for w in cases]
    for s, w in zip(sims, cases):
        s.init(w.sdf, w.c1_tilde, w.c2_tilde)
    stream = sims[0].stream
    b = Batch(sims)
    if args.tiling:
        tw, th = (int(v) for v in args.tiling.lower().split("x"))
        b.set_tiling(tw, th)
        tune = dict(b.tiling(), cached=False, trials=[], fixed=True)
    else:
        tune = b.autotune(steps_per_trial=10)
    b.step(max(3, args.warmup))
    b.sync()

    phys = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if \
        os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    sampler = ClockSampler(int(phys) if phys.isdigit() else local)
    sampler.start()
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    b.sync()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    value = whole_job_mlups(world, cells, args.steps, ms)

    # the same cases, each stepped by its own launches, one case after another
    per_steps = min(args.steps, 500)
    torch.cuda.synchronize(dev)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for s in sims:
        s.step(per_steps)
    p1.record(stream)
    torch.cuda.synchronize(dev)
    per_case = cells * per_steps / (p0.elapsed_time(p1) * 1e-3) / 1e6

    bytes_per_cell = 2 * 28 * 4 + 2 * 5 * 4
    launch_s = ms * 1e-3 / args.steps
    achieved = bytes_per_cell * cells / launch_s / 1e9
    peak, peak_kind = hbm_peak()

    e2e = None
    if not args.no_e2e:
        sdf_host = [torch.from_numpy(np.ascontiguousarray(w.sdf)).pin_memory() for w in cases]
        outs = [torch.empty((6, w.params["ny"], w.params["nx"]), dtype=torch.float32).pin_memory()
                for w in cases]
        names = ("phi", "ux", "uy", "p", "c1", "c2")
        # one untimed pass through the same buffers first (first touches of newly
        # page-locked host memory)
        for s, w, h in zip(sims, cases, sdf_host):
            s.init(h, w.c1_tilde, w.c2_tilde)
        b.step(max(3, args.warmup))
        for s, o in zip(sims, outs):
            s.fields(names=names, dtype="f32", out=o.numpy())
        barrier()
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s, w, h in zip(sims, cases, sdf_host):
            s.init(h, w.c1_tilde, w.c2_tilde)
        b.step(args.steps)
        for s, o in zip(sims, outs):
            s.fields(names=names, dtype="f32", out=o.numpy())
        t1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ems = max_over_ranks(t0.elapsed_time(t1), world, dev)
        e2e = {"value": whole_job_mlups(world, cells, args.steps, ems), "unit": "MLUPS",
               "h2d_bytes_per_step": cells * 8 / args.steps,
               "d2h_bytes_per_step": 6 * cells * 4 / args.steps}
        b.sync()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, 64 * 64, "one case of the batch,")

    if rank == 0:
        graphs, rest = divmod(args.steps, 32)
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched256", "cases": len(cases), "cells": cells,
                       "sides": "64..512 step 32", "bc": "periodic", "scalar_q": 5,
                       "precision": "fp32", "l2": "state larger than L2 (no flush)",
                       "tiling": {k: tune[k] for k in ("tile_w", "tile_h", "tiles", "ctas")},
                       "per_case_launches_mlups": per_case, "per_case_steps": per_steps,
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": peak_kind, "bytes_per_cell": bytes_per_cell},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": graphs + (1 if rest else 0),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    b.close()
    for s in sims:
        s.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched256":
        run_batched(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
