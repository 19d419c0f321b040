#!/usr/bin/env python3
"""Throughput of the fused EVD lattice Boltzmann step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload stratification|tube|tubes|adjoint] [--precision fp32|fp64|fp16]

One bench step is one time step of the whole hot path (gather with
interpolation and wall scheme, moments, tau_ij, collision with forcing) over
the whole lattice.  The default workload is the 256^3 D3Q19 ternary closed box
under gravity (the stratification case, the one whose working set exceeds L2,
so HBM bandwidth is the bound and no L2 flush is needed between steps), FP32.

Metric: species-site updates per second, GLUPS = N_species * sites * steps /
time / 1e9, whole job over all ranks.  Every rank runs an independent replica
(the path is single-GPU; there is no data-path collective), so scaling is weak.

``--workload adjoint`` times instead the loss and exact gradient of the
mole-fraction misfit (evd_loss_gradient, FP64 reverse sweep) over a horizon of
``--horizon`` steps (20000) of the 128 x 512 ternary D2Q9 tube with gravity of
the inverse problem, one GPU, with the FP64 and the FP32 forward pass.

Prints one JSON line on rank 0.  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead (the paper publishes no
implementation to run).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_07059_gb300 import workloads as W  # noqa: E402

METRIC = "species-site updates/s (GLUPS)"
UNIT = "GLUPS"
FALLBACK_HBM_GBS = 6800.0

# dram__bytes_read.sum + dram__bytes_write.sum of one step-kernel launch, keyed
# by (digest of KERNEL_SOURCES, workload, cube side, precision), from an ncu
# capture of the kernel sources with this digest (summaries under profiles/).
# A change to those sources changes the digest and the entry no longer applies.
NCU_TRAFFIC = {
    # 128^3 captures (k_step_tma, one-row tiles), x8 for a 256^3 launch: FP32
    # 537.9 MB read + 439.9 MB written (1.023 x the algorithmic 956.3 MB), FP16
    # storage 258.1 MB read + 213.8 MB written
    ("8227cc2459e25752", "stratification", 256, "fp32"): 7823.0e6,
    ("8227cc2459e25752", "stratification", 256, "fp16"): 3775.3e6,
    # the batched sweep: k_step_batch on the first 64 tubes, 204.5 MB read + 180.2 MB written
    # = 0.99943 x the algorithmic 384.9 MB, the same ratio applied to the 512-tube launch
    ("324794d064f54151", "tubes", 512, "fp32"): 3461.8e6,
}


# Floating-point operations per species-site update of a step kernel, from
# the ncu thread-instruction counters of one launch (dadd + dmul + 2 dfma for
# double; fadd + fmul + 2 ffma, doubled for the f32x2 forms, for float), keyed
# like NCU_TRAFFIC.  They place the compute-bound paths on their arithmetic
# roof.  FP64: the general step on a 64^3 copy of the workload (wall nodes,
# whose lumps add arithmetic, are 9 % of its sites against 2 % at 256^3);
# FP32 and FP16 storage: k_step_tma on a 128^3 copy.
NCU_FLOPS = {
    ("8227cc2459e25752", "stratification", "fp64"): 614.2,
    ("8227cc2459e25752", "stratification", "fp32"): 632.0,
    ("8227cc2459e25752", "stratification", "fp16"): 749.5,
}


def flops_for(digest: str, workload: str, precision: str):
    return NCU_FLOPS.get((digest, workload, precision))


def measure_alu_peaks(torch, dev, stream, device_id) -> dict:
    """Arithmetic throughput of this GPU: the FMA-chain kernel in double,
    float and float pairs (CUDA events), with the SM clock sampled meanwhile."""
    from paper_2504_07059_gb300 import evd
    out = {}
    with ClockSampler(device_id) as clocks:
        for name, kind, iters in (("fp64", 0, 1 << 15), ("fp32", 1, 1 << 20), ("fp32x2", 2, 1 << 19)):
            flops, ms = evd.evd_fma_rate(kind, iters, stream)
            out[name + "_tflops"] = flops / (ms * 1e-3) / 1e12
    out["clocks"] = clocks.summary()
    out["how"] = ("8 independent FMA chains per thread, 8 blocks of 256 threads per SM, one launch timed with "
                  "CUDA events after a warm-up launch")
    return out


# The sources that define the step kernels and their launch configuration
# (the device code, the TMA step, the launchers and the D3Q19 units).
KERNEL_SOURCES = ("evd_device.cuh", "evd_tma.cuh", "evd_tma_launch.cuh", "evd_launch.cuh",
                  "evd_fp32_d3q19.cu", "evd_fp16_d3q19.cu", "evd_fp64_d3q19.cu")


# The sources of the batched step kernel (FP32 D2Q9 storage).
BATCH_SOURCES = ("evd_device.cuh", "evd_batch_kernels.cuh", "evd_batch_fp32_d2q9.cu")


def kernel_digest(sources: tuple = KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_2504_07059_gb300", "csrc", name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(digest: str, workload: str, size: int, precision: str):
    """ncu DRAM bytes of one step launch captured from kernel sources with
    this digest, or None (sources changed since the capture, or none)."""
    return NCU_TRAFFIC.get((digest, workload, size, precision))


def measured_peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def make_workload(name: str, size: int = 256) -> W.Workload:
    if name == "stratification":
        return W.stratification_3d(n=size)
    if name == "tube":
        return W.loschmidt_ternary_gravity()
    raise ValueError(name)


def bytes_per_ssu(wl: W.Workload, precision: str) -> int:
    """Algorithmic HBM bytes per species-site update: each population read
    once and written once (ping-pong)."""
    elem = {"fp64": 8, "fp32": 4, "fp16": 2}[precision]
    # half storage also reads and writes the node's stored density
    return 2 * wl.Q * elem + (2 * elem if precision == "fp16" else 0)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.device_id = device_id
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.device_id:
            cmd += ["-i", self.device_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        loaded = sorted(sm)[len(sm) // 4:] or sm   # drop the idle tail of the window
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_device_id(torch, dev: int) -> str | None:
    p = torch.cuda.get_device_properties(dev)
    for attr in ("pci_bus_id",):
        v = getattr(p, attr, None)
        if v:
            return str(v)
    u = getattr(p, "uuid", None)
    if u:
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    return None


def oracle_all_cores():
    """Context for timing the oracle on every host core: its OpenMP build
    (bitwise the serial arithmetic) where the compiler has OpenMP, else the
    serial build.  Yields the number of threads a step runs on."""
    import contextlib

    from oracle import oracle as O

    @contextlib.contextmanager
    def ctx():
        so = O.build_omp()
        if so is None:
            yield O.threads()
            return
        with O.swapped_library(so):
            yield O.threads()
    return ctx()


def time_oracle_sample(side: int, steps: int, warmup: int = 0) -> tuple[float, int, float]:
    """The FP64 oracle on a side^3 copy of the stratification workload (same
    recipe and seed).  Returns (seconds for ``steps`` steps, species-site
    updates, seconds per step)."""
    from oracle import oracle as O
    wl = W.stratification_3d(shape=(side, side, side))
    o = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g)
    o.init(wl.x)
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return dt, wl.ns * wl.nsites * steps, dt / max(steps, 1)


def _oracle_rate(side: int, budget_s: float) -> tuple[float, int, float]:
    """(GLUPS, steps, seconds) of the oracle on a side^3 copy, as many steps as
    fit in about budget_s seconds (at least 2)."""
    _, _, per = time_oracle_sample(side, 1)
    steps = max(2, int(budget_s / max(per, 1e-6)))
    dt, ssu, _ = time_oracle_sample(side, steps)
    return ssu / dt / 1e9, steps, dt


def cpu_baseline(budget_s: float = 10.0) -> dict:
    """Bounded samples of the oracle on the 32^3 copy of the workload: on
    every host core (the OpenMP build), and single-threaded beside it."""
    with oracle_all_cores() as threads:
        v_all, steps_all, dt_all = _oracle_rate(32, budget_s)
    v_one, steps_one, dt_one = _oracle_rate(32, budget_s)
    sample = "stratification-d3q19-32x32x32 (same recipe and seed), FP64 C oracle"
    return {"value": v_all, "unit": UNIT, "cores": threads, "kind": "oracle",
            "nproc": os.cpu_count(),
            "sample": f"{sample}, {steps_all} steps on {threads} threads (OpenMP), {dt_all:.1f} s",
            "single_thread": {"value": v_one, "unit": UNIT, "cores": 1,
                              "sample": f"{sample}, {steps_one} steps single-threaded, {dt_one:.1f} s"}}


def time_oracle_tubes(budget_s: float, steps: int | None = None, warmup: int = 0) -> tuple[float, int, str]:
    """The FP64 oracle on the first tubes of the sweep (same recipe and seed),
    one after another, until about budget_s seconds of stepping (or ``steps``
    steps per tube on as many tubes as fit).  Returns (seconds, species-site
    updates, description)."""
    from oracle import oracle as O
    tubes = W.batched_tubes()
    t_total, ssu, used, k_used = 0.0, 0, 0, 0
    for wl in tubes:
        o = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g)
        o.init(wl.x)
        if warmup:
            o.step(warmup)
        k = steps
        if k is None:   # as many steps as fit in what is left of the budget, at least 2
            t0 = time.perf_counter()
            o.step(1)
            per = time.perf_counter() - t0
            t_total += per
            ssu += wl.ns * wl.nsites
            k = max(2, int((budget_s - t_total) / max(per, 1e-6)))
        t0 = time.perf_counter()
        o.step(k)
        t_total += time.perf_counter() - t0
        ssu += wl.ns * wl.nsites * k
        used += 1
        k_used = k
        if t_total >= budget_s:
            break
    return t_total, ssu, f"first {used} tube(s) of the sweep, up to {k_used} steps each, FP64 single-threaded C"


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    with oracle_all_cores() as threads:
        if args.workload == "tubes":
            # bounded: each step a pass over as many tubes as fit in ~60 s / (W + K)
            dt, ssu, what = time_oracle_tubes(60.0 / (args.steps + args.warmup) * args.steps)
            value = ssu / dt / 1e9
            what = what.replace("single-threaded", f"{threads} thread(s)")
            ssu_step = sum(t.ns * t.nsites for t in W.batched_tubes())
            out = {
                "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ssu_step / (value * 1e9) * 1e3,   # one step of the whole sweep at this rate
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": dict(tubes_config(), precision="fp64", sample=what),
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": what},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            }
            print(json.dumps(out), flush=True)
            return
        # choose the sample cube so that warmup + steps end within about a minute
        _, _, per16 = time_oracle_sample(16, 1)
        total = args.steps + args.warmup
        side = 16
        for s in (48, 40, 32, 24, 16, 12, 8):
            if per16 * (s / 16.0) ** 3 * total <= 60.0:
                side = s
                break
        dt, ssu, _ = time_oracle_sample(side, args.steps, args.warmup)
    value = ssu / dt / 1e9
    wl = make_workload(args.workload, args.size)
    out = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(wl.describe(), precision="fp64",
                       sample=f"{side}x{side}x{side} copy of the workload (same recipe and seed)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "nproc": os.cpu_count(),
                         "sample": f"stratification-d3q19-{side}^3, {args.steps} steps after {args.warmup} "
                                   f"warm-up, FP64 C oracle on {threads} thread(s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def replica_throughput(ms_local: float, ssu_rank: int, device) -> tuple[float, float]:
    """Whole-job throughput of independent replicas: every rank processed
    ``ssu_rank`` species-site updates in ``ms_local`` milliseconds; the job
    takes as long as the slowest rank.  Returns (max ms over ranks, GLUPS of
    all ranks together).  With torch.distributed initialised this is one MAX
    all-reduce on ``device`` (NCCL on the GPU, gloo on CPU); otherwise one rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * ssu_rank / (ms_max * 1e-3) / 1e9


def tubes_config(members: int = 512) -> dict:
    return {"workload": f"batched-tubes-d2q9-{members}x32", "lattice": "D2Q9", "members": members, "width": 32,
            "length": "log-uniform [128, 4096]", "species": "2 or 3", "mass_ratio": "U[1, 10]",
            "diffusivity": "binary members U[0.01, 0.1]; ternary members U[0.06, 0.1] (narrowed from "
                           "U[0.01, 0.1]: ternary tubes with a mass ratio near 10 and D_ij below ~0.05 "
                           "diverge in the FP64 oracle itself)",
            "walls": ["y-", "y+"], "seed": W.SEED}


def measure_tubes(torch, dev, stream, prec: str, steps: int, warmup: int, members: int = 512,
                  schedule: str = "", e2e: bool = True, fp64: bool = True, sync=None) -> dict:
    """The batched sweep: ``members`` independent tubes advanced by one
    persistent launch per step, replayed from CUDA graphs, schedule picked by
    the autotuner (or given) before the timed region.  ``sync`` runs around
    the timed region (the ranks' barrier)."""
    from paper_2504_07059_gb300 import evd
    sync = sync or (lambda: None)
    tubes = W.batched_tubes()[:members]
    b = evd.Batch(tubes, prec, stream)
    x_all = np.concatenate([t.x.ravel() for t in tubes])
    evd.evd_batch_set_fields(b.b, x_all)   # host path once, for the mass targets
    t0 = time.perf_counter()
    if schedule:
        sched = tuple(int(v) for v in schedule.split(","))
        evd.evd_batch_set_schedule(b.b, *sched)
    else:
        sched = evd.evd_batch_autotune(b.b, 8)
    tune_s = time.perf_counter() - t0
    ssu_step = sum(t.ns * t.nsites for t in tubes)
    bpl = sum(t.ns * t.nsites * bytes_per_ssu(t, prec) for t in tubes)
    evd.evd_batch_step(b.b, warmup)
    torch.cuda.synchronize(dev)
    sync()
    torch.cuda.synchronize(dev)
    launches0 = evd.evd_batch_launch_count(b.b)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    evd.evd_batch_step(b.b, steps)
    stop.record(stream)
    torch.cuda.synchronize(dev)
    sync()
    torch.cuda.synchronize(dev)
    ms = start.elapsed_time(stop)
    evd.evd_batch_check(b.b)
    launches = evd.evd_batch_launch_count(b.b) - launches0
    peak, peak_kind = measured_peaks()
    achieved = bpl / (ms / steps * 1e-3) / 1e9
    res = {"ms": ms, "ms_per_step": ms / steps, "ssu_step": ssu_step, "bytes_per_launch": bpl,
           "value": ssu_step * steps / (ms * 1e-3) / 1e9, "achieved": achieved, "peak": peak,
           "peak_source": peak_kind, "frac": achieved / peak, "launches": launches,
           "schedule": {"item_sites": sched[0], "ctas_per_sm": sched[1],
                        "autotune_s": None if schedule else tune_s}}
    if e2e:
        # end to end through the public API: upload the initial mole fractions
        # from pinned host memory, run the steps, read the mole fractions back
        x_host = torch.from_numpy(x_all).pin_memory()
        out_host = torch.empty_like(x_host).pin_memory()
        times = []
        for _ in range(2):
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            evd.evd_batch_set_fields(b.b, x_host.data_ptr())
            evd.evd_batch_step(b.b, steps)
            evd.evd_batch_get_mole_fractions(b.b, out_host.data_ptr())
            times.append(time.perf_counter() - t1)
        res["e2e_s"] = min(times)
        res["h2d"] = x_host.numel() * 8
        res["d2h"] = out_host.numel() * 8
    b.close()
    if fp64 and prec != "fp64":
        b64 = evd.Batch(tubes, "fp64", stream)
        evd.evd_batch_set_fields(b64.b, x_all)
        evd.evd_batch_step(b64.b, 8)
        torch.cuda.synchronize(dev)
        n64 = 16
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        evd.evd_batch_step(b64.b, n64)
        z.record(stream)
        torch.cuda.synchronize(dev)
        evd.evd_batch_check(b64.b)
        ms64 = a.elapsed_time(z) / n64
        b64.close()
        res["fp64"] = {"ms_per_step": ms64, "value": ssu_step / (ms64 * 1e-3) / 1e9, "unit": UNIT, "steps": n64,
                       "speedup": ms64 / (ms / steps)}
    return res


def run_tubes(args, torch, dev, world, rank, local) -> None:
    """The batched sweep as the bench's workload (one JSON line)."""
    stream = torch.cuda.current_stream(dev)
    sync = (lambda: torch.distributed.barrier()) if world > 1 else None
    with ClockSampler(gpu_device_id(torch, local)) as clocks:
        r = measure_tubes(torch, dev, stream, args.precision, args.steps, args.warmup, args.members, args.schedule,
                          e2e=not args.no_e2e, fp64=not args.no_fp64, sync=sync)
    ms_max, value = replica_throughput(r["ms"], r["ssu_step"] * args.steps, dev)
    e2e_value = float("nan")
    if "e2e_s" in r:
        _, e2e_value = replica_throughput(r["e2e_s"] * 1e3, r["ssu_step"] * args.steps, dev)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        with oracle_all_cores() as threads:
            dt, ssu, what = time_oracle_tubes(15.0)
        cpu = {"value": ssu / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": what.replace("single-threaded", f"{threads} thread(s)")}
    if rank == 0:
        prec = args.precision
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f32 (f16 storage)"}[prec],
            "data": "synthetic",
            "config": dict(tubes_config(args.members), precision=prec, parallelism=f"replicas{world}",
                           schedule=r["schedule"], graph_steps=8, l2="inputs larger than L2 (no flush needed)"),
            "roofline": {"bound": "hbm", "achieved": r["achieved"], "peak": r["peak"], "unit": "GB/s",
                         "frac": r["frac"], "traffic": traffic_for(kernel_digest(BATCH_SOURCES), "tubes", args.members, prec),
                         "peak_source": r["peak_source"],
                         "kernel": "k_step_batch", "bytes_per_launch": r["bytes_per_launch"],
                         "timing": "CUDA events around the timed steps, divided by the steps "
                                   "(includes the small mass-correction reductions)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": r.get("h2d", 0),
                    "d2h_bytes_per_step": r.get("d2h", 0), "steps_per_e2e_step": args.steps,
                    "what": "evd_batch_set_fields(pinned host x) + evd_batch_step(steps) + "
                            "evd_batch_get_mole_fractions(pinned host)"},
            "gpu_launches": r["launches"],
            "clocks": clocks.summary(),
        }
        if "fp64" in r:
            out["vs_fp64_gpu"] = r["fp64"]
        if cpu is not None:
            out["cpu_baseline"] = cpu
        print(json.dumps(out), flush=True)


def measure_single(torch, dev, stream, wl, prec: str, x_dev, steps: int, warmup: int,
                   workload: str = "", size: int = 0) -> dict:
    """One lattice in another storage: CUDA-event time per step over ``steps``
    steps after ``warmup``, the roofline of its step kernel (algorithmic bytes
    of that storage) and the kernel that ran."""
    from paper_2504_07059_gb300 import evd
    sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, prec, stream)
    evd.evd_set_fields_device(sim.ctx, x_dev, None)
    evd.evd_step(sim.ctx, warmup)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    evd.evd_step(sim.ctx, steps)
    b.record(stream)
    torch.cuda.synchronize(dev)
    evd.evd_check(sim.ctx)
    ms = a.elapsed_time(b) / steps
    kernel = "k_step_tma" if evd.evd_get_kernel(sim.ctx) == evd.EVD_KERNEL_TMA else "k_step"
    sim.close()
    peak, peak_kind = measured_peaks()
    bpl = bytes_per_ssu(wl, prec) * wl.ns * wl.nsites
    achieved = bpl / (ms * 1e-3) / 1e9
    return {"precision": prec, "ms_per_step": ms, "value": wl.ns * wl.nsites / (ms * 1e-3) / 1e9, "unit": UNIT,
            "steps": steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind, "kernel": kernel,
                         "bytes_per_launch": bpl,
                         "traffic": traffic_for(kernel_digest(), workload, size, prec) if kernel == "k_step_tma" else None}}


def run_adjoint(args, torch, dev) -> None:
    """Loss and gradient per step of the horizon: forward steps with
    checkpoints, recomputation and the reverse sweep, through the C ABI call
    (host inputs and outputs, allocations included), over ``--horizon`` steps
    with the FP64 and with the FP32 forward pass; the dual-number cross-check
    over a shorter horizon; the FP64 forward step on the same lattice beside
    them (CUDA events)."""
    from paper_2504_07059_gb300 import adjoint as ADJ, evd
    wl = W.loschmidt_ternary_gravity(nx=128, ny=512)
    nsteps = args.horizon
    d = [wl.D[0, 1], wl.D[0, 2], wl.D[1, 2]]
    g = (0.0, wl.g[1])
    stream = torch.cuda.current_stream(dev)

    def problem(n, mode=evd.EVD_ADJOINT_REVERSE, forward="fp64"):
        # target: the same run with every diffusivity x 1.1 and the force x 0.9
        sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, 1.1 * wl.D, wl.tau1,
                             (0.0, 0.9 * wl.g[1]), "fp64", stream)
        sim.set_fields(wl.x)
        sim.step(n)
        target = sim.mole_fractions()[:, 0].mean(axis=2)
        sim.close()
        return ADJ.Problem(wl.shape[:2], wl.wall_mask, wl.M, wl.tau1, wl.x, target, n, mode=mode, forward=forward)

    sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, "fp64", stream)
    sim.set_fields(wl.x)
    evd.evd_step(sim.ctx, args.warmup)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    evd.evd_step(sim.ctx, nsteps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sim.check()
    fwd_ms = e0.elapsed_time(e1) / nsteps
    sim.close()

    def timed(prob):
        warm = ADJ.Problem(prob.shape, prob.wall_mask, prob.molar_mass, prob.tau1, prob.x0, prob.target,
                           args.warmup, mode=prob.mode, forward=prob.forward)
        ADJ.loss_and_gradient(warm, d, g)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        loss, dd, dg = ADJ.loss_and_gradient(prob, d, g)
        return (time.perf_counter() - t0) * 1e3 / prob.nsteps, loss, np.concatenate([dd, dg])

    def rel(a, b):
        return float(np.max(np.abs(a - b) / np.abs(b)))

    full = problem(nsteps)
    ms, loss, grad = timed(full)
    full.forward = "fp32"
    ms32, loss32, grad32 = timed(full)
    nshort = min(nsteps, args.dual_horizon)
    short = problem(nshort)
    ms_rs, _, grad_rs = timed(short)
    short.mode = evd.EVD_ADJOINT_DUAL
    ms_dual, _, grad_dual = timed(short)
    ssu = wl.ns * wl.nsites
    print(json.dumps({
        "metric": "adjoint species-site updates/s (GLUPS)", "value": ssu / (ms * 1e-3) / 1e9, "unit": UNIT,
        "n_gpus": 1, "steps": nsteps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "inverse-problem tube 128x512 ternary D2Q9, gravity, loss + gradient "
                               "w.r.t. 3 D_ij and g", "horizon": nsteps, "checkpoint_every": "ceil(sqrt(steps))"},
        "forward_fp64_ms_per_step": fwd_ms, "reverse_over_forward": ms / fwd_ms,
        "loss": loss, "dL_dD": list(map(float, grad[:3])), "dL_dg": list(map(float, grad[3:])),
        "fp32_forward": {"ms_per_step": ms32, "loss_rel_diff": abs(loss32 - loss) / abs(loss),
                         "grad_norm_rel_diff": float(np.linalg.norm(grad32 - grad) / np.linalg.norm(grad)),
                         "grad_rel_diff": [float(v) for v in np.abs(grad32 - grad) / np.abs(grad)],
                         "note": "per component [dL/dD12, dL/dD13, dL/dD23, dL/dg_x, dL/dg_y]; dL/dg_x is six to "
                                 "nine orders below the others and cancels out of larger terms"},
        "dual_check": {"horizon": nshort, "reverse_ms_per_step": ms_rs, "dual_ms_per_step": ms_dual,
                       "max_rel_diff": rel(grad_rs, grad_dual)},
    }), flush=True)


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2504_07059_gb300 import build, evd
    build.build()
    if args.workload == "adjoint":
        if rank == 0:
            run_adjoint(args, torch, dev)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == "tubes":
        run_tubes(args, torch, dev, world, rank, local)
        if world > 1:
            dist.destroy_process_group()
        return
    wl = make_workload(args.workload, args.size)
    prec = args.precision
    ns, nsites = wl.ns, wl.nsites

    stream = torch.cuda.current_stream(dev)
    sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, prec, stream)
    if args.tile_rows:
        evd.evd_set_tile_rows(sim.ctx, args.tile_rows)
    # inputs resident in HBM before the timed region
    x_dev = torch.from_numpy(np.ascontiguousarray(wl.x)).to(dev)
    evd.evd_set_fields_device(sim.ctx, x_dev, None)
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    evd.evd_step(sim.ctx, args.warmup)
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    launches0 = evd.evd_launch_count(sim.ctx)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_device_id(torch, local)) as clocks:
        start.record(stream)
        evd.evd_step(sim.ctx, args.steps)
        stop.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    ms = start.elapsed_time(stop)
    evd.evd_check(sim.ctx)
    launches = evd.evd_launch_count(sim.ctx) - launches0

    ssu_rank = ns * nsites * args.steps
    ms_max, value = replica_throughput(ms, ssu_rank, dev)

    # roofline of the dominant (only) kernel of the step: algorithmic bytes per
    # launch over the average launch duration (one launch per step)
    peak, peak_kind = measured_peaks()
    bpl = bytes_per_ssu(wl, prec) * ns * nsites
    achieved = bpl / (ms / args.steps * 1e-3) / 1e9
    digest = kernel_digest()
    traffic = traffic_for(digest, args.workload, args.size, prec)

    # end to end through the public API with pinned host buffers: upload the
    # initial mole fractions, run the same number of steps, read the mole
    # fractions back
    x_host = torch.from_numpy(np.ascontiguousarray(wl.x)).pin_memory()
    out_host = torch.empty_like(x_host).pin_memory()
    e2e_times = []
    for _ in range(0 if args.no_e2e else 2):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        evd.evd_set_fields(sim.ctx, x_host, None)
        evd.evd_step(sim.ctx, args.steps)
        evd.evd_get_mole_fractions(sim.ctx, out_host)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = min(e2e_times) if e2e_times else float("nan")
    _, e2e_value = replica_throughput(e2e_s * 1e3, ssu_rank, dev)
    h2d = x_host.numel() * 8
    d2h = out_host.numel() * 8

    kernel_name = "k_step_tma" if evd.evd_get_kernel(sim.ctx) == evd.EVD_KERNEL_TMA else "k_step"
    sim.close()

    # the same workload advanced by the plain FP64 step on the same GPU (a few
    # steps; the FP64 path is ALU-bound on this part)
    fp64 = None
    if prec != "fp64" and not args.no_fp64:
        s64 = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, "fp64", stream)
        evd.evd_set_fields_device(s64.ctx, x_dev, None)
        n64 = max(3, min(args.steps, 20))
        evd.evd_step(s64.ctx, 3)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        evd.evd_step(s64.ctx, n64)
        b.record(stream)
        torch.cuda.synchronize(dev)
        evd.evd_check(s64.ctx)
        ms64 = a.elapsed_time(b) / n64
        s64.close()
        fp64 = {"ms_per_step": ms64, "value": ns * nsites / (ms64 * 1e-3) / 1e9, "unit": UNIT,
                "steps": n64, "speedup": ms64 / (ms / args.steps)}
        # the FP64 step against the double-precision arithmetic roof
        alu = measure_alu_peaks(torch, dev, stream, gpu_device_id(torch, local))
        f64 = flops_for(kernel_digest(), args.workload, "fp64")
        fp64["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "peak": alu["fp64_tflops"],
                            "peak_source": "measured (evd_fma_rate, double FMA chains)",
                            "flops_per_ssu": f64,
                            "achieved": None if f64 is None else f64 * ns * nsites / (ms64 * 1e-3) / 1e12}
        if f64 is not None:
            fp64["roofline"]["frac"] = fp64["roofline"]["achieved"] / alu["fp64_tflops"]
        fp64["alu_peaks"] = alu

    # the other storage and the batched sweep, measured after the headline's
    # timed region: FP16 storage on the same workload, and the 512-tube sweep
    # in FP32 with its FP64 batch beside it
    extras = {}
    if not args.no_extras and args.workload == "stratification" and prec == "fp32":
        extras["fp16"] = measure_single(torch, dev, stream, wl, "fp16", x_dev, min(args.steps, 300), 5,
                                        args.workload, args.size)
        if fp64 is not None:
            extras["fp16"]["speedup_over_fp64"] = fp64["ms_per_step"] / extras["fp16"]["ms_per_step"]
            f32 = flops_for(kernel_digest(), args.workload, "fp16")
            peak32 = max(fp64["alu_peaks"]["fp32_tflops"], fp64["alu_peaks"]["fp32x2_tflops"])
            if f32 is not None:
                a32 = f32 * ns * nsites / (extras["fp16"]["ms_per_step"] * 1e-3) / 1e12
                extras["fp16"]["alu"] = {"bound": "alu", "unit": "TFLOP/s", "flops_per_ssu": f32, "achieved": a32,
                                         "peak": peak32, "frac": a32 / peak32}
        r = measure_tubes(torch, dev, stream, "fp32", min(args.steps, 300), 5, e2e=False, fp64=True)
        extras["tubes"] = {"workload": tubes_config()["workload"], "precision": "fp32",
                           "ms_per_step": r["ms_per_step"], "value": r["value"], "unit": UNIT,
                           "roofline": {"bound": "hbm", "achieved": r["achieved"], "peak": r["peak"],
                                        "unit": "GB/s", "frac": r["frac"], "kernel": "k_step_batch",
                                        "bytes_per_launch": r["bytes_per_launch"],
                                        "traffic": traffic_for(kernel_digest(BATCH_SOURCES), "tubes", 512, "fp32")},
                           "schedule": r["schedule"], "graph_steps": 8,
                           "fp64_ms_per_step": r["fp64"]["ms_per_step"], "speedup_over_fp64": r["fp64"]["speedup"],
                           "config": tubes_config()}

    cpu = cpu_baseline() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    if rank == 0:
        cl = clocks.summary()
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f32 (f16 storage)"}[prec],
            "data": "synthetic",
            "config": dict(wl.describe(), precision=prec, parallelism=f"replicas{world}",
                           l2="inputs larger than L2 (no flush needed)" if bpl > 129e6
                           else "working set fits in L2 (HBM fraction not meaningful)"),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                         "kernel": kernel_name, "bytes_per_launch": bpl,
                         "timing": "CUDA events around the timed steps, divided by the steps "
                                   "(includes the small mass-correction reductions)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps_per_e2e_step": args.steps,
                    "what": "evd_set_fields(pinned host x) + evd_step(steps) + "
                            "evd_get_mole_fractions(pinned host)"},
            "gpu_launches": launches,
            "clocks": cl,
        }
        if fp64 is not None:
            out["vs_fp64_gpu"] = fp64
        out.update(extras)
        if cpu is not None:
            out["cpu_baseline"] = cpu
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["stratification", "tube", "tubes", "adjoint"], default="stratification",
                    help="stratification: 256^3 D3Q19 closed box; tube: 64x1024 ternary D2Q9 tube; "
                         "tubes: the batched sweep of 512 D2Q9 tubes; adjoint: loss and gradient on the "
                         "128x512 ternary inverse-problem tube (one GPU)")
    ap.add_argument("--precision", choices=["fp32", "fp64", "fp16"], default="fp32")
    ap.add_argument("--size", type=int, default=256, help="cube side of the stratification workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip timing the FP64 step for comparison")
    ap.add_argument("--members", type=int, default=512, help="tubes workload: the first N tubes of the sweep")
    ap.add_argument("--schedule", default="", help="tubes workload: 'item_sites,ctas_per_sm' instead of autotuning")
    ap.add_argument("--tile-rows", type=int, default=0, help="rows per tile of the TMA step (1, 2 or 4)")
    ap.add_argument("--horizon", type=int, default=20000, help="adjoint workload: steps of the loss horizon")
    ap.add_argument("--dual-horizon", type=int, default=1000,
                    help="adjoint workload: horizon of the dual-number cross-check")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP16-storage and batched-sweep measurements after the headline")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
