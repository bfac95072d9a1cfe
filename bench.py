#!/usr/bin/env python
"""Benchmark of the sparse-state quantum walk (arXiv 2303.06890) on GB300.

Workload: the quantum walk on a random symmetric N = 16384 matrix with at most
16 non-zeros per column (s = 16), Q1.15 values, random normalised |b>,
complex64 amplitudes (FP32 arithmetic with error-free products and sums in
the merges; FP64 norm and renormalisation), at the size
of the paper's largest walk (Table 1 row E, N = 16384).  One benchmark step
= one walk step W = S T~ P T~^dag of the whole state.

Prints one JSON line: walk steps/s (value), branch entries/s, the plain
FP64-amplitude path on the same workload, the roofline of the step kernel,
the end-to-end rate through the C ABI with host buffers, the CPU oracle's rate
and the SM clocks seen during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own copy of the walk (weak
scaling, no data exchange); the reported time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walk steps/s and sparse-state entries/s at n=16384, FP32 vs FP64; HBM GB/s vs peak"
UNIT = "walk steps/s"
PROFILE = os.path.join(ROOT, "profiles", "k_walk_n16384_s16.md")
PROFILE_SLOT = os.path.join(ROOT, "profiles", "k_walk_slot_n16384_s16.md")
PROFILE_POS = os.path.join(ROOT, "profiles", "k_walk_pos_n16384_s16.md")
KERNEL_SRC = [os.path.join(ROOT, "paper_2303_06890_gb300", "csrc", f) for f in ("qw_kernels.cu", "qw_device.cuh")]
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--fp64-steps", type=int, default=1000)
    p.add_argument("--e2e-jobs", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batched-steps", type=int, default=300)
    p.add_argument("--no-table1", action="store_true")
    p.add_argument("--no-qls", action="store_true")
    p.add_argument("--no-mmax", action="store_true")
    p.add_argument("--no-configs", action="store_true", help="skip the N=16 and N=1024 walk legs")
    p.add_argument("--no-partition", action="store_true", help="skip the row-partitioned walk leg")
    p.add_argument("--no-schedules", action="store_true",
                   help="skip the flat and register-faithful schedule leg")
    p.add_argument("--variant", type=int, default=-1,
                   help="step-kernel variant for both precisions instead of the autotuner's choice (profiling)")
    p.add_argument("--shard", action="store_true",
                   help="under torchrun: one N=16384 walk split in row blocks over the ranks (strong scaling), "
                        "S's sends exchanged by an all-to-all each step, instead of replicas")
    return p.parse_args()


def dist_env():
    from paper_2303_06890_gb300 import ranks
    return ranks.env()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_hash() -> str:
    h = hashlib.sha256()
    for path in KERNEL_SRC:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


VARIANTS = ("rows", "rows, pipelined", "segments", "segments, pipelined", "slot lanes")


def kernel_name(variant: int, amp: str = "float2", s: int = 16) -> str:
    """The step kernel that walk_variant ``variant`` launches."""
    if variant == 4:
        return f"k_walk_slot<{amp}, s = {s}>"
    if variant == 7:
        return f"k_walk_pos<{amp}, s = {s}>"
    return f"k_walk<{amp}, {VARIANTS[variant]}>"


def profiled_traffic(precision: str, variant: int = 0):
    """DRAM bytes per launch of the step kernel (k_walk_pos for variant 7,
    k_walk_slot for variant 4, else k_walk) from the committed ncu summary,
    or None when the kernel source changed since the capture."""
    try:
        text = open({4: PROFILE_SLOT, 7: PROFILE_POS}.get(variant, PROFILE)).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != kernel_hash():
        return None
    key = f"dram_bytes_per_launch_{precision}"
    try:
        return int(float(vals[key]))
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="qw_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def timed_walk(sim, steps: int, torch, flush) -> tuple[float, list[float]]:
    """Per-step device time (CUDA events on the simulator's stream) with an
    untimed L2 flush (a 256 MiB write) before every timed step."""
    stream = torch.cuda.current_stream()
    evs = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.enqueue_walk_steps(1)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    sim.sync()
    ms = [a.elapsed_time(b) for a, b in evs]
    return sum(ms) / 1000.0, ms


def algorithmic_bytes(stats: dict, nb: int, amp_bytes: int) -> tuple[float, float]:
    """Per step: the bytes the interference ops of the step stream if each
    reads its input and writes its output once (R^dag, H P H, R), with
    W_live = ceil((4 nb + 18) / 64) key words; and the bytes the fused kernel
    must move at least (the state read once and written once)."""
    steps = max(1, stats["steps"])
    w_live = -(-(4 * nb + 18) // 64)
    entry = 8 * w_live + amp_bytes
    ops = [(stats["in"], stats["after_rdag"]), (stats["after_rdag"], stats["after_hph"]),
           (stats["after_hph"], stats["out"])]
    if stats["after_h1"]:
        ops = [(stats["in"], stats["after_rdag"]), (stats["after_rdag"], stats["after_h1"]),
               (stats["after_h1"], stats["after_hph"]), (stats["after_hph"], stats["out"])]
    b_alg = sum(i + o for i, o in ops) * entry / steps
    b_min = (stats["in"] + stats["out"]) * (8 + amp_bytes) / steps
    return b_alg, b_min


def _canonical(regs, amps):
    import numpy as np
    regs = np.ascontiguousarray(regs[:, :7], dtype=np.uint64)
    order = np.lexsort(tuple(regs[:, c] for c in range(6, -1, -1)))
    return regs[order], np.asarray(amps)[order]


def state_error(gpu, ref) -> dict:
    """Error of a GPU state against the oracle's, over the union of keys (a
    key held by one side only counts as amplitude 0 on the other): max |da|,
    ||da||_2, and how many keys (and the largest |a| among them) one side
    alone holds."""
    import numpy as np
    (kg, ag), (kr, ar) = _canonical(*gpu), _canonical(*ref)
    both = np.concatenate([kg, kr])
    _, inv = np.unique(both.view(np.dtype((np.void, 56))).ravel(), return_inverse=True)
    inv = inv.ravel()
    m = int(inv.max()) + 1 if inv.size else 0
    vg, vr = np.zeros(m, complex), np.zeros(m, complex)
    hg, hr = np.zeros(m, bool), np.zeros(m, bool)
    vg[inv[:len(kg)]], hg[inv[:len(kg)]] = ag, True
    vr[inv[len(kg):]], hr[inv[len(kg):]] = ar, True
    d = vg - vr
    one = hg ^ hr
    return {"max_abs": float(np.abs(d).max()) if m else 0.0, "l2": float(np.linalg.norm(d)),
            "keys": m, "keys_equal": bool(not one.any()), "one_sided": int(one.sum()),
            "one_sided_max_abs": float((np.abs(vg) + np.abs(vr))[one].max()) if one.any() else 0.0}


def gpu_walk_state(w, precision, steps: int, variant: int | None = None):
    """(regs, amps) of the GPU walk T~ then ``steps`` walk steps (fresh simulator)."""
    from paper_2303_06890_gb300 import qwalk
    kw = {} if variant is None else {"walk_variant": variant}
    sim = qwalk.Sim(w.matrix, s_pad=w.s, precision=precision, **kw)
    sim.state_init(w.b, apply_T=True)
    sim.apply_walk_step(steps)
    keys, amps = sim.state_export(key_words=2 if 4 * sim.nb + 34 <= 128 else 10)
    regs = sim.unpack(keys)
    sim.close()
    return regs, amps


def oracle_walk(w, steps: int):
    """The oracle (plain C, FP64, one thread) on T~ then ``steps`` walk steps:
    its state and its walk-step rate."""
    import oracle
    o = oracle.Oracle(w.matrix, w.s)
    o.init_b(w.b)
    o.apply("T")
    t0 = time.perf_counter()
    for _ in range(steps):
        o.apply("W")
    dt = time.perf_counter() - t0
    return o, dt


def run_sharded(args, rank, world, local_rank):
    """--shard under torchrun: one N = 16384 walk split in row blocks over the
    ranks (one simulator per rank), S's sends exchanged each step by an
    all-to-all (paper_2303_06890_gb300.partition.walk_partitioned over NCCL);
    the metric is walk steps/s of the one walk (strong scaling)."""
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2303_06890_gb300 import partition, qwalk, ranks
    from paper_2303_06890_gb300 import workloads as wl
    w = wl.walk_n16384()
    sim = qwalk.Sim(w.matrix, s_pad=w.s, precision=qwalk.QW_FP32_AMP, walk_variant=4, nparts=world, part=rank)
    sim.state_init(w.b)
    eng = partition.SimEngine(sim, world, rank)
    partition.walk_partitioned(eng, args.warmup)
    torch.cuda.synchronize()
    ranks.barrier()
    t0 = time.perf_counter()
    partition.walk_partitioned(eng, args.steps)
    torch.cuda.synchronize()
    ranks.barrier()
    t = ranks.max_over_ranks(time.perf_counter() - t0, device="cuda")
    sim.close()
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": args.steps / t, "unit": UNIT, "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps,
                          "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                          "data": "synthetic",
                          "config": {"workload": w.name, "n": w.n, "s": w.s, "parallelism": f"row blocks x{world}",
                                     "l2": "not flushed (host-clock timing of whole steps with their exchange)"}}),
              flush=True)
    dist.destroy_process_group()


def run_ours(args, rank, world, local_rank):
    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2303_06890_gb300 import qwalk
    from paper_2303_06890_gb300 import workloads as wl

    w = wl.walk_n16384()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    from paper_2303_06890_gb300 import ranks

    def barrier():
        torch.cuda.synchronize()
        ranks.barrier()

    def max_over_ranks(x: float) -> float:
        return ranks.max_over_ranks(x, device="cuda")

    # --- the benchmarked path: complex64 amplitudes, FP64 merge/norm/renorm ---
    def tuned(precision):
        """a simulator of the workload in T~|b~> with the autotuner's (or the
        requested) step-kernel variant"""
        if args.variant >= 0:
            sm = qwalk.Sim(w.matrix, s_pad=w.s, precision=precision, walk_variant=args.variant)
            sm.state_init(w.b, apply_T=True)
            return sm, args.variant, []
        sm = qwalk.Sim(w.matrix, s_pad=w.s, precision=precision)
        sm.state_init(w.b, apply_T=True)
        v, us = sm.autotune(max(2, args.warmup // 2))  # warm-up steps, all variants
        return sm, v, us

    sim, variant, tune_us = tuned(qwalk.QW_FP32_AMP)
    sim.apply_walk_step(args.warmup)
    sim.step_stats(reset=True)
    launches0 = sim.launch_count()
    clocks = ClockSampler(local_rank)
    barrier()
    t_dev, per_step = timed_walk(sim, args.steps, torch, flush)
    barrier()
    clk = clocks.stop()
    gpu_launches = sim.launch_count() - launches0
    stats = sim.step_stats(reset=True)
    t_max = max_over_ranks(t_dev)
    value = world * args.steps / t_max
    ms_step = 1000.0 * t_max / args.steps
    entries_per_step = (stats["in"] + stats["after_rdag"] + stats["after_hph"]) / max(1, stats["steps"])
    b_alg, b_min = algorithmic_bytes(stats, sim.nb, 8)
    mean_step_s = statistics.mean(per_step) / 1000.0
    peak, peak_kind = peaks()
    achieved = b_alg / mean_step_s / 1e9
    traffic = profiled_traffic("fp32", variant)
    live_entries = stats["out"] / max(1, stats["steps"])
    sim.close()

    # --- the plain FP64 path on the same workload ---
    sim64, variant64, tune64 = tuned(qwalk.QW_FP64)
    sim64.apply_walk_step(args.warmup)
    sim64.step_stats(reset=True)
    barrier()
    t64, per64 = timed_walk(sim64, args.fp64_steps, torch, flush)
    barrier()
    t64 = max_over_ranks(t64)
    stats64 = sim64.step_stats(reset=True)
    b_alg64, _ = algorithmic_bytes(stats64, sim64.nb, 16)
    fp64 = {"value": world * args.fp64_steps / t64, "unit": UNIT, "steps": args.fp64_steps,
            "variant": variant64, "autotune_us_per_step": tune64,
            "ms_per_step": 1000.0 * t64 / args.fp64_steps,
            "entries_per_s": world * (stats64["in"] + stats64["after_rdag"] + stats64["after_hph"]) / t64,
            "achieved_gbs": b_alg64 / statistics.mean(per64) * 1000.0 / 1e9,
            "traffic": profiled_traffic("fp64", variant64)}
    sim64.close()

    # --- end to end through the C ABI with host buffers ---
    import numpy as np
    b_host = torch.from_numpy(np.ascontiguousarray(w.b)).pin_memory()
    probs_host = torch.empty(w.n, dtype=torch.float64).pin_memory()
    sim_e = qwalk.Sim(w.matrix, s_pad=w.s, precision=qwalk.QW_FP32_AMP, walk_variant=variant)
    steps_per_job = w.steps
    sim_e.state_init(b_host.numpy(), apply_T=True)
    sim_e.apply_walk_step(2)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_jobs):
        sim_e.state_init(b_host.numpy(), apply_T=True)  # H2D of |b> from pinned memory
        sim_e.enqueue_walk_steps(steps_per_job)
        sim_e.measure_register("j", w.n, out=probs_host.numpy())  # D2H of the marginal, synchronises
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    sim_e.close()
    e2e = {"value": world * args.e2e_jobs * steps_per_job / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": w.n * 8 / steps_per_job,
           "d2h_bytes_per_step": w.n * 8 / steps_per_job,
           "job": f"qw_state_init(|b> from pinned host memory, T~) + qw_enqueue_walk_steps({steps_per_job}) "
                  f"+ qw_measure_register(j) into pinned host memory"}

    batched = None if args.no_batched else batched_leg(args, torch, flush, barrier, max_over_ranks,
                                                       world, rank)

    table1 = None if args.no_table1 else table1_leg(torch, barrier, max_over_ranks)
    part = None if (args.no_partition or world > 1) else partition_leg(torch)
    sched = None if args.no_schedules else schedules_leg(torch)
    qls = None if args.no_qls else qls_leg(torch, barrier, max_over_ranks)
    mmax = None if args.no_mmax else mmax_leg()

    cpu, err = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle walks the benchmarked workload (T~ + its 20 steps, ~10 s on
        # one core): its rate is the CPU baseline, its state the reference of
        # the per-result error of both GPU precisions (fresh walks of 20 steps,
        # outside every timed region)
        o, dt = oracle_walk(w, w.steps)
        cpu = {"value": w.steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the whole {w.steps}-step N=16384 walk after T~ ({dt:.1f} s, {o.size()} branches), "
                         f"plain C FP64 register-level oracle, one thread"}
        ref = o.export()
        err = {"walk_n16384_complex64_20_steps": state_error(gpu_walk_state(w, qwalk.QW_FP32_AMP, w.steps, variant),
                                                              ref),
               "walk_n16384_complex128_20_steps": state_error(gpu_walk_state(w, qwalk.QW_FP64, w.steps), ref),
               "walk_n16384_flat_complex128_20_steps": state_error(gpu_walk_state(w, qwalk.QW_FP64, w.steps, 5),
                                                                   ref),
               "walk_n16384_faithful_complex128_20_steps": state_error(
                   gpu_walk_state(w, qwalk.QW_FP64, w.steps, 6), ref),
               "bounds": {"complex128": "keys equal, max |da| <= 1e-12",
                          "complex64": "max |da| <= 2e-6, ||da||_2 <= 1e-5 over the union of keys"}}
        del o
        if not args.no_configs:
            err.update(configs_leg(torch))

    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "s": w.s, "nnz": int(w.matrix.nnz),
                   "amplitudes": "complex64 in HBM; FP32 arithmetic with error-free products and "
                                 "sums (~48-bit float pairs) in the rotations and the reflection sum; "
                                 "FP64 norm and renormalisation",
                   "steps_per_walk": w.steps, "branches_per_step": live_entries,
                   "l2": "flushed before every timed step (256 MiB write, untimed)",
                   "parallelism": f"replicas x{world}"},
        "entries_per_s": world * entries_per_step / (t_max / args.steps),
        "fp64": fp64,
        "fp32_speedup_vs_fp64": value / fp64["value"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": kernel_name(variant),
                     "autotune_us_per_step": tune_us,
                     "algorithmic_bytes_per_launch": b_alg,
                     "state_bytes_per_launch": b_min,
                     "state_gbs": b_min / mean_step_s / 1e9},
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clk,
    }
    if batched is not None:
        line["batched"] = batched
    if table1 is not None:
        line["table1"] = table1
    if qls is not None:
        line["qls"] = qls
    if mmax is not None:
        line["mmax"] = mmax
    if part is not None:
        line["partitioned"] = part
    if sched is not None:
        line["schedules"] = sched
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if err is not None:
        line["error_vs_oracle"] = err
    print(json.dumps(line), flush=True)


def batched_leg(args, torch, flush, barrier, max_over_ranks, world, rank) -> dict:
    """256 independent walks (N log-uniform in [64, 4096], s = 8) advanced
    together, one k_walk launch per step: kernel time per step (L2 flushed
    before each timed step), the whole 50-step walk as CUDA-graph replays,
    and the same instances walked one at a time by the plain complex128 path
    and by the complex64 path (the gain of batching alone).
    Each rank runs its own 256 instances (weak scaling)."""
    from paper_2303_06890_gb300 import qwalk
    from paper_2303_06890_gb300 import ranks
    from paper_2303_06890_gb300 import workloads as wl

    ws = wl.batched(256, first=ranks.instance_seed_offset(rank, 256))
    sim = qwalk.Sim([w.matrix for w in ws], s_pad=8, precision=qwalk.QW_FP32_AMP)
    nb = sim.nb
    for i, w in enumerate(ws):
        sim.state_init(w.b, inst=i)
    variant, tune = sim.autotune(3)
    sim.apply_walk_step(6)
    sim.step_stats(reset=True)
    barrier()
    t_dev, per = timed_walk(sim, args.batched_steps, torch, flush)
    barrier()
    stats = sim.step_stats(reset=True)
    t_dev = max_over_ranks(t_dev)
    # whole walks: re-initialise, 50 steps issued as graph replays, one event pair
    for i, w in enumerate(ws):
        sim.state_init(w.b, inst=i)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e0.record()
    sim.enqueue_walk_steps(50)
    e1.record()
    torch.cuda.synchronize()
    sim.sync()
    t_walk = max_over_ranks(e0.elapsed_time(e1) / 1000.0)
    sim.close()
    # the same instances walked one at a time, by the plain complex128 path and
    # by the complex64 path (instances after the first 64 are timed on a
    # stride-4 sample and scaled by the instance count)
    def sequential(precision) -> float:
        t = 0.0
        sample = list(range(0, 256, 4))
        for i in sample:
            w = ws[i]
            s1 = qwalk.Sim(w.matrix, s_pad=8, precision=precision)
            s1.state_init(w.b)
            s1.apply_walk_step(2)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            s1.enqueue_walk_steps(50)
            a1.record()
            torch.cuda.synchronize()
            s1.sync()
            t += a0.elapsed_time(a1) / 1000.0
            s1.close()
        return max_over_ranks(t * 256 / len(sample))

    t_seq = sequential(qwalk.QW_FP64)
    t_seq32 = sequential(qwalk.QW_FP32_AMP)
    # error of the complex64 batched walk against each instance's oracle, on
    # the smallest, a middle and the largest instance (after 50 steps)
    err = {}
    if rank == 0:
        sim = qwalk.Sim([w.matrix for w in ws], s_pad=8, precision=qwalk.QW_FP32_AMP, walk_variant=variant)
        for i, w in enumerate(ws):
            sim.state_init(w.b, inst=i)
        sim.apply_walk_step(50)
        by_size = sorted(range(len(ws)), key=lambda i: ws[i].n)
        for i in (by_size[0], by_size[len(ws) // 2], by_size[-1]):
            keys, amps = sim.state_export(inst=i)
            o, _ = oracle_walk(ws[i], 50)
            err[f"instance_{i}_n{ws[i].n}"] = state_error((sim.unpack(keys), amps), o.export())
        sim.close()
    steps = max(1, stats["steps"])
    b_alg, _ = algorithmic_bytes(stats, nb, 8)
    t_step = t_dev / args.batched_steps
    return {"workload": "batched_256_n64-4096_s8", "instances": 256,
            "branches_per_step": stats["out"] / steps,
            "entries_per_s": world * (stats["in"] + stats["after_rdag"] + stats["after_hph"]) / steps / t_step,
            "achieved_gbs": world * b_alg / t_step / 1e9,
            "steps_per_s": world * args.batched_steps / t_dev,
            "instance_steps_per_s": world * 256 * args.batched_steps / t_dev,
            "ms_per_step": 1000.0 * t_dev / args.batched_steps,
            "variant": variant, "autotune_us_per_step": tune,
            "walk_50_steps_ms_graph": 1000.0 * t_walk,
            "sequential_fp64_walk_50_steps_ms": 1000.0 * t_seq,
            "speedup_vs_sequential_fp64": t_seq / t_walk,
            "sequential_fp32_walk_50_steps_ms": 1000.0 * t_seq32,
            "speedup_vs_sequential_same_precision": t_seq32 / t_walk,
            "error_vs_oracle_complex64_50_steps": err}


# Table 1: average time per walk step of the paper's simulator on one core of
# a Xeon E5-2680 (context only: another machine, and the paper's matrices).
TABLE1_PAPER_S_PER_STEP = {"A": 1.1e-3, "B": 12e-3, "C": 1.2, "D": 14.0, "E": 66.0}


def _events_time(torch, fn) -> float:
    """Device seconds of the work ``fn`` enqueues on the current stream."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0


def mmax_leg(steps: int = 12) -> dict:
    """The largest number of branches M_max the walk reaches (the state after
    T~ and after each interference op of every step, counted on the device),
    against N at fixed s and against s at fixed N, on full positive band
    matrices (Sec. V-B), complex128 -- the scan of Fig. 10 -- with the log-log
    slopes between the ends of each scan."""
    import math
    import numpy as np
    from paper_2303_06890_gb300 import qwalk
    from paper_2303_06890_gb300 import workloads as wl

    def m_max(n: int, s: int) -> int:
        m = wl.band_positive(n, s // 2 - 1, 8, seed=900 + n + s)
        b = np.random.default_rng(901 + n).uniform(0.0, 1.0, n)
        sim = qwalk.Sim(m, s_pad=s)
        sim.state_init(b / np.linalg.norm(b))
        best = sim.state_size()
        sim.step_stats(reset=True)
        for _ in range(steps):
            sim.apply_walk_step(1)
            st = sim.step_stats(reset=True)
            best = max(best, st["in"], st["after_rdag"], st["after_hph"], st["out"])
        sim.close()
        return int(best)

    def slope(xs, ys):
        return math.log(ys[-1] / ys[0]) / math.log(xs[-1] / xs[0])

    out = {"steps": steps, "versus_n": {}, "versus_s": {}}
    for s in (4, 8):
        ns = [256, 1024, 4096, 16384]
        ms = [m_max(n, s) for n in ns]
        out["versus_n"][f"s={s}"] = {"n": ns, "m_max": ms, "slope": slope(ns, ms)}
    ss = [4, 8, 16, 32, 64]
    ms = [m_max(4096, s) for s in ss]
    out["versus_s"]["n=4096"] = {"s": ss, "m_max": ms, "slope": slope(ss, ms)}
    return out


def table1_leg(torch, barrier, max_over_ranks) -> dict:
    """Walk steps on the band matrices shaped like Table 1 (A..E, Sec. V-B),
    complex128 and complex64, autotuned, steps issued back to back as graph
    replays (the state stays resident; no L2 flush: consecutive steps of one
    walk), beside the paper's single-core time per step; and the same walk on
    the paper's literal schedule (flat path and register-faithful, complex128,
    wall clock per step)."""
    from paper_2303_06890_gb300 import qwalk
    from paper_2303_06890_gb300 import workloads as wl

    out = {}
    for name in "ABCDE":
        w = wl.table1(name)
        steps = 600 if w.n <= 1024 else 60
        row = {"n": w.n, "s": w.s, "word": wl.TABLE1[name][1], "nnz": int(w.matrix.nnz),
               "paper_s_per_step": TABLE1_PAPER_S_PER_STEP[name]}
        for label, prec in (("fp64", qwalk.QW_FP64), ("fp32", qwalk.QW_FP32_AMP)):
            sim = qwalk.Sim(w.matrix, s_pad=w.s, precision=prec)
            sim.state_init(w.b)
            variant, _ = sim.autotune(2 if w.n > 1024 else 6)
            sim.apply_walk_step(6)
            sim.step_stats(reset=True)
            barrier()
            t = max_over_ranks(_events_time(torch, lambda: sim.enqueue_walk_steps(steps)))
            sim.sync()
            st = sim.step_stats(reset=True)
            sim.close()
            row[label] = {"us_per_step": 1e6 * t / steps, "variant": variant,
                          "branches_per_step": st["out"] / max(1, st["steps"]),
                          "entries_per_s": (st["in"] + st["after_rdag"] + st["after_hph"]) / t}
        row["paper_over_fp64"] = row["paper_s_per_step"] / (row["fp64"]["us_per_step"] * 1e-6)
        # the paper's own schedule (complex128): the flat path and the
        # register-faithful one, whose keys hold Alg. 1's registers and stack
        # as the paper's simulator does; wall clock (the host synchronises
        # between their stages)
        for label, variant in (("flat", 5), ("faithful", 6)):
            sim = qwalk.Sim(w.matrix, s_pad=w.s, walk_variant=variant)
            sim.state_init(w.b)
            sim.apply_walk_step(2)
            sim.step_stats(reset=True)
            nst = 4
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.apply_walk_step(nst)
            torch.cuda.synchronize()
            dt = max_over_ranks(time.perf_counter() - t0)
            st = sim.step_stats(reset=True)
            sim.close()
            row[label] = {"ms_per_step": 1e3 * dt / nst, "branches_per_step": st["out"] / max(1, st["steps"])}
        row["paper_over_faithful"] = row["paper_s_per_step"] / (row["faithful"]["ms_per_step"] * 1e-3)
        out[name] = row
    return out


def _cks_theory(w, coeffs):
    """Y_j = sum_{i<=j} a_i T_{2i+1}(A/s) b and p_j = ||Y_j||^2 in FP64 (the
    identity before Eq. (fx)), by the three-term recurrence on the sparse A/s."""
    import numpy as np
    import scipy.sparse as sp
    m = w.matrix
    a = sp.csc_matrix((m.val_q15.astype(np.float64) / 32768.0 / w.s, m.rowidx, m.colptr), shape=(m.n, m.n)).tocsr()
    t_prev, t_cur = w.b.astype(np.float64), a @ w.b
    y = coeffs[0] * t_cur
    p = np.empty(len(coeffs))
    p[0] = y @ y
    for j in range(1, len(coeffs)):
        t_prev, t_cur = t_cur, 2.0 * (a @ t_cur) - t_prev
        t_prev, t_cur = t_cur, 2.0 * (a @ t_cur) - t_prev
        y = y + coeffs[j] * t_cur
        p[j] = y @ y
    return y, p


def qls_leg(torch, barrier, max_over_ranks) -> dict:
    """The CKS solver (Sec. IV, Eq. (fx)) end to end through qw_apply_qls:
    * the cond(A) = 100 N = 1024 system with complex64 amplitudes, at its own
      j0 and at Table 1 C's kappa = 5000 (j0 = 106122, the 212245 walk steps
      the paper ran for 70 h on one core); the wider interval [1/5000, 1]
      still covers the spectrum, so the solution stays accurate;
    * matrix C of Table 1 (N = 1024, s = 32, kappa 4907) in complex128 at its
      own j0.
    Fidelity |<x|y>|^2 / ||y||^2 against x = A^-1 b / ||A^-1 b|| from a dense
    FP64 solve (numpy); p_succ = ||Y||^2 / (sum |a_j|)^2."""
    import numpy as np
    from paper_2303_06890_gb300 import qwalk
    from paper_2303_06890_gb300 import workloads as wl

    runs = [("qls_n1024_own_j0", wl.qls_n1024(), None, qwalk.QW_FP32_AMP),
            ("qls_n1024_kappa5000", wl.qls_n1024(), 5000.0, qwalk.QW_FP32_AMP),
            ("table1_C_own_j0", wl.table1("C", steps=0), None, qwalk.QW_FP64)]
    out = {}
    for label, w, kappa, prec in runs:
        kappa = w.kappa if kappa is None else kappa
        coeffs, j0, _ = qwalk.cks_coefficients(kappa, 1e-3)
        sim = qwalk.Sim(w.matrix, s_pad=w.s, precision=prec)
        sim.state_init(w.b)
        variant, _ = sim.autotune(2)  # the step kernel the solve runs
        sim.step_stats(reset=True)
        barrier()
        t0 = time.perf_counter()
        sim.state_init(w.b)
        y, p = sim.apply_qls(coeffs)
        t = max_over_ranks(time.perf_counter() - t0)
        st = sim.step_stats(reset=True)
        sim.close()
        x = np.linalg.solve(w.matrix.dense(), w.b)
        x /= np.linalg.norm(x)
        fid = float(abs(np.vdot(x, y)) ** 2 / np.vdot(y, y).real)
        # the dense FP64 theory of the same run: Y = sum_j a_j T_{2j+1}(A/s) b
        # by the Chebyshev recurrence (sparse A/s), p_j = ||Y_j||^2 at every j
        y_th, p_th = _cks_theory(w, coeffs)
        fid_th = float(abs(np.vdot(x, y_th)) ** 2 / np.vdot(y_th, y_th).real)
        out[label] = {"n": w.n, "s": w.s, "kappa_walk": w.kappa, "kappa_coefficients": kappa,
                      "j0": j0, "walk_steps": 2 * (j0 + 1),
                      "precision": "complex64" if prec == qwalk.QW_FP32_AMP else "complex128",
                      "seconds": t, "walk_steps_per_s": 2 * (j0 + 1) / t, "variant": variant,
                      "entries_per_s": (st["in"] + st["after_rdag"] + st["after_hph"]) / t,
                      "fidelity": fid,
                      "p_succ": float(p[-1] / np.abs(coeffs).sum() ** 2),
                      "error_vs_dense_theory": {
                          "abs_dF": abs(fid - fid_th),
                          "max_rel_dp_j": float(np.max(np.abs(p - p_th) / p_th)),
                          "rel_dY": float(np.linalg.norm(y - y_th) / np.linalg.norm(y_th))}}
    return out


def partition_leg(torch, steps: int = 24) -> dict:
    """The N = 16384 walk split in row blocks among P simulators of this
    process on one device (qw_part_walk: each step runs every part's step
    kernel, then appends S's sends to each part straight from the others'
    outboxes and sets the renormalisation from the summed norms, all on the
    device; one synchronisation per call), complex64: walk steps/s of the
    whole walk and the branches each part holds.  An emulation of the
    multi-GPU partition on one device: the parts share its SMs."""
    from paper_2303_06890_gb300 import partition, qwalk
    from paper_2303_06890_gb300 import workloads as wl
    w = wl.walk_n16384()
    out = {"workload": w.name, "precision": "complex64", "steps": steps}
    for nparts in (2, 4):
        sims = [qwalk.Sim(w.matrix, s_pad=w.s, precision=qwalk.QW_FP32_AMP, walk_variant=4, nparts=nparts, part=p)
                for p in range(nparts)]
        for sim in sims:
            sim.state_init(w.b)
        partition.walk_in_process(sims, 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        partition.walk_in_process(sims, steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sizes = [sim.state_size() for sim in sims]
        for sim in sims:
            sim.close()
        out[f"p{nparts}"] = {"walk_steps_per_s": steps / dt, "ms_per_step": 1000.0 * dt / steps,
                             "branches_per_part": sizes}
    return out


def schedules_leg(torch, steps: int = 6) -> dict:
    """The N = 16384 walk (complex128) on the paper's literal schedule: the
    flat path (walk_variant 5: one list of 16-byte keys, every interference
    op a global radix sort, a per-group transform and a compaction) and the
    register-faithful one (walk_variant 6: 80-byte keys holding the QRAM
    address and Alg. 1's registers and stack, the 58 sub-operations of W).
    Wall-clock per step (the host synchronises between stages), branches
    through the step per second, and the key bytes a branch carries."""
    from paper_2303_06890_gb300 import qwalk
    from paper_2303_06890_gb300 import workloads as wl
    w = wl.walk_n16384()
    out = {"workload": w.name, "precision": "complex128", "steps": steps}
    for variant, name, key_bytes in ((5, "flat", 16), (6, "faithful", 80)):
        sim = qwalk.Sim(w.matrix, s_pad=w.s, walk_variant=variant)
        sim.state_init(w.b)
        sim.apply_walk_step(2)
        sim.step_stats(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.apply_walk_step(steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = sim.step_stats(reset=True)
        row = {"ms_per_step": 1000.0 * dt / steps, "walk_steps_per_s": steps / dt,
               "branches_per_s": (st["in"] + st["after_rdag"] + st["after_h1"] + st["after_hph"]) / dt,
               "key_bytes_per_branch": key_bytes}
        if variant == 6:
            row.update(sim.faithful_info())
        sim.close()
        out[name] = row
    return out


def configs_leg(torch) -> dict:
    """The two small walk workloads: N = 16 (10 steps, complex128) and N = 1024
    (100 steps, complex128 and complex64).  Per workload and precision: the
    autotuned step kernel, the device time per step of the whole walk issued
    as graph replays (state resident), and the error of the final state
    (a fresh walk on that kernel) against the oracle's."""
    from paper_2303_06890_gb300 import qwalk
    from paper_2303_06890_gb300 import workloads as wl
    out = {}
    for w, precs in ((wl.walk_n16(), (qwalk.QW_FP64,)), (wl.walk_n1024(), (qwalk.QW_FP64, qwalk.QW_FP32_AMP))):
        o, dt = oracle_walk(w, w.steps)
        ref = o.export()
        row = {"n": w.n, "s": w.s, "steps": w.steps, "oracle_s_per_step": dt / w.steps}
        for prec in precs:
            label = "complex128" if prec == qwalk.QW_FP64 else "complex64"
            sim = qwalk.Sim(w.matrix, s_pad=w.s, precision=prec)
            sim.state_init(w.b)
            variant, _ = sim.autotune(2)
            sim.apply_walk_step(6)
            sim.step_stats(reset=True)
            reps = 20
            t = _events_time(torch, lambda: [sim.enqueue_walk_steps(w.steps) for _ in range(reps)])
            sim.sync()
            st = sim.step_stats(reset=True)
            b_alg, _ = algorithmic_bytes(st, sim.nb, 8 if prec == qwalk.QW_FP32_AMP else 16)
            sim.close()
            us = 1e6 * t / (reps * w.steps)
            row[label] = {"us_per_step": us, "variant": variant,
                          "entries_per_s": (st["in"] + st["after_rdag"] + st["after_hph"]) / t,
                          "achieved_gbs": b_alg / us * 1e6 / 1e9,
                          "error": state_error(gpu_walk_state(w, prec, w.steps, variant), ref)}
        out[w.name] = row
    return out


def run_reference(args, rank, world):
    """The oracle timed as the reference arm: rank 0 only, bounded sample."""
    if rank != 0:
        return
    from paper_2303_06890_gb300 import workloads as wl
    import oracle

    w = wl.walk_n16384()
    o = oracle.Oracle(w.matrix, w.s)
    o.init_b(w.b)
    o.apply("T")
    for _ in range(min(args.warmup, 1)):
        o.apply("W")
    budget = 60.0
    steps, t0 = 0, time.perf_counter()
    while steps < max(1, args.steps) and (steps < 1 or time.perf_counter() - t0 < budget):
        o.apply("W")
        steps += 1
    dt = time.perf_counter() - t0
    v = steps / dt
    sample = (f"{steps} of the requested {args.steps} walk steps (60 s budget) of the N=16384 walk, "
              f"after T~ and {min(args.warmup, 1)} warm-up step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": min(args.warmup, 1), "ms_per_step": 1000.0 * dt / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "n": w.n, "s": w.s},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse_args()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.shard and world > 1:
        run_sharded(args, rank, world, local_rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
