"""Benchmark of the minimal-Tersoff hot path on one GB300 (or N replicas under torchrun).

Workload (the GA fitness batch): P = 200 parameter sets (genes uniform within +-30 % of Table 2) x
C = 300 periodic 64-atom diamond-Si cells (strain +-2 %, displacements sigma = 0.1 A), targets = the
FP64 E/F/W of the Table 2 parameters plus Gaussian noise (1 meV/atom, 5 meV/atom, 0.02 eV/A).

One step = one GA generation's fitness evaluation done from scratch: neighbour build and geometry
cache of all 300 cells, then E/F/W and the fitness Z of every parameter set (FP32 pair arithmetic,
FP64 reductions). metric = atom-evals/s (P x total atoms per step / time).

Prints one JSON line (rank 0). The roofline block rates the batched E/F/W kernel, timed alone by CUDA
events on its stream, against the FP32 ALU peak (the kernel does no dense contraction and reads a few
MB of geometry per launch).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "atom-evals/sec (E+F+W)"
UNIT = "atom-evals/s"
L2_BYTES = 129 * 1024 * 1024

# Algorithmic operations of one atom evaluation, counted by running the formula listing of the method
# (site terms of Eq. 2-10, the derivative of the site energy with respect to its bond vectors, the
# force gather, the virial and the force residual) through an op-counting scalar (oracle/flops.py;
# tests/test_flop_model.py checks these constants against it). +, -, *, / count 1 FLOP (an FMA 2);
# exp and log are transcendental (XU) ops. For an atom with m bonds:
#   FLOP = FLOP_PER_BOND m + FLOP_PER_TRIPLET m (m - 1) + FLOP_PER_ATOM, plus FLOP_PER_CONFIG per
#   configuration; XU = XU_PER_BOND m.  Diamond (m = 4): 654 FLOP and 24 XU ops per atom-evaluation.
FLOP_PER_BOND = 50.0
FLOP_PER_TRIPLET = 37.0
FLOP_PER_ATOM = 10.0
FLOP_PER_CONFIG = -2
XU_PER_BOND = 6
# The MD-scale call computes the bond geometry every step (bond vector, length, unit vector, pair
# cosines; its cells have every bond inside R1): 744 FLOP and 28 XU ops per 4-neighbour atom.
MD_FLOP_PER_BOND = 65.0
MD_FLOP_PER_TRIPLET = 39.5
MD_FLOP_PER_ATOM = 10.0
MD_XU_PER_BOND = 7
# Algorithmic bytes of the MD-scale call per atom: FP64 positions in, forces out (FP32 or FP64).
MD_BYTES_IN = 24
# The parameter gradient as forward-mode dual arithmetic with the six parameter tangents over the same
# listing (the plain method of Sec. III's loss gradient): 9398 FLOP per 4-neighbour atom-evaluation.
ADJ_FLOP_PER_BOND = 718.0
ADJ_FLOP_PER_TRIPLET = 541.0
ADJ_FLOP_PER_ATOM = 34.0
ADJ_FLOP_PER_CONFIG = -14
ADJ_XU_PER_BOND = 6

# ncu summary holding the batched kernel's DRAM bytes per launch, valid while these sources are unchanged
TRAFFIC_PROFILE = "batch_kernel_ga_fitness_P200_C300.md"
TRAFFIC_SOURCES = ("batch_kernel.cuh", "batch.cu", "batch_launch.cuh", "common.cuh", "dual.cuh", "ctx.hpp")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if ts < t0 or ts > t1:
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_sources_digest():
    """SHA-256 over the sources the batched kernel is compiled from."""
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1909_11474_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic():
    """DRAM bytes per launch of the batched kernel from the committed ncu summary, or None when the
    kernel's sources changed after that capture."""
    p = os.path.join(ROOT, "profiles", TRAFFIC_PROFILE)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        for line in f:
            m = re.match(r"^traffic: dram_bytes_per_launch=(\d+) kernel_sources_sha256=([0-9a-f]{64})\s*$", line)
            if m:
                return int(m.group(1)) if m.group(2) == kernel_sources_digest() else None
    return None


def executed_block(b_time, fp32_peak):
    """The FP32 arithmetic the kernel executes (not the algorithmic model) against the same peak: how
    busy the FP32 lanes are. The kernel folds the method's formulas (sums of unit vectors before the
    projection, constants folded), so it executes fewer FLOP than the formula listing counts."""
    ex = profiled_executed_flop()
    if ex is None:
        return None
    a = ex / b_time / 1e12
    return {"flop_per_launch": ex, "achieved": round(a, 3), "frac": round(a / fp32_peak, 4),
            "source": "ncu thread-instruction counters of the committed profile (FFMA, FADD, FMUL and packed forms)"}


def profiled_executed_flop():
    """FP32 FLOP the batched kernel executes per launch (ncu instruction counters, committed in the
    profile summary: 2 FFMA + FADD + FMUL + 4 FFMA2 + 2 FADD2 + 2 FMUL2 per thread instruction), or None
    when the kernel's sources changed after that capture."""
    p = os.path.join(ROOT, "profiles", TRAFFIC_PROFILE)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        for line in f:
            m = re.match(r"^executed_fp32: flop_per_launch=(\d+) kernel_sources_sha256=([0-9a-f]{64})\s*$", line)
            if m:
                return int(m.group(1)) if m.group(2) == kernel_sources_digest() else None
    return None


def flop_model(ctx, P):
    """Algorithmic FLOP and XU ops of one fitness evaluation over all (p, c), and the bond and ordered
    bond-pair counts of the build."""
    N, B, _ = ctx.build_info()
    cnt = np.minimum(ctx.export_neighbors()[0].astype(np.int64), ctx.max_nbr)
    triplets = int((cnt * (cnt - 1)).sum())
    flop = P * (FLOP_PER_BOND * B + FLOP_PER_TRIPLET * triplets + FLOP_PER_ATOM * N + FLOP_PER_CONFIG * ctx.C)
    xu = P * XU_PER_BOND * B
    return flop, xu, B, triplets


def run_ours(args):
    import torch

    from paper_1909_11474_gb300 import binding
    from paper_1909_11474_gb300 import inputs as I

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = I.workload_ga_batch(P=args.P, C=args.C)
    cs = w["configs"]
    P = len(w["params"])
    ctx = binding.Context(local)
    pos = torch.tensor(cs.pos, device=dev)
    box = torch.tensor(cs.box, device=dev)
    params = torch.tensor(w["params"], device=dev)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    # targets: FP64 E/F/W of the hidden (Table 2) parameter set from the library's FP64 path
    Eh, Fh, Wh = ctx.eval(torch.tensor(w["hidden"][None, :], device=dev), precision=64)
    natoms = torch.tensor(cs.natoms, device=dev, dtype=torch.float64)
    ne, nw, nf = w["noise"]
    tg = {"E": (Eh[0] / natoms + torch.tensor(ne, device=dev)).contiguous(),
          "W": (Wh[0] / natoms[:, None] + torch.tensor(nw, device=dev)).contiguous(),
          "F": (Fh[0] + torch.tensor(nf, device=dev)).contiguous(),
          "mask": torch.full((cs.C,), 7, dtype=torch.uint8, device=dev)}
    flop, xu, nbonds, ntrip = flop_model(ctx, P)
    atom_evals = P * cs.Ntot
    # arithmetic throughput of this device by the library's microbenchmarks (FFMA, FP64, XU chains)
    mpeaks = binding.measure_peaks(local)
    # the library's E/F/W of every (p, c) in FP32 and FP64, compared with the oracle on the CPU baseline's
    # sample after the timed region
    want_cpu = rank == 0 and ws == 1 and not args.no_cpu
    gpu_out = None
    if want_cpu:
        gpu_out = {}
        for prec in (32, 64):
            E_, F_, W_ = ctx.eval(params, precision=prec)
            gpu_out[prec] = (E_.cpu().numpy(), F_.double().cpu().numpy(), W_.cpu().numpy())
        E_, F_, W_ = ctx.eval(torch.tensor(w["hidden"][None, :], device=dev), precision=32)
        gpu_out["hidden32"] = (E_.cpu().numpy(), F_.double().cpu().numpy(), W_.cpu().numpy())
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    Zbuf = (torch.empty(P, dtype=torch.float64, device=dev), torch.empty((P, 3), dtype=torch.float64, device=dev),
            torch.empty((P, 3), dtype=torch.float64, device=dev))

    def step():
        ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
        ctx.fitness(params, tg, precision=32, out=Zbuf)

    def fitness_only():
        ctx.fitness(params, tg, precision=32, out=Zbuf)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    # the library's schedule autotuner, once per (build, P), before the timed region; or a fixed
    # schedule (tile, warps, items per configuration, narrow), e.g. to profile one variant
    if args.schedule:
        tile, warps, items, narrow = (int(v) for v in args.schedule.split(","))
        ctx.set_schedule(P, tile=tile, items_per_config=items, narrow=bool(narrow), precision=32, warps=warps)
        tuned_ms, tuned_tried = float("nan"), 0
    else:
        tuned_ms, tuned_tried = ctx.autotune(params, tg, precision=32, reps=3)
    for _ in range(2):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    sampler.start()
    time.sleep(0.5)
    t_clock0 = time.time()
    # soak: keep the GPU under the same load for a moment so the clock samples see it
    t_end = time.time() + args.soak
    while time.time() < t_end:
        for _ in range(20):
            fitness_only()
        torch.cuda.synchronize()

    def timed(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a, b in ev:
            flush.fill_(1.0)                       # L2 flush between timed iterations
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    n0 = ctx.kernel_launches()
    t_step = timed(step, args.steps)
    launches = ctx.kernel_launches() - n0
    t_build = timed(lambda: ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16), args.steps)
    ctx.build_info()                              # the host side of the last build
    t_fit = timed(fitness_only, args.steps)       # the fitness call as a user makes it (graph replay)
    ctx.profile(True)                             # CUDA events around the batched kernel alone
    timed(fitness_only, args.steps)               # (direct launches while the events are on)
    n_kern, ms_kern = ctx.profile_read()
    ctx.profile(False)
    torch.cuda.synchronize()
    t_clock1 = time.time()
    clocks = sampler.stop(t_clock0, t_clock1)
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_step, t_fit], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step, t_fit = float(tt[0]), float(tt[1])

    ms_step = 1e3 * t_step / args.steps
    value = ws * atom_evals * args.steps / t_step
    fit_value = ws * atom_evals * args.steps / t_fit

    # end to end: host buffers -> device, full step, Z back to host (pinned memory). The step's inputs
    # (positions, boxes, parameters, targets) sit in one pinned host buffer and go over in one copy
    # into one device buffer, whose slices are the arrays the calls take
    host_arrays = [("pos", torch.tensor(cs.pos)), ("box", torch.tensor(cs.box)), ("params", torch.tensor(w["params"]))]
    host_arrays += [("tg_" + k, v.cpu()) for k, v in tg.items()]
    offs, total = [], 0
    for _, a in host_arrays:
        offs.append(total)
        total += (a.numel() * a.element_size() + 255) // 256 * 256
    h_in = torch.zeros(total, dtype=torch.uint8).pin_memory()
    d_in = torch.empty(total, dtype=torch.uint8, device=dev)
    views = {}
    for (name, a), o in zip(host_arrays, offs):
        nb = a.numel() * a.element_size()
        h_in[o:o + nb].copy_(a.contiguous().view(-1).view(torch.uint8))
        views[name] = d_in[o:o + nb].view(a.dtype).view(a.shape)
    e_pos, e_box, e_par = views["pos"], views["box"], views["params"]
    d_tg = {k: views["tg_" + k] for k in tg}
    h_Z = torch.empty(P, dtype=torch.float64).pin_memory()

    def e2e_step():
        d_in.copy_(h_in, non_blocking=True)
        ctx.build_neighbors(cs.atom_off, e_pos, e_box, 2.8, 3.2, 16)
        ctx.fitness(e_par, d_tg, precision=32, out=Zbuf)
        h_Z.copy_(Zbuf[0], non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    assert torch.equal(h_Z, Zbuf[0].cpu())
    t_e2e = timed(e2e_step, args.steps)
    h2d = total
    d2h = h_Z.numel() * 8

    # dominant kernel: the batched E/F/W + residual kernel, its launches timed by CUDA events that the
    # library records on the launching stream
    k_time = t_fit / args.steps                   # whole fitness call: prep + batched kernel + finalize
    if n_kern != args.steps:
        raise RuntimeError(f"expected {args.steps} timed batched-kernel launches, got {n_kern}")
    b_time = ms_kern / 1e3 / n_kern
    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = props.multi_processor_count
    fp32_peak = nsm * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s: SMs x FP32 lanes x 2 (FMA) x clock
    achieved = flop / b_time / 1e12
    xu_rate = xu / b_time / 1e12
    info = ctx.schedule_info(32)[0]
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_peak, 3), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak, 4), "traffic": profiled_traffic(),
                "kernel": "tsf::batch_kernel<{t},4,0,{m},float,{w}> (every cell of the workload has m <= 4; "
                          "variant {how})".format(how="fixed by --schedule" if args.schedule else "chosen by the autotuner",
                                                  t=info["tile"], w=info["warps"], m=3 if info["tile"] == 16 else 2),
                "kernel_ms": round(1e3 * b_time, 4), "flop_per_launch": flop,
                "flop_model": "op-counted formula listing: %g m + %g m(m-1) + %g per atom, %g per config "
                              "(654 FLOP per 4-neighbour atom)" % (FLOP_PER_BOND, FLOP_PER_TRIPLET, FLOP_PER_ATOM,
                                                                  FLOP_PER_CONFIG),
                "peak_source": f"{nsm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (sm_max_mhz from "
                               f"MEASURED_PEAKS.json, {peak_src}); measured FFMA chains "
                               f"{mpeaks['fp32_fma_flops'] / 1e12:.2f} TFLOP/s",
                "frac_of_measured_ffma": round(achieved * 1e12 / mpeaks["fp32_fma_flops"], 4),
                "executed": executed_block(b_time, fp32_peak),
                "xu": {"achieved_tops": round(xu_rate, 4), "ops_per_launch": xu,
                       "peak_tops": round(mpeaks["xu_ex2_ops"] / 1e12, 3),
                       "frac": round(xu_rate * 1e12 / mpeaks["xu_ex2_ops"], 4),
                       "peak_source": "measured ex2.approx chains (32 per SM per clock on this device)"},
                "fitness_call_frac": round(flop / k_time / 1e12 / fp32_peak, 4)}
    measured = {k: round(v / 1e12, 4) for k, v in mpeaks.items()}
    measured["unit"] = "T op/s (FLOP/s for the FMA kinds)"

    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "GA fitness batch: P=200 parameter sets x C=300 periodic 64-atom diamond Si "
                                  "cells (strain +-2%, sigma=0.1 A), neighbour build + geometry + E/F/W + Z per step",
                      "P": P, "C": cs.C, "atoms": cs.Ntot, "bonds": nbonds, "ordered_bond_pairs": ntrip,
                      "precision": "FP32 pair math, FP64 reductions", "l2": "flushed between timed steps",
                      "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
           "fitness_evals_per_s": round(ws * P * args.steps / t_step, 1),
           "fitness_only": {"value": round(fit_value, 1), "unit": UNIT, "ms": round(1e3 * k_time, 4),
                            "fitness_evals_per_s": round(ws * P / k_time, 1),
                            "note": "per GA generation after the first: geometry cache resident"},
           "e2e": {"value": round(ws * atom_evals * args.steps / t_e2e, 1), "unit": UNIT,
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
           "build_only": {"ms": round(1e3 * t_build / args.steps, 4),
                          "note": "neighbour build and FP32 geometry of the 300 cells, counts read back beside it"},
           "gpu_launches": int(launches), "roofline": roofline, "measured_peaks": measured, "clocks": clocks,
           "autotune": {"candidates": tuned_tried, "tuned_launch_ms": None if args.schedule else round(tuned_ms, 4),
                        "schedule": ctx.schedule_info(32)}}
    if not args.quick:
        rows = {
            "adjoint": lambda: bench_adjoint(ctx_dev=dev, steps=max(3, args.steps // 5), flush=flush, stream=stream),
            "plain_fp64_vs_batched": lambda: bench_plain(ctx, params, tg, dev, cs, flush, stream, k_time),
            "uneven_batch": lambda: bench_uneven(dev, flush, stream),
            "md_force": lambda: bench_md(dev, flush, stream, steps=max(3, args.steps // 5)),
            "ga_fit": lambda: bench_ga(ctx, tg, w),
            "elastic": bench_elastic,
            "tersoff_form": lambda: bench_tersoff_form(dev, flush, stream, w, steps=max(3, args.steps // 5)),
        }
        pick = [r for r in args.rows.split(",") if r] or list(rows)
        unknown = [r for r in pick if r not in rows]
        if unknown:
            raise SystemExit(f"unknown rows {unknown}; choose from {list(rows)}")
        out["rows"] = {r: rows[r]() for r in pick}
    if want_cpu:
        out["cpu_baseline"], out["error_vs_oracle"] = cpu_baseline(w, gpu_out, budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _fp32_peak(dev):
    """Nominal FP32 peak (TFLOP/s): SMs x 128 lanes x 2 (FMA) x sm_max_mhz of MEASURED_PEAKS.json."""
    import torch
    peaks, _ = measured_peaks()
    return torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2 * \
        float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def _counts(cnt, M):
    """Bonds kept, ordered bond pairs and atoms of neighbour counts cnt (lists cut at M entries)."""
    m = np.minimum(np.asarray(cnt, dtype=np.int64), M)
    return int(m.sum()), int((m * (m - 1)).sum()), len(m)


def _time(fn, k, flush, stream, warmup=2):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for a, b in ev:
        flush.fill_(1.0)
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / 1e3 / k


def _targets_from_fp64(ctx, w, cs, dev):
    """Targets = the library's FP64 E/F/W at the hidden (Table 2) parameters + the workload's noise."""
    import torch
    Eh, Fh, Wh = ctx.eval(torch.tensor(w["hidden"][None, :], device=dev), precision=64)
    natoms = torch.tensor(cs.natoms, device=dev, dtype=torch.float64)
    ne, nw, nf = w["noise"]
    return {"E": (Eh[0] / natoms + torch.tensor(ne, device=dev)).contiguous(),
            "W": (Wh[0] / natoms[:, None] + torch.tensor(nw, device=dev)).contiguous(),
            "F": (Fh[0] + torch.tensor(nf, device=dev)).contiguous(),
            "mask": torch.full((cs.C,), 7, dtype=torch.uint8, device=dev)}


def bench_adjoint(ctx_dev, steps, flush, stream):
    """Loss gradient over the six parameters: P = 64 x C = 100 64-atom cells (FP32, FP64 accumulation)."""
    import torch

    from paper_1909_11474_gb300 import binding
    from paper_1909_11474_gb300 import inputs as I
    w = I.workload_adjoint()
    cs = w["configs"]
    ctx = binding.Context(ctx_dev.index or 0)
    ctx.build_neighbors(cs.atom_off, torch.tensor(cs.pos, device=ctx_dev), torch.tensor(cs.box, device=ctx_dev))
    tg = _targets_from_fp64(ctx, w, cs, ctx_dev)
    params = torch.tensor(w["params"], device=ctx_dev)
    t = _time(lambda: ctx.param_grad(params, tg), steps, flush, stream)
    tf = _time(lambda: ctx.fitness(params, tg), steps, flush, stream)
    P = len(w["params"])
    B, T, N = _counts(ctx.export_neighbors()[0], ctx.max_nbr)
    flop = P * (ADJ_FLOP_PER_BOND * B + ADJ_FLOP_PER_TRIPLET * T + ADJ_FLOP_PER_ATOM * N + ADJ_FLOP_PER_CONFIG * cs.C)
    peak = _fp32_peak(ctx_dev)
    return {"workload": "P=64 x C=100 64-atom cells, dL/dx over 6 parameters", "ms": round(1e3 * t, 4),
            "value": round(P * cs.Ntot / t, 1), "unit": "atom-evals/s (forward + 6-parameter gradient)",
            "gradients_per_s": round(P / t, 1), "cost_vs_fitness": round(t / tf, 2),
            "roofline": {"bound": "alu", "achieved": round(flop / t / 1e12, 3), "peak": round(peak, 3),
                         "unit": "TFLOP/s", "frac": round(flop / t / 1e12 / peak, 4), "flop_per_call": flop,
                         "flop_model": "forward-mode dual arithmetic (six tangents) over the op-counted listing: "
                                       "%g m + %g m(m-1) + %g per atom" % (ADJ_FLOP_PER_BOND, ADJ_FLOP_PER_TRIPLET,
                                                                           ADJ_FLOP_PER_ATOM),
                         "timed": "whole call (preparation, forward and tangent passes, finalize)"}}


def bench_plain(ctx, params, tg, dev, cs, flush, stream, t_fit32):
    """The plain FP64 path (one launch per (p, c), no cache) on a sample of the GA batch, and the
    batched path in FP64 and FP32 on the whole batch."""
    import torch
    Ps = 2
    sub = params[:Ps].contiguous()
    t_plain = _time(lambda: ctx.eval_plain(sub), 2, flush, stream, warmup=1)
    t_b64 = _time(lambda: ctx.eval(params, precision=64), 3, flush, stream)
    t_b32 = _time(lambda: ctx.eval(params, precision=32), 5, flush, stream)
    P = params.shape[0]
    v_plain = Ps * cs.Ntot / t_plain
    return {"plain_fp64": {"value": round(v_plain, 1), "unit": "atom-evals/s",
                           "sample": f"{Ps} parameter sets x {cs.C} cells = {Ps * cs.C} launches"},
            "batched_fp64_eval": {"value": round(P * cs.Ntot / t_b64, 1), "unit": "atom-evals/s"},
            "batched_fp32_eval": {"value": round(P * cs.Ntot / t_b32, 1), "unit": "atom-evals/s"},
            "batched_fp32_fitness": {"value": round(P * cs.Ntot / t_fit32, 1), "unit": "atom-evals/s"},
            "speedup_fitness_vs_plain_fp64": round(P * cs.Ntot / t_fit32 / v_plain, 1)}


def bench_uneven(dev, flush, stream):
    """Uneven batch: P = 1000 x C = 500 cells of 8..512 atoms (thread-block clusters for large cells)."""
    import torch

    from paper_1909_11474_gb300 import binding
    from paper_1909_11474_gb300 import inputs as I
    w = I.workload_uneven()
    cs = w["configs"]
    ctx = binding.Context(dev.index or 0)
    ctx.build_neighbors(cs.atom_off, torch.tensor(cs.pos, device=dev), torch.tensor(cs.box, device=dev))
    tg = _targets_from_fp64(ctx, w, cs, dev)
    params = torch.tensor(w["params"], device=dev)
    t_untuned = _time(lambda: ctx.fitness(params, tg, precision=32), 3, flush, stream)
    tuned_ms, tried = ctx.autotune(params, tg, precision=32, reps=2)
    t32 = _time(lambda: ctx.fitness(params, tg, precision=32), 3, flush, stream)
    t64 = _time(lambda: ctx.fitness(params, tg, precision=64), 1, flush, stream, warmup=1)
    P = len(w["params"])
    flop, _, _, _ = flop_model(ctx, P)
    peaks, _ = measured_peaks()
    fp32_peak = torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2 * \
        float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    return {"workload": "P=1000 x C=500 cells of 7..512 atoms", "atoms": cs.Ntot,
            "fitness_call_roofline_frac": round(flop / t32 / fp32_peak, 4),
            "fp32": {"value": round(P * cs.Ntot / t32, 1), "unit": "atom-evals/s", "ms": round(1e3 * t32, 3),
                     "fitness_evals_per_s": round(P / t32, 1), "ms_before_autotune": round(1e3 * t_untuned, 3),
                     "autotune": {"candidates": tried, "tuned_launch_ms": round(tuned_ms, 3)}},
            "fp64": {"value": round(P * cs.Ntot / t64, 1), "unit": "atom-evals/s", "ms": round(1e3 * t64, 3)}}


def bench_ga(ctx, tg, w):
    """The paper's GA run on the bench workload (Sec. III.B): N_pop = 200, N_par = 100, 1000 generations,
    mutation rate 0.2 -> 0, each generation one fitness call plus one GA kernel on the device; then
    the damped-Newton gradient polish of the best individual (30 iterations, adjoint gradients)."""
    import torch

    from paper_1909_11474_gb300 import inputs as I
    from paper_1909_11474_gb300.ga import GeneticFit, polish
    lo = I.TABLE2_PARAMS - 0.3 * np.abs(I.TABLE2_PARAMS)
    hi = I.TABLE2_PARAMS + 0.3 * np.abs(I.TABLE2_PARAMS)
    fit = GeneticFit(ctx, tg, lo, hi, n_pop=200, n_par=100, seed=1)
    fit.run(n_gen=5)                                   # warm-up (graph capture of the fitness call)
    fit = GeneticFit(ctx, tg, lo, hi, n_pop=200, n_par=100, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = fit.run(n_gen=1000)
    torch.cuda.synchronize()
    t_ga = time.perf_counter() - t0
    t0 = time.perf_counter()
    x, L0, L1 = polish(ctx, res["params"], tg, lo, hi, steps=30)
    torch.cuda.synchronize()
    t_pol = time.perf_counter() - t0
    hidden = torch.tensor(w["hidden"][None, :], device="cuda")
    L_hidden = float(ctx.param_grad(hidden, tg)[0][0])
    Z_hidden = float(ctx.fitness(hidden, tg, precision=32)[0][0])
    Z_pol = float(ctx.fitness(torch.tensor(x[None, :], device="cuda"), tg, precision=32)[0][0])
    rel = (x - w["hidden"]) / np.abs(w["hidden"])
    return {"workload": "P=200 x C=300 64-atom cells, noisy targets of the Table 2 parameters",
            "generations": 1000, "wall_s": round(t_ga, 3), "ms_per_generation": round(1e3 * t_ga / 1000, 4),
            "best_Z": round(res["Z"], 6),
            "polish": {"method": "damped Newton, 30 iterations", "wall_s": round(t_pol, 3), "loss_before": L0,
                       "loss_after": L1, "loss_at_hidden": L_hidden, "Z_after": round(Z_pol, 6),
                       "Z_at_hidden": round(Z_hidden, 6)},
            "rel_error_vs_hidden": [round(float(v), 6) for v in rel],
            "max_rel_error_vs_hidden": round(float(np.abs(rel).max()), 6),
            "note": "targets carry noise, so the loss minimum sits near, not at, the hidden parameters",
            "paper": "1000 generations take a few minutes on one Tesla P100 (Sec. III.C; context only)"}


def bench_tersoff_form(dev, flush, stream, w, steps):
    """Fitness of P=200 parameter sets of the nine-parameter Tersoff form (Eq. 8 angular function, free S)
    on the bench workload, against the minimal form on the same context and targets."""
    import torch

    from paper_1909_11474_gb300 import binding
    cs = w["configs"]
    ctx = binding.Context(dev.index or 0)
    pos = torch.tensor(cs.pos, device=dev)
    box = torch.tensor(cs.box, device=dev)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    rng = np.random.default_rng(23)
    x9 = np.array([3.2, 1.45, 2.25, 1.9, 0.65, -0.6, 0.06, 20.0, 3.0])[None, :] * rng.uniform(0.9, 1.1, (200, 9))
    p9 = torch.tensor(x9, device=dev)
    p6 = torch.tensor(w["params"], device=dev)
    Eh, Fh, Wh = ctx.eval(torch.tensor(w["hidden"][None, :], device=dev), precision=64)
    natoms = torch.tensor(cs.natoms, device=dev, dtype=torch.float64)
    tg = {"E": (Eh[0] / natoms).contiguous(), "W": (Wh[0] / natoms[:, None]).contiguous(), "F": Fh[0].contiguous(),
          "mask": torch.full((cs.C,), 7, dtype=torch.uint8, device=dev)}
    out = (torch.empty(200, dtype=torch.float64, device=dev), None, None)
    t6 = _time(lambda: ctx.fitness(p6, tg, precision=32, out=out), steps, flush, stream)
    ctx.set_form(binding.FORM_TERSOFF)
    t9 = _time(lambda: ctx.fitness(p9, tg, precision=32, out=out), steps, flush, stream)
    assert ctx.get_status() == 0
    n = 200 * cs.Ntot
    return {"workload": "P=200 x C=300 64-atom cells, FP32 fitness call (default schedule)", "unit": "atom-evals/s",
            "tersoff_form": {"value": round(n / t9, 1), "ms": round(1e3 * t9, 4)},
            "minimal_form": {"value": round(n / t6, 1), "ms": round(1e3 * t6, 4)},
            "cost_ratio": round(t9 / t6, 3)}


def bench_elastic():
    """Table 3 through the device path: lattice constant, C11, C12 and the relaxed C44 of the Table 2
    parameters by zero-temperature stress-strain (batched FP64 evaluation of strained 8-atom cells)."""
    import torch

    from paper_1909_11474_gb300 import inputs as I
    from paper_1909_11474_gb300.elastic import elastic_constants
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c = elastic_constants(I.TABLE2_PARAMS)
    wall = time.perf_counter() - t0
    return {"workload": "8-atom conventional cell, strains +-1e-4, C44 with the internal shift relaxed",
            "a0_A": round(c["a0"], 6), "C11_GPa": round(c["C11"], 3), "C12_GPa": round(c["C12"], 3),
            "C44_GPa": round(c["C44"], 3), "C44_unrelaxed_GPa": round(c["C44_unrelaxed"], 3),
            "device_calls": c["device_calls"], "wall_s": round(wall, 3),
            "paper": {"C11": 148, "C12": 65, "C44": 75, "source": "Table 3, mini-Tersoff"}}


def bench_md(dev, flush, stream, steps):
    """MD-scale force call: 512,000 atoms, cell-list rebuild + E/F/W per call."""
    import torch

    from paper_1909_11474_gb300 import binding
    from paper_1909_11474_gb300 import inputs as I
    w = I.workload_md()
    cs = w["configs"]
    ctx = binding.Context(dev.index or 0)
    pos = torch.tensor(cs.pos, device=dev)
    N = cs.Ntot
    out32 = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty((N, 3), dtype=torch.float32, device=dev),
             torch.empty(6, dtype=torch.float64, device=dev))
    out64 = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty((N, 3), dtype=torch.float64, device=dev),
             torch.empty(6, dtype=torch.float64, device=dev))
    t32 = _time(lambda: ctx.md_force(pos, cs.box[0], w["params"][0], precision=32, out=out32), steps, flush, stream)
    t64 = _time(lambda: ctx.md_force(pos, cs.box[0], w["params"][0], precision=64, out=out64), steps, flush, stream)
    # velocity-Verlet NVE on the same cell at 300 K: 100 steps of 1 fs per call, FP32 forces
    rng = np.random.default_rng(17)
    m = np.full(N, I.SI_MASS)
    vel0 = torch.tensor(I.thermal_velocities(rng, m, 300.0), device=dev)
    mass = torch.tensor(m, device=dev)
    p = pos.clone()
    v = vel0.clone()
    nst = 100
    nve_out = (torch.empty(nst + 1, dtype=torch.float64, device=dev), torch.empty(nst + 1, dtype=torch.float64, device=dev),
               torch.empty((N, 3), dtype=torch.float32, device=dev), torch.empty(6, dtype=torch.float64, device=dev))

    def nve():
        p.copy_(pos)
        v.copy_(vel0)
        ctx.md_nve(p, v, mass, cs.box[0], w["params"][0], 1.0, nst, precision=32, out=nve_out)

    tn = _time(nve, max(2, steps // 2), flush, stream, warmup=1)
    Et = (nve_out[0] + nve_out[1]).cpu().numpy()
    ctx.md_force(pos, cs.box[0], w["params"][0], precision=32, out=out32)
    B, T, _ = _counts(ctx.md_export_neighbors()[0], ctx.md_M)
    flop = MD_FLOP_PER_BOND * B + MD_FLOP_PER_TRIPLET * T + MD_FLOP_PER_ATOM * N
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    fp32 = _fp32_peak(dev)

    def roof(t, fbytes):
        byt = N * (MD_BYTES_IN + fbytes)
        return {"fp32": {"achieved": round(flop / t / 1e12, 3), "peak": round(fp32, 3), "unit": "TFLOP/s",
                         "frac": round(flop / t / 1e12 / fp32, 4)},
                "hbm": {"achieved": round(byt / t / 1e9, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(byt / t / 1e9 / hbm, 4), "bytes_per_call": byt}}
    return {"workload": "40^3 conventional cells = 512,000 atoms, sigma = 0.08 A", "unit": "atom-steps/s",
            "fp32": {"value": round(N / t32, 1), "ms": round(1e3 * t32, 4), "roofline": roof(t32, 12)},
            "fp64": {"value": round(N / t64, 1), "ms": round(1e3 * t64, 4), "roofline": roof(t64, 24)},
            "roofline_model": {"flop_per_call": flop, "bonds": B, "ordered_bond_pairs": T,
                               "flop": "op-counted listing with the bond geometry computed in the call: "
                                       "%g m + %g m(m-1) + %g per atom" % (MD_FLOP_PER_BOND, MD_FLOP_PER_TRIPLET,
                                                                           MD_FLOP_PER_ATOM),
                               "bytes": "algorithmic: FP64 positions in (24 B) and forces out (12 B FP32, "
                                        "24 B FP64) per atom; HBM peak %s (MEASURED_PEAKS.json)" % peak_src},
            "nve_fp32": {"steps_per_call": nst, "dt_fs": 1.0, "T0_K": 300.0,
                         "value": round(N * nst / tn, 1), "ms_per_step": round(1e3 * tn / nst, 4),
                         "max_energy_deviation_eV_per_atom": float(np.abs(Et - Et[0]).max() / N),
                         "note": "one extra force call at the start of each call is included"}}


def host_cores():
    """Host cores this process may run on, and the CPU model (lscpu, else /proc/cpuinfo)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    return n, model or "unknown"


def _oracle_worker_init():
    import torch
    torch.set_num_threads(1)                       # one core per worker process


def _oracle_job(job):
    """Evaluate (p, c, pos, box, x) items with the FP64 oracle: (p, c, E, W, F, E_scale, W_scale, F_scale)
    each (the scales are the summed magnitudes of the terms of E, W and each atom's force)."""
    import oracle
    out = []
    for p, c, pos, box, x in job:
        r = oracle.evaluate(pos, box, x)
        out.append((p, c, r["E"], r["W"], r["F"], r["E_scale"], r["W_scale"], r["F_scale"]))
    return out


class OraclePool:
    """The oracle (as it stands) on every host core: one spawned worker process per core, each with one
    thread, over (parameter set, configuration) items; spawned, not forked, because CUDA is initialised
    in the parent."""

    def __init__(self):
        import multiprocessing as mp
        self.cores, self.model = host_cores()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init)

    def run(self, items, chunk=8):
        jobs = [items[k:k + chunk] for k in range(0, len(items), chunk)]
        t0 = time.perf_counter()
        res = [r for part in self.pool.map(_oracle_job, jobs, chunksize=1) for r in part]
        return res, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def _items(w, pairs, hidden=False):
    cs = w["configs"]
    out = []
    for p, c in pairs:
        pos, box = cs.config(c)
        out.append((p, c, pos, box, w["hidden"] if hidden else w["params"][p]))
    return out


def cpu_baseline(w, gpu_out, budget_s=15.0):
    """The FP64 oracle on all host cores over a bounded, seeded sample of the workload's (p, c) items
    (sized from a calibration round to about budget_s of wall time), and the error of the library's
    FP32 and FP64 E/F/W against it on that sample."""
    cs = w["configs"]
    P = len(w["params"])
    pool = OraclePool()
    try:
        rng = np.random.default_rng(20191125)
        order = [(int(k) % P, int(k) // P) for k in rng.permutation(P * cs.C)]
        pool.run(_items(w, order[:pool.cores]), chunk=1)                 # start-up: imports in every worker
        _, t_cal = pool.run(_items(w, order[:4 * pool.cores]), chunk=4)
        n = int(min(len(order), max(pool.cores, 4 * pool.cores * budget_s / max(t_cal, 1e-3))))
        res, dt = pool.run(_items(w, order[:n]))
        hidden_pairs = [(0, c) for c in range(min(cs.C, pool.cores))]
        res_h, _ = pool.run(_items(w, hidden_pairs, hidden=True), chunk=1)
    finally:
        pool.close()
    atoms = sum(int(cs.natoms[c]) for _, c, *_ in res)
    base = {"value": round(atoms / dt, 1), "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "cpu": pool.model,
            "sample": f"{n} seeded (parameter set, 64-atom cell) evaluations of the same workload in {dt:.1f} s, "
                      f"FP64 torch CPU with autograd forces/virial, one worker process per core"}
    err = {}
    FLOOR = 0.1
    for prec in (32, 64):
        E, F, W = gpu_out[prec]
        e_rel = w_rel = f_abs = f_scl = 0.0
        for p, c, Er, Wr, Fr, ES, WS, FS in res:
            a = int(cs.atom_off[c])
            e_rel = max(e_rel, abs(E[p, c] - Er) / max(abs(Er), FLOOR * ES))
            w_rel = max(w_rel, float(np.linalg.norm(W[p, c] - Wr) / max(np.linalg.norm(Wr), FLOOR * WS)))
            dF = np.abs(F[p, a:a + len(Fr)] - Fr)
            f_abs = max(f_abs, float(dF.max()))
            mag = np.maximum(np.abs(Fr).max(-1), FLOOR * FS)
            f_scl = max(f_scl, float((dF.max(-1) / np.maximum(1.0, mag / 10.0)).max()))
        err[f"fp{prec}"] = {"E_rel_max": e_rel, "W_rel_max": w_rel, "F_abs_max_eV_per_A": f_abs,
                            "F_scaled_max": f_scl}
    E, F, W = gpu_out["hidden32"]
    f_h = e_h = 0.0
    for _, c, Er, Wr, Fr, ES, WS, FS in res_h:
        a = int(cs.atom_off[c])
        f_h = max(f_h, float(np.abs(F[0, a:a + len(Fr)] - Fr).max()))
        e_h = max(e_h, abs(E[0, c] - Er) / abs(Er))
    err["fp32_table2_parameters"] = {"E_rel_max": e_h, "F_abs_max_eV_per_A": f_h, "configs": len(res_h)}
    err["sample"] = f"{n} seeded (p, c) items of the workload ({len(res_h)} cells at the Table 2 parameters)"
    err["bars"] = {"E_rel": 1e-5, "W_rel": 1e-5, "F_abs_eV_per_A": 1e-4, "F_scaled": 1e-4,
                   "reading": "E and W relative to max(|X|, 0.1 x the summed magnitudes of their terms); "
                              "F_scaled = |dF_i| / max(1, max(|F_i|, 0.1 x the summed magnitudes of atom i's "
                              "bond terms) / 10 eV/A), so 1e-4 eV/A absolute up to 10 eV/A and 1e-5 relative "
                              "above; F_abs against 1e-4 applies to the Table 2 parameters (physical forces)"}
    return base, err


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    from paper_1909_11474_gb300 import inputs as I
    w = I.workload_ga_batch(P=args.P, C=args.C)
    cs = w["configs"]
    P = len(w["params"])
    n_pairs = max(1, int(args.ref_pairs))
    order = [(p, c) for c in range(cs.C) for p in range(P)]
    pool = OraclePool()
    times = []
    try:
        pool.run(_items(w, order[:pool.cores]), chunk=1)       # start-up: imports in every worker
        k = 0
        for s in range(args.warmup + args.steps):
            pairs = [order[(k + q) % len(order)] for q in range(n_pairs)]
            k += n_pairs
            res, dt = pool.run(_items(w, pairs))
            if s >= args.warmup:
                times.append((sum(int(cs.natoms[c]) for _, c, *_ in res), dt))
    finally:
        pool.close()
    atoms = sum(a for a, _ in times)
    dt = sum(t for _, t in times)
    v = atoms / dt
    out = {"metric": METRIC, "value": round(v, 1), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": "GA fitness batch: P=200 x C=300 64-atom cells; each step a bounded sample "
                                  f"of {n_pairs} (parameter set, cell) evaluations", "P": P, "C": cs.C},
           "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                            "cpu": pool.model,
                            "sample": f"{n_pairs} (parameter set, 64-atom cell) evaluations per step, one "
                                      "worker process per core"},
           "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--P", type=int, default=200)
    ap.add_argument("--C", type=int, default=300)
    ap.add_argument("--soak", type=float, default=2.0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-pairs", type=int, default=800)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--quick", action="store_true", help="main step only (no per-row measurements)")
    ap.add_argument("--rows", default="", help="comma-separated subset of the extra rows (default: all)")
    ap.add_argument("--schedule", default="", help="fixed batched schedule 'tile,warps,items,narrow' instead of "
                                                   "the autotuner (e.g. 32,12,1,1)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
