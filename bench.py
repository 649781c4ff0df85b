#!/usr/bin/env python
"""Benchmark one CCSD iteration on the GPU (and the CPU oracle as the reference arm).

A step is one full CCSD iteration: the Appendix A residual (all contractions,
ladder included), the denominator update, the norms and DIIS, replayed as one
CUDA graph through the C ABI (ccsd_iterate). Default workload: o = 20 occupied,
v = 120 virtual spinors, naux = 400 DF functions (seeded synthetic system),
complex FP64, <ab||cd> stored packed. The iteration uses a 20 Eh level shift in
the denominators (the paper's remedy for hard-to-converge cases) so that every
timed iteration stays finite on this strongly correlated synthetic system; the
work per iteration does not depend on it.

Printed JSON line: value = seconds per CCSD iteration (lower is better), the
ladder GEMM roofline against the FP64 peak, the end-to-end time through host
buffers, the oracle's CPU time per iteration, clocks during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config o20v120|o10v30|o40v240|o60v400|batch64]
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "o20v120": dict(o=20, v=120, naux=400, seed=2, level_shift=20.0, precision="fp64",
               name="ccsd_fp64_o20_v120_naux400_storedW"),
    "o10v30": dict(o=10, v=30, naux=120, seed=1, level_shift=0.0, precision="fp64",
               name="ccsd_fp64_o10_v30_naux120"),
    "o40v240": dict(o=40, v=240, naux=800, seed=3, level_shift=40.0, precision="split",
               name="ccsd_split_o40_v240_naux800_storedW"),
    "batch64": dict(nsys=64, seed=4, level_shift=0.0, precision="fp64", tol=1e-10,
               name="ccsd_batch64_o4-16_v16-64_naux3v"),
    "o60v400": dict(o=60, v=400, naux=1200, seed=5, level_shift=120.0, precision="split", store_w=False,
               name="ccsd_split_o60_v400_naux1200_dfW"),
}
SPLIT_SLICES = 8  # 5-bit e4m3 digits: 39 bits of each row scale
SPLIT_BITS = 5
METRIC = "CCSD iteration time (s)"
FP64_OVER_BF16_NOMINAL = 1.25 / 2250.0  # dense FP64 vs dense BF16 tensor rate (nominal)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def split_ladder_frac(lad_ms, o: int, v: int, slices: int):
    """Fraction of the e4m3 peak (2 x the measured bf16 burst rate) reached by a split ladder launch
    of lad_ms ms: s(s+1)/2 digit pairs x 8 P(o) P(v)^2 e4m3 flops (packed pairs, stored <ab||cd>)."""
    if not lad_ms:
        return None
    from paper_2103_08473_gb300 import flops
    peaks, _ = load_peaks()
    fl = slices * (slices + 1) // 2 * 8.0 * float(flops.pairs(o)) * float(flops.pairs(v)) ** 2
    return fl / (lad_ms * 1e-3) / 1e12 / (peaks["bf16_tflops"] * 2.0)


def recorded_traffic(kernel_file: str, key: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    prof = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_2103_08473_gb300", "csrc", kernel_file)
    if not (os.path.exists(prof) and os.path.exists(src)):
        return None
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for line in open(prof):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == key and parts[1] == digest:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            cols = [c.strip() for c in line.split(",")]
            if len(cols) < 9:
                continue
            try:
                sm.append(float(cols[1]))
                smax.append(float(cols[2]))
            except ValueError:
                continue
            for nm, val in zip(names, cols[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(ms: float, device: str = "cuda") -> float:
    """The slowest rank's timed region (replicas: every rank runs the whole workload)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def seconds_per_step(ms: float, steps: int) -> float:
    """Seconds per step of the slowest rank. Replicas do not make one system iterate faster, so
    the per-iteration time is not divided by the number of GPUs; the whole job's rate is
    ``replica_throughput``."""
    return ms / 1e3 / steps


def replica_throughput(ms: float, steps: int, world: int) -> dict:
    """N replicas each doing `steps` steps within the slowest rank's time: steps/s of the job."""
    return {"steps_per_s": world * steps / (ms / 1e3), "replicas": world,
            "note": "independent replicas of the same system, one per GPU; no data-path collective"}


def oracle_iteration_time(wl, steps: int = 1, method: str = "ccsd"):
    """Time the CPU oracle on the same workload: integrals untimed, then `steps` full iterations."""
    import numpy as np
    from oracle import ccsd_ref as R
    from paper_2103_08473_gb300 import inputs

    s = inputs.make_system(wl["o"], wl["v"], wl["naux"], wl["seed"])
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, s.o)
    D1, D2 = R.denominators(f, s.o, wl["level_shift"])
    t1, t2 = inputs.random_amplitudes(s.o, s.v, wl["seed"] + 77, scale=0.01)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        S1, S2 = (R.residual_cc2 if method == "cc2" else R.residual)(f, V, t1, t2)
        d1, d2 = S1 / D1, S2 / D2
        t1, t2 = t1 + d1, t2 + d2
        _ = max(np.max(np.abs(d1)), np.max(np.abs(d2)))
        times.append(time.perf_counter() - t0)
    return times


def oracle_ladder_rows_time(wl, npairs: int):
    """Time the oracle's ladder on a sample of (a, b) rows at full size (<ab||cd> rows formed from
    B^Q, contracted with the full tau) and extrapolate by the number of a < b rows: the ladder
    term alone, a lower bound on one oracle iteration. Returns (seconds, sample description)."""
    import numpy as np
    from oracle import ccsd_ref as R
    from paper_2103_08473_gb300 import inputs

    s = inputs.make_system(wl["o"], wl["v"], wl["naux"], wl["seed"])
    t1, t2 = inputs.random_amplitudes(s.o, s.v, wl["seed"] + 77, scale=0.01)
    tau = R.tau(t1, t2)
    del t2
    rng = np.random.default_rng(9)
    pairs = []
    while len(pairs) < npairs:
        a, b = int(rng.integers(s.v)), int(rng.integers(s.v))
        if a < b:
            pairs.append((a, b))
    R.ladder_rows(s.B, s.o, tau, pairs[:1])  # first touch of tau and B
    t0 = time.perf_counter()
    R.ladder_rows(s.B, s.o, tau, pairs)
    dt = time.perf_counter() - t0
    rows = s.v * (s.v - 1) // 2
    est = dt / npairs * rows
    return est, (f"the oracle's ladder term only: {npairs} sampled (a<b) rows of 1/2 sum_cd <ab||cd> tau^cd_ij "
                 f"at every (i, j), <ab||cd> formed from B^Q (numpy complex128), {dt:.1f} s, extrapolated by "
                 f"the {rows} rows; a lower bound on one oracle iteration of {wl['name']}")


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    total = args.warmup + args.steps
    times = oracle_iteration_time(wl, total)[args.warmup:]
    value = sum(times) / len(times)
    cores = os.cpu_count()
    sample = (f"{args.steps} full oracle iterations (Appendix A residual + denominator update, numpy complex128 "
              f"einsum) of the {wl['name']} workload after {args.warmup} warm-up iterations; integrals untimed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "o": wl["o"], "v": wl["v"], "naux": wl["naux"],
                       "level_shift": wl["level_shift"]},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_ctx(ccmod, s, wl, precision, slices, stream, profile=1, complex_4m=0, method=0):
    kw = dict(level_shift=wl["level_shift"], tol=0.0, diis_dim=8, profile=profile, stream=stream.cuda_stream,
              complex_4m=complex_4m, store_w=1 if wl.get("store_w", True) else 0, method=method)
    if precision == "split":
        kw.update(precision=ccmod.PREC_SPLIT, slices=slices, digit_bits=SPLIT_BITS)
    return ccmod.CCSD(s.o, s.v, s.eps, B=s.B, **kw)


def timed_iterations(ccmod, cc, stream, warmup, steps, barrier=lambda: None, sampler=None):
    """warm-up, then `steps` iterations bracketed by CUDA events on the library's stream."""
    import torch
    for _ in range(warmup):
        st, _, _ = cc.iterate(1)
        if st == ccmod.ERR_DIVERGED:
            raise RuntimeError("iteration diverged during warm-up")
    cc.timings()  # reset the per-op averages
    if sampler:
        sampler.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        st, _, _ = cc.iterate(1)
        if st == ccmod.ERR_DIVERGED:
            raise RuntimeError("iteration diverged in the timed region")
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    ops = {}
    for name, t in cc.timings():
        ops[name] = ops.get(name, 0.0) + t
    return e0.elapsed_time(e1), ops, clocks


def split_target_companion(ccmod, inputs, flops, stream, local, meth, n_cmp=2, n_time=3):
    """The o40/v240/naux800 workload in both precisions on fresh contexts from the MP2 guess:
    n_cmp iterations each (the split-vs-FP64 energy and amplitude difference after them, and
    the FP64 time per iteration), then n_time more split iterations timed on their own (the
    split time per iteration and its ladder launch). Contexts are created one after the other
    so that only one holds device memory at a time."""
    import numpy as np
    wl3 = WORKLOADS["o40v240"]
    s3 = inputs.make_system(wl3["o"], wl3["v"], wl3["naux"], wl3["seed"])
    o, v = s3.o, s3.v
    sampler = ClockSampler(local)
    t0 = time.perf_counter()
    cs = make_ctx(ccmod, s3, wl3, "split", SPLIT_SLICES, stream, method=meth)
    create_split = time.perf_counter() - t0
    ms_cmp_s, _, _ = timed_iterations(ccmod, cs, stream, 0, n_cmp)
    e_s, t_s = cs.energy(), cs.get_amplitudes()
    ms_s, opd_s, clocks_s = timed_iterations(ccmod, cs, stream, 0, n_time, sampler=sampler)
    bytes_s = cs.query("device_bytes")
    cs.close()
    t0 = time.perf_counter()
    cf = make_ctx(ccmod, s3, wl3, "fp64", None, stream, method=meth)
    create_fp64 = time.perf_counter() - t0
    ms_f, _, clocks_f = timed_iterations(ccmod, cf, stream, 0, n_cmp, sampler=sampler)
    e_f, t_f = cf.energy(), cf.get_amplitudes()
    bytes_f = cf.query("device_bytes")
    cf.close()
    peaks, peak_kind = load_peaks()
    lad_ms = opd_s.get("ladder:gemm")
    pairs = SPLIT_SLICES * (SPLIT_SLICES + 1) // 2
    fp8_fl = pairs * 8.0 * float(flops.pairs(o)) * flops.pairs(v) ** 2
    fp8_peak = peaks["bf16_tflops"] * 2.0
    lad_frac = fp8_fl / (lad_ms * 1e-3) / 1e12 / fp8_peak if lad_ms else None
    amp = float(max(np.max(np.abs(t_s[0] - t_f[0])), np.max(np.abs(t_s[1] - t_f[1]))))
    return {"workload": wl3["name"], "o": o, "v": v, "naux": wl3["naux"], "level_shift": wl3["level_shift"],
            "slices": SPLIT_SLICES, "bits_per_slice": SPLIT_BITS, "digit_type": "e4m3",
            "split_s_per_iteration": ms_s / 1e3 / n_time, "fp64_s_per_iteration": ms_f / 1e3 / n_cmp,
            "speedup_split_vs_fp64": (ms_f / n_cmp) / (ms_s / n_time),
            "iterations_compared": n_cmp, "abs_dE_split_vs_fp64": abs(e_s - e_f), "max_amp_err_split_vs_fp64": amp,
            "energy_fp64": [e_f.real, e_f.imag],
            "ladder_ms": lad_ms, "ladder_e4m3_frac": lad_frac,
            "ladder_peak_basis": f"{peak_kind} bf16_tflops (burst) x 2 (nominal dense FP8/BF16 ratio)",
            "top_ops_ms": {k: round(t, 3) for k, t in sorted(opd_s.items(), key=lambda kv: -kv[1])[:10]},
            "device_bytes": {"split": bytes_s, "fp64": bytes_f},
            "create_s": {"split": create_split, "fp64": create_fp64},
            "clocks": {"split": clocks_s, "fp64": clocks_f}}


def run_ours(args, wl):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2103_08473_gb300 import build, flops, inputs
    from paper_2103_08473_gb300 import ccsd as ccmod

    ccmod.load(build.build())
    s = inputs.make_system(wl["o"], wl["v"], wl["naux"], wl["seed"])
    o, v = s.o, s.v
    precision = args.precision or wl["precision"]
    slices = args.slices or SPLIT_SLICES
    stream = torch.cuda.Stream()  # a real stream: the library captures its iteration graph on it
    m4 = 1 if args.complex_4m else 0
    meth = {"ccsd": ccmod.METHOD_CCSD, "ccd": ccmod.METHOD_CCD, "cc2": ccmod.METHOD_CC2}[args.method]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(local)[0]
    cc = make_ctx(ccmod, s, wl, precision, slices, stream, complex_4m=m4, method=meth)
    torch.cuda.synchronize()
    # device memory of the context: what its allocations add up to, and what the free memory
    # reported by the driver fell by (the latter includes allocator rounding)
    memory = {"ctx_device_bytes": cc.query("device_bytes"),
              "free_memory_drop_bytes": float(free0 - torch.cuda.mem_get_info(local)[0])}
    for key in ("plan_scratch_bytes", "plan_cached_bytes", "gemm_workspace_bytes", "split_workspace_bytes",
                "diis_bytes"):
        memory[key] = cc.query(key)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    sampler = ClockSampler(local)
    ms, opd, clocks = timed_iterations(ccmod, cc, stream, args.warmup, args.steps, barrier, sampler)
    ms = max_over_ranks(ms)
    kernels = int(cc.query("kernels_per_iteration"))
    e_main = cc.energy()
    t_main = cc.get_amplitudes()

    # end to end through the C ABI with host buffers: H2D of the step's amplitudes from pinned
    # memory, the iteration, D2H of the norm and the energy
    t1h = torch.empty((o, v), dtype=torch.complex128, pin_memory=True)
    t2h = torch.empty((o, o, v, v), dtype=torch.complex128, pin_memory=True)
    cc.get_amplitudes((t1h.numpy(), t2h.numpy()))
    e2e_steps = max(2, args.steps)
    barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        cc.set_amplitudes(t1h.numpy(), t2h.numpy())
        cc.iterate(1)
        cc.energy()
    torch.cuda.synchronize()
    e2e = (time.perf_counter() - w0) / e2e_steps
    cc.timings()
    cc.close()
    h2d = 16 * (o * v + o * o * v * v)
    d2h = 16 + 16

    # companion: the other precision on the same workload and the same iteration count, for the
    # split-precision speedup and its energy / amplitude error against the FP64 GPU path
    companion = None
    if precision == "fp64" and not args.no_split_companion:
        cs = make_ctx(ccmod, s, wl, "split", slices, stream, method=meth)
        ms2, opd2, _ = timed_iterations(ccmod, cs, stream, args.warmup, args.steps)
        e_split = cs.energy()
        t_split = cs.get_amplitudes()
        cs.close()
        companion = {"precision": "split", "slices": slices, "bits_per_slice": SPLIT_BITS, "digit_type": "e4m3",
                     "ms_per_step": ms2 / args.steps, "speedup_vs_fp64": ms / ms2,
                     "abs_dE_vs_fp64_gpu": abs(e_split - e_main),
                     "max_amp_err_vs_fp64_gpu": float(max(np.max(np.abs(t_split[0] - t_main[0])),
                                                          np.max(np.abs(t_split[1] - t_main[1])))),
                     "iterations_compared": args.warmup + args.steps,
                     "ladder_ms": opd2.get("ladder:gemm"),
                     "ladder_e4m3_frac": (split_ladder_frac(opd2.get("ladder:gemm"), o, v, slices)
                                          if args.method == "ccsd" and wl.get("store_w", True) else None),
                     "top_ops_ms": {k: round(t, 4) for k, t in sorted(opd2.items(), key=lambda kv: -kv[1])[:10]}}

    # opt-in: both precisions from the MP2 guess for the same number of iterations on fresh
    # contexts (the split-vs-FP64 error after N iterations, and both iteration times)
    after_n = None
    if args.fp64_companion > 0 and precision == "split":
        n = args.fp64_companion
        res = {}
        for prec in ("split", "fp64"):
            cx = make_ctx(ccmod, s, wl, prec, slices, stream, method=meth)
            ms_n, _, _ = timed_iterations(ccmod, cx, stream, 0, n)
            res[prec] = (ms_n / n, cx.energy(), cx.get_amplitudes())
            cx.close()
        (ms_s, e_s, t_s), (ms_f, e_f, t_f) = res["split"], res["fp64"]
        after_n = {"iterations": n, "split_ms_per_step": ms_s, "fp64_ms_per_step": ms_f,
                   "speedup_split_vs_fp64": ms_f / ms_s, "abs_dE_split_vs_fp64": abs(e_s - e_f),
                   "max_amp_err_split_vs_fp64": float(max(np.max(np.abs(t_s[0] - t_f[0])),
                                                          np.max(np.abs(t_s[1] - t_f[1])))),
                   "energy_fp64": [e_f.real, e_f.imag]}

    # the split-precision target workload (o40/v240/naux800): split against FP64 on the same GPU
    target = None
    if args.config == "o20v120" and world == 1 and not args.no_split_target and precision == "fp64":
        target = split_target_companion(ccmod, inputs, flops, stream, local, meth)

    if rank != 0:
        return
    value = seconds_per_step(ms, args.steps)
    peaks, peak_kind = load_peaks()
    lad_ms = opd.get("ladder:gemm")
    lad_fl = flops.ladder_flops_packed(o, v)
    lad_tf = lad_fl / (lad_ms * 1e-3) / 1e12 if lad_ms else None
    gemm_ms = sum(t for n, t in opd.items() if n.endswith(":gemm"))
    total_op_ms = sum(opd.values())
    if precision == "fp64":
        fp64_peak = peaks["bf16_tflops_sustained"] * FP64_OVER_BF16_NOMINAL
        # FP64 operations the kernel executes: 3M = three real GEMMs (6 flops per complex
        # multiply-add), 4M = four (8 flops); the fragment sums of 3M are left out (< 3%)
        ex_fl = lad_fl * (1.0 if m4 else 0.75)
        ach = ex_fl / (lad_ms * 1e-3) / 1e12 if lad_ms else None
        roofline = {"kernel": f"zgemm_dmma_kernel<{'4M' if m4 else '3M'}> (ladder launch, M=o(o-1)/2, "
                              f"N=K=v(v-1)/2)", "bound": "tensor",
                    "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": (ach / fp64_peak) if ach else None,
                    "peak_basis": f"{peak_kind} bf16_tflops_sustained x 1.25/2250 (nominal dense FP64/BF16 ratio)",
                    "algorithmic_flops_per_launch": ex_fl, "launch_ms": lad_ms,
                    "zgemm_equivalent_tflops": lad_tf,
                    "traffic": recorded_traffic("zgemm_f64.cu", f"ladder_{wl['name']}")}
    else:
        # the split ladder launch executes P = s(s+1)/2 digit pairs x 4 real e4m3 GEMMs of 2 M N K each;
        # without stored <ab||cd> the ladder op also rebuilds (ac|bd) over Q in blocks of a
        pairs = slices * (slices + 1) // 2
        M, N = flops.pairs(o), flops.pairs(v)
        cplx = float(M) * N * N + (0.0 if wl.get("store_w", True) else flops.df_rebuild_cmacs(v, wl["naux"]))
        fp8_fl = pairs * 8.0 * cplx
        fp8_peak = peaks["bf16_tflops"] * 2.0
        ach = fp8_fl / (lad_ms * 1e-3) / 1e12 if lad_ms else None
        lad_name = ("split_kernel<e4m3> (ladder: digits of tau x cached digits of <ab||cd>)"
                    if wl.get("store_w", True) else
                    "split_kernel<e4m3> (ladder op: (ac|bd) rebuilt over Q per block of a, then tau x <ab||cd> rows)")
        roofline = {"kernel": lad_name,
                    "bound": "tensor", "achieved": ach, "peak": fp8_peak, "unit": "TFLOP/s",
                    "frac": (ach / fp8_peak) if ach else None,
                    "peak_basis": f"{peak_kind} bf16_tflops (burst) x 2 (nominal dense FP8/BF16 ratio)",
                    "algorithmic_flops_per_launch": fp8_fl, "launch_ms": lad_ms,
                    "fp64_equivalent_tflops": lad_tf,
                    "traffic": recorded_traffic("zgemm_split.cu", f"ladder_{wl['name']}")}
    if args.method == "cc2":
        # CC2 has no ladder: its largest GEMM is (ai|bj)~ over the T1-dressed factors, M = N = ov, K = naux
        j_ms = opd.get("cc2:J")
        cm = float(o * v) ** 2 * wl["naux"]
        if precision == "fp64":
            ex_fl, peak = 6.0 * cm, peaks["bf16_tflops_sustained"] * FP64_OVER_BF16_NOMINAL
            kname, basis = "zgemm_dmma_kernel<3M> (CC2 (ai|bj)~ launch)", roofline["peak_basis"]
        else:
            ex_fl, peak = slices * (slices + 1) // 2 * 8.0 * cm, peaks["bf16_tflops"] * 2.0
            kname, basis = "split_kernel<e4m3> (CC2 (ai|bj)~ launch)", roofline["peak_basis"]
        ach = ex_fl / (j_ms * 1e-3) / 1e12 if j_ms else None
        roofline = {"kernel": kname, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": (ach / peak) if ach else None, "peak_basis": basis,
                    "algorithmic_flops_per_launch": ex_fl, "launch_ms": j_ms, "traffic": None}
    top = sorted(opd.items(), key=lambda kv: -kv[1])[:8]
    cores = os.cpu_count()
    cpu = None
    if world == 1 and not args.no_cpu_baseline and wl["o"] * wl["v"] <= 2400:
        ct = oracle_iteration_time(wl, 1, args.method)
        cpu = {"value": ct[0], "unit": "s", "cores": cores, "kind": "oracle",
               "sample": f"one full oracle iteration ({'CC2' if args.method == 'cc2' else 'Appendix A'} residual + update, numpy complex128) of the "
                         f"{wl['name']} workload, integrals untimed"}
    elif world == 1 and not args.no_cpu_baseline:
        est, sample = oracle_ladder_rows_time(wl, 12 if wl["v"] <= 240 else 3)
        cpu = {"value": est, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample}
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "e4m3 digits, f32 accumulate, f64",
            "data": "synthetic",
            "config": {"workload": wl["name"], "o": o, "v": v, "naux": wl["naux"], "precision": precision,
                       "slices": slices if precision == "split" else None,
                       "complex_mult": "4M" if m4 else "3M", "method": args.method,
                       "store_w": wl.get("store_w", True), "level_shift": wl["level_shift"], "diis_dim": 8,
                       "l2": "inputs larger than L2 (packed <ab||cd> and vovv exceed 129 MB)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "ladder_tflops": lad_tf,
            "gemm_share_of_iteration": gemm_ms / total_op_ms if total_op_ms else None,
            "roofline": roofline, "split": companion, "fp64_after_n": after_n, "split_o40v240": target,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": clocks, "gpu_launches": kernels * args.steps,
            "throughput": replica_throughput(ms, args.steps, world) if world > 1 else None,
            "energy": [e_main.real, e_main.imag], "device_memory": memory,
            "top_ops_ms": {k: round(t, 4) for k, t in top}}
    print(json.dumps(line), flush=True)


def oracle_triples_time(wl, ntriples: int = 2):
    """Time the oracle's per-pair triples on the last pairs (one triple each) at full size and
    extrapolate by the number of triples i<j<k. Returns (seconds, sample description)."""
    from oracle import ccsd_ref as R
    from oracle import triples_ref as T3
    from paper_2103_08473_gb300 import inputs

    s = inputs.make_system(wl["o"], wl["v"], wl["naux"], wl["seed"])
    o, v = s.o, s.v
    f = R.fock_matrix(s.eps)
    t1, t2 = inputs.random_amplitudes(o, v, wl["seed"] + 77, scale=0.01)
    V = {k: R.antisym_block(s.B, o, k) for k in ("oovv", "ooov", "vovv")}
    pairs = [(o - 3 - n, o - 2) for n in range(ntriples)]  # j = o-2: the single triple k = o-1
    t0 = time.perf_counter()
    for i, j in pairs:
        T3.pair_contributions(f, V, t1, t2, i, j)
    dt = time.perf_counter() - t0
    nt = o * (o - 1) * (o - 2) // 6
    return dt / len(pairs) * nt, (f"the oracle's triples (numpy complex128, per-pair form): {len(pairs)} triples "
                                  f"(i, {o - 2}, {o - 1}) at full size in {dt:.1f} s, extrapolated by the {nt} "
                                  f"triples i<j<k of {wl['name']}; integral blocks untimed")


def run_triples(args, wl):
    """One step = one evaluation of E(+T), E((T)), E(-T) (FP64) at the workload's MP2 amplitudes
    with random singles; the amplitudes' values do not change the work."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2103_08473_gb300 import build, flops, inputs
    from paper_2103_08473_gb300 import ccsd as ccmod

    ccmod.load(build.build())
    s = inputs.make_system(wl["o"], wl["v"], wl["naux"], wl["seed"])
    o, v = s.o, s.v
    stream = torch.cuda.Stream()
    precision = args.precision or "fp64"
    cc = make_ctx(ccmod, s, wl, precision, SPLIT_SLICES, stream)
    t1, _ = inputs.random_amplitudes(o, v, wl["seed"] + 77, scale=0.01)
    _, t2 = cc.get_amplitudes()
    cc.set_amplitudes(t1, t2)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        cc.triples()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    eg = mg = en = 0.0
    for _ in range(args.steps):
        res = cc.triples()
        eg += cc.query("triples_egemm_ms")
        mg += cc.query("triples_mgemm_ms")
        en += cc.query("triples_energy_ms")
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    launches = int(cc.query("triples_launches"))
    batches = int(cc.query("triples_batches"))
    nb = int(cc.query("triples_batch"))

    # end to end through the C ABI with host buffers: H2D of the amplitudes from pinned memory, the
    # evaluation, the three energies back
    t1h = torch.from_numpy(t1).pin_memory()
    t2h = torch.from_numpy(t2).pin_memory()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(max(2, args.steps)):
        cc.set_amplitudes(t1h.numpy(), t2h.numpy())
        cc.triples()
    e2e = (time.perf_counter() - w0) / max(2, args.steps)
    cc.close()
    if rank != 0:
        return
    cm = flops.triples_cmacs(o, v)
    peaks, peak_kind = load_peaks()
    eg_s = eg / args.steps * 1e-3
    nt = o * (o - 1) * (o - 2) // 6
    if precision == "fp64":
        fp64_peak = peaks["bf16_tflops_sustained"] * FP64_OVER_BF16_NOMINAL
        ex_fl = 6.0 * cm["e"]  # 3M: three real GEMMs per complex GEMM
        ach = ex_fl / eg_s / 1e12 if eg_s > 0 else None
        nl = 3 * batches
        roofline = {"kernel": "zgemm_dmma_kernel<3M> (triples e-terms: M = v(v-1)/2, N = K = v, batched over k)",
                    "bound": "tensor", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": (ach / fp64_peak) if ach else None,
                    "peak_basis": f"{peak_kind} bf16_tflops_sustained x 1.25/2250 (nominal dense FP64/BF16 ratio)",
                    "traffic": recorded_traffic("zgemm_f64.cu", f"triples_egemm_{wl['name']}")}
    else:
        # per triple and term: s(s+1)/2 digit pairs x 4 real e4m3 GEMMs of 2 M N K flops
        pairs = SPLIT_SLICES * (SPLIT_SLICES + 1) // 2
        ex_fl = pairs * 8.0 * cm["e"]
        fp8_peak = peaks["bf16_tflops"] * 2.0
        ach = ex_fl / eg_s / 1e12 if eg_s > 0 else None
        nl = 3 * batches
        roofline = {"kernel": "split_smallk_kernel<e4m3> (triples e-terms: one launch per batch of k and term, "
                              "M = nk v(v-1)/2 or v(v-1)/2, N = v or nk v, K = v)",
                    "bound": "tensor", "achieved": ach, "peak": fp8_peak, "unit": "TFLOP/s",
                    "frac": (ach / fp8_peak) if ach else None,
                    "peak_basis": f"{peak_kind} bf16_tflops (burst) x 2 (nominal dense FP8/BF16 ratio)",
                    "traffic": recorded_traffic("zgemm_split.cu", f"triples_egemm_{wl['name']}")}
    roofline.update({"algorithmic_flops_per_launch": ex_fl / nl, "launch_ms": eg / args.steps / nl,
                     "launches_per_step": nl,
                     "zgemm_equivalent_tflops": 8.0 * cm["e"] / eg_s / 1e12 if eg_s > 0 else None})
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        est, sample = oracle_triples_time(wl)
        cpu = {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample}
    value = seconds_per_step(ms, args.steps)
    line = {"metric": "triples corrections time (s)", "value": value, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "e4m3 digits, f32 accumulate, f64 (e- and m-terms); f64 (rest)",
            "data": "synthetic",
            "config": {"workload": f"{wl['name']} triples", "o": o, "v": v, "naux": wl["naux"],
                       "precision": precision, "slices": SPLIT_SLICES if precision == "split" else None,
                       "amplitudes": "MP2 doubles, random singles (scale 0.01)", "max_batch": nb,
                       "batches": batches,
                       "l2": "inputs larger than L2 (packed vovv and the W batch exceed 129 MB)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "step_ms_split": {"e_gemm": eg / args.steps, "m_gemm": mg / args.steps, "energy": en / args.steps},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": 16 * (o * v + o * o * v * v),
                    "d2h_bytes_per_step": 3 * 8},
            "clocks": clocks, "gpu_launches": launches * args.steps,
            "throughput": replica_throughput(ms, args.steps, world) if world > 1 else None,
            "energies": res}
    print(json.dumps(line), flush=True)


def run_lambda(args, wl):
    """One step = one iteration of the Lambda equations at the workload's amplitudes (FP64 or split);
    the amplitudes' values do not change the work. Each timed call runs the residual plan once
    to refresh the intermediates, then `steps` Lambda iterations."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2103_08473_gb300 import build, flops, inputs
    from paper_2103_08473_gb300 import ccsd as ccmod

    ccmod.load(build.build())
    s = inputs.make_system(wl["o"], wl["v"], wl["naux"], wl["seed"])
    o, v = s.o, s.v
    precision = args.precision or "fp64"
    stream = torch.cuda.Stream()
    cc = make_ctx(ccmod, s, wl, precision, SPLIT_SLICES, stream)
    cc.lambda_iterate(args.warmup)
    nops = cc.query("lambda_iterations")
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cc.lambda_iterate(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    lad_ms = cc.query("lambda_op_ms:L:ladder:gemm")
    lkern = int(cc.query("lambda_kernels_per_iteration"))
    lops = {}
    for name, t in cc.timings():
        if name.startswith("L:"):
            lops[name] = lops.get(name, 0.0) + t
    # end to end through the C ABI: multipliers in from pinned host memory, one residual, out
    l1, l2 = cc.get_lambda()
    l1h = torch.from_numpy(l1).pin_memory()
    l2h = torch.from_numpy(l2).pin_memory()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(max(2, args.steps)):
        cc.lambda_residual(l1h.numpy(), l2h.numpy())
    e2e = (time.perf_counter() - w0) / max(2, args.steps)
    cc.close()
    if rank != 0:
        return
    peaks, peak_kind = load_peaks()
    lad_fl = flops.ladder_flops_packed(o, v)  # lambda . <ab||cd>: the forward ladder's shape
    if precision == "fp64":
        ex_fl, peak = 0.75 * lad_fl, peaks["bf16_tflops_sustained"] * FP64_OVER_BF16_NOMINAL
        kname = "zgemm_dmma_kernel<3M> (Lambda ladder adjoint, lambda . <ab||cd>)"
        basis = f"{peak_kind} bf16_tflops_sustained x 1.25/2250 (nominal dense FP64/BF16 ratio)"
    else:
        ex_fl = SPLIT_SLICES * (SPLIT_SLICES + 1) // 2 * lad_fl
        peak = peaks["bf16_tflops"] * 2.0
        kname = "split_kernel<e4m3> (Lambda ladder adjoint, lambda . <ab||cd>)"
        basis = f"{peak_kind} bf16_tflops (burst) x 2 (nominal dense FP8/BF16 ratio)"
    ach = ex_fl / (lad_ms * 1e-3) / 1e12 if lad_ms else None
    cpu = None
    if world == 1 and not args.no_cpu_baseline and o * v <= 2400:
        from oracle import ccsd_ref as R
        from oracle import lambda_ref as L
        f = R.fock_matrix(s.eps)
        V = R.integrals(s.B, o)
        t1, t2 = inputs.random_amplitudes(o, v, wl["seed"] + 77, scale=0.01)
        t0 = time.perf_counter()
        L.lagrangian_gradient(f, V, t1, t2, l1, l2)
        cpu = {"value": time.perf_counter() - t0, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one Lambda residual of the oracle (torch autograd through the Appendix-A residual, "
                         f"CPU complex128) at {wl['name']}"}
    line = {"metric": "Lambda iteration time (s)", "value": seconds_per_step(ms, args.steps),
            "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "e4m3 digits, f32 accumulate, f64", "data": "synthetic",
            "config": {"workload": f"{wl['name']} lambda", "o": o, "v": v, "naux": wl["naux"],
                       "precision": precision, "amplitudes": "MP2 guess",
                       "timed": "one call: a residual-plan refresh, then steps Lambda iterations",
                       "l2": "inputs larger than L2 (packed <ab||cd> exceeds 129 MB)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "lambda_plan_ms": {"ladder_adjoint": lad_ms,
                               "top_ops": {k: round(t, 4) for k, t in sorted(lops.items(), key=lambda kv: -kv[1])[:12]}},
            "roofline": {"kernel": kname, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": (ach / peak) if ach else None, "peak_basis": basis,
                         "algorithmic_flops_per_launch": ex_fl, "launch_ms": lad_ms, "traffic": None},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": 16 * (o * v + o * o * v * v),
                    "d2h_bytes_per_step": 16 * (o * v + o * o * v * v)},
            "clocks": clocks, "gpu_launches": lkern * args.steps, "lambda_iterations_before": nops,
            "throughput": replica_throughput(ms, args.steps, world) if world > 1 else None}
    print(json.dumps(line), flush=True)


def run_batch(args, wl):
    """64 uneven systems solved to convergence in one batch vs one after another. Under torchrun
    the systems are partitioned across the ranks by their o^2 v^4 (no exchange while solving);
    the per-system results come to every rank with one all_gather at the end."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2103_08473_gb300 import build, inputs, shard
    from paper_2103_08473_gb300 import ccsd as ccmod

    ccmod.load(build.build())
    shapes = inputs.batch_shapes(wl["nsys"], wl["seed"])
    n = len(shapes)
    parts = shard.partition([shard.ladder_cost(o, v) for (o, v, _, _) in shapes], world)
    mine = parts[rank]
    systems = {k: inputs.make_system(*shapes[k]) for k in mine}
    spec = [(systems[k].o, systems[k].v, systems[k].eps, systems[k].B) for k in mine]
    tol, maxit = wl["tol"], 200
    precision = args.precision or wl["precision"]
    slices = args.slices or SPLIT_SLICES
    # split batches route GEMMs from 3e7 flops up (the library default is 1e8): measured on the 64
    # systems, 33.8 systems/s against 31.5 (1e8) and 21.1 (1e9)
    popts = (dict(precision=ccmod.PREC_SPLIT, slices=slices, digit_bits=SPLIT_BITS, split_min_flops=3e7)
             if precision == "split" else {})

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # warm-up (module load, first graph instantiation)
    with ccmod.Batch(spec[:4], tol=tol, max_iter=maxit, **popts) as b:
        b.iterate(3)
    sampler = ClockSampler(local)
    # batched, end to end from host arrays: create (H2D, integral blocks, MP2 guess, autotune),
    # iterate to convergence, energies back to the host
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt = ccmod.Batch(spec, tol=tol, max_iter=maxit, autotune=0 if precision == "split" else 1, **popts)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    sampler.start()
    barrier()
    t1 = time.perf_counter()
    st, its, norms, sts = bt.iterate()
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t1
    barrier()
    clocks = sampler.stop()
    eb = bt.energies()
    t_e2e = time.perf_counter() - t0
    bt.close()
    # sequential plain solves of the same systems (contexts created beforehand, cost-model tiles)
    ctxs = [ccmod.CCSD(o, v, e, B=B, tol=tol, max_iter=maxit) for (o, v, e, B) in spec]
    barrier()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    seq_it = []
    for c in ctxs:
        r = c.iterate()
        seq_it.append(r[1])
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t2
    seq_e = [c.energy() for c in ctxs]
    launches = [c.query("kernels_per_iteration") * k for c, k in zip(ctxs, its)]
    for c in ctxs:
        c.close()
    # per-system rows: batch energy (re, im), status, iterations, sequential energy (re, im),
    # sequential iterations, kernel launches of the batch solve
    rows = {k: [eb[q].real, eb[q].imag, sts[q], its[q], seq_e[q].real, seq_e[q].imag, seq_it[q], launches[q]]
            for q, k in enumerate(mine)}
    table = shard.gather_results(rows, n, 8)
    t_solve = max_over_ranks(t_solve * 1e3) / 1e3
    t_seq = max_over_ranks(t_seq * 1e3) / 1e3
    t_e2e = max_over_ranks(t_e2e * 1e3) / 1e3
    t_create = max_over_ranks(t_create * 1e3) / 1e3
    if rank != 0:
        return
    e_batch = table[:, 0] + 1j * table[:, 1]
    e_seq = table[:, 4] + 1j * table[:, 5]
    dE = float(np.max(np.abs(e_batch - e_seq)))  # batch (this precision) vs sequential plain FP64
    all_conv = bool(np.all(table[:, 2] == ccmod.OK))
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        from oracle import ccsd_ref as R
        # the three systems nearest the median ladder cost o^2 v^4, solved fully by the oracle
        cost = sorted(range(n), key=lambda k: shard.ladder_cost(shapes[k][0], shapes[k][1]))
        pick = cost[n // 2 - 1:n // 2 + 2]
        tc = time.perf_counter()
        for k in pick:
            sk = systems[k]
            R.solve(R.fock_matrix(sk.eps), R.integrals(sk.B, sk.o), sk.o, sk.v, max_iter=maxit, tol=tol)
        tc = time.perf_counter() - tc
        cpu = {"value": len(pick) / tc, "unit": "systems/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "the 3 systems nearest the median o^2 v^4 of the 64 ("
                         + ", ".join(f"o={shapes[k][0]} v={shapes[k][1]}" for k in pick)
                         + f") solved to {tol:g} by the oracle, integrals included"}
    h2d = int(sum(16 * sh[2] * (sh[0] + sh[1]) ** 2 + 8 * (sh[0] + sh[1]) for sh in shapes))
    par = ("one fork/join CUDA graph per batch iteration" if world == 1 else
           f"{world} GPUs: systems partitioned by o^2 v^4 (largest first, to the least-loaded rank), one "
           f"fork/join CUDA graph per batch iteration on each; no exchange while solving, one all_gather "
           f"of the per-system results")
    line = {"metric": "systems/s (64 uneven systems solved to convergence)", "value": n / t_solve,
            "unit": "systems/s", "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": t_solve * 1e3,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "e4m3 digits, f32 accumulate, f64", "data": "synthetic",
            "config": {"workload": wl["name"], "nsys": n, "tol": tol, "autotune": precision == "fp64",
                       "precision": precision, "slices": slices if precision == "split" else None,
                       "iterations_max": int(np.max(table[:, 3])), "iterations_total": int(np.sum(table[:, 3])),
                       "all_converged": all_conv, "parallelism": par,
                       "systems_per_rank": [len(p) for p in parts],
                       "cost_per_rank": [sum(shard.ladder_cost(shapes[k][0], shapes[k][1]) for k in p)
                                         for p in parts]},
            "sequential": {"systems_per_s": n / t_seq, "seconds": t_seq,
                           "iterations_total": int(np.sum(table[:, 6]))},
            "speedup_vs_sequential": t_seq / t_solve, "max_abs_dE_batch_vs_sequential_fp64": dE,
            "create_s": t_create, "roofline": None, "cpu_baseline": cpu,
            "e2e": {"value": n / t_e2e, "unit": "systems/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 16 * n + 24 * n},
            "clocks": clocks, "gpu_launches": int(np.sum(table[:, 7]))}
    print(json.dumps(line), flush=True)


def batch_once(args, wl):
    """One batch iteration with all systems active (after creation and two iterations), inside the
    NVTX range "batch_iteration" and timed with CUDA events on the batch stream, for a launch
    list of one batch iteration."""
    import torch
    from paper_2103_08473_gb300 import build, inputs
    from paper_2103_08473_gb300 import ccsd as ccmod

    ccmod.load(build.build())
    systems = inputs.make_batch(wl["nsys"], wl["seed"])
    spec = [(s.o, s.v, s.eps, s.B) for s in systems]
    precision = args.precision or wl["precision"]
    slices = args.slices or SPLIT_SLICES
    # split batches route GEMMs from 3e7 flops up (the library default is 1e8): measured on the 64
    # systems, 33.8 systems/s against 31.5 (1e8) and 21.1 (1e9)
    popts = (dict(precision=ccmod.PREC_SPLIT, slices=slices, digit_bits=SPLIT_BITS, split_min_flops=3e7)
             if precision == "split" else {})
    stream = torch.cuda.Stream()
    with ccmod.Batch(spec, tol=wl["tol"], max_iter=200, stream=stream.cuda_stream, **popts) as b:
        b.iterate(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("batch_iteration")
        e0.record(stream)
        st, its, norms, sts = b.iterate(1)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    active = sum(1 for k in its if k == 3)
    print(json.dumps({"batch_iteration_ms": e0.elapsed_time(e1), "systems_active": active,
                      "precision": precision, "workload": wl["name"]}), flush=True)


def residual_once(wl, precision, slices):
    """One eager residual on the workload (NVTX range per op, e.g. "ladder_gemm")."""
    from paper_2103_08473_gb300 import build, inputs
    from paper_2103_08473_gb300 import ccsd as ccmod

    ccmod.load(build.build())
    s = inputs.make_system(wl["o"], wl["v"], wl["naux"], wl["seed"])
    kw = dict(level_shift=wl["level_shift"])
    if precision == "split":
        kw.update(precision=ccmod.PREC_SPLIT, slices=slices, digit_bits=SPLIT_BITS)
    with ccmod.CCSD(s.o, s.v, s.eps, B=s.B, **kw) as cc:
        cc.residual()
    print("residual evaluated", flush=True)


def gemm_once(kind, M, N, K, reps=3):
    """One complex GEMM C = A B^T (A: M x K, B: N x K, row-major, random) through the C ABI, timed
    with CUDA events after two warm-up calls: a small case for profiling either GEMM kernel."""
    import torch
    from paper_2103_08473_gb300 import build, flops
    from paper_2103_08473_gb300 import ccsd as ccmod

    ccmod.load(build.build())
    g = torch.Generator(device="cuda").manual_seed(7)
    a = torch.randn((M, K), dtype=torch.complex128, device="cuda", generator=g)
    b = torch.randn((N, K), dtype=torch.complex128, device="cuda", generator=g)
    c = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.Stream()

    def run():
        if kind == "split":
            ccmod.split_zgemm(a, b, c, transB=True, bits=SPLIT_BITS, slices=SPLIT_SLICES, stream=stream)
        else:
            ccmod.zgemm(a, b, c, transB=True, stream=stream)

    for _ in range(2):
        run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    conv = 8.0 * M * N * K
    pairs = SPLIT_SLICES * (SPLIT_SLICES + 1) // 2
    executed = conv * pairs if kind == "split" else conv * 0.75
    print(json.dumps({"gemm": kind, "M": M, "N": N, "K": K, "ms": ms,
                      "zgemm_equivalent_tflops": conv / ms / 1e9,
                      "executed_tflops": executed / ms / 1e9,
                      "executed": "e4m3 flops of 36 digit pairs x 4 real GEMMs (slicing included in the time)"
                      if kind == "split" else "FP64 flops of 3 real GEMMs (3M)"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(WORKLOADS), default="o20v120")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "split"], default=None,
                    help="default: fp64 for o10v30/o20v120/batch64, split for o40v240/o60v400")
    ap.add_argument("--slices", type=int, default=0, help=f"split digits per operand (default {SPLIT_SLICES})")
    ap.add_argument("--no-split-companion", action="store_true")
    ap.add_argument("--no-split-target", action="store_true",
                    help="o20v120: skip the o40v240 split-vs-FP64 companion (split_o40v240 in the line)")
    ap.add_argument("--fp64-companion", type=int, default=0, metavar="N",
                    help="split runs: also run N iterations from the MP2 guess in split and in FP64 and compare")
    ap.add_argument("--gemm-once", nargs=4, metavar=("KIND", "M", "N", "K"),
                    help="one GEMM (KIND fp64 or split) of M x N x K for profiling, then exit")
    ap.add_argument("--method", choices=["ccsd", "ccd", "cc2"], default="ccsd",
                    help="ccd: the doubles equations with t1 held at zero; cc2: the CC2 doubles")
    ap.add_argument("--complex-4m", action="store_true",
                    help="FP64 GEMMs with four real products per complex product instead of three")
    ap.add_argument("--triples", action="store_true",
                    help="time the triples corrections E(+T), E((T)), E(-T) on the workload instead of an iteration")
    ap.add_argument("--lambda", dest="lam", action="store_true",
                    help="time iterations of the Lambda equations on the workload instead of the amplitudes'")
    ap.add_argument("--batch-once", action="store_true",
                    help="batch64: one profiled batch iteration (NVTX range batch_iteration), then exit")
    ap.add_argument("--residual-once", action="store_true",
                    help="create the context and evaluate one residual eagerly (for ncu captures), no timing")
    args = ap.parse_args()
    if args.gemm_once:
        kind, M, N, K = args.gemm_once[0], int(args.gemm_once[1]), int(args.gemm_once[2]), int(args.gemm_once[3])
        gemm_once(kind, M, N, K)
        return
    args.warmup = max(args.warmup, 3)  # timing rule: at least 3 untimed warm-up steps
    wl = WORKLOADS[args.config]
    if args.config == "batch64" and args.batch_once:
        batch_once(args, wl)
    elif args.config == "batch64":
        run_batch(args, wl)
    elif args.residual_once:
        residual_once(wl, args.precision or wl["precision"], args.slices or SPLIT_SLICES)
    elif args.triples and args.impl == "ours":
        run_triples(args, wl)
    elif args.lam and args.impl == "ours":
        run_lambda(args, wl)
    elif args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
