#!/usr/bin/env python
"""Throughput of the matrix-P total-count estimator on GB300.

One step = one pass of the whole estimator over one batch of E synthetic
trajectories of the named workload, on a network already resident on the
device: sampler -> propagation GEMM + occupation epilogue -> per-trajectory
finalize -> generating functions summed per sub-ensemble -> inverse DFT and
statistics of P(m).  Metric: trajectories per second (whole job).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbs|reference]
       [--workload m8000] [--precision bf16x3]
The default workload is the largest single-GPU configuration, m8000
(N = M = 8000, r = 1, T = sqrt(0.99) U, E = 2^20 per step, K+1 = 16384).
Under torchrun (N > 1, --gpus N must equal WORLD_SIZE) every rank runs the
same per-rank workload on its own GPU with disjoint trajectory ranges (weak
scaling); gloo carries the barriers and the one sum of sub-ensemble sums
after the timed region.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "matrix-P samples/sec and binned-P(m) wall time per N-mode network at |dP|/sigma<=1"
UNIT = "samples/s"

# DRAM bytes (read + write) of the GEMM kernel per trajectory, from ncu
# captures (dram__bytes_read.sum + dram__bytes_write.sum of one launch,
# divided by its trajectories; the operands grow in proportion to them),
# keyed by (workload, precision, whether the GEMM also runs the next chunk's
# sampler, CTA pair 1/2, band, keep_a bits).  An entry holds only for the kernel version
# it was captured on: the table is emptied whenever the kernel changes, and a
# run without an entry reports traffic null.
GEMM_TRAFFIC_BYTES_PER_SAMPLE = {
    ("m8000", "bf16x3", True, 2, 16, 8): (
        (19.29e9 + 1.11e9) / 16768,
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 16768-trajectory sampling "
        "launch with aligned waves (profiles/k_gemm_tc_pair_m8000.md), scaled to the average "
        "launch"),
    ("m8000", "bf16x3", True, 2, 16, 24): (
        (19.29e9 + 1.11e9) / 16768,
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 16768-trajectory sampling "
        "launch with aligned waves and the 5-stage operand ring "
        "(profiles/k_gemm_tc_pair_m8000.md), scaled to the average launch"),
    ("m8000", "bf16x3", True, 2, 16, 0): (
        (67.03e9 + 1.11e9) / 16768,
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 16768-trajectory sampling "
        "launch without aligned waves (profiles/k_gemm_tc_pair_m8000.md), scaled to the "
        "average launch"),
    ("m4000", "bf16x3", True, 2, 16, 9): (
        (8.53e9 + 1.11e9) / 33408,
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 33408-trajectory sampling "
        "launch with aligned waves and the evict-last policy on A, scaled to the average launch"),
    ("m4000", "bf16x3", True, 2, 16, 8): (
        (8.54e9 + 1.11e9) / 33408,
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 33408-trajectory sampling "
        "launch with aligned waves, scaled to the average launch"),
    ("m1000", "bf16x3", True, 2, 0, 0): (
        (1.28e9 + 1.09e9) / 131072,
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 131072-trajectory sampling "
        "launch (profiles/k_gemm_tc_pair_m1000.md), scaled to the average launch"),
}

# FP32 lane-operation slots of the FMA pipe per evaluated (trajectory, k)
# pair of the double-float generating-function kernel (k_gf_df): the FMA
# pipe's elapsed share (ncu sm__pipe_fma_cycles_active, 54.67 %) x elapsed
# SM cycles (7.188e5) x 152 SMs x 128 FP32 lanes, divided by the launch's
# in-window pairs (131072 trajectories x 290.9 pairs per trajectory, counted
# by gbs_debug_windows): 200.5.  A packed FP32x2 instruction occupies two
# lane slots.  Capture: m1000 chunk of 131072 trajectories
# (profiles/k_gf_df_m1000.md); valid for that kernel version only.
GF_FP32_OPS_PER_PAIR = 200.5

# FP64 peak: the FMA-chain probe (gbs_measure_fp64_rate, CUDA events; 8 to
# 32 independent chains per thread, 128 to 1024 threads per block, 1 to 8
# blocks per SM, outer-product and recurrence operand patterns) tops out at
# 1.057 TFLOP/s on GB300, below the 1.25 the FP64 GEMM itself sustains on
# m8000 (8MN FLOP per trajectory over CUDA-event kernel time), so the
# larger of the probe and GB300's nominal FP64 rate is the peak.
FP64_NOMINAL_TFLOPS = 1.25
# FP32 FMA peak from unit counts: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz
FP32_UNIT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_PEAK_SOURCE = "unit counts: 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2.07 GHz (maximum clock)"
FP64_PEAK_SOURCE = ("max(gbs_measure_fp64_rate, nominal GB300 FP64 1.25 TFLOP/s): the "
                    "FMA-chain probe reads below the rate the FP64 GEMM sustains")


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        top = max(sm)
        loaded = [s for s in sm if s >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def run_oracle_sample(T, r, seed, e0, E, n_sub, K1, threads=0):
    """The oracle's per-trajectory work on E trajectories (samples + GF sums)."""
    import oracle
    n, nS = oracle.samples(T, r, seed, e0, E, threads)
    oracle.accumulate_gf(n, nS, e0, n_sub, K1, threads)


def _oracle_samples(wl_def, seconds):
    """Trajectories for about `seconds` of oracle work on 16 host cores (the
    oracle's propagation runs at roughly 9.4e10 FLOP/s there, 8 M N FLOP per
    trajectory), a power of two in [64, 131072]."""
    e = seconds * 9.4e10 / (8.0 * wl_def.M * wl_def.N)
    return int(min(131072, max(64, 1 << int(round(math.log2(max(e, 1.0)))))))


def reference_arm(args, wl_def):
    """The oracle timed on the host cores on bounded samples of the workload."""
    import oracle
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    oracle.build()
    use_dev = False
    if wl_def.N >= 2000:
        try:
            import torch
            use_dev = torch.cuda.is_available()
        except Exception:
            use_dev = False
    # the network's QR on the GPU where there is one (input generation, not timed)
    net = wl_def.network(device=use_dev)
    cores = oracle.max_threads()
    Es = args.ref_samples or _oracle_samples(wl_def, 2.5)
    for s in range(args.warmup):
        run_oracle_sample(net.T, net.r, net.seed_s, s * Es, Es, wl_def.n_sub, wl_def.K1)
    t0 = time.perf_counter()
    for s in range(args.steps):
        run_oracle_sample(net.T, net.r, net.seed_s, (args.warmup + s) * Es, Es, wl_def.n_sub,
                          wl_def.K1)
    dt = time.perf_counter() - t0
    value = Es * args.steps / dt
    sample = (f"{Es} trajectories per step of {wl_def.name} (sampling, propagation and "
              f"generating-function sums; the one-off inverse DFT is excluded)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl_def.name, "precision": "fp64 (CPU oracle)",
                   "samples_per_step": Es},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _network(wl_def, cache=None):
    """The workload's network; large ones take their QR on the GPU.  With a
    cache path, T is read from it when it exists and written to it
    otherwise (profiling runs load T without the GPU linear-algebra
    library)."""
    import numpy as np
    import workloads as wl
    if cache and os.path.exists(cache):
        T = np.load(cache)
        return wl.Network(T=T, r=wl_def.squeezing(), t2=wl_def.t2,
                          seed_s=wl.SEED_S_BASE + wl_def.index)
    net = wl_def.network(device=wl_def.N >= 2000)
    if cache:
        np.save(cache, net.T)
    return net


def _window_pairs(w, K1):
    """Per trajectory, the k of the K1 roots of unity at which the
    generating-function kernel evaluates a term: cyclic distance to k = 0 at
    most w1, or to k = K1/2 at most w2 (w[:, 0], w[:, 1]; -1 = none,
    >= K1/2 = all)."""
    import numpy as np
    half = K1 // 2
    w1 = w[:, 0].astype(np.int64)
    w2 = w[:, 1].astype(np.int64)

    def count_within(wv):
        return np.where(wv < 0, 0, np.where(wv >= half, K1, 2 * wv + 1))

    def count_dist(lo, hi):  # k whose distance to k = 0 lies in [lo, hi] (0 <= lo, hi <= half)
        n = 2 * (hi - lo + 1) - (lo == 0) - (hi == half)
        return np.where(hi >= lo, n, 0)

    both = np.where((w1 >= 0) & (w2 >= 0),
                    count_dist(np.maximum(half - np.minimum(w2, half), 0), np.minimum(w1, half)), 0)
    return count_within(w1) + count_within(w2) - both


def _fp64_samples(wl_def, n_sub):
    """Trajectories of the FP64-path comparison: about 4e12 FLOP of FP64
    propagation (a few seconds on GB300's FP64 pipe), a power of two, at
    least 32 per sub-ensemble and at most the workload's E."""
    target = 4e12 / (8.0 * wl_def.M * wl_def.N)
    e = 1 << max(0, int(round(math.log2(max(target, 1.0)))))
    return int(min(wl_def.E, max(e, 32 * n_sub)))


def gbs_arm(args, wl_def):
    import numpy as np
    import torch

    import paper_2503_12749_gb300 as gbs
    from paper_2503_12749_gb300 import distributed as gdist

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world != args.gpus:
        sys.stderr.write(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}; launch N > 1 "
                         "GPUs as torchrun --nproc-per-node N bench.py --gpus N\n")
        return 2
    dist = None
    if world > 1:
        # gloo (host memory) carries the barriers, the max over ranks and the
        # one sum of sub-ensemble sums: there is no device collective
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend="gloo")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    def barrier():
        if dist:
            dist.barrier()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    gbs.build()
    precision = args.precision or wl_def.precision
    stream = torch.cuda.Stream()
    sptr = stream.cuda_stream
    netdef = _network(wl_def, args.t_cache)
    E, n_sub, K1 = wl_def.E, wl_def.n_sub, wl_def.K1
    if args.samples:
        E = args.samples
    net = gbs.gbs_make_network(netdef.T, netdef.r, precision, sptr)
    if args.sampler_fusion is not None:
        gbs.gbs_set_sampler_fusion(net, args.sampler_fusion)
    if args.pair_autotune is not None:
        gbs.gbs_set_pair_autotune(bool(args.pair_autotune))
    if args.gemm_pair is not None and precision not in ("fp64", "fp32"):
        gbs.gbs_set_gemm_config(net, args.gemm_pair, args.gemm_band, args.gemm_keep_a)
    out = torch.empty(4 * K1, dtype=torch.float64, device="cuda")
    seed = netdef.seed_s
    # rank r draws trajectories [r * R, (r + 1) * R) with R = (W + K + 2) * E
    # (warm-up, timed and 2 phase-timing steps)
    base, _ = gdist.rank_range(rank, world, (args.warmup + args.steps + 2) * E)

    def step(s):
        gbs.gbs_sample(net, seed, base + s * E, E, n_sub, K1)
        gbs.gbs_binned_counts_device(net, 0, out.data_ptr())

    with torch.cuda.stream(stream):
        for s in range(args.warmup):
            step(s)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    ev0.record(stream)
    for s in range(args.steps):
        step(args.warmup + s)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1))
    # kernel times per phase: further steps with phase timing on (events
    # around every phase), scaled to the timed steps
    nprof = 2
    gbs.gbs_profile_enable(net, True)
    for s in range(nprof):
        step(args.warmup + args.steps + s)
    torch.cuda.synchronize()
    prof = gbs.gbs_profile_read(net)
    gbs.gbs_profile_enable(net, False)
    prof = {k: (v[0] * args.steps / nprof, v[1] * args.steps // nprof) for k, v in prof.items()}
    if dist:
        # combine sub-ensemble sums of all ranks (the estimator's one exchange)
        _, _, acc, cnt = gbs.gbs_get_accumulators(net)
        acc_all, cnt_all = gdist.combine_accumulators(acc, cnt)
        gbs.gbs_set_accumulators(net, acc_all, cnt_all)
    ms_step = ms_total / args.steps
    value = world * E * args.steps / (ms_total / 1e3)

    # the run's P(m) over all warm-up and timed trajectories (its agreement
    # with the exact distribution at this size is gated by
    # tests/test_gpu_fullsize.py)
    P = gbs.gbs_binned_counts(net, 0, K1)
    acc_summary = {"sum_P": float(np.sum(P[0])), "max_sigma_mP": float(np.max(P[1])),
                   "max_sigma_plusP": float(np.max(P[3])),
                   "trajectories": int(world * (args.warmup + args.steps + nprof) * E)}

    # roofline of the dominant kernel (the propagation GEMM)
    peaks, peak_kind = _peaks()
    gemm_ms, gemm_launches = prof["gemm"]
    flops = 8.0 * netdef.M * netdef.N * E * args.steps
    tc_path = precision not in ("fp64", "fp32")
    P_products = {"bf16x3": 3, "bf16x6": 6}.get(precision, 1)
    folded = bool(tc_path and gbs.gbs_sampler_fusion(net))
    if tc_path:
        achieved = flops / (gemm_ms / 1e3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        pair, band, keep_a = gbs.gbs_gemm_config(net)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": f"{peak_kind} bf16 sustained (kernel timed inside a long step)",
                "algorithmic_flops_per_sample": 8 * netdef.M * netdef.N,
                "mma_products": P_products, "mma_issued_frac": P_products * achieved / peak,
                "kernel": "k_gemm_tc", "launches": gemm_launches,
                "gemm_config": {"cta_pair": pair == 2, "band": band,
                                "keep_a_in_l2": bool(keep_a & 1),
                                "b_evict_first": bool(keep_a & 2),
                                "waves_aligned": bool(keep_a & 8),
                                "ring": "one stage shallower" if keep_a & 16 else "deepest"},
                "avg_launch_ms": gemm_ms / max(gemm_launches, 1),
                "sm_mhz_median": clk.get("sm_mhz"),
                "achieved_at_max_clock": (achieved * clk["sm_max_mhz"] / clk["sm_mhz"]
                                          if clk.get("sm_mhz") else None)}
        if folded:
            roof["kernel"] = "k_gemm_tc (sampling variant: its spare warps also draw the " \
                             "next chunk's samples)"
        # per trajectory: the sample operand (alpha and beta rows, 2 BF16
        # planes each) and one n_S partial (16 B) per 64-mode tile; per
        # launch: the T planes the products read
        planes = 2 if precision == "bf16x3" else 3
        per_traj = 2 * planes * 2 * netdef.N + 16 * (-(-netdef.M // 64))
        if folded:
            # the next chunk's operand and n[] written by the sampler warps
            per_traj += 2 * planes * 2 * netdef.N + 8
        roof["algorithmic_bytes"] = per_traj * E * args.steps / max(gemm_launches, 1) + \
            planes * 2 * netdef.M * netdef.N * 2
        key = (wl_def.name.split(":")[0], precision, folded, pair, band, keep_a)
        per_sample = GEMM_TRAFFIC_BYTES_PER_SAMPLE.get(key)
        if per_sample is not None:
            roof["traffic"] = per_sample[0] * E * args.steps / max(gemm_launches, 1)
            roof["traffic_source"] = per_sample[1]
        else:
            roof["traffic_source"] = "no ncu capture of this kernel version, workload and " \
                                     "configuration"
    elif precision == "fp32":
        achieved = flops / (gemm_ms / 1e3) / 1e12
        peak = FP32_UNIT_TFLOPS
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_gemm_fp64<float>",
                "peak_source": FP32_PEAK_SOURCE}
    else:
        achieved = flops / (gemm_ms / 1e3) / 1e12
        probe = gbs.gbs_measure_fp64_rate(sptr)
        peak = max(probe, FP64_NOMINAL_TFLOPS)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "traffic": None,
                "kernel": "k_gemm_fp64", "fp64_probe_tflops": probe,
                "peak_source": FP64_PEAK_SOURCE}
    phases = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
              for k, v in prof.items()}
    launches = int(sum(v[1] for v in prof.values()))

    # the generating-function phase: in-window (trajectory, k) pairs per
    # second, the pairs counted from the kernels' own windows on a sample
    roof_gf = None
    if tc_path and prof["gf"][0] > 0:
        nw = min(E, 65536)
        w = gbs.gbs_debug_windows(net, seed, base, nw)
        ppt = float(np.mean(_window_pairs(w, K1)))
        pairs_s = ppt * E * args.steps / (prof["gf"][0] / 1e3)
        fma_peak = 152 * 128 * (clk.get("sm_max_mhz") or 2070.0) * 1e6
        roof_gf = {"bound": "alu", "kernel": "k_gf_df", "unit": "pairs/s",
                   "pairs_per_trajectory": ppt, "achieved_pairs_per_s": pairs_s,
                   "pairs_sample": nw, "fp32_ops_per_pair": GF_FP32_OPS_PER_PAIR,
                   "peak_fp32_lane_ops_per_s": fma_peak,
                   "peak_source": "152 SMs x 128 FP32 lanes x max SM clock"}
        if GF_FP32_OPS_PER_PAIR:
            roof_gf["achieved_fp32_lane_ops_per_s"] = pairs_s * GF_FP32_OPS_PER_PAIR
            roof_gf["frac"] = pairs_s * GF_FP32_OPS_PER_PAIR / fma_peak

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x3": "bf16x3 split (fp32 accumulate, f64 sums)",
                  "bf16x6": "bf16x6 split (fp32 accumulate, f64 sums)",
                  "fp32": "f32 GEMM (fp32 accumulate, f64 sums)"}.get(precision, "f64"),
        "data": "synthetic",
        "config": {"workload": wl_def.name, "precision": precision, "samples_per_step": E,
                   "n_sub": n_sub, "K1": K1, "N": netdef.N, "M": netdef.M,
                   "l2": "inputs larger than L2 (sample operand of a chunk > 129 MB, "
                         "written and read every chunk)",
                   "network": "Haar U (QR of seeded complex Gaussian, phase-fixed), "
                              f"T = sqrt({wl_def.t2}) U",
                   "binned_P_wall_ms": ms_step,
                   "phases_from": "2 further steps with phase timing (CUDA events around "
                                  "each phase), scaled to the timed steps",
                   "sampler": ("drawn in the spare warps of the previous chunk's GEMM"
                               if folded else "one launch per chunk")},
        "roofline": roof,
        "roofline_gf": roof_gf,
        "phases": phases,
        "result": acc_summary,
        "gpu_launches": launches,
        "clocks": clk,
    }

    # the plain FP64-GPU path on the same network and trajectories: its rate,
    # the split path's speed-up over it and |dP| / sigma_FP64 between the two
    if tc_path and not args.no_fp64_path and world == 1:
        Ef = args.fp64_samples or _fp64_samples(wl_def, n_sub)
        f0 = base + (args.warmup + args.steps + nprof) * E
        res = {}
        fp64_gemm_ms = None
        for prec in ("fp64", precision):
            n2 = gbs.gbs_make_network(netdef.T, netdef.r, prec, sptr)
            gbs.gbs_sample(n2, seed, f0, min(Ef, 4 * n_sub), n_sub, K1)  # warm-up, tuning
            gbs.gbs_reset(n2)
            torch.cuda.synchronize()
            if prec == "fp64":
                gbs.gbs_profile_enable(n2, True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gbs.gbs_sample(n2, seed, f0, Ef, n_sub, K1)
            e1.record(stream)
            torch.cuda.synchronize()
            if prec == "fp64":
                fp64_gemm_ms = gbs.gbs_profile_read(n2)["gemm"][0]
                gbs.gbs_profile_enable(n2, False)
            res[prec] = (e0.elapsed_time(e1), gbs.gbs_binned_counts(n2, 0, K1))
            gbs.gbs_free_network(n2)
        (ms64, P64), (msb, Pb) = res["fp64"], res[precision]
        sig = np.maximum(P64[1], 1e-13)
        fp64_probe = gbs.gbs_measure_fp64_rate(sptr)
        fp64_peak = max(fp64_probe, FP64_NOMINAL_TFLOPS)
        fp64_gemm_tflops = 8.0 * netdef.M * netdef.N * Ef / (fp64_gemm_ms / 1e3) / 1e12
        line["fp64_path"] = {
            "samples": Ef, "value": Ef / (ms64 / 1e3), "unit": UNIT,
            "gemm_ms": fp64_gemm_ms, "gemm_tflops": fp64_gemm_tflops,
            "fp64_peak_tflops": fp64_peak, "fp64_probe_tflops": fp64_probe,
            "fp64_peak_source": FP64_PEAK_SOURCE,
            "gemm_frac_of_fp64_peak": fp64_gemm_tflops / fp64_peak if fp64_peak else None,
            "speedup_of_split_path": value / (Ef / (ms64 / 1e3)),
            "max_abs_dP_over_sigma_fp64": float(np.max(np.abs(Pb[0] - P64[0]) / sig)),
            "max_abs_dP_plusP_over_sigma_fp64": float(np.max(np.abs(Pb[2] - P64[2]) /
                                                             np.maximum(P64[3], 1e-13))),
            "what": f"gbs_sample of {Ef} trajectories on a GBS_FP64 network (FP64 sampler, "
                    "SIMT FP64 GEMM, FP64 generating functions; CUDA events) and on a "
                    f"{precision} network, the same trajectories; speed-up = the timed "
                    "split-path value / this FP64 rate"}

    # end to end through the C ABI with host buffers: upload the network,
    # sample, invert and read P(m) back, every step, as many steps as the
    # device leg
    if not args.no_e2e:
        # the step's inputs in pinned host memory
        Tn = torch.empty(2 * netdef.T.size, dtype=torch.float64, pin_memory=True).numpy()
        Tn = Tn.view(np.complex128).reshape(netdef.T.shape)
        Tn[:] = netdef.T
        rn = torch.empty(netdef.r.size, dtype=torch.float64, pin_memory=True).numpy()
        rn[:] = netdef.r
        h2d = Tn.nbytes + rn.nbytes
        d2h = 4 * K1 * 8

        parts = {"make": 0.0, "sample_invert_read": 0.0, "free": 0.0}

        def e2e_step(s):
            ta = time.perf_counter()
            n2 = gbs.gbs_make_network(Tn, rn, precision, sptr)
            if args.sampler_fusion is not None:
                gbs.gbs_set_sampler_fusion(n2, args.sampler_fusion)
            if args.gemm_pair is not None and precision not in ("fp64", "fp32"):
                gbs.gbs_set_gemm_config(n2, args.gemm_pair, args.gemm_band, args.gemm_keep_a)
            tb = time.perf_counter()
            gbs.gbs_sample(n2, seed, base + s * E, E, n_sub, K1)
            res = gbs.gbs_binned_counts(n2, 0, K1)
            tc = time.perf_counter()
            gbs.gbs_free_network(n2)
            td = time.perf_counter()
            parts["make"] += tb - ta
            parts["sample_invert_read"] += tc - tb
            parts["free"] += td - tc
            return res

        e2e_step(0)
        for k in parts:
            parts[k] = 0.0
        barrier()
        eclocks = ClockSampler(dev)
        eclocks.start()
        t0 = time.perf_counter()
        ne = args.steps
        for s in range(ne):
            e2e_step(1 + s)
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0)
        eclk = eclocks.stop()
        line["e2e"] = {"value": world * E * ne / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "steps": ne,
                       "clocks": {"sm_mhz": eclk.get("sm_mhz"), "reasons": eclk.get("reasons")},
                       "ms_per_step": {k: 1e3 * v / ne for k, v in parts.items()},
                       "what": "gbs_make_network (pinned host T, r) + gbs_sample + "
                               "gbs_binned_counts (host outputs) + gbs_free_network per step, "
                               "wall clock, max over ranks"}

    if not args.no_cpu_baseline and rank == 0 and world == 1:
        import oracle
        oracle.build()
        Es = args.cpu_samples or _oracle_samples(wl_def, 12.0)
        run_oracle_sample(netdef.T, netdef.r, seed, 0, 64, n_sub, K1)
        t0 = time.perf_counter()
        run_oracle_sample(netdef.T, netdef.r, seed, 0, Es, n_sub, K1)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {
            "value": Es / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{Es} trajectories of {wl_def.name}: sampling, propagation and "
                      f"generating-function sums ({dt:.1f} s); inverse DFT excluded"}

    gbs.gbs_free_network(net)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def batch_arm(args):
    """64 uneven Haar networks in one batch (the batched-networks workload)."""
    import numpy as np
    import torch

    import paper_2503_12749_gb300 as gbs
    import workloads as wl

    torch.cuda.set_device(0)
    gbs.build()
    stream = torch.cuda.Stream()
    sptr = stream.cuda_stream
    wls = wl.batched_networks(count=args.batch_count)
    defs = [w.network() for w in wls]
    E = [args.samples or w.E for w in wls]
    n_sub = [w.n_sub for w in wls]
    K1s, offs = [], []
    for w, d in zip(wls, defs):
        k1, off = wl.count_window(d.r, w.t2)
        K1s.append(k1)
        offs.append(off)
    nets = [gbs.gbs_make_network(d.T, d.r, "bf16x3", sptr) for d in defs]
    batch = gbs.gbs_make_batch(nets)
    outs = [torch.empty(4 * k1, dtype=torch.float64, device="cuda") for k1 in K1s]
    seeds = [d.seed_s for d in defs]

    def step(s):
        gbs.gbs_sample_batch(batch, seeds, [s * e for e in E], E, n_sub, K1s)
        for i, net in enumerate(nets):
            gbs.gbs_binned_counts_device(net, offs[i], outs[i].data_ptr())

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for s in range(args.steps):
        step(args.warmup + s)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    (pair, band, stages), rounds, tiles = gbs.gbs_batch_info(batch)
    # kernels per step: per network and chunk a finalize, a generating-
    # function launch and a sampler (networks of >= 900 output modes with
    # more than one chunk: round 0 only, the grouped GEMMs draw the rest);
    # per round one grouped GEMM; per network the inversion (prep, log2 K1
    # FFT passes, statistics)
    chunks = [-(-e // gbs.gbs_network_info(n)[3]) for e, n in zip(E, nets)]
    samplers = [1 if (c > 1 and d.M >= 900) else c for c, d in zip(chunks, defs)]
    launches_per_step = 2 * sum(chunks) + sum(samplers) + rounds + \
        sum(int(math.log2(k)) + 2 for k in K1s)
    # kernel times: extra steps with phase timing on every network (the
    # rounds are then issued one by one rather than as a graph; the grouped
    # GEMM is attributed to the first network, each network's generating
    # functions to itself)
    for n in nets:
        gbs.gbs_profile_enable(n, True)
    nprof = 2
    for s in range(nprof):
        step(args.warmup + args.steps + s)
    profs = [gbs.gbs_profile_read(n) for n in nets]
    for n in nets:
        gbs.gbs_profile_enable(n, False)
    gemm_ms = profs[0]["gemm"][0] * args.steps / nprof
    gf_ms = sum(p["gf"][0] for p in profs) * args.steps / nprof
    total = sum(E) * args.steps
    flops = sum(8.0 * d.M * d.N * e for d, e in zip(defs, E)) * args.steps
    peaks, peak_kind = _peaks()
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    achieved = flops / (gemm_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": total / (ms_total / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3 split (fp32 accumulate, f64 sums)", "data": "synthetic",
        "config": {"workload": f"batch{len(wls)}: {len(wls)} Haar networks, N=M log-uniform "
                               "[100,2000], r_j~U[0.5,1.5], t~U[0.5,0.995], E=2^18 each",
                   "N": [d.N for d in defs], "K1": K1s, "n_sub": n_sub[0],
                   "samples_per_step": sum(E), "gemm_config_chosen": {"cta_pair": pair == 2, "band": band,
                                                          "ring_stages": stages},
                   "rounds": rounds,
                   "gemm_tiles_per_call": tiles,
                   "note": "one CUDA graph per gbs_sample_batch call; GEMM kernel time from "
                           "2 further steps issued without the graph under phase timing"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": f"{peak_kind} bf16 sustained",
                     "mma_issued_frac": 3 * achieved / peak, "kernel": "k_gemm_tc (grouped)",
                     "gemm_ms_per_step": gemm_ms / args.steps},
        "phases": {"gemm": {"ms_per_step": gemm_ms / args.steps},
                   "gf": {"ms_per_step": gf_ms / args.steps,
                          "note": "sum over the networks' generating-function launches, which "
                                  "run side by side on 8 branches (so the sum exceeds their "
                                  "share of the wall time)"}},
        "gpu_launches": launches_per_step * args.steps, "clocks": clk,
    }
    gbs.gbs_free_batch(batch)
    for n in nets:
        gbs.gbs_free_network(n)
    print(json.dumps(line))
    return 0


def bin2d_arm(args):
    """The paper's two-bin example ("Higher-dimensional binning", Fig. 3):
    lossless 200-mode Haar network, r = 0.5, bins {1..100} and {101..200},
    E = 1.2e6 per step, K1 = K2 = 128, N_R = 100, BF16x3 propagation,
    double-float generating functions.  One step = gbs_sample_2d of E trajectories and the
    two-dimensional inversion."""
    import numpy as np
    import torch

    import paper_2503_12749_gb300 as gbs
    import workloads as wl

    torch.cuda.set_device(0)
    gbs.build()
    stream = torch.cuda.Stream()
    M, r, E, n_sub, K = 200, 0.5, args.samples or 1_200_000, 100, 128
    U = wl.haar_unitary(M, wl.SEED_U_BASE + 200)
    bins = [0] * 100 + [1] * 100
    net = gbs.gbs_make_network_binned(U, np.full(M, r), bins, "bf16x3", stream.cuda_stream)
    seed = wl.SEED_S_BASE + 200

    def step(s):
        gbs.gbs_sample_2d(net, seed, s * E, E, n_sub, K, K)
        return gbs.gbs_binned_counts_2d(net, K, K)

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    for s in range(args.steps):
        P = step(args.warmup + s)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms_step = 1e3 * wall / args.steps
    # kernel launches per step: one further step with phase timing
    gbs.gbs_reset(net)
    gbs.gbs_profile_enable(net, True)
    step(args.warmup + args.steps)
    prof = gbs.gbs_profile_read(net)
    gbs.gbs_profile_enable(net, False)
    launches_per_step = sum(v[1] for v in prof.values())
    line = {
        "metric": "two-bin matrix-P samples/s (joint P(m1, m2) of the paper's 200-mode example)",
        "value": E / (ms_step / 1e3), "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3 GEMM, double-float generating functions, f64 sums and DFT",
        "data": "synthetic",
        "config": {"workload": "bin2d: N=M=200 Haar lossless, r=0.5, bins 100+100, E=1.2e6, "
                               "K1=K2=128, N_R=100", "samples_per_step": E,
                   "timing": "wall clock per step; each step ends with the synchronous "
                             "gbs_binned_counts_2d"},
        "result": {"max_sigma": float(P[1].max()), "paper_max_sigma": 3e-5,
                   "sum_P": float(P[0].sum()),
                   "max_abs_P_odd_total": float(np.max(np.abs(
                       P[0][(np.add.outer(np.arange(K), np.arange(K)) % 2) == 1])))},
        "roofline": {"bound": "alu", "achieved": None, "peak": None, "unit": None,
                     "frac": None, "traffic": None, "kernel": "k_gf2d_df",
                     "note": "issue-bound double-float generating functions on the FP32 "
                             "pipes, like the one-bin k_gf_df (see profiles/); not measured "
                             "separately for this workload"},
        "phases": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1]},
        "gpu_launches": launches_per_step * args.steps, "clocks": clk,
    }
    gbs.gbs_free_network(net)
    print(json.dumps(line))
    return 0


def moments_arm(args):
    """Normally-ordered moments <:n_j^m:> (m = 1..4) and single-mode
    marginals P_j(c) (c = 0..7) of every output mode of the m1000 network
    (Eq. moment, Eq. projection_op with S = {j}): BF16x3 propagation with
    the per-mode occupations written by the GEMM, 10^6 trajectories per
    step, N_R = 100.  One step = one gbs_moments call (synchronous)."""
    import numpy as np
    import torch

    import oracle.moments as orc_mo
    import paper_2503_12749_gb300 as gbs
    import workloads as wl

    torch.cuda.set_device(0)
    gbs.build()
    stream = torch.cuda.Stream()
    w = wl.M1000
    netdef = w.network()
    E = args.samples or w.E
    n_sub, mmax, cmax = w.n_sub, 4, 7
    net = gbs.gbs_make_network(netdef.T, netdef.r, "bf16x3", stream.cuda_stream)
    seed = netdef.seed_s

    def step(s):
        return gbs.gbs_moments(net, seed, s * E, E, n_sub, mmax, cmax)

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    for s in range(args.steps):
        res = step(args.warmup + s)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms_step = 1e3 * wall / args.steps
    nprof = 2
    gbs.gbs_profile_enable(net, True)
    for s in range(nprof):
        step(args.warmup + args.steps + s)
    prof = gbs.gbs_profile_read(net)
    gbs.gbs_profile_enable(net, False)
    phases = {k: {"ms_per_step": v[0] / nprof, "launches_per_step": v[1] / nprof}
              for k, v in prof.items() if v[1]}
    mom_ms = phases["moments"]["ms_per_step"]
    # the run's agreement with the exact Gaussian moments (E1)
    emom = orc_mo.exact_moments(netdef.T, netdef.r, mmax)
    z = (res[0][0] - emom) / np.maximum(res[1][0], 1e-300)
    cpu = None
    if not args.no_cpu_baseline:
        Ec = 256
        t0 = time.perf_counter()
        orc_mo.run(netdef.T, netdef.r, seed, 0, Ec, 16, mmax, cmax)
        dt = time.perf_counter() - t0
        cpu = {"value": Ec / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
               "sample": f"{Ec} trajectories of the same network (oracle/moments.py: C "
                         "sampler and propagation, numpy moments and projectors)"}
    elements = float(E) * w.M
    line = {
        "metric": "normally-ordered moments (m<=4) and single-mode marginals (c<=7) of every "
                  "output mode: matrix-P samples/s",
        "value": E / (ms_step / 1e3), "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3 GEMM, f32 per-mode values (f64 beyond |n'| = 40), f64 sums",
        "data": "synthetic",
        "config": {"workload": "moments: m1000 network N=M=1000 r=1 t2=0.98, E=10^6 per step, "
                               "N_R=100, mmax=4, cmax=7", "samples_per_step": E,
                   "timing": "wall clock per step; gbs_moments is synchronous",
                   "l2": "occupation planes (8 GB per step) larger than L2"},
        "phases": phases,
        "roofline": {"bound": "alu", "kernel": "k_moments<float, 4, 7>",
                     "elements_per_s": elements / (mom_ms / 1e3), "ms_per_step": mom_ms,
                     "achieved": None, "peak": None, "unit": None, "frac": None,
                     "traffic": None,
                     "note": "issue-bound FP32 evaluation, 8 B of occupations read per "
                             "(mode, trajectory); the step's largest phase is the GEMM "
                             "(tensor); see profiles/"},
        "result": {"max_abs_z_matrixP_moments": float(np.max(np.abs(z))),
                   "mean_z2": float(np.mean(z ** 2))},
        "cpu_baseline": cpu,
        "gpu_launches": int(round(sum(v[1] for v in prof.values()) / nprof * args.steps)),
        "clocks": clk,
    }
    gbs.gbs_free_network(net)
    print(json.dumps(line))
    return 0


# Appendix B, Fig. 6: m_max (total-count probability 1e-7) for M = 128 ... 8192
# (left, lossless r = 0.89, with m_min) and for M = 16 ... 1024 (right caption)
FIG6_LEFT = {"M": [128, 256, 512, 1024, 2048, 4096, 8192],
             "m_max": [273, 450, 776, 1388, 2562, 4831, 9267],
             "m_min": [37, 122, 318, 755, 1678, 3605, 7561]}
FIG6_RIGHT = {"M": [16, 32, 64, 128, 256, 512, 1024],
              "m_max": [85, 118, 174, 273, 450, 776, 1388]}


def fig6_arm(args):
    """Appendix B's scaling experiments with E_S = 1.2e6 samples per network
    (N_R = 120 sub-ensembles): left, the time per network of lossless Haar
    networks with r = 0.89 for M = 128 ... 8192 over the window [m_min,
    m_max]; right, max sigma_T of the matrix-P P(m) for M = 16 ... 1024 with
    r_i = 0.89 + 0.1 w_i (w_i standard normal) and amplitude transmissions
    t = 1, 0.995 and 1 - 1/m_max."""
    import numpy as np
    import torch

    import paper_2503_12749_gb300 as gbs
    import workloads as wl

    torch.cuda.set_device(0)
    gbs.build()
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    E = args.samples or 1_200_000
    n_sub = 120

    def pow2(v):
        return 1 << int(math.ceil(math.log2(max(v, 2))))

    left = []
    for M, mx, mn in zip(FIG6_LEFT["M"], FIG6_LEFT["m_max"], FIG6_LEFT["m_min"]):
        # U is produced on the network's stream: the conversion kernel is
        # ordered only after earlier work on that stream
        with torch.cuda.stream(stream):
            U = wl.haar_unitary_device(M, wl.SEED_U_BASE + 7000 + M).contiguous()
        K1 = pow2(mx - mn + 1)
        net = gbs.gbs_make_network_device(U.data_ptr(), M, M, np.full(M, 0.89), "bf16x3", sp)
        del U
        seed = wl.SEED_S_BASE + 7000 + M
        # warm-up over 3 chunks, so that both GEMM variants (the sampling one
        # runs from the second chunk on) are tuned before the timed call
        chunk = gbs.gbs_network_info(net)[3]
        gbs.gbs_sample(net, seed, 0, 3 * chunk, n_sub, K1)
        gbs.gbs_reset(net)
        torch.cuda.synchronize()
        # phase events (a few per chunk) count the kernel launches of the run
        gbs.gbs_profile_enable(net, True)
        t0 = time.perf_counter()
        gbs.gbs_sample(net, seed, 0, E, n_sub, K1)
        P = gbs.gbs_binned_counts(net, mn, K1)
        dt = time.perf_counter() - t0
        prof = gbs.gbs_profile_read(net)
        gbs.gbs_free_network(net)
        left.append({"M": M, "K1": K1, "m_off": mn, "seconds": dt, "samples_per_s": E / dt,
                     "max_sigma": float(P[1].max()),
                     "launches": sum(v[1] for v in prof.values())})
    right = []
    for M, mx in zip(FIG6_RIGHT["M"], FIG6_RIGHT["m_max"]):
        U = wl.haar_unitary(M, wl.SEED_U_BASE + 8000 + M)
        w = np.random.default_rng(wl.SEED_U_BASE + 8000 + M + wl.SEED_R_OFFSET).standard_normal(M)
        r = np.maximum(0.89 + 0.1 * w, 0.0)
        K1 = pow2(mx + 1)
        row = {"M": M, "m_max": mx, "K1": K1}
        for name, t in (("t=1", 1.0), ("t=0.995", 0.995), ("t=1-1/m_max", 1.0 - 1.0 / mx)):
            net = gbs.gbs_make_network(t * U, r, "bf16x3", sp)
            gbs.gbs_sample(net, wl.SEED_S_BASE + 8000 + M, 0, E, n_sub, K1)
            P = gbs.gbs_binned_counts(net, 0, K1)
            gbs.gbs_free_network(net)
            row[name] = float(P[1].max())
        right.append(row)
    big = left[-1]
    line = {
        "metric": "Appendix B scaling: matrix-P time per 1.2e6-sample network vs M, and max "
                  "sampling error vs M",
        "value": big["samples_per_s"], "unit": "samples/s (M = 8192 network)", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": 1e3 * big["seconds"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 split (fp32 accumulate, f64 sums)",
        "data": "synthetic",
        "config": {"workload": "fig6: E_S=1.2e6, N_R=120; left: lossless Haar r=0.89, "
                               "M=128..8192, window [m_min, m_max]; right: r_i=0.89+0.1 w_i, "
                               "t in {1, 0.995, 1-1/m_max}, M=16..1024",
                   "timing": "wall clock of gbs_sample + gbs_binned_counts per network, "
                             "network resident"},
        "left": left, "right": right,
        "result": {"max_sigma_decreases_with_M": {
            k: bool(right[-1][k] < right[0][k]) for k in ("t=1", "t=0.995", "t=1-1/m_max")}},
        "roofline": None, "gpu_launches": big["launches"],
    }
    print(json.dumps(line))
    return 0


SUR_METRIC = "surrogate binned-P(m) predictions/s on held-out networks, judged by matrix-P runs"


def surrogate_arm(args):
    """The learned surrogate at scale: trained on 2000 method-generated
    distributions (N = M log-uniform [500, 8000]), judged against plain
    matrix-P runs on 50 held-out Haar networks plus the N = M = 8000, r = 1,
    t^2 = 0.99 network at E = 2^20.  Timed step: one surrogate prediction of
    all judged networks (features, standardisation, MLP forward, decode)."""
    import numpy as np
    import torch

    import paper_2503_12749_gb300 as gbs
    from paper_2503_12749_gb300 import surrogate as S
    import workloads as wl

    torch.cuda.set_device(0)
    gbs.build()
    stream = torch.cuda.Stream()
    E_train = args.sur_train_samples
    train = wl.surrogate_networks(args.sur_train)
    fourier = lambda n: (n.t * wl.fourier_unitary_device(n.N, n.seed_u)).contiguous()
    cache = {}

    def haar(n):
        if n.seed_u not in cache:
            cache[n.seed_u] = (n.t * wl.haar_unitary_device(n.N, n.seed_u)).contiguous()
        return cache[n.seed_u]

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P, _, ld = S.method_distributions(train, E_train, 64, fourier, stream=stream)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    sur = S.Surrogate(max_batch=args.sur_train, stream=stream)
    t0 = time.perf_counter()
    fit = sur.fit(train, P, ld, steps=400, lr_max=1e-3, rounds=40)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    del P

    held = wl.surrogate_networks(args.sur_heldout, seed=wl.SUR_HELDOUT_SEED)
    big = wl.M8000
    r8 = np.full(big.N, 1.0)
    K8, off8 = wl.dft_window(big.N, 1.0, big.t2, math.sinh(1.0) ** 2)
    net8 = wl.SurrogateNet(big.N, r8, math.sqrt(big.t2), K8, off8, wl.SEED_U_BASE + big.index,
                           wl.SEED_S_BASE + big.index)
    judged = held + [net8]
    # judges: E_judge trajectories per held-out network, 2^20 for the 8000-mode one
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Pj, Sj, ldj = S.method_distributions(held, args.sur_judge_samples, 64, haar, stream=stream)
    torch.cuda.synchronize()
    t_judge = time.perf_counter() - t0
    t0 = time.perf_counter()
    P8, S8, ld8 = S.method_distributions([net8], big.E, 64, haar, stream=stream)
    torch.cuda.synchronize()
    t_big = time.perf_counter() - t0
    ldj = max(ldj, ld8)
    PJ = torch.zeros(len(judged), ldj, dtype=torch.float64, device="cuda")
    PJ[:len(held), :Pj.shape[1]] = Pj
    PJ[len(held), :ld8] = P8[0]
    sig = [float(Sj[i, :n.K1].max() / Pj[i, :n.K1].max()) for i, n in enumerate(held)]
    sig.append(float(S8[0, :K8].max() / P8[0, :K8].max()))

    def errs(Pa, nets):
        return np.array([float((Pa[i, :n.K1] - PJ[i, :n.K1]).abs().max() / PJ[i, :n.K1].max())
                         for i, n in enumerate(nets)])

    # the method without the surrogate: error of shorter runs against the judges
    curve = {}
    for Ec in (2 ** 12, 2 ** 14, 2 ** 16):
        Pc, _, _ = S.method_distributions(held, Ec, 64, haar, stream=stream)
        curve[Ec] = float(np.median(errs(Pc, held)))
        del Pc
    cache.clear()

    # timed: surrogate predictions of all judged networks
    def step():
        return sur.predict(judged, ldj)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        Ps, _, dom = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms_dev = ev0.elapsed_time(ev1)
    ms_step = 1e3 * wall / args.steps     # predict() synchronises: wall clock per step
    e_sur = errs(Ps, judged)
    med = float(np.median(e_sur[:len(held)]))
    # samples a plain run needs for the surrogate's median error (error ~ E^-1/2
    # through the measured curve's largest E)
    E_eq = 2 ** 16 * (curve[2 ** 16] / med) ** 2
    per_sample_s = t_judge / (len(held) * args.sur_judge_samples)
    flops = 2.0 * (10 * 512 + 2 * 512 * 512 + 512 * 512) * len(judged)
    peaks, peak_kind = _peaks()
    line = {
        "metric": SUR_METRIC, "value": len(judged) / (ms_step / 1e3), "unit": "networks/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 weights, fp32 accumulate (activations as bf16 hi+lo)",
        "data": "synthetic",
        "config": {"workload": f"surrogate: 4-layer width-512 MLP trained on {args.sur_train} "
                               f"matrix-P distributions (N=M log-uniform [500,8000], E={E_train} "
                               f"each), judged on {len(held)} held-out Haar networks "
                               f"(E={args.sur_judge_samples}) + N=M=8000 r=1 t^2=0.99 (E={big.E})",
                   "judged_networks": len(judged), "l2": "inputs smaller than L2 (latency-bound)"},
        "surrogate": {
            "train_data_s": t_data, "fit_s": t_fit, "best_round": fit["best_round"],
            "rounds": fit["rounds"], "val_loss_best": float(np.min(fit["val_loss"])),
            "heldout_error_median": med,
            "heldout_error_p90": float(np.percentile(e_sur[:len(held)], 90)),
            "heldout_error_max": float(np.max(e_sur[:len(held)])),
            "m8000_error": float(e_sur[-1]), "judge_sigma_median": float(np.median(sig)),
            "m8000_judge_sigma": sig[-1],
            "method_error_median_at_E": {str(k): v for k, v in curve.items()},
            "method_samples_equivalent": E_eq,
            "method_seconds_per_network_at_equivalent": E_eq * per_sample_s,
            "surrogate_seconds_per_network": ms_step / 1e3 / len(judged),
            "gain_time_at_equal_error": E_eq * per_sample_s / (ms_step / 1e3 / len(judged)),
            "in_domain": int(dom.sum()), "m8000_wall_s": t_big,
            "error": "max_m |P - P_judge| / max_m P_judge"},
        "roofline": {"bound": "latency", "achieved": flops / (ms_dev / args.steps / 1e3) / 1e12,
                     "peak": peaks.get("bf16_tflops"), "unit": "TFLOP/s",
                     "frac": flops / (ms_dev / args.steps / 1e3) / 1e12 / peaks.get("bf16_tflops"),
                     "traffic": None, "kernel": "k_mlp_gemm (4 launches per prediction)",
                     "note": f"{len(judged)} rows per GEMM: launch/latency bound by construction"},
        "gpu_launches": args.steps * 8,
        "clocks": clk,
    }
    # end to end: the same predictions with the distributions read back to
    # host memory every step
    if not args.no_e2e:
        t0 = time.perf_counter()
        for _ in range(max(1, min(3, args.steps))):
            Ph = step()[0].cpu().numpy()
        dt = (time.perf_counter() - t0) / max(1, min(3, args.steps))
        line["e2e"] = {"value": len(judged) / dt, "unit": "networks/s",
                       "h2d_bytes_per_step": int(sum(8 * n.N + 40 for n in judged)),
                       "d2h_bytes_per_step": int(Ph.nbytes),
                       "what": "surrogate prediction from host r arrays to host P(m) arrays"}
    if not args.no_cpu_baseline:
        import oracle.surrogate as osur
        params = gbs.gbs_mlp_get_params(sur.mlp).astype(np.float64)
        dims = [10, 512, 512, 512, 512]
        layers, o = [], 0
        for i in range(4):
            W = params[o:o + dims[i + 1] * dims[i]].reshape(dims[i + 1], dims[i])
            o += W.size
            b = params[o:o + dims[i + 1]]
            o += dims[i + 1]
            layers.append((osur.bf16_round(W), b))
        st = sur.stats.cpu().numpy()
        sample = judged
        t0 = time.perf_counter()
        for n in sample:
            u = osur.features(n.N, n.M, n.r, n.t, n.K1)
            mu, sd = osur.count_moments(n.r, n.t)
            x = np.where(st[1] > 1e-12, (u - st[0]) / np.where(st[1] > 1e-12, st[1], 1.0), 0.0)
            y, _ = osur.forward(layers, x[None, :])
            osur.decode(y[0], n.m_off, n.K1, mu, sd)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(sample) / dt, "unit": "networks/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"all {len(sample)} judged networks: features, "
                                          f"FP64 MLP forward, decode ({dt:.2f} s)"}
    print(json.dumps(line))
    sur.close()
    return 0


def main():
    import workloads as wl
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbs", choices=["gbs", "reference"])
    ap.add_argument("--workload", default="m8000",
                    choices=sorted(wl.NAMED) + ["batch64", "surrogate", "bin2d", "fig6", "moments"])
    ap.add_argument("--sur-train", type=int, default=2000)
    ap.add_argument("--sur-train-samples", type=int, default=2 ** 16)
    ap.add_argument("--sur-heldout", type=int, default=50)
    ap.add_argument("--sur-judge-samples", type=int, default=2 ** 18)
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "bf16x3", "bf16x6"])
    ap.add_argument("--samples", type=int, default=0, help="override trajectories per step")
    ap.add_argument("--ref-samples", type=int, default=0,
                    help="trajectories per reference-arm step (default: about 2 s of oracle "
                         "work on 16 cores)")
    ap.add_argument("--cpu-samples", type=int, default=0,
                    help="trajectories of the cpu_baseline sample (default: about 10-20 s of "
                         "oracle work on 16 cores)")
    ap.add_argument("--fp64-samples", type=int, default=0)
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--gemm-pair", type=int, choices=[0, 1, 2], default=None,
                    help="gbs_set_gemm_config: 1 = one CTA per tile, 2 = CTA pairs, 0 = "
                         "autotuned (the default)")
    ap.add_argument("--gemm-band", type=int, default=0,
                    help="gbs_set_gemm_config band (with --gemm-pair 1 or 2)")
    ap.add_argument("--gemm-keep-a", type=int, choices=list(range(32)), default=0,
                    help="gbs_set_gemm_config keep_a (with --gemm-pair 1 or 2)")
    ap.add_argument("--pair-autotune", type=int, choices=[0, 1], default=None,
                    help="gbs_set_pair_autotune before the run")
    ap.add_argument("--sampler-fusion", type=int, choices=[0, 1, 2], default=None,
                    help="gbs_set_sampler_fusion mode of the timed network (default: the "
                         "library's, 1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--t-cache", default=None,
                    help="read T from this .npy file if it exists, else write it there")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "batch64":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference",
                              "unavailable": "the reference arm is defined for the single-network workloads"}))
            return 0
        return batch_arm(args)
    if args.workload == "fig6":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference",
                              "unavailable": "the reference arm is defined for the single-network workloads"}))
            return 0
        return fig6_arm(args)
    if args.workload == "bin2d":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference",
                              "unavailable": "the reference arm is defined for the single-network workloads"}))
            return 0
        return bin2d_arm(args)
    if args.workload == "moments":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference",
                              "unavailable": "the reference arm is defined for the single-network workloads"}))
            return 0
        return moments_arm(args)
    if args.workload == "surrogate":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference",
                              "unavailable": "the reference arm is defined for the single-network workloads"}))
            return 0
        return surrogate_arm(args)
    wl_def = wl.NAMED[args.workload]
    if args.impl == "reference":
        return reference_arm(args, wl_def)
    return gbs_arm(args, wl_def)


if __name__ == "__main__":
    sys.exit(main())
