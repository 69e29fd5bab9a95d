#!/usr/bin/env python
"""Benchmark of the Gaussian-state -> MPS hot path on GB300.

One step = the whole path on one synthetic state shaped like the paper's
144-mode lossy-experiment workload (144 modes, squeezing r~U(0.1,0.4), depth-12
brick-wall interferometer, d = 6, chi = 256, eps = 1e-12): input check, GSVD
chain, kept bases, PCO tensor build, environments and normalisation, then
100,000 photon-pattern samples (in-kernel Philox uniforms).  Inputs are
resident in device memory when the timed region starts; the tensors (0.9 GB)
and sampling work buffers (several GB) exceed the 129 MB L2, so no flush is
needed between steps.  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun every rank runs its own replica (weak scaling, no collective on
the data path); rank 0 prints the line with the max time over ranks.
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
sys.path.insert(0, ROOT)

METRIC = "MPS tensors/s & samples/s vs plain FP64 GPU path at fixed fidelity; p50/p99 latency"
WORKLOAD = "n144_d6_chi256"
WORKLOAD_DESC = ("144-mode pure Gaussian state: squeezed vacua r~U(0.1,0.4) through a depth-12 "
                 "brick-wall beamsplitter network; d=6, chi=256, eps=1e-12, lambda2_freeze=1e-9")
# DRAM bytes (read + write) per launch from one-kernel ncu captures of the
# current kernels (profiles/): the sampler GEMM at 100,000 samples (the mean
# of a site's pre-pass launch, 169.6 MB, and its rest launch, 13.5 MB), and
# the environment products of the 144-mode workload (one product pass:
# slicing, GEMM and k-split reduction, the mean over two steps' four passes;
# cold-cache, so an upper bound: the bench run keeps them in L2)
TRAFFIC_BYTES_PER_LAUNCH = 91.6e6
ENV_TRAFFIC_BYTES_PER_LAUNCH = 25.8e6
# slice pairs (s, t), s + t <= 6, of seven-slice operands: the bf16 products
# the environment GEMM issues per real multiply-add
ENV_SLICE_PAIRS = 28
# the PCO build's DRAM bytes per launch (one launch per 144-mode build), from
# a one-kernel capture of the current kernel: (1704.4 + 1979.8) MB
PCO_TRAFFIC_BYTES_PER_LAUNCH = 3.6842e9
# A double-float multiply-add (2 flops of the FP64 algorithm) costs 12 FP32
# instructions: the exact product by FMA (4, with the low words) and Knuth's
# TwoSum into the (hi, lo) accumulator (6) plus the low-word update (2)
DF64_FP32_INSTR_PER_FMA = 12
FP32_LANES_PER_SM = 128


def pco_update_count(occ_l, occ_r, d, Q=None):
    """Algorithmic work of one PCO tensor build as the paper's algorithms do
    it (Sec. II C, App. B Algs. 2, 4, 5 and the physical-mode PCOs): the
    number of (target, source) complex updates over the tensor
    C[alpha, p, beta] summed over every PCO zeta <= zeta' with a nonzero
    coupling Q[zeta, zeta'] (all of them when Q is None).  With
    N_q(k) = #{states with n_q >= k} (d - k for the physical mode) a cross
    PCO between two index spaces makes sum_k N_q(k) N_q'(k) x (size of the
    third space) updates, an intra PCO (Alg. 4, composed vector set)
    sum_k #{n_q >= k and n_q' >= k} x (the other two), a duplicate PCO
    (Alg. 5) sum_{k even} N_q(k) x (the other two).  occ_l (D_l, n_l) and
    occ_r (D_r, n_r) are the kept occupation vectors of the two bonds."""
    import numpy as np
    occ_l = np.asarray(occ_l, dtype=np.int64).reshape(len(occ_l), -1)
    occ_r = np.asarray(occ_r, dtype=np.int64).reshape(len(occ_r), -1)
    Dl, nl = occ_l.shape
    Dr, nr = occ_r.shape
    K = max(d, int(occ_l.max(initial=0)), int(occ_r.max(initial=0)))
    ks = np.arange(1, K + 1)

    def nge(col):
        return (col[None, :] >= ks[:, None]).sum(axis=1)

    Nl = [nge(occ_l[:, q]) for q in range(nl)]
    Nr = [nge(occ_r[:, q]) for q in range(nr)]
    Np = np.maximum(d - ks, 0)
    a = nl
    on = (lambda z1, z2: True) if Q is None else (lambda z1, z2: Q[z1, z2] != 0)
    U = 0
    for q in range(nl):
        if on(q, a):
            U += int((Nl[q] * Np).sum()) * Dr
    for q in range(nr):
        if on(a, a + 1 + q):
            U += int((Nr[q] * Np).sum()) * Dl
    if on(a, a):
        U += int(Np[1::2].sum()) * Dl * Dr
    for q in range(nl):
        for qq in range(nr):
            if on(q, a + 1 + qq):
                U += int((Nl[q] * Nr[qq]).sum()) * d
    for occ, N, off, other in ((occ_l, Nl, 0, d * Dr), (occ_r, Nr, a + 1, d * Dl)):
        n = occ.shape[1]
        for q in range(n):
            for qq in range(q + 1, n):
                if on(off + q, off + qq):
                    both = np.minimum(occ[:, q], occ[:, qq])
                    U += int(nge(both).sum()) * other
            if on(off + q, off + q):
                U += int(N[q][1::2].sum()) * other
    return U


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbsmps", choices=["gbsmps", "reference"])
    ap.add_argument("--samples", type=int, default=100_000)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="time the steps one after another instead of as one stream "
                         "(the next state's chain beside the current state's sampling)")
    ap.add_argument("--batch-states", type=int, default=64)
    ap.add_argument("--ref-budget", type=float, default=20.0,
                    help="seconds of oracle work behind the CPU baseline / reference arm")
    ap.add_argument("--serving-requests", type=int, default=100,
                    help="requests per arrival rate")
    ap.add_argument("--serving-rates", default="3,6,12",
                    help="comma-separated Poisson arrival rates (1/s), one serving run each")
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-batch", type=int, default=8,
                    help="most queued requests one serving slot builds in one batched call")
    ap.add_argument("--latency-runs", type=int, default=100,
                    help="one-state runs behind latency_ms (p99 is then not the maximum)")
    ap.add_argument("--large", type=int, default=1,
                    help="1: add the 1024-mode configuration (build + 1M samples) to the line")
    ap.add_argument("--filter-states", type=int, default=152,
                    help="lossy 64-mode states decomposed in one batched call (0: skip)")
    ap.add_argument("--profile-pass", default=None, choices=["build", "sample", "filter"],
                    help="run one build of the workload (and one sampling of --samples) on "
                         "cuda:0 and exit without a JSON line: a short, fixed launch sequence "
                         "for profiler captures")
    return ap.parse_args()


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return 0, 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, local, ws, dist


def replica_stream(rank, step, samples):
    """(seed, counter0) of one replica's sampling in one step: every rank has
    its own Philox key and every step its own counter range, so the replicas
    draw disjoint streams and no step repeats another's draws."""
    return 1234 + rank, step * samples


def max_over_ranks(x, dist):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank, local, ws, dist):
    import numpy as np
    import torch

    import paper_2512_10643_gb300 as g
    import workloads as wl

    dev = local
    torch.cuda.set_device(dev)
    w = wl.config(WORKLOAD)
    N, S = w.N, args.samples
    prec = g.PREC_MIXED if args.precision == "mixed" else g.PREC_FP64
    opts = dict(d=w.d, chi_max=w.chi, eps_trunc=w.eps, lambda2_freeze=w.freeze, precision=prec)
    stream = torch.cuda.Stream(device=dev)
    ctx = g.Context(dev, stream.cuda_stream)
    gam = torch.from_numpy(np.ascontiguousarray(w.gamma)).to(f"cuda:{dev}")
    out = torch.empty((S, N), dtype=torch.uint8, device=f"cuda:{dev}")

    def step(i, sample_count=S, precision=prec, dst=out):
        m = g.MPS.from_cov(ctx, gam, **dict(opts, precision=precision))
        seed, counter0 = replica_stream(rank, i, sample_count)
        m.sample(sample_count, seed=seed, counter0=counter0, out=dst[:sample_count])
        m.release()

    out2 = torch.empty_like(out)
    o_struct = g.opts_default(**opts)

    def stream_steps(i0, K, gam_src=None, outs=None):
        """K steps as one stream: build k+1's chain runs beside sampling k."""
        ks = range(i0, i0 + K)
        keys = [replica_stream(rank, i, S) for i in ks]
        g.gbsmps_build_sample_stream(
            ctx.h, [gam if gam_src is None else gam_src] * K, [o_struct] * K, S,
            [k[0] for k in keys], [k[1] for k in keys],
            outs if outs is not None else [(out, out2)[j % 2] for j in range(K)])

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    pipelined = not args.no_pipeline
    if pipelined:
        stream_steps(0, args.warmup)
    else:
        for i in range(args.warmup):
            step(i)
    barrier()
    n0 = g.gbsmps_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with Clocks(dev) as clk:
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            if pipelined:
                stream_steps(args.warmup, args.steps)
                ev[args.steps].record(stream)
            else:
                for i in range(args.steps):
                    step(args.warmup + i)
                    ev[i + 1].record(stream)
        barrier()
    launches = g.gbsmps_launch_count() - n0
    total_ms = ev[0].elapsed_time(ev[args.steps])
    total_s = max_over_ranks(total_ms / 1e3, dist)
    value = N * args.steps * ws / total_s
    samples_per_s = S * args.steps * ws / total_s
    # latency of one state alone (build + sampling, nothing overlapped), over
    # enough runs that the 99th percentile is not simply the largest one
    nlat = max(args.latency_runs, 1)
    lat = [torch.cuda.Event(enable_timing=True) for _ in range(nlat + 1)]
    barrier()
    with torch.cuda.stream(stream):
        lat[0].record(stream)
        for i in range(nlat):
            step(args.warmup + args.steps + i)
            lat[i + 1].record(stream)
    barrier()
    step_ms = [lat[i].elapsed_time(lat[i + 1]) for i in range(nlat)]

    # dominant kernel, traced over one extra step outside the timed region
    g.gbsmps_trace(ctx.h, True)
    step(10_000)
    torch.cuda.synchronize(dev)
    tr = g.gbsmps_trace_read_kernel(ctx.h, 0)
    te = g.gbsmps_trace_read_kernel(ctx.h, 1)
    tp = g.gbsmps_trace_read_kernel(ctx.h, 2)
    g.gbsmps_trace(ctx.h, False)
    # the PCO build's algorithmic work: the paper's update count from the
    # kept bases of the same state
    mb = g.MPS.from_cov(ctx, gam, **opts)
    occs = [g.gbsmps_get_basis(mb.h, b)[0] for b in range(N + 1)]
    mb.release()
    U = sum(pco_update_count(occs[m], occs[m + 1], w.d) for m in range(N))
    out_entries = sum(occs[m].shape[0] * w.d * occs[m + 1].shape[0] for m in range(N))
    peaks, src = measured_peaks()
    step_ms_avg = total_ms / args.steps
    # the sampler GEMM against the tensor roof
    ach_tflops = tr["flops"] / (tr["ms"] / 1e3) / 1e12 if tr["ms"] > 0 else 0.0
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    n_launch = max(tr["launches"], 1)
    roof_s = {"kernel": "canon_gemm_tc_kernel (persistent tcgen05 split-FP16 complex GEMM over "
                        "both photon-parity groups, A rows gathered by sample index, B by TMA; two "
                        "launches per site: W_0 = Vt At^m[0] for every sample, written as the next "
                        "state, then W = Vt At^m for the samples the p = 0 pre-pass leaves; 100k samples)",
              "bound": "tensor", "achieved": round(ach_tflops, 3), "peak": peak,
              "peak_source": (f"bf16_tflops_sustained of {src} MEASURED_PEAKS.json x 1 "
                              "(nominal dense fp16/bf16 ratio)"),
              "unit": "TFLOP/s", "frac": round(ach_tflops / peak, 5),
              "traffic": (None if TRAFFIC_BYTES_PER_LAUNCH is None or S != 100_000
                          else TRAFFIC_BYTES_PER_LAUNCH),
              "algorithmic_flops_per_launch": tr["flops"] / n_launch,
              "algorithmic_bytes_per_launch": tr["bytes"] / n_launch,
              "algorithmic_flops_def": ("8 real flops per complex product of the nonzero parity blocks "
                                        "the sampler multiplies: block p = 0 of every sample "
                                        "(8 D_{m-1,c} D_{m,c}) plus all blocks of the samples the p = 0 "
                                        "pre-pass leaves (8 D_{m-1,c} sum_p D_{m,c^(p&1)}); two launches "
                                        "per site"),
              "avg_launch_ms": tr["ms"] / n_launch,
              "launches_per_step": tr["launches"],
              "ms_per_state": round(tr["ms"], 3),
              "share_of_step": round(tr["ms"] / step_ms_avg, 4),
              "split_products": 3,
              "issued_fp16_tflops": round(3 * ach_tflops, 3),
              "issued_frac": round(3 * ach_tflops / peak, 5)}
    if roof_s["traffic"] is not None and tr["ms"] > 0:
        hbm = peaks.get("hbm_gbs", 6800.0)
        gbs = roof_s["traffic"] / (tr["ms"] / n_launch / 1e3) / 1e9
        roof_s.update(dram_gbs=round(gbs, 1), dram_frac=round(gbs / hbm, 4),
                      dram_peak_source=f"hbm_gbs of {src} MEASURED_PEAKS.json")
    ne = max(te["launches"], 1)
    ach_e = te["flops"] / (te["ms"] / 1e3) / 1e12 if te["ms"] > 0 else 0.0
    env_common = {
        "algorithmic_flops_per_launch": te["flops"] / ne,
        "algorithmic_bytes_per_launch": te["bytes"] / ne,
        "algorithmic_flops_def": ("8 real flops per complex multiply-add of the parity-block "
                                  "products: X_c[:, p] = Ahat_c[:, p] R_{c^(p&1)} (kl_c kr^2 "
                                  "per block) and R_c = X_c Ahat_c^dag on its lower triangle "
                                  "(kl_c (kl_c + 1) / 2 K_c)"),
        "avg_launch_ms": te["ms"] / ne,
        "launches_per_step": te["launches"],
        "ms_per_state": round(te["ms"], 3),
        "share_of_step": round(te["ms"] / step_ms_avg, 4)}
    if os.environ.get("GBSMPS_ENV_TC", "1") != "0":
        # the exact-accumulation tensor-core products: algorithmic flops
        # counted once against the sustained bf16 rate; the slices' products
        # that the tensor cores actually run (28 slice pairs per real
        # multiply-add) shown apart
        roof_e = {"kernel": ("envtc_kernel (tcgen05: complex products as real ones, seven bf16 "
                             "integer slices per operand row/column exponent, 28 slice-pair MMAs "
                             "of M = 128, N = 96 into four exact FP32 tensor-memory "
                             "accumulators and one for the low-order pairs, double-float "
                             "epilogue; right-environment chain R_m = sum_p Ahat^m[p] R_{m+1} "
                             "Ahat^m[p]^dag on the parity blocks; two product passes per site, "
                             "each timed from its operands' slicing through the GEMM to its "
                             "in-order k-split reduction)"),
                  "bound": "tensor", "achieved": round(ach_e, 4), "peak": peak,
                  "peak_source": (f"bf16_tflops_sustained of {src} MEASURED_PEAKS.json (the "
                                  "kernel runs inside a long step)"),
                  "unit": "TFLOP/s", "frac": round(ach_e / peak, 5),
                  "slice_pairs": ENV_SLICE_PAIRS,
                  "issued_tflops": round(ENV_SLICE_PAIRS * ach_e, 3),
                  "issued_frac": round(ENV_SLICE_PAIRS * ach_e / peak, 4),
                  "issued_frac_def": ("bf16 tensor flops of the slice-pair products (28 per real "
                                      "multiply-add; tile padding and the upper triangles of the "
                                      "Hermitian products not counted) over the sustained bf16 rate"),
                  "traffic": ENV_TRAFFIC_BYTES_PER_LAUNCH}
    else:
        # the double-float GEMM against the FP32 pipes it runs on: algorithmic
        # flops counted once (x1), the emulation cost shown apart
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        fmax = (clk.summary().get("sm_max_mhz") or 2070.0) * 1e6
        fp32_peak = nsm * FP32_LANES_PER_SM * fmax * 2.0 / 1e12
        roof_e = {"kernel": "zgemm_df64_grouped_kernel (double-float complex GEMM on the FP32 pipes, "
                            "right-environment chain on the parity blocks; two grouped launches per "
                            "site, split-K partials summed in k order by each tile's last CTA)",
                  "bound": "alu", "achieved": round(ach_e, 4), "peak": round(fp32_peak, 3),
                  "peak_source": (f"derived: {nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                  f"{fmax / 1e6:.0f} MHz (max SM clock) x 2 flops per FMA"),
                  "unit": "TFLOP/s", "frac": round(ach_e / fp32_peak, 5) if fp32_peak > 0 else None,
                  "issued_fp32_instr_per_fma": DF64_FP32_INSTR_PER_FMA,
                  "issued_frac": round(ach_e * DF64_FP32_INSTR_PER_FMA / 2.0 / (fp32_peak / 2.0), 4)
                  if fp32_peak > 0 else None,
                  "traffic": None}
    roof_e.update(env_common)
    # the PCO tensor build against the HBM roof of the paper's algorithm:
    # U (target, source) updates, each a source read, a target read and a
    # target write of one complex number in the pass precision (complex64 in
    # mixed builds, complex128 in FP64 ones), plus the tensors written once
    # as complex128
    cbytes = 8 if prec == g.PREC_MIXED else 16
    alg_b = U * 3 * cbytes + out_entries * 16
    hbm = peaks.get("hbm_gbs", 6800.0)
    ach_p = alg_b / (tp["ms"] / 1e3) / 1e9 if tp["ms"] > 0 else 0.0
    roof_p = {"kernel": ("pco_kernel<%s> (one CTA of 1024 threads per site: one-sided PCOs on "
                         "vectors, cross PCOs in place by level, physical PCOs as d - 1 passes of "
                         "l_L + l_R with odd-parity entries skipped; FP32 passes with FP64 plane "
                         "sums in mixed builds)") % ("float" if prec == g.PREC_MIXED else "double"),
              "bound": "hbm", "achieved": round(ach_p, 1), "peak": hbm,
              "peak_source": f"hbm_gbs of {src} MEASURED_PEAKS.json", "unit": "GB/s",
              "frac": round(ach_p / hbm, 4),
              "traffic": PCO_TRAFFIC_BYTES_PER_LAUNCH,
              "updates_per_state": U, "updates_per_s": round(U / (tp["ms"] / 1e3), 1) if tp["ms"] > 0 else None,
              "algorithmic_bytes_per_launch": alg_b / max(tp["launches"], 1),
              "algorithmic_bytes_def": ("the paper's update count U (Algs. 2, 4, 5 and the physical "
                                        "PCOs: (target, source, kappa) trip counts of the vector sets "
                                        "with the kappa match, counted from the kept bases) x (source "
                                        f"read + target read + target write) x {cbytes} B + the "
                                        "tensors written once (d D_l D_r x 16 B)"),
              "paper_estimate": "O(n_e^2 n~ d D^2) per tensor (Sec. II C)",
              "avg_launch_ms": tp["ms"] / max(tp["launches"], 1),
              "launches_per_step": tp["launches"], "ms_per_state": round(tp["ms"], 3),
              "share_of_step": round(tp["ms"] / step_ms_avg, 4),
              "note": ("the kernel regroups the PCOs (one-sided products on vectors, the physical "
                       "PCOs as d - 1 combined passes) and keeps its working set on chip and in "
                       "L2, so it moves far fewer bytes than the paper's algorithm would: frac "
                       "near or above 1 means it runs at or faster than that algorithm at the "
                       "HBM roof; traffic is its measured DRAM bytes per launch")}
    # the roofline object follows the kernel with the most device time per
    # state on the step's critical path (the Gaussian-SVD chains run on one
    # SM beside the step), the other is reported beside it
    if te["ms"] >= tr["ms"]:
        roof, roof_other = roof_e, dict(roof_s, name="sampler")
    else:
        roof, roof_other = roof_s, dict(roof_e, name="environments")

    # build-only throughput and the FP64 GPU path for comparison
    res = {}
    if rank == 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            m = g.MPS.from_cov(ctx, gam, **opts)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        res["build_ms"] = e0.elapsed_time(e1)
        pats = wl.random_patterns(256, N, w.d, seed=3)
        pats[0] = 0
        pats_d = torch.from_numpy(pats).to(f"cuda:{dev}")
        amp_mixed = m.amplitudes(pats)
        m.release()
        if not args.no_fp64:
            S64 = 2000
            with torch.cuda.stream(stream):
                e0.record(stream)
                m64 = g.MPS.from_cov(ctx, gam, **dict(opts, precision=g.PREC_FP64))
                e1.record(stream)
            torch.cuda.synchronize(dev)
            b64 = e0.elapsed_time(e1)
            e2 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                m64.sample(S64, seed=1234, counter0=0, out=out[:S64])
                e2.record(stream)
            torch.cuda.synchronize(dev)
            s64 = e1.elapsed_time(e2)
            s64_ms_step = b64 + s64 * (S / S64)
            amp64 = m64.amplitudes(pats)
            rel = np.abs(amp_mixed - amp64) / np.maximum(np.abs(amp64), 1e-300)
            big = np.abs(amp64) >= 1e-3 * np.abs(amp64).max()
            # shared-seed sample agreement between the two paths
            mref = g.MPS.from_cov(ctx, gam, **opts)
            s_a = torch.empty((S64, N), dtype=torch.uint8, device=f"cuda:{dev}")
            mref.sample(S64, seed=99, counter0=0, out=s_a)
            s_b = torch.empty_like(s_a)
            m64.sample(S64, seed=99, counter0=0, out=s_b)
            agree = float((s_a == s_b).all(dim=1).float().mean().item())
            mref.release()
            m64.release()
            res["fp64_gpu"] = {
                "build_ms": round(b64, 3), "sample_ms_per_1k": round(s64 / S64 * 1e3, 3),
                "ms_per_step_extrapolated": round(s64_ms_step, 1),
                "tensors_per_s": round(N / (s64_ms_step / 1e3), 3),
                "samples_per_s": round(S / (s64_ms_step / 1e3), 1),
                "sample": f"FP64 build timed in full; sampling timed on {S64} samples and scaled to {S}",
                "note": ("the plain FP64 GPU path: FP64 PCO passes, dense FP64 environments (no "
                         "parity blocks, no energy gauge), sampling by dense w R w^dag per sample "
                         "(no right-canonical form, no p = 0 pre-pass); the ratio to the mixed "
                         "path includes these algorithmic changes as well as the precision"),
                "mixed_vs_fp64_amp_max_rel_err": float(rel[big].max()),
                "mixed_vs_fp64_amp_max_abs_err_rel_to_max": float(np.abs(amp_mixed - amp64).max() / np.abs(amp64).max()),
                "shared_seed_sample_agreement": agree}
        del pats_d

    # end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        gam_h = torch.from_numpy(np.ascontiguousarray(w.gamma)).pin_memory()
        out_h = torch.empty((S, N), dtype=torch.uint8).pin_memory()
        K2 = max(1, args.steps)
        out_h2 = torch.empty_like(out_h).pin_memory()
        barrier()
        t0 = time.perf_counter()
        if pipelined:
            stream_steps(20_000, K2, gam_src=gam_h, outs=[(out_h, out_h2)[j % 2] for j in range(K2)])
        else:
            for i in range(K2):
                m = g.MPS.from_cov(ctx, gam_h, **opts)
                m.sample(S, seed=4321 + rank, counter0=i * S, out=out_h)
                m.release()
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        te = max_over_ranks(t1 - t0, dist)
        e2e = {"value": round(N * K2 * ws / te, 3), "unit": "tensors/s",
               "samples_per_s": round(S * K2 * ws / te, 1),
               "h2d_bytes_per_step": int(gam_h.numel() * 8), "d2h_bytes_per_step": int(S * N),
               "steps": K2}
    ctx.close()
    return dict(value=value, samples_per_s=samples_per_s, step_ms=step_ms, launches=launches,
                ms_per_step=total_s * 1e3 / args.steps, pipelined=pipelined,
                roof=roof, roof_other=roof_other, roof_pco=roof_p, clocks=clk.summary(), e2e=e2e,
                **res)


# --------------------------------------------------------------------------- large configuration
def run_large(args, dev):
    """The 1024-mode configuration (r~U(0.05,0.25), depth-32 brick wall,
    d = 4, chi = 512) in mixed precision: one build and 1,000,000 samples,
    each timed with CUDA events on the launching stream, and the sampler
    GEMM traced over the sampling (its tensor-roof fraction)."""
    import numpy as np
    import torch

    import paper_2512_10643_gb300 as g
    import workloads as wl

    w = wl.config("n1024_d4_chi512")
    S = 1_000_000
    stream = torch.cuda.Stream(device=dev)
    ctx = g.Context(dev, stream.cuda_stream)
    gam = torch.from_numpy(np.ascontiguousarray(w.gamma)).to(f"cuda:{dev}")
    out = torch.empty((S, w.N), dtype=torch.uint8, device=f"cuda:{dev}")
    opts = dict(d=w.d, chi_max=w.chi, eps_trunc=w.eps, lambda2_freeze=w.freeze,
                precision=g.PREC_MIXED)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize(dev)
    g.gbsmps_trace(ctx.h, True)
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        m = g.MPS.from_cov(ctx, gam, **opts)
        ev[1].record(stream)
        m.sample(S, seed=77, counter0=0, out=out)
        ev[2].record(stream)
    torch.cuda.synchronize(dev)
    tr = g.gbsmps_trace_read_kernel(ctx.h, 0)
    g.gbsmps_trace(ctx.h, False)
    build_ms, sample_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    photons = out.to(torch.int64).sum(dim=1)
    even = bool((photons % 2 == 0).all().item())
    mean_ph = float(photons.float().mean().item())
    dims = [int(x) for x in m.info["bond_dims"]]
    # out of core: the sampler planes in pinned host memory, streamed site by
    # site through a three-slot device ring; the same patterns
    free0 = torch.cuda.mem_get_info(dev)[0]
    host_bytes = m.offload()
    free1 = torch.cuda.mem_get_info(dev)[0]
    out2 = torch.empty_like(out)
    with torch.cuda.stream(stream):
        ev[1].record(stream)
        m.sample(S, seed=77, counter0=0, out=out2)
        ev[2].record(stream)
    torch.cuda.synchronize(dev)
    ooc_ms = ev[1].elapsed_time(ev[2])
    same = bool(torch.equal(out, out2))
    m.release()
    ctx.close()
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    ach = tr["flops"] / (tr["ms"] / 1e3) / 1e12 if tr["ms"] > 0 else 0.0
    return {"workload": ("1024-mode pure Gaussian state: squeezed vacua r~U(0.05,0.25) through a "
                         "depth-32 brick-wall network; d=4, chi=512, eps=1e-12, lambda2_freeze=1e-9; "
                         "mixed precision; Gamma on the device"),
            "build_ms": round(build_ms, 2), "sample_ms": round(sample_ms, 2), "samples": S,
            "tensors_per_s_build": round(w.N / (build_ms / 1e3), 1),
            "samples_per_s": round(S / (sample_ms / 1e3), 1),
            "tensors_per_s_whole": round(w.N / ((build_ms + sample_ms) / 1e3), 1),
            "max_bond_dim": max(dims), "mean_photons": round(mean_ph, 3),
            "all_samples_even": even,
            "out_of_core": {"sample_ms": round(ooc_ms, 2),
                            "samples_per_s": round(S / (ooc_ms / 1e3), 1),
                            "host_plane_bytes": host_bytes,
                            "h2d_gbs": round(host_bytes / (ooc_ms / 1e3) / 1e9, 1),
                            "device_bytes_freed": int(free1 - free0),
                            "same_patterns_as_resident": same,
                            "def": ("gbsmps_offload: sampler planes in pinned host memory, "
                                    "streamed through three device slots by a copy stream")},
            "sampler_gemm": {"ms": round(tr["ms"], 2), "launches": tr["launches"],
                             "achieved_tflops": round(ach, 3), "peak": peak,
                             "frac": round(ach / peak, 5), "issued_frac": round(3 * ach / peak, 5),
                             "share_of_sampling": round(tr["ms"] / sample_ms, 4) if sample_ms > 0 else None,
                             "peak_source": f"bf16_tflops_sustained of {src} MEASURED_PEAKS.json"}}


# --------------------------------------------------------------------------- mixed -> pure
def run_filtration(args, dev):
    """The step before the path (Sec. III Eq. (decompose), App. C): lossy
    64-mode covariances (squeezed vacua r~U(0.3,0.8) through a depth-16
    brick wall, then uniform loss eta = 0.5: Gamma_th = eta Gamma +
    (1 - eta) I / 2, shaped like the paper's 64-mode configuration) split
    into a pure part and noise by the App. C descent (alpha = 0.01, eps =
    1e-10), all states in one batched call (one state per SM).  The oracle is
    timed on a bounded number of steps of one state beside it."""
    import numpy as np
    import torch

    import paper_2512_10643_gb300 as g
    import workloads as wl

    N, count, alpha, eps = 64, args.filter_states, 0.01, 1e-10
    gths = np.stack([wl.lossy(N, 3000 + i, eta=0.5, depth=16)[0] for i in range(count)])
    stream = torch.cuda.Stream(device=dev)
    ctx = g.Context(dev, stream.cuda_stream)
    gd = torch.from_numpy(gths).to(f"cuda:{dev}")
    g.gbsmps_filter(ctx.h, gd[:1], alpha, eps=eps, max_iter=2)          # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        e0.record(stream)
        S, iters, loss = g.gbsmps_filter(ctx.h, gd, alpha, eps=eps, max_iter=100000)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    ctx.close()
    Sh = S.cpu().numpy()
    n_eff = [0.5 * np.trace(0.5 * x @ x.T) - 0.5 * N for x in Sh]
    n = 2 * N
    # per step: the tridiagonalisation (4/3 n^3), the Sturm multisection
    # (11 rounds x 32 points x 3n), the back transformation and gradient step
    # (~18 n^2), the recomputation of W every 64 steps (n^3)
    fl_step = 4.0 / 3.0 * n ** 3 + 11 * 32 * 3 * n + 18 * n ** 2 + n ** 3 / 64
    flops = fl_step * float(np.sum(iters))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_peak = nsm * 2 * 2 * 2.07e9 / 1e12        # 2 FP64 FMA per clock per SM
    # the CPU baseline: the oracle on a bounded number of steps of one state,
    # scaled by the steps a state takes
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import filtration as F
        t = time.perf_counter()
        K = 20
        F.filtration(gths[0], alpha, eps=0.0, max_iter=K)
        per_step = (time.perf_counter() - t) / K
        ora_state_s = per_step * float(np.mean(iters))
        cpu = {"s_per_state": round(ora_state_s, 2), "value": round(1.0 / ora_state_s, 4),
               "unit": "states/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{K} steps of one state (numpy eigh + expm per step), scaled to the "
                         "mean step count of the GPU run"}
    return {"workload": ("lossy 64-mode covariances: squeezed vacua r~U(0.3,0.8) through a depth-16 "
                         "brick-wall network, uniform transmission eta = 0.5; App. C descent with "
                         "alpha = 0.01, eps = 1e-10"),
            "states": count, "ms": round(ms, 2), "states_per_s": round(count / (ms / 1e3), 2),
            "steps_mean": float(np.mean(iters)), "steps_max": int(np.max(iters)),
            "converged": int(np.sum(loss <= eps)), "n_eff_mean": round(float(np.mean(n_eff)), 5),
            "roofline": {"bound": "alu", "achieved": round(flops / (ms / 1e3) / 1e12, 4),
                         "peak": round(fp64_peak, 3), "unit": "TFLOP/s",
                         "frac": round(flops / (ms / 1e3) / 1e12 / fp64_peak, 4),
                         "peak_source": (f"derived: {nsm} SMs x 2 FP64 FMA per clock x 2 flops x "
                                         "2070 MHz (GB300's FP64 rate)"),
                         "algorithmic_flops_def": ("per step 4/3 n^3 (tridiagonalisation) + "
                                                   "11 x 32 x 3n (Sturm counts) + 18 n^2 (back "
                                                   "transformation, gradient, rank-2 updates) + "
                                                   "n^3 / 64 (W recomputed every 64 steps), n = 2N")},
            "cpu_baseline": cpu}


# --------------------------------------------------------------------------- batched build
def run_batched(args, dev):
    """Many independent states built in one batched call (all GSVD chains in
    one launch, all PCO tensors together, the environment chains in one
    persistent launch) against the same states built one call at a time."""
    import numpy as np
    import torch

    import paper_2512_10643_gb300 as g
    import workloads as wl

    states = wl.batch(args.batch_states)
    stream = torch.cuda.Stream(device=dev)
    ctx = g.Context(dev, stream.cuda_stream)
    gams = [torch.from_numpy(np.ascontiguousarray(w.gamma)).to(f"cuda:{dev}") for w in states]
    opts = [dict(d=w.d, chi_max=w.chi, eps_trunc=w.eps, lambda2_freeze=w.freeze,
                 precision=g.PREC_MIXED) for w in states]
    tensors = sum(w.N for w in states)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            e0.record(stream)
            ms = fn()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        for m in ms:
            m.release()
        return e0.elapsed_time(e1)

    batch_fn = lambda: g.MPS.batch(ctx, gams, opts)
    seq_fn = lambda: [g.MPS.from_cov(ctx, x, **o) for x, o in zip(gams, opts)]
    timed(batch_fn)                                   # warm-up
    n0 = g.gbsmps_launch_count()
    t_b = min(timed(batch_fn) for _ in range(2))
    n_b = (g.gbsmps_launch_count() - n0) // 2
    n0 = g.gbsmps_launch_count()
    t_s = timed(seq_fn)
    n_s = g.gbsmps_launch_count() - n0
    ctx.close()
    return {"states": len(states), "tensors": tensors,
            "batched_ms": round(t_b, 2), "sequential_ms": round(t_s, 2),
            "tensors_per_s_batched": round(tensors / (t_b / 1e3), 1),
            "tensors_per_s_sequential": round(tensors / (t_s / 1e3), 1),
            "speedup": round(t_s / t_b, 2), "launches_batched": int(n_b),
            "launches_sequential": int(n_s),
            "workload": ("N~U{16..144}, r~U(0.1,0.5), brick-wall depth N/8, d=6, "
                         "chi in {32,64,128,256}, eps 1e-12, lambda2_freeze 1e-9; mixed precision; "
                         "build only (Gamma on the device)")}


# --------------------------------------------------------------------------- serving
def run_serving(args, dev, rate):
    """Poisson-arriving build + sampling requests through the library's
    request loop (gbsmps_server_*): N log-uniform in [32, 512], r~U(0.05,0.4),
    depth N/16, d in {4, 6}, chi in {64..512}, 1e3..1e5 samples each.
    Reports latency quantiles and throughput over the busy period."""
    import paper_2512_10643_gb300 as g
    import workloads as wl

    reqs = wl.serving(args.serving_requests, rate)
    t0 = time.perf_counter()
    ids = []
    with g.Server(dev, slots=args.serving_slots, batch_max=args.serving_batch) as srv:
        start = time.perf_counter()
        for t_arr, w, S in reqs:
            delay = t_arr - (time.perf_counter() - start)
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(w.gamma, S, seed=17, counter0=0, d=w.d, chi_max=w.chi,
                                  eps_trunc=w.eps, lambda2_freeze=w.freeze,
                                  precision=g.PREC_MIXED))
        srv.drain()
        infos = [srv.wait(i)[1] for i in ids]
        st = srv.stats()
    busy = st["busy_s"]
    return {"requests": len(reqs), "arrival_rate_hz": rate,
            "slots": args.serving_slots, "batch_max": args.serving_batch,
            "mean_batch": round(sum(x["batch"] for x in infos) / max(len(infos), 1), 2),
            "completed": st["completed"], "failed": st["failed"],
            "latency_ms": {"p50": round(st["p50_ms"], 2), "p99": round(st["p99_ms"], 2),
                           "mean": round(st["mean_ms"], 2)},
            "tensors_per_s": round(st["tensors"] / busy, 2) if busy > 0 else None,
            "samples_per_s": round(st["samples"] / busy, 1) if busy > 0 else None,
            "busy_s": round(busy, 3), "wall_s": round(time.perf_counter() - t0, 3),
            "max_concurrent": max(sum(1 for y in infos if y["t_admit"] <= x["t_admit"] < y["t_done"])
                                  for x in infos) if infos else 0,
            "hbm_peak_gb": round(st["hbm_peak"] / 1e9, 2),
            "workload": ("Poisson arrivals; N log-U[32,512], r~U(0.05,0.4), brick-wall depth N/16, "
                         "d in {4,6}, chi in {64,128,256,512}, samples U{1e3..1e5}; mixed precision; "
                         "latency = submit -> patterns in host memory")}


# --------------------------------------------------------------------------- oracle (CPU)
def oracle_step_estimate(budget_s=20.0):
    """Time the FP64 oracle on a bounded sample of the same workload and scale
    to one step (all 144 tensors + 100k samples)."""
    import numpy as np

    import workloads as wl
    from oracle import basis as B
    from oracle import gaussian as G
    from oracle import mps as M
    from oracle import pco as P

    w = wl.config(WORKLOAD)
    t0 = time.perf_counter()
    cuts = G.gsvd_chain(w.gamma, lambda2_freeze=w.freeze)
    bases = [M.vacuum_basis()] + [B.kept_basis(c.lam2, w.chi, w.eps) for c in cuts[:-1]] + [M.vacuum_basis()]
    t_chain = time.perf_counter() - t0
    sites = [71, 36, 108, 72, 20, 124]
    t_pco, n_pco, tensors = 0.0, 0, {}
    for s in sites:
        t = time.perf_counter()
        tensors[s] = P.local_tensor(cuts[s].Q, bases[s], bases[s + 1], w.d, cuts[s].c)
        t_pco += time.perf_counter() - t
        n_pco += 1
        if t_pco > budget_s * 0.5:
            break
    per_site_pco = t_pco / n_pco
    A = tensors[71]
    Dl, Dr = A.shape[0], A.shape[2]
    # one right-environment step through a central tensor
    t = time.perf_counter()
    for _ in range(3):
        M.environments([A, np.ones((Dr, 1, 1), dtype=np.complex128)])
    per_site_env = (time.perf_counter() - t) / 3
    # conditional sampling through the same tensor: a 1 x 1 x Dl opening
    # tensor then A, with identity environments (cost is shape-determined)
    S0 = 200
    u = wl.uniforms(S0, 2, seed=1)
    TT = [np.ones((1, 1, Dl), dtype=np.complex128) / np.sqrt(Dl), A]
    Rs = [None, np.eye(Dl, dtype=np.complex128), np.eye(Dr, dtype=np.complex128)]
    t = time.perf_counter()
    M.sample(TT, u, R=Rs)
    per_sample_site = (time.perf_counter() - t) / S0
    full_sites = sum(1 for b in bases[1:-1] if b.D == w.chi)
    step_s = (t_chain + w.N * (per_site_pco + per_site_env) + 100_000 * full_sites * per_sample_site)
    sample_desc = (f"oracle GSVD chain + kept bases over all {w.N - 1} cuts ({t_chain:.2f}s), PCO build of "
                   f"{n_pco} central sites ({per_site_pco:.2f}s/site), one environment step and "
                   f"{S0} conditional samples through one central site, scaled to {w.N} sites and "
                   f"100000 samples per step")
    return {"step_s": step_s, "value": w.N / step_s, "samples_per_s": 100_000 / step_s,
            "sample": sample_desc, "cores": os.cpu_count(), "measured_s": time.perf_counter() - t0}


def oracle_config_timings(budget_s=8.0):
    """The FP64 oracle timed on the small configuration (the 8-mode state
    through a Haar unitary, d = 8, chi = 64: the full build) and on the
    64-site prefix of the 1024-mode configuration (its GSVD chain over all
    cuts, the kept bases of bonds 1..64, and the PCO build of prefix sites
    at the full bond dimension within budget_s, scaled to the 64 sites)."""
    import workloads as wl
    from oracle import basis as B
    from oracle import gaussian as G
    from oracle import mps as M
    from oracle import pco as P

    out = {}
    w = wl.config("pr1_n8")
    t0 = time.perf_counter()
    mps = M.build_mps(w.gamma, d=w.d, chi=w.chi)
    M.normalise(mps.tensors)
    t = time.perf_counter() - t0
    out["c1"] = {"tensors_per_s": round(w.N / t, 3), "build_s": round(t, 3),
                 "sample": f"full oracle build of the {w.N}-mode state (d = {w.d}, chi = {w.chi})"}
    w = wl.config("n1024_d4_chi512")
    K = 64
    t0 = time.perf_counter()
    cuts = G.gsvd_chain(w.gamma, lambda2_freeze=w.freeze)
    t_chain = time.perf_counter() - t0
    bases = [M.vacuum_basis()] + [B.kept_basis(c.lam2, w.chi, w.eps) for c in cuts[:K]]
    t_bases = time.perf_counter() - t0 - t_chain
    t_pco, n_pco = 0.0, 0
    for s in range(K - 1, -1, -1):          # the last prefix sites: full bond dimension
        t = time.perf_counter()
        P.local_tensor(cuts[s].Q, bases[s], bases[s + 1], w.d, cuts[s].c)
        t_pco += time.perf_counter() - t
        n_pco += 1
        if t_pco > budget_s:
            break
    prefix_s = t_chain + t_bases + K * t_pco / n_pco
    out["c4_prefix"] = {"tensors_per_s": round(K / prefix_s, 4),
                        "gsvd_cuts_per_s": round((w.N - 1) / t_chain, 1),
                        "prefix_s": round(prefix_s, 2),
                        "sample": (f"oracle GSVD chain over all {w.N - 1} cuts ({t_chain:.2f}s), kept bases "
                                   f"of bonds 1..{K} ({t_bases:.2f}s), PCO build of the last {n_pco} prefix "
                                   f"sites at D = {bases[K].D} ({t_pco / n_pco:.2f}s/site), scaled to the "
                                   f"{K}-site prefix")}
    return out


def profile_pass(args):
    """One build (and one sampling) of the workload, nothing else timed or
    printed but a checksum: the launch sequence a profiler capture skips
    into (the kernel launches of one build, then 2 per site of sampling)."""
    import numpy as np
    import torch

    import paper_2512_10643_gb300 as g
    import workloads as wl

    if args.profile_pass == "filter":
        # eight lossy 64-mode states, 20 steps of the App. C descent
        gths = np.stack([wl.lossy(64, 3000 + i, eta=0.5, depth=16)[0] for i in range(8)])
        ctx = g.Context(0)
        S, it, loss = g.gbsmps_filter(ctx.h, gths, 0.01, eps=1e-10, max_iter=20)
        ctx.close()
        print("steps", int(it.sum()), "loss", float(loss.max()))
        return
    w = wl.config(WORKLOAD)
    ctx = g.Context(0)
    prec = g.PREC_MIXED if args.precision == "mixed" else g.PREC_FP64
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=w.d, chi_max=w.chi, eps_trunc=w.eps,
                       lambda2_freeze=w.freeze, precision=prec)
    try:
        if args.profile_pass == "sample":
            out = torch.empty((args.samples, w.N), dtype=torch.uint8, device="cuda:0")
            m.sample(args.samples, seed=1, counter0=0, out=out)
            torch.cuda.synchronize()
            print("photons", int(out.sum()))
        else:
            print("bond dims", m.info["bond_dims"][w.N // 2])
    finally:
        m.release()
        ctx.close()


def main():
    args = parse()
    if args.profile_pass:
        profile_pass(args)
        return
    rank, local, ws, dist = dist_init()
    base = {"metric": METRIC, "unit": "tensors/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic (seeded Philox; paper's experimental data not available)"}
    cfg = {"workload": WORKLOAD_DESC, "name": WORKLOAD, "samples_per_step": args.samples,
           "precision": args.precision, "inputs": "device-resident; working set > L2 (no flush needed)",
           "parallelism": f"replicas x{ws}"}
    if args.impl == "reference":
        if rank != 0:
            return
        est = oracle_step_estimate(args.ref_budget)
        line = dict(base, impl="reference", value=round(est["value"], 6),
                    ms_per_step=round(est["step_s"] * 1e3, 1), dtype="f64", config=cfg,
                    samples_per_s=round(est["samples_per_s"], 3),
                    cpu_baseline={"value": round(est["value"], 6), "unit": "tensors/s",
                                  "cores": est["cores"], "kind": "oracle", "sample": est["sample"]},
                    e2e={"value": round(est["value"], 6), "unit": "tensors/s",
                         "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
        print(json.dumps(line))
        return
    r = run_gpu(args, rank, local, ws, dist)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        est = oracle_step_estimate(args.ref_budget)
        cpu = {"value": round(est["value"], 6), "unit": "tensors/s", "cores": est["cores"],
               "kind": "oracle", "sample": est["sample"],
               "samples_per_s": round(est["samples_per_s"], 3),
               "configs": oracle_config_timings()}
    sm = sorted(r["step_ms"])
    if r["pipelined"]:
        cfg["pipeline"] = ("one stream of steps: the next states' Gaussian-SVD chains (one SM) and "
                           "the next state's environments and canonical form run beside the current sampling; "
                           "latency_ms is one state alone, build + sampling")
    line = dict(base, value=round(r["value"], 3), ms_per_step=round(r["ms_per_step"], 3),
                dtype=("f64 gsvd + f32 pco (f64 plane sums) + exact bf16-slice tensor-core env + fp16x2 (3 products)/fp32 tensor-core sampling"
                       if args.precision == "mixed" else "f64"),
                config=cfg, samples_per_s=round(r["samples_per_s"], 1),
                latency_ms={"p50": round(statistics.median(sm), 3),
                            "p99": round(sm[min(len(sm) - 1, max(0, int(math.ceil(0.99 * len(sm))) - 1))], 3),
                            "runs": len(sm), "max": round(sm[-1], 3),
                            "def": "one state alone: build + 100k samples, nothing overlapped; "
                                   "nearest-rank quantiles"},
                build_ms=round(r.get("build_ms", 0.0), 3),
                roofline=r["roof"], roofline_other=r["roof_other"], roofline_pco=r["roof_pco"],
                cpu_baseline=cpu, e2e=r["e2e"],
                gpu_launches=r["launches"],
                clocks=r["clocks"])
    if "fp64_gpu" in r:
        line["fp64_gpu"] = r["fp64_gpu"]
    # supplementary sections: a failure is recorded in the line, not fatal
    if ws == 1 and args.batch_states > 0:
        try:
            line["batched"] = run_batched(args, local)
        except Exception as e:          # noqa: BLE001
            line["batched"] = {"error": f"{type(e).__name__}: {e}"}
    if ws == 1 and args.filter_states > 0:
        try:
            line["filtration"] = run_filtration(args, local)
        except Exception as e:          # noqa: BLE001
            line["filtration"] = {"error": f"{type(e).__name__}: {e}"}
    if ws == 1 and args.large:
        try:
            line["large"] = run_large(args, local)
        except Exception as e:          # noqa: BLE001
            line["large"] = {"error": f"{type(e).__name__}: {e}"}
    if ws == 1 and args.serving_requests > 0:
        sweep = []
        for rate in [float(x) for x in args.serving_rates.split(",") if x.strip()]:
            try:
                sweep.append(run_serving(args, local, rate))
            except Exception as e:          # noqa: BLE001
                sweep.append({"arrival_rate_hz": rate, "error": f"{type(e).__name__}: {e}"})
        line["serving"] = sweep
    print(json.dumps(line))


if __name__ == "__main__":
    main()
