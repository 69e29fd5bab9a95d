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
# DRAM bytes (read + write) per launch from an ncu capture of the current
# kernels (None until one is taken): the sampler GEMM at 100,000 samples, and
# the environment GEMM of the 144-mode workload (the same at any sample count)
TRAFFIC_BYTES_PER_LAUNCH = 92.3e6          # (69032.0 + 37278.6) MB over 1152 launches
ENV_TRAFFIC_BYTES_PER_LAUNCH = 5.01e6       # (7214.2 + 0.1) MB over 1440 launches
# A double-float multiply-add (2 flops of the FP64 algorithm) costs 12 FP32
# instructions: the exact product by FMA (4, with the low words) and Knuth's
# TwoSum into the (hi, lo) accumulator (6) plus the low-word update (2)
DF64_FP32_INSTR_PER_FMA = 12
FP32_LANES_PER_SM = 128


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
    ap.add_argument("--serving-requests", type=int, default=24)
    ap.add_argument("--serving-rate", type=float, default=4.0)
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--profile-pass", default=None, choices=["build", "sample"],
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
    if pipelined:
        # latency of one state alone (build + sampling, nothing overlapped)
        lat = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        barrier()
        with torch.cuda.stream(stream):
            lat[0].record(stream)
            for i in range(args.steps):
                step(args.warmup + args.steps + i)
                lat[i + 1].record(stream)
        barrier()
        step_ms = [lat[i].elapsed_time(lat[i + 1]) for i in range(args.steps)]
    else:
        step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]

    # dominant kernel, traced over one extra step outside the timed region
    g.gbsmps_trace(ctx.h, True)
    step(10_000)
    torch.cuda.synchronize(dev)
    tr = g.gbsmps_trace_read_kernel(ctx.h, 0)
    te = g.gbsmps_trace_read_kernel(ctx.h, 1)
    g.gbsmps_trace(ctx.h, False)
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
    # the environment GEMM against the FP32 pipe's double-float roof
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fmax = (clk.summary().get("sm_max_mhz") or 2070.0) * 1e6
    df_peak = nsm * FP32_LANES_PER_SM * fmax * 2.0 / DF64_FP32_INSTR_PER_FMA / 1e12
    ne = max(te["launches"], 1)
    ach_df = te["flops"] / (te["ms"] / 1e3) / 1e12 if te["ms"] > 0 else 0.0
    roof_e = {"kernel": "zgemm_df64_grouped_kernel (double-float complex GEMM on the FP32 pipes, "
                        "right-environment chain R_m = sum_p Ahat^m[p] R_{m+1} Ahat^m[p]^dag on the "
                        "parity blocks; two grouped launches per site, split-K partials summed in k "
                        "order by each tile's last CTA)",
              "bound": "alu", "achieved": round(ach_df, 4), "peak": round(df_peak, 3),
              "peak_source": (f"derived: {nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                              f"{fmax / 1e6:.0f} MHz (max SM clock) x 2 flops / "
                              f"{DF64_FP32_INSTR_PER_FMA} FP32 instructions per double-float "
                              "multiply-add"),
              "unit": "TFLOP/s", "frac": round(ach_df / df_peak, 5) if df_peak > 0 else None,
              "traffic": ENV_TRAFFIC_BYTES_PER_LAUNCH,
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
                roof=roof, roof_other=roof_other, clocks=clk.summary(), e2e=e2e, **res)


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
def run_serving(args, dev):
    """Poisson-arriving build + sampling requests through the library's
    request loop (gbsmps_server_*): N log-uniform in [32, 512], r~U(0.05,0.4),
    depth N/16, d in {4, 6}, chi in {64..512}, 1e3..1e5 samples each.
    Reports latency quantiles and throughput over the busy period."""
    import paper_2512_10643_gb300 as g
    import workloads as wl

    reqs = wl.serving(args.serving_requests, args.serving_rate)
    t0 = time.perf_counter()
    ids = []
    with g.Server(dev, slots=args.serving_slots) as srv:
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
    return {"requests": len(reqs), "arrival_rate_hz": args.serving_rate,
            "slots": args.serving_slots, "completed": st["completed"], "failed": st["failed"],
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


def profile_pass(args):
    """One build (and one sampling) of the workload, nothing else timed or
    printed but a checksum: the launch sequence a profiler capture skips
    into (the kernel launches of one build, then 2 per site of sampling)."""
    import numpy as np
    import torch

    import paper_2512_10643_gb300 as g
    import workloads as wl

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
               "samples_per_s": round(est["samples_per_s"], 3)}
    sm = sorted(r["step_ms"])
    if r["pipelined"]:
        cfg["pipeline"] = ("one stream of steps: the next states' Gaussian-SVD chains (one SM) and "
                           "the next state's environments and canonical form run beside the current sampling; "
                           "latency_ms is one state alone, build + sampling")
    line = dict(base, value=round(r["value"], 3), ms_per_step=round(r["ms_per_step"], 3),
                dtype=("f64 gsvd + f32 pco (f64 plane sums) + df64 env + fp16x2 (3 products)/fp32 tensor-core sampling"
                       if args.precision == "mixed" else "f64"),
                config=cfg, samples_per_s=round(r["samples_per_s"], 1),
                latency_ms={"p50": round(statistics.median(sm), 3),
                            "p99": round(sm[min(len(sm) - 1, int(0.99 * len(sm)))], 3)},
                build_ms=round(r.get("build_ms", 0.0), 3),
                roofline=r["roof"], roofline_other=r["roof_other"], cpu_baseline=cpu, e2e=r["e2e"],
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
    if ws == 1 and args.serving_requests > 0:
        try:
            line["serving"] = run_serving(args, local)
        except Exception as e:          # noqa: BLE001
            line["serving"] = {"error": f"{type(e).__name__}: {e}"}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
