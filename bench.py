"""Benchmark of the EPWI + SERTA transport hot path on GB300.

One step = the whole hot path on the Al-like metal at a 48^3 k and q grid (seeded synthetic
inputs resident on the device): H(k)/D(q) eigensolves -> +-0.3 eV window -> sieve ->
q-batched g(k,q) interpolation with SERTA delta sums -> sigma.  The step time is the
time-to-sigma; ``value`` is the sieved (k,q) pairs per second of that step.
``e2e`` repeats the step through the C ABI from host buffers (setup copies H, Phi, g from
the host; the rates, states and sigma come back to the host) inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl reference]
Under torchrun (N > 1) every rank runs an independent copy of the workload (weak scaling,
no data-path collective); rank 0 prints the line with the max time over ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "el-ph (k,q)-pairs/s and time-to-σ, mixed-precision vs FP64 at stated error"
WORKLOAD = dict(workload="al_like_48", system="Al-like fcc, nw=4, 3 modes, 5^3 WS-weighted Re/Rp",
                grid=48, window_eV=0.3, smear_eV=0.02, T_K=300.0, mu="band centre", seed=2)
CHOSEN = "fp32"
DTYPE = {"fp64": "f64", "tf32x3": "tf32x3 (f32 acc, f64 sums)", "bf16x3": "bf16x3 (f32 acc, f64 sums)",
         "fp16x3": "fp16x3 (f32 acc, f64 sums)", "fp32": "f32 (sum-factorised, f64 sums)"}
L2_BYTES = 129 * 2 ** 20
# DRAM bytes (read + write) per (k,q) pair of the dominant kernel, from one ncu capture each:
# k_scatter_tc (fp16x3) at 24^3, 255 MB / 19.6 M pairs (ncu --set full); k_scatter_sf (fp32,
# band-major k+q tables) at 32^3, 624.1 + 4.2 MB / 110.2 M pairs (ncu --set full).  Traffic grows
# with the pairs processed, so a launch's traffic is this times its pairs.  Valid for the kernel
# versions of those captures.
TRAFFIC_BYTES_PER_PAIR = {"fp16x3": 13.0, "fp32": 5.70}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return mp, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def fma_peaks(device=0, stream=None):
    """FP32 and FP64 FMA peaks (TFLOP/s) measured live by the library's throughput probe
    (epwi_fma_peak: register-only FMA chains on every SM, best of three ~50 ms launches).
    Falls back to the unit-count figures only if the probe fails."""
    from paper_2306_16493_gb300 import epwi
    out = {}
    for name, fp64, derived in (("fp32", False, FP32_PEAK_TFLOPS), ("fp64", True, FP64_PEAK_TFLOPS)):
        try:
            tf, ms = epwi.epwi_fma_peak(fp64, device, stream)
            out[name] = (tf, f"measured: FMA probe epwi_fma_peak ({name}, best of 3 launches of {ms:.0f} ms)")
        except Exception as e:                     # noqa: BLE001
            out[name] = (derived, f"derived from unit counts x 2.07 GHz (probe failed: {e})")
    return out


def roofline_for(precision, stats, per_launch_traffic=None, simt_peaks=None):
    """Dominant kernel: the fused Rp->q + rotation + delta kernel (one launch per chunk)."""
    mp, src = peaks()
    flops = stats["scatter_flops"]
    ms = stats["ms_scatter"]
    simt = simt_peaks or {"fp32": (FP32_PEAK_TFLOPS, "derived from unit counts"),
                          "fp64": (FP64_PEAK_TFLOPS, "derived from unit counts")}
    if precision in ("fp64", "fp32"):
        # CUDA-core FMA work: FP64 path, or the sum-factorised FP32 kernel
        peak, note = simt[precision]
        bound, unit = "alu", "TFLOP/s"
        achieved = flops / (ms * 1e-3) / 1e12
    else:
        ratio = 0.5 if precision == "tf32x3" else 1.0
        peak = mp["bf16_tflops"] * ratio
        bound, unit = "tensor", "TFLOP/s"
        achieved = 3.0 * flops / (ms * 1e-3) / 1e12      # three split products
        note = f"{src} bf16 burst peak x {ratio}"
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": per_launch_traffic, "traffic_unit": "bytes per launch",
            "kernel": ("k_scatter_sf (sum-factorised Rp->q + rotations + delta sum)" if precision == "fp32"
                       else "k_scatter (fused Rp->q GEMM + rotations + delta sum)"),
            "launches_per_step": stats["n_chunks"], "peak_source": note}


class ClockSampler:
    def __init__(self, out):
        self.out = out
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()
            self.f.close()

    def summary(self, device=0):
        try:
            rows = [r.split(",") for r in open(self.out).read().strip().splitlines()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = [[x.strip() for x in r] for r in rows if r and r[0].strip() == str(device)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------------- oracle arm
def oracle_sample(sysm, gr, nkp_sample, seed, T, eta, mu, full=False):
    """Times the FP64 CPU oracle on a seeded sample of k-points of the workload.  Returns
    (pairs, seconds), or (pairs, seconds, oracle result) with ``full``."""
    from oracle import epwi_oracle as O
    ik_all, _ = gr.window_states(mu - WORKLOAD["window_eV"], mu + WORKLOAD["window_eV"])
    kp = np.unique(ik_all)
    pick = np.random.default_rng(seed).choice(kp, nkp_sample, replace=False)
    t0 = time.perf_counter()
    r = O.serta(gr, T, mu, eta, mu - WORKLOAD["window_eV"], mu + WORKLOAD["window_eV"],
                k_subset=pick)
    dt = time.perf_counter() - t0
    return (r["n_pairs"], dt, r) if full else (r["n_pairs"], dt)


def group_rel_error(ik, n, r, ref_ik, ref_n, ref_r, eps, tol=1e-6):
    """Largest relative error of 1/tau over degenerate groups (states at one k whose energies
    differ by < tol eV; only their sums are gauge invariant), over the states of the reference.
    Each group's error is relative to its own reference rate.  Returns (max, groups)."""
    def groups(ik_, n_, r_):
        o = np.lexsort((n_, ik_))
        ik_, n_, r_ = ik_[o], n_[o], r_[o]
        out, i = {}, 0
        while i < len(ik_):
            j = i + 1
            while j < len(ik_) and ik_[j] == ik_[i] and abs(eps[ik_[j], n_[j]] - eps[ik_[j - 1], n_[j - 1]]) < tol:
                j += 1
            out[(int(ik_[i]), int(n_[i]))] = float(r_[i:j].sum())
            i = j
        return out
    ref = groups(np.asarray(ref_ik), np.asarray(ref_n), np.asarray(ref_r))
    sel = np.isin(ik, np.unique(ref_ik))
    got = groups(np.asarray(ik)[sel], np.asarray(n)[sel], np.asarray(r)[sel])
    if got.keys() != ref.keys():
        return float("inf"), len(ref)
    scale = max((abs(v) for v in ref.values()), default=1.0)
    worst = max((abs(got[k] - v) / max(abs(v), 1e-12 * scale) for k, v in ref.items()), default=0.0)
    return float(worst), len(ref)


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def build_oracle_grid():
    from oracle import epwi_oracle as O
    from paper_2306_16493_gb300 import synth
    s = synth.al_like_system(WORKLOAD["seed"])
    N = WORKLOAD["grid"]
    gr = O.Grids(s, (N, N, N))
    return s, gr


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.destroy_process_group()
            return
    s, gr = build_oracle_grid()
    mu = gr.band_centre()
    T, eta = WORKLOAD["T_K"], WORKLOAD["smear_eV"]
    nsample = args.ref_kpoints
    for w in range(args.warmup):
        oracle_sample(s, gr, max(1, nsample // 4), 1000 + w, T, eta, mu)
    tot_pairs, tot_t = 0, 0.0
    for k in range(args.steps):
        p, dt = oracle_sample(s, gr, nsample, 2000 + k, T, eta, mu)
        tot_pairs += p
        tot_t += dt
    val = tot_pairs / tot_t
    line = {"metric": METRIC, "value": val, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": dict(WORKLOAD, precision="fp64 CPU oracle",
                           sample=f"{nsample} seeded k-points per step (all their q) of the 48^3 workload"),
            "cpu_baseline": {"value": val, "unit": "pairs/s", "cores": cores_used(), "kind": "oracle",
                             "sample": f"{nsample} k-points x {args.steps} steps, numpy FP64"},
            "e2e": {"value": val, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2306_16493_gb300 import epwi, synth

    precision = args.precision
    s = synth.al_like_system(WORKLOAD["seed"])
    N = args.grid
    T, eta, win = WORKLOAD["T_K"], WORKLOAD["smear_eV"], WORKLOAD["window_eV"]
    stream = torch.cuda.current_stream()
    ctx = epwi.Context(precision=precision, device=local, stream=stream.cuda_stream)
    ctx.setup(s)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        ctx.eigs(N)
        lo, hi = ctx.band_range()
        mu = 0.5 * (lo + hi)
        ns, npairs = ctx.scatter_rates(T, mu, eta, mu - win, mu + win)
        sig = ctx.conductivity()
        return npairs, sig

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    pairs_total = 0
    sc_ms, sc_flops, chunks = 0.0, 0.0, 0
    launches0 = epwi.epwi_kernel_launches()
    clocks_path = os.path.join(tempfile.gettempdir(), f"epwi_clocks_{os.getpid()}.csv")
    with ClockSampler(clocks_path) as cs:
        time.sleep(0.3)
        for k in range(args.steps):
            flush.zero_()                        # L2 flush between timed steps (not timed)
            ev[k][0].record(stream)
            npairs, sig = step()
            ev[k][1].record(stream)
            pairs_total += npairs
            st = ctx.stats()
            sc_ms += st["ms_scatter"]
            sc_flops += st["scatter_flops"]
            chunks += st["n_chunks"]
        torch.cuda.synchronize()
    launches = (epwi.epwi_kernel_launches() - launches0) // args.steps
    if world > 1:
        torch.distributed.barrier()
    gpu_k, gpu_b, gpu_r = ctx.rates()            # the last timed step's rates (not timed)
    gpu_sig = sig
    mu_step = 0.5 * sum(ctx.band_range())
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max = reduce_max_over_ranks(ms, world)
    pairs_all = reduce_sum_over_ranks(float(pairs_total), world)
    value = pairs_all / (ms_max * 1e-3)
    clocks = cs.summary(local)
    stats = dict(ctx.stats(), scatter_flops=sc_flops / args.steps, ms_scatter=sc_ms / args.steps,
                 n_chunks=chunks // args.steps)
    pairs_per_launch = pairs_total / args.steps / max(1, stats["n_chunks"])
    tb = TRAFFIC_BYTES_PER_PAIR.get(precision)
    simt = fma_peaks(local, stream.cuda_stream)
    roof = roofline_for(precision, stats,
                        per_launch_traffic=None if tb is None else tb * pairs_per_launch, simt_peaks=simt)

    # ---- e2e through the C ABI with host buffers
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 3))
    h2d = sum(a.nbytes for a in (s.mass, s.Re, s.we, s.H, s.Rp, s.wp, s.Phi, s.g))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_pairs, d2h = 0, 0
    for _ in range(e2e_steps):
        ctx.setup(s)
        npairs, sig = step()
        k_idx, band, rates = ctx.rates()
        e2e_pairs += npairs
        d2h = k_idx.nbytes + band.nbytes + rates.nbytes + sig.nbytes
    torch.cuda.synchronize()
    e2e_t = max(time.perf_counter() - t0, 1e-30)
    e2e_t = reduce_max_over_ranks(e2e_t, world)
    e2e_pairs = reduce_sum_over_ranks(float(e2e_pairs), world)

    # ---- the same workload on the FP64 GPU path: time-to-sigma and the error of this precision
    fp64 = None
    if rank == 0 and world == 1 and not args.no_fp64_leg and precision != "fp64":
        ctx64 = epwi.Context(precision="fp64", device=local, stream=stream.cuda_stream)
        ctx64.setup(s)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        ctx64.eigs(N)
        lo64, hi64 = ctx64.band_range()
        mu64 = 0.5 * (lo64 + hi64)
        _, np64 = ctx64.scatter_rates(T, mu64, eta, mu64 - win, mu64 + win)
        sig64 = ctx64.conductivity()
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        k64, b64, r64 = ctx64.rates()
        eps64 = ctx64.bands()[0]
        err64, ng64 = group_rel_error(gpu_k, gpu_b, gpu_r, k64, b64, r64, eps64)
        fp64 = {"time_to_sigma_ms": ms64, "value": np64 / (ms64 * 1e-3), "unit": "pairs/s",
                "speedup_of_this_precision": ms64 / (ms_max / args.steps),
                "pairs": int(np64), "same_pairs": int(np64) == int(pairs_total // args.steps),
                "rate_max_rel_error_vs_fp64": err64, "rate_groups_compared": ng64,
                "sigma_rel_frobenius_vs_fp64": float(np.linalg.norm(gpu_sig - sig64) / np.linalg.norm(sig64)),
                "stated_tolerance": {"inv_tau": 1e-4, "sigma": 1e-4},
                "steps": 1, "note": "one step of the FP64 path (FP64 Re->k, FP64 Rp->q + rotations + "
                                    "delta sum) on the same grid, window and smearing, L2 flushed first"}
        ctx64.close()

    line = None
    if rank == 0:
        cpu, err_oracle = None, None
        if world == 1 and not args.no_cpu_baseline:
            _, gr = build_oracle_grid()
            mu = gr.band_centre()
            p, dt, ref = oracle_sample(s, gr, args.ref_kpoints, 7, T, eta, mu, full=True)
            cpu = {"value": p / dt, "unit": "pairs/s", "cores": cores_used(), "kind": "oracle",
                   "sample": f"{args.ref_kpoints} seeded k-points of the 48^3 workload with all their q "
                             f"({p} pairs, {dt:.1f} s, numpy FP64; grid eigensolves excluded)"}
            if N == WORKLOAD["grid"]:
                e, ng = group_rel_error(gpu_k, gpu_b, gpu_r, ref["ik"], ref["n"], ref["inv_tau"], gr.eps)
                err_oracle = {"inv_tau_max_rel_error": e, "groups_compared": ng,
                              "kpoints": args.ref_kpoints, "mu_abs_diff_eV": abs(mu - mu_step),
                              "stated_tolerance": 1e-4,
                              "how": "the last timed step's 1/tau against the FP64 oracle on the "
                                     "cpu_baseline sample, per degenerate group, relative to each "
                                     "group's own rate"}
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "time_to_sigma_ms": ms_max / args.steps, "pairs_per_step": pairs_total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[precision], "data": "synthetic",
                "config": dict(WORKLOAD, grid=N, workload=f"al_like_{N}", precision=precision,
                               l2="flushed between timed steps (256 MiB write)",
                               parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
                "gpu_launches": int(launches),
                "stage_ms": {k: stats[k] for k in ("ms_eigs", "ms_sieve", "ms_restage", "ms_scatter", "ms_reduce")},
                "roofline": roof, "clocks": clocks, "cpu_baseline": cpu,
                "simt_peaks_tflops": {k: v[0] for k, v in simt.items()},
                "error_vs_oracle": err_oracle, "fp64_gpu": fp64,
                "e2e": None if args.no_e2e else
                       {"value": e2e_pairs / e2e_t, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)}}
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- other workloads
BATCH = dict(workload="batch64", systems="64 seeded cells s = 16a+4b+c: nat=[1,2,4,6][c], "
             "nw=[4,8,16,24][b], grid=[24,36,48,60][a]^3 / scale, R cube side=[3,5,7][(a+b+c)%3]",
             window_eV=0.2, smear_eV=0.02, T_K=300.0, mu="band centre per system")
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # fallback only: 152 SM x 128 FP32 lanes x FMA x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12     # fallback only: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz


def run_batch(args):
    """64 uneven systems, one graph launch per step (persistent work-queue kernel)."""
    import torch
    from paper_2306_16493_gb300 import epwi, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()             # the batch's graph runs on this stream
    torch.cuda.set_stream(stream)
    T, eta, win = BATCH["T_K"], BATCH["smear_eV"], BATCH["window_eV"]
    t0 = time.perf_counter()
    b = epwi.Batch(stream=stream.cuda_stream)
    h2d, grids = 0, []
    members = [int(x) for x in args.batch_systems.split(",")] if args.batch_systems else range(64)
    for s in members:
        sysm, N = synth.batch_system(s)
        Nr = max(2, N // args.batch_scale)
        b.add(sysm, (Nr, Nr, Nr))
        h2d += sum(a.nbytes for a in (sysm.mass, sysm.Re, sysm.we, sysm.H, sysm.Rp, sysm.wp,
                                      sysm.Phi, sysm.g))
        grids.append(Nr)
        del sysm
    t_setup = time.perf_counter() - t0
    nsys = len(grids)
    mu = np.array([0.5 * sum(b.band_range(s)) for s in range(nsys)])
    t1 = time.perf_counter()
    npairs = b.plan(T, mu, eta, mu - win, mu + win, autotune=not args.no_autotune)
    sig = b.run()
    t_first = time.perf_counter() - t1
    for _ in range(args.warmup):
        b.run()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    pers = []
    clocks_path = os.path.join(tempfile.gettempdir(), f"epwi_clocks_{os.getpid()}.csv")
    with ClockSampler(clocks_path) as cs:
        time.sleep(0.3)
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            sig = b.run()
            ev[k][1].record(stream)
            pers.append(b.stats()["ms_persistent"])
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(c) for a, c in ev) / args.steps
    st = b.stats()
    ms_p = sum(pers) / len(pers)
    achieved = st["scatter_flops"] / (ms_p * 1e-3) / 1e12
    fp32_peak, fp32_src = fma_peaks(0, stream.cuda_stream)["fp32"]
    tiles = [b.tile(s) for s in range(nsys)]
    line = {"metric": "batched el-ph (k,q)-pairs/s over 64 uneven systems (one graph launch per step)",
            "value": npairs / (ms * 1e-3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "time_to_sigma_ms": ms, "pairs_per_step": npairs,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (f64 sums)", "data": "synthetic",
            "config": dict(BATCH, scale=args.batch_scale, grids=grids, members=list(members),
                           l2="flushed between timed steps (256 MiB write)"),
            # one graph launch per step; its nodes are this library's kernels plus a few
            # memset and event-record nodes
            "gpu_launches": int(b.stats()["graph_nodes"]),
            "graph": {"nodes": st["graph_nodes"], "persistent_ctas": st["persistent_ctas"],
                      "items": st["n_items"], "smem_bytes": st["smem_bytes"]},
            "stage_ms": {"persistent": ms_p, "rest_of_graph": ms - ms_p, "plan": st["ms_plan"]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                         "kernel": "k_batch_scatter (persistent, FP32 SIMT)",
                         "peak_source": fp32_src},
            "restage_flops": st["restage_flops"],
            "tiles": {"autotuned": sum(1 for t in tiles if t[2] in (1, 2)),
                      "shapes": sorted({f"{t[0]}x{t[1]}" for t in tiles})},
            "clocks": cs.summary(0),
            "e2e": {"value": npairs / (t_setup + t_first), "unit": "pairs/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": nsys * 9 * 8,
                    "note": "host arrays -> sigma once: setup of 64 systems + plan (autotune) + first run"},
            "cpu_baseline": None}
    b.close()
    print(json.dumps(line), flush=True)


def run_learned(args):
    """Learned q-proposal on the Si-like system: train at 24^3, importance-sample 1/tau at
    100^3, compare with the full-grid FP64 and fp16x3 results."""
    import torch
    from paper_2306_16493_gb300 import epwi, synth
    torch.cuda.set_device(0)
    sysm = synth.si_like_system(3)
    T, eta = 300.0, 0.01
    ctx = epwi.Context()
    ctx.setup(sysm)
    ctx.eigs(24)
    mu24 = ctx.find_mu(T, 1e18, sysm.n_valence)
    _, cbm24 = ctx.band_edges(sysm.n_valence)
    t0 = time.perf_counter()
    loss = ctx.mlp_train(T, mu24, 4 * eta, cbm24 - 0.05, cbm24 + 0.3, seed=2)
    t_train = time.perf_counter() - t0
    ntrain = len(epwi.epwi_mlp_get_training_set(ctx.h)[1])
    N = args.learned_grid
    ctx.eigs(N)
    mu = ctx.find_mu(T, 1e18, sysm.n_valence)
    _, cbm = ctx.band_edges(sysm.n_valence)
    lo, hi = cbm, cbm + 0.25

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t

    res = {}
    for prec in ("fp64", "fp16x3"):
        ctx.set_precision(prec)
        ctx.scatter_rates(T, mu, eta, lo, hi)             # warm-up
        dt = timed(lambda: ctx.scatter_rates(T, mu, eta, lo, hi))
        r = ctx.rates()[2]
        if prec == "fp64":
            full = r
        res[prec] = {"s": dt, "pairs": ctx.stats()["n_pairs"],
                     "rms_rel_err": float(np.sqrt(np.mean(((r - full) / full) ** 2)))}
    ctx.set_precision(args.learned_precision)      # evaluation kernels of the drawn pairs
    for S in args.learned_samples:
        for name, kw in (("uniform", dict(proposal="uniform")),
                         ("learned", dict(proposal="learned", alpha=0.1, cell_stride=args.learned_stride))):
            errs, dts = [], []
            for seed in range(2):
                dts.append(timed(lambda: ctx.scatter_rates_is(T, mu, eta, lo, hi, S, seed=11 + seed, **kw)))
                r = ctx.rates()[2]
                errs.append(float(np.sqrt(np.mean(((r - full) / full) ** 2))))
            st = ctx.stats()
            res[f"{name}_S{S}"] = {"s": min(dts), "pairs": st["n_pairs"], "rms_rel_err": float(np.mean(errs)),
                                   "ms_proposal": st["ms_proposal"], "ms_sampling": st["ms_sampling"],
                                   "ms_scatter": st["ms_scatter"],
                                   "proposal_tflops": st["proposal_flops"] / max(1e-9, st["ms_proposal"]) / 1e9}
    S = args.learned_samples[-1]
    line = {"metric": "importance-sampled 1/tau with the learned q-proposal: time and rms error vs the "
                      "full-grid FP64 rates", "value": res[f"learned_S{S}"]["s"] * 1e3, "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": 2, "warmup": 1, "data": "synthetic",
            "dtype": "bf16 weights f32 network, f64 estimator", "vs_baseline": None,
            "config": {"workload": f"si_like_{N}_learned", "train_grid": 24, "train_smear_eV": 4 * eta,
                       "is_precision": args.learned_precision,
                       "smear_eV": eta, "T_K": T, "n_c_cm3": 1e18, "window": "[CBM, CBM+0.25]",
                       "cell_stride": args.learned_stride, "alpha": 0.1, "samples_per_k": args.learned_samples},
            "training": {"samples": ntrain, "loss": loss, "s": t_train},
            "results": res}
    ctx.close()
    print(json.dumps(line), flush=True)


IBTE = dict(workload="al_like_tr_48_ibte",
            system="Al-like fcc, nw=4, 3 modes, 5^3 WS-weighted Re/Rp, real H(R) and g (time-reversal "
                   "symmetric)", grid=48, window_eV=0.3, smear_eV=0.02, T_K=300.0, mu="band centre", seed=2)


def run_ibte(args):
    """Iterative BTE on the time-reversal-symmetric Al-like metal: one step = eigensolves ->
    window -> sieve -> interpolation with 1/tau and the Gamma capture -> iterations to the
    tolerance -> sigma from F.  value = sieved pairs / step time."""
    import torch
    from paper_2306_16493_gb300 import epwi, synth
    torch.cuda.set_device(0)
    precision = args.ibte_precision
    s = synth.time_reversal_symmetric(synth.al_like_system(IBTE["seed"]))
    N = args.grid
    T, eta, win = IBTE["T_K"], IBTE["smear_eV"], IBTE["window_eV"]
    stream = torch.cuda.current_stream()
    ctx = epwi.Context(precision=precision, device=0, stream=stream.cuda_stream)
    ctx.setup(s)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        ctx.eigs(N)
        lo, hi = ctx.band_range()
        mu = 0.5 * (lo + hi)
        it, ch = ctx.ibte(T, mu, eta, mu - win, mu + win, max_iter=args.ibte_iters, tol=args.ibte_tol)
        sig = ctx.ibte_transport()[0]
        return ctx.ibte_stats(), sig, mu

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = epwi.epwi_kernel_launches()
    sts = []
    clocks_path = os.path.join(tempfile.gettempdir(), f"epwi_clocks_{os.getpid()}.csv")
    with ClockSampler(clocks_path) as cs:
        time.sleep(0.3)
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            st, sig, mu = step()
            ev[k][1].record(stream)
            sts.append(dict(st, ms_scatter=ctx.stats()["ms_scatter"], scatter_flops=ctx.stats()["scatter_flops"],
                            n_chunks=ctx.stats()["n_chunks"]))
        torch.cuda.synchronize()
    launches = (epwi.epwi_kernel_launches() - launches0) // args.steps
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    st = sts[-1]
    pairs = st["n_pairs"]
    mp, src = peaks()
    ms_step = statistics.mean(x["ms_step"] for x in sts)
    achieved = st["bytes_per_step"] / (ms_step * 1e-3) / 1e9
    roof_step = {"bound": "hbm", "achieved": achieved, "peak": mp["hbm_gbs"], "unit": "GB/s",
                 "frac": achieved / mp["hbm_gbs"], "traffic": None,
                 "kernel": "k_ib_step (one BTE iteration: q list, Gamma blocks, F gathers)",
                 "launches_per_step": st["iters"], "peak_source": f"{src} HBM copy bandwidth"}
    roof_sc = roofline_for(precision, dict(scatter_flops=statistics.mean(x["scatter_flops"] for x in sts),
                                           ms_scatter=statistics.mean(x["ms_scatter"] for x in sts),
                                           n_chunks=st["n_chunks"]), simt_peaks=fma_peaks(0, stream.cuda_stream))
    it_ms = statistics.mean(x["ms_step"] * x["iters"] for x in sts)
    sc_ms = statistics.mean(x["ms_scatter"] for x in sts)
    roof, roof_other = (roof_sc, roof_step) if sc_ms >= it_ms else (roof_step, roof_sc)

    # e2e: host arrays -> sigma and F on the host, through the C ABI
    e2e_steps = max(1, min(args.steps, 2))
    h2d = sum(a.nbytes for a in (s.mass, s.Re, s.we, s.H, s.Rp, s.wp, s.Phi, s.g))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        ctx.setup(s)
        st_e, sig, _ = step()
        F = ctx.mfp()
        d2h = F.nbytes + sig.nbytes
    torch.cuda.synchronize()
    e2e_t = (time.perf_counter() - t0) / e2e_steps

    cpu = None
    if not args.no_cpu_baseline:
        from oracle import epwi_oracle as O
        n_cpu = 12
        gr = O.Grids(s, (n_cpu,) * 3)
        mu_c = gr.band_centre()
        t0 = time.perf_counter()
        ref = O.ibte(gr, T, mu_c, eta, mu_c - win, mu_c + win, max_iter=args.ibte_iters, tol=args.ibte_tol)
        dt = time.perf_counter() - t0
        npairs_c = int(sum(len(O.sieve_k(gr, int(k), ref["n"][ref["ik"] == k], eta)) for k in np.unique(ref["ik"])))
        cpu = {"value": npairs_c / dt, "unit": "pairs/s", "cores": cores_used(), "kind": "oracle",
               "sample": f"the whole oracle solve at {n_cpu}^3 ({npairs_c} pairs, {ref['iters']} iterations, "
                         f"{dt:.1f} s, numpy FP64; the iteration couples every k-point, so no k subset)"}
    line = {"metric": "el-ph (k,q)-pairs/s and time-to-σ of the iterative BTE", "value": pairs / (ms * 1e-3),
            "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[precision],
            "data": "synthetic",
            "config": dict(IBTE, grid=N, workload=f"al_like_tr_{N}_ibte", precision=precision,
                           max_iter=args.ibte_iters, tol=args.ibte_tol,
                           l2="flushed between timed steps (256 MiB write)", parallelism="single GPU"),
            "gpu_launches": int(launches),
            "ibte": {"iters": st["iters"], "change": st["change"], "n_states": st["n_states"],
                     "n_pairs": pairs, "gamma_entries": st["n_entries"], "entry_bytes": st["entry_bytes"],
                     "ms_rates": statistics.mean(x["ms_rates"] for x in sts),
                     "ms_iterate": statistics.mean(x["ms_iterate"] for x in sts), "ms_step_kernel": ms_step,
                     "bytes_per_step_kernel": st["bytes_per_step"],
                     "sigma_diag_S_per_m": [float(sig[i, i]) for i in range(3)]},
            "roofline": roof, "roofline_other": roof_other, "clocks": cs.summary(0), "cpu_baseline": cpu,
            "e2e": {"value": pairs / e2e_t, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)}}
    ctx.close()
    print(json.dumps(line), flush=True)


SI = dict(workload="si_like_100", system="Si-like diamond, nw=8 (4v+4c), 6 modes, 7^3 WS-weighted Re/Rp, "
          "1.1 eV gap", grid=100, window="[CBM, CBM+0.25 eV]", n_c_cm3=1e18, smear_eV=0.01, T_K=300.0, seed=3)


def run_si(args):
    """Si-like semiconductor mobility: one step = eigensolves -> mu(n_c) -> window above the
    CBM -> sieve -> interpolation + SERTA -> mobility tensor.  value = sieved pairs / step
    time (time-to-mobility).  The fp32 mode is timed over the steps; one FP64 step and the
    FP64 oracle on sampled k-points give its error."""
    import torch
    from paper_2306_16493_gb300 import epwi, synth
    torch.cuda.set_device(0)
    s = synth.si_like_system(SI["seed"])
    N = args.si_grid
    T, eta, n_c, nv = SI["T_K"], SI["smear_eV"], SI["n_c_cm3"], s.n_valence
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def make(prec):
        ctx = epwi.Context(precision=prec, device=0, stream=stream.cuda_stream)
        ctx.setup(s)
        return ctx

    def step(ctx):
        ctx.eigs(N)
        mu = ctx.find_mu(T, n_c, nv)
        _, cbm = ctx.band_edges(nv)
        _, npairs = ctx.scatter_rates(T, mu, eta, cbm, cbm + 0.25)
        ctx.conductivity()
        return npairs, ctx.mobility(n_c), mu, cbm

    ctx = make(args.precision)
    for _ in range(args.warmup):
        step(ctx)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sts = []
    launches0 = epwi.epwi_kernel_launches()
    clocks_path = os.path.join(tempfile.gettempdir(), f"epwi_clocks_{os.getpid()}.csv")
    with ClockSampler(clocks_path) as cs:
        time.sleep(0.3)
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            npairs, mob, mu, cbm = step(ctx)
            ev[k][1].record(stream)
            sts.append(ctx.stats())
        torch.cuda.synchronize()
    launches = (epwi.epwi_kernel_launches() - launches0) // args.steps
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    gk, gb, gr_ = ctx.rates()
    st = sts[-1]
    stats = dict(st, scatter_flops=statistics.mean(x["scatter_flops"] for x in sts),
                 ms_scatter=statistics.mean(x["ms_scatter"] for x in sts))
    roof = roofline_for(args.precision, stats, simt_peaks=fma_peaks(0, stream.cuda_stream))
    # one FP64 step on the same workload
    fp64 = None
    if not args.no_fp64_leg and args.precision != "fp64":
        c64 = make("fp64")
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        np64, mob64, _, _ = step(c64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        k64, b64, r64 = c64.rates()
        err64, ng = group_rel_error(gk, gb, gr_, k64, b64, r64, c64.bands()[0])
        fp64 = {"time_to_mobility_ms": ms64, "value": np64 / (ms64 * 1e-3), "unit": "pairs/s",
                "speedup_of_this_precision": ms64 / ms, "same_pairs": int(np64) == int(npairs),
                "rate_max_rel_error_vs_fp64": err64, "rate_groups_compared": ng,
                "mobility_rel_frobenius_vs_fp64": float(np.linalg.norm(mob - mob64) / np.linalg.norm(mob64)),
                "stated_tolerance": {"inv_tau": 1e-4, "mobility": 1e-4}}
        c64.close()
    # FP64 oracle on sampled k-points of the window
    err_oracle, cpu = None, None
    if not args.no_cpu_baseline:
        from oracle import epwi_oracle as O
        t0 = time.perf_counter()
        gro = O.Grids(s, (N, N, N))
        t_grid = time.perf_counter() - t0
        kp = np.unique(gk)
        pick = np.random.default_rng(5).choice(kp, min(len(kp), args.ref_kpoints), replace=False)
        t0 = time.perf_counter()
        ref = O.serta(gro, T, mu, eta, cbm, cbm + 0.25, k_subset=pick)
        dt = time.perf_counter() - t0
        e, ng = group_rel_error(gk, gb, gr_, ref["ik"], ref["n"], ref["inv_tau"], gro.eps)
        err_oracle = {"inv_tau_max_rel_error": e, "groups_compared": ng, "kpoints": len(pick),
                      "stated_tolerance": 1e-4, "oracle_grid_s": t_grid}
        cpu = {"value": ref["n_pairs"] / dt, "unit": "pairs/s", "cores": cores_used(), "kind": "oracle",
               "sample": f"{len(pick)} seeded window k-points of the {N}^3 workload with all their q "
                         f"({ref['n_pairs']} pairs, {dt:.1f} s, numpy FP64; grid eigensolves excluded)"}
    line = {"metric": "el-ph (k,q)-pairs/s and time-to-mobility, mixed-precision vs FP64 at stated error",
            "value": npairs / (ms * 1e-3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "time_to_sigma_ms": ms, "pairs_per_step": npairs,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": dict(SI, grid=N, workload=f"si_like_{N}", precision=args.precision,
                           l2="flushed between timed steps (256 MiB write)", parallelism="single GPU"),
            "gpu_launches": int(launches), "n_states": st["n_states"], "n_kpoints": st["n_kpoints"],
            "mu_eV": mu, "cbm_eV": cbm, "mobility_cm2_per_Vs_diag": [float(mob[i, i]) for i in range(3)],
            "stage_ms": {k: st[k] for k in ("ms_eigs", "ms_sieve", "ms_restage", "ms_scatter", "ms_reduce")},
            "roofline": roof, "clocks": cs.summary(0), "cpu_baseline": cpu, "error_vs_oracle": err_oracle,
            "fp64_gpu": fp64}
    ctx.close()
    print(json.dumps(line), flush=True)


def run_sym(args):
    """Symmetry-reduced k grid (Sec. III A) on the Al-like crystal symmetrised under the fcc
    point group (48 operations): one step = eigs -> window -> sieve + rates for one k-point per
    star -> expansion to every window state -> sigma, timed against the same step on the full
    grid (both in the chosen precision)."""
    import torch
    from paper_2306_16493_gb300 import epwi, synth
    torch.cuda.set_device(0)
    s = synth.al_like_sym_system(WORKLOAD["seed"])
    kops = synth.kpoint_ops(synth.point_group(s.lattice))
    N = args.grid
    T, eta, win = WORKLOAD["T_K"], WORKLOAD["smear_eV"], WORKLOAD["window_eV"]
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    res = {}
    for mode in ("full", "reduced"):
        ctx = epwi.Context(precision=args.precision, device=0, stream=stream.cuda_stream)
        ctx.setup(s)
        if mode == "reduced":
            ctx.set_symmetry(kops)

        def step():
            ctx.eigs(N)
            lo, hi = ctx.band_range()
            mu = 0.5 * (lo + hi)
            _, npairs = ctx.scatter_rates(T, mu, eta, mu - win, mu + win)
            return npairs, ctx.conductivity()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with ClockSampler(os.path.join(tempfile.gettempdir(), f"epwi_clocks_{os.getpid()}_{mode}.csv")) as cs:
            time.sleep(0.3)
            for k in range(args.steps):
                flush.zero_()
                ev[k][0].record(stream)
                npairs, sig = step()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        st = ctx.stats()
        k_, b_, r_ = ctx.rates()
        res[mode] = {"time_to_sigma_ms": ms, "pairs_computed": int(npairs), "n_states": st["n_states"],
                     "states_computed": st["sym_states"] or st["n_states"], "stage_ms": {
                         x: st[x] for x in ("ms_eigs", "ms_sieve", "ms_restage", "ms_scatter")},
                     "sigma": sig, "rates": (k_, b_, r_), "eps": ctx.bands()[0], "clocks": cs.summary(0)}
        ctx.close()
    f, r = res["full"], res["reduced"]
    err, ng = group_rel_error(r["rates"][0], r["rates"][1], r["rates"][2], f["rates"][0], f["rates"][1],
                              f["rates"][2], f["eps"])
    for m in res.values():
        for key in ("rates", "eps"):
            m.pop(key)
    sig_err = float(np.linalg.norm(r["sigma"] - f["sigma"]) / np.linalg.norm(f["sigma"]))
    for m in res.values():
        m["sigma_diag_S_per_m"] = [float(m["sigma"][i, i]) for i in range(3)]
        m.pop("sigma")
    line = {"metric": "time-to-sigma with the symmetry-reduced k grid vs the full grid",
            "value": f["time_to_sigma_ms"] / r["time_to_sigma_ms"], "unit": "x", "higher_is_better": True,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": DTYPE[args.precision],
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": f"al_like_sym_{N}", "system": "Al-like fcc, nw=4, 3 modes, Wigner-Seitz R-sets "
                       "of the 4^3 supercell (93 vectors), symmetrised under the 48 operations of Oh",
                       "grid": N, "window_eV": win, "smear_eV": eta, "T_K": T, "precision": args.precision,
                       "operations": len(kops), "l2": "flushed between timed steps (256 MiB write)"},
            "full": f, "reduced": r, "rate_max_rel_error_reduced_vs_full": err, "rate_groups_compared": ng,
            "sigma_rel_frobenius_reduced_vs_full": sig_err}
    print(json.dumps(line), flush=True)


def run_kbatch(args):
    """Ordering ablation (Sec. III C, Table 3): the same FP64 rates call with the q-batch and
    the k-batch interpolation order on the Al-like metal."""
    import torch
    from paper_2306_16493_gb300 import epwi, synth
    torch.cuda.set_device(0)
    s = synth.al_like_system(WORKLOAD["seed"])
    N = args.ablation_grid
    T, eta, win = WORKLOAD["T_K"], WORKLOAD["smear_eV"], WORKLOAD["window_eV"]
    stream = torch.cuda.current_stream()
    res = {}
    for ordering in ("q-batch", "k-batch"):
        ctx = epwi.Context(precision="fp64", device=0, stream=stream.cuda_stream, ordering=ordering)
        ctx.setup(s)
        ctx.eigs(N)
        lo, hi = ctx.band_range()
        mu = 0.5 * (lo + hi)
        for _ in range(args.warmup):
            ctx.scatter_rates(T, mu, eta, mu - win, mu + win)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        sts = []
        for k in range(args.steps):
            ev[k][0].record(stream)
            ctx.scatter_rates(T, mu, eta, mu - win, mu + win)
            ev[k][1].record(stream)
            sts.append(ctx.stats())
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        st = sts[-1]
        interp = statistics.mean(x["ms_restage"] + x["ms_scatter"] for x in sts)
        res[ordering] = {"ms_rates_call": ms, "ms_interpolation": interp,
                         "ms_restage": statistics.mean(x["ms_restage"] for x in sts),
                         "ms_scatter": statistics.mean(x["ms_scatter"] for x in sts),
                         "pairs": st["n_pairs"], "pairs_per_s": st["n_pairs"] / (ms * 1e-3),
                         "tiles": st["n_tiles"], "interp_tflops": st["scatter_flops"] / (interp * 1e-3) / 1e12,
                         "rates": ctx.rates()[2], "n_k": st["n_states"] / max(1, st["n_kpoints"])}
        ctx.close()
    q, k = res["q-batch"], res["k-batch"]
    k.pop("n_k")
    rq, rk = q.pop("rates"), k.pop("rates")
    rel = float(np.abs(rq - rk).max() / np.abs(rq).max())
    nbar = q.pop("n_k")
    line = {"metric": "k-batch / q-batch time of the interpolation stages (Re->k + Rp->q), FP64",
            "value": k["ms_interpolation"] / q["ms_interpolation"], "unit": "x", "higher_is_better": True,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
            "vs_baseline": None,
            "config": dict(WORKLOAD, grid=N, workload=f"al_like_{N}_ordering_ablation", precision="fp64"),
            "rates_call_ratio": k["ms_rates_call"] / q["ms_rates_call"],
            "q_batch": q, "k_batch": k, "max_rel_rate_difference": rel,
            "mean_window_bands_n_k": nbar,
            "predicted_mac_ratio": (s.nw / nbar) * (len(s.Re) / len(s.Rp))}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default=CHOSEN, choices=["fp64", "tf32x3", "bf16x3", "fp16x3", "fp32"])
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ref-kpoints", type=int, default=40)
    ap.add_argument("--grid", type=int, default=WORKLOAD["grid"],
                    help="k and q grid per axis (48 is the benchmark; smaller sizes are for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-leg", action="store_true", help="skip the FP64 GPU comparison step")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (large one-off grids)")
    ap.add_argument("--workload", default="al_like",
                    choices=["al_like", "si_like", "al_like_sym", "batch64", "si_like_learned",
                             "al_like_ibte", "ordering_ablation"],
                    help="al_like: the benchmark; batch64 and si_like_learned: the batched and "
                         "learned-proposal workloads (reported separately)")
    ap.add_argument("--batch-scale", type=int, default=3, help="batch64: grid divisor")
    ap.add_argument("--batch-systems", default="", help="batch64: comma-separated subset (profiling)")
    ap.add_argument("--no-autotune", action="store_true", help="batch64: default tile shapes")
    ap.add_argument("--learned-grid", type=int, default=100)
    ap.add_argument("--learned-stride", type=int, default=2)
    ap.add_argument("--learned-precision", default="fp16x3", choices=["fp64", "fp16x3"])
    ap.add_argument("--learned-samples", type=int, nargs="+", default=[10000, 100000])
    ap.add_argument("--ibte-iters", type=int, default=200, help="al_like_ibte: iteration cap")
    ap.add_argument("--ibte-tol", type=float, default=1e-6, help="al_like_ibte: max |dF| / max |F|")
    ap.add_argument("--ibte-precision", default="fp32", choices=["fp64", "tf32x3", "bf16x3", "fp16x3", "fp32"],
                    help="al_like_ibte: precision of the rates and Gamma capture")
    ap.add_argument("--ablation-grid", type=int, default=24, help="ordering_ablation: grid per axis")
    ap.add_argument("--si-grid", type=int, default=100, help="si_like: grid per axis")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "si_like_learned":
        run_learned(args)
    elif args.workload == "al_like_ibte":
        run_ibte(args)
    elif args.workload == "ordering_ablation":
        run_kbatch(args)
    elif args.workload == "si_like":
        run_si(args)
    elif args.workload == "al_like_sym":
        run_sym(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
