#!/usr/bin/env python
"""Benchmark: deflated MG-FGMRES solves/s to true relative residual 1e-8 on one GB300.

Workload (one step): one new complex-Gaussian right-hand side on each of 10
seeded beta = 6.0 quenched U(1) configurations of a 256^2 lattice (m0 tuned so
the smallest real part of the spectrum of D is 1e-3), each solved by FGMRES(8)
preconditioned by the three-grid V-cycle (4^2 blocking, 12 chirally doubled
near-null vectors, GMRES(2) smoothing, coarse GMRES-DR(30,10) then
GMRES-Proj(30,10)).  The ten hierarchies and their coarse deflation spaces are
built during set-up and warm-up and stay resident in HBM.  The default arm is
mixed precision (FP32 V-cycle, FP64 outer FGMRES and true residual); the plain
FP64 path is timed beside it on the same work.

--impl reference times the FP64 CPU oracle (the only reference this method has)
on a bounded sample of the same workload on the host cores.

Multi-GPU: every solve is independent, so N ranks are N replicas, each solving
its own right-hand sides on its own copy of the ten hierarchies (weak scaling,
no collective on the data path).
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
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MG-FGMRES solves/s to true rel-res 1e-8 (mixed vs FP64); p50/p99 latency"
L = 256
NCONF = 10
TOL = 1e-8
H_DR_M = 30  # GMRES-DR / GMRES-Proj m (k = 10)
WORKLOAD = ("256^2 x 10 configs x 1 RHS per step, deflated MG-FGMRES(8), GMRES-DR(30,10)/GMRES-Proj(30,10), "
            "tol 1e-8 true FP64 residual; mixed: FP32 V-cycle (coarsest operator streamed as an FP16 copy), FP64 outer")
LR_SITE = 24 * 24 + 4 * 2 * 4 * 24  # complex entries a site of the factored intermediate-grid stencil


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--configs", type=int, default=NCONF)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-arms", action="store_true", help="skip the CGNE and fine GMRES-DR comparison arms")
    ap.add_argument("--no-serving", action="store_true", help="skip the served-stream sample")
    ap.add_argument("--no-partial", action="store_true", help="skip the partial-intermediate-solve variant")
    ap.add_argument("--no-batching", action="store_true", help="skip the 64-right-hand-side batching sample")
    ap.add_argument("--no-scale", action="store_true", help="skip the 1024^2 x 16-right-hand-side block solve")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests per phase of the served stream")
    ap.add_argument("--serve-budget-gib", type=float, default=64.0,
                    help="HBM budget of the server's resident hierarchies (below the stream's total need)")
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--coarse-mma", type=int, choices=[0, 1], default=1,
                    help="mixed-precision handles: coarse GMRES-Proj apply on tensor cores (1) or FP32 FMAs (0)")
    ap.add_argument("--micro", choices=["bstencil", "coarse_block", "stencil", "wilson"], default=None,
                    help="time one kernel alone (the target of the ncu captures) instead of the benchmark")
    ap.add_argument("--micro-lattice", type=int, default=256)
    ap.add_argument("--micro-nrhs", default="8,64", help="comma-separated block sizes")
    ap.add_argument("--micro-reps", type=int, default=10)
    ap.add_argument("--micro-level", type=int, default=1, help="grid of the block stencil (1 or 2)")
    ap.add_argument("--micro-fp16", action="store_true", help="FP16 instead of BF16 operator")
    ap.add_argument("--micro-dense", action="store_true", help="dense intermediate-grid hop blocks (lowrank_hops 0)")
    ap.add_argument("--micro-f64", action="store_true", help="--micro stencil in FP64 instead of FP32")
    ap.add_argument("--study", choices=["table1", "massgap"], default=None,
                    help="counter study of the paper's Section 3 instead of the benchmark")
    ap.add_argument("--study-sizes", default="64,128,256", help="the paper's lattice sizes")
    ap.add_argument("--study-gaps", default="1e-1,1e-2,1e-3,1e-4")
    ap.add_argument("--study-configs", type=int, default=2)
    return ap.parse_args()


SERVE_SIZES = (64, 128, 256, 512)
SERVE_CONFIGS = 10
SERVE_RATES = (0.5, 0.9, 1.2)  # offered load as a fraction of the measured saturated rate


def run_serving(mg, torch, np, dev, rank):
    """Served stream over a pool of 10 configurations at each of 64^2, 128^2,
    256^2 and 512^2 (40 operators), each request carrying U{1..32} complex-
    Gaussian right-hand sides at tol 1e-8, keys drawn uniformly.  The server runs
    the block precision (BF16 tensor-core block products, FP32 V-cycle, FP64
    outer): queued right-hand sides of one operator, from any request, are
    solved together.  Hierarchies are admitted under an HBM budget below what
    keeping all 40 resident would take, so the stream evicts and rebuilds.

    Phases, each a fresh draw of requests: a saturated one (every request
    submitted at once; right-hand sides per second over the makespan), then
    Poisson arrivals offering 0.5x, 0.9x and 1.2x that saturated rate.  Per
    phase: right-hand sides per second from the first submission to the last
    completion, p50/p99 request latency (submission to completion), cold starts
    and evictions.  The plain FP64 sequential reference time of each phase's
    requests is estimated from warm FP64 GPU solves at each lattice size."""
    import synth
    args = parse()
    nreq = args.serve_requests
    budget = int(args.serve_budget_gib * (1 << 30))
    rng = np.random.default_rng(1234 + rank)
    keys = [(L_, c) for L_ in SERVE_SIZES for c in range(SERVE_CONFIGS)]
    t0 = time.perf_counter()
    fields = {k: synth.gauge_field(k[0], k[1], gpu=True) for k in keys}
    gen_s = time.perf_counter() - t0
    fp_ok = all(synth.check_fingerprint(k[0], k[1], fields[k]) for k in keys)
    starts = {k: (torch.from_numpy(synth.nullvec_starts(k[0], k[1], 0, 12, k[0] * k[0] * 2)),
                  torch.from_numpy(synth.nullvec_starts(k[0], k[1], 1, 12, (k[0] // 4) ** 2 * 24))) for k in keys}
    gauges = {k: torch.from_numpy(fields[k]) for k in keys}

    def key_id(k):
        return k[0] * 1000 + k[1]

    def plan_of(n):
        return [(keys[rng.integers(len(keys))], int(rng.integers(1, 33))) for _ in range(n)]

    def run_phase(srv, plan, gaps, seed0):
        # the requests' right-hand sides, in pinned host memory, made before the clock starts
        bufs = []
        for i, (k, n) in enumerate(plan):
            b = torch.from_numpy(synth.rhs(k[0], k[1], seed0 + i, nrhs=n)).pin_memory()
            bufs.append((b, torch.zeros_like(b).pin_memory()))
        s0 = srv.stats()
        tickets = []
        t_start = time.perf_counter()
        arrive = np.concatenate([[0.0], np.cumsum(gaps[1:])]) if gaps is not None else np.zeros(len(plan))
        for i, ((k, n), (b, x)) in enumerate(zip(plan, bufs)):
            wait = t_start + arrive[i] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            t = srv.submit(key_id(k), gauges[k], k[0], k[0], synth.m0_for(k[0], k[1]), b, x, n, TOL,
                           starts0=starts[k][0], starts1=starts[k][1])
            tickets.append((t, n))
        lat, worst, solved = [], 0.0, 0
        for t, n in tickets:
            st, it, rr, l = srv.wait(t, n)
            lat.append(l)
            worst = max(worst, max(rr))
            solved += n
        t_end = time.perf_counter()
        s1 = srv.stats()
        assert worst <= TOL, f"a served solve missed the tolerance: {worst}"
        return {"solves_per_s": solved / (t_end - t_start), "rhs": solved, "requests": len(plan),
                "wall_s": t_end - t_start,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "cold_starts": int(s1["cold_starts"] - s0["cold_starts"]),
                "evictions": int(s1["evictions"] - s0["evictions"]),
                "batches": int(s1["batches"] - s0["batches"]), "max_batch": int(s1["max_batch"])}

    params = mg.default_params(precision=mg.MG_MIXED_BF16, rhs_block=32)
    srv = mg.Server(params, hbm_budget_bytes=budget, workers=args.serve_workers)
    phases, plans = {}, {}
    try:
        # cold starts first: one single-right-hand-side request per operator, so the
        # saturated phase measures solving rather than set-up (the budget still evicts)
        plans["warm"] = [(k, 1) for k in keys]
        warm = run_phase(srv, plans["warm"], None, 300000)
        plans["saturated"] = plan_of(nreq)
        sat = run_phase(srv, plans["saturated"], None, 100000)
        phases["saturated"] = sat
        mean_rhs = 16.5
        for j, frac in enumerate(SERVE_RATES):
            rate = frac * sat["solves_per_s"] / mean_rhs
            plan = plan_of(nreq)
            gaps = rng.exponential(1.0 / rate, size=nreq)
            ph = run_phase(srv, plan, gaps, 200000 + 10000 * j)
            ph["offered_req_per_s"] = rate
            ph["offered_fraction_of_saturated"] = frac
            phases[f"rate_{frac:g}x"] = ph
            plans[f"rate_{frac:g}x"] = plan
        info = srv.stats()
    finally:
        srv.close()
    # FP64 sequential reference: warm per-right-hand-side time at each size (one solve
    # after the deflation-building one)
    per_rhs = {}
    for L_ in SERVE_SIZES:
        k = (L_, 0)
        h = mg.mg_setup(gauges[k].to(dev), L_, L_, synth.m0_for(L_, 0),
                        params=mg.default_params(precision=mg.MG_FP64),
                        starts0=starts[k][0].to(dev), starts1=starts[k][1].to(dev))
        b = torch.from_numpy(synth.rhs(L_, 0, 90000, nrhs=2)).to(dev)
        x = torch.zeros_like(b)
        mg.mg_solve(h, b[0], x[0], 1, TOL)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        mg.mg_solve(h, b[1], x[1], 1, TOL)
        per_rhs[L_] = time.perf_counter() - ts
        h.close()
    for name, ph in phases.items():
        seq = sum(per_rhs[k[0]] * n for k, n in plans[name])
        ph["fp64_sequential_est_s"] = seq
        ph["fp64_sequential_est_solves_per_s"] = ph["rhs"] / seq
    phases["cold_start"] = warm
    served = phases[f"rate_{SERVE_RATES[1]:g}x"]
    return {"value": served["solves_per_s"], "unit": "solves/s", "what": f"Poisson stream at {SERVE_RATES[1]:g}x "
            "the saturated rate", "p50_ms": served["p50_ms"], "p99_ms": served["p99_ms"],
            "phases": phases, "operators": len(keys), "sizes": list(SERVE_SIZES), "configs_per_size": SERVE_CONFIGS,
            "nrhs": "U{1..32}", "tol": TOL, "precision": "mixed, BF16 tensor-core block products",
            "workers": args.serve_workers, "rhs_block": 32,
            "hbm_budget_bytes": budget, "demand_bytes_all_resident": int(info["demand_bytes"]),
            "cold_starts": int(info["cold_starts"]), "evictions": int(info["evictions"]),
            "fp64_seq_ms_per_rhs": {str(k): 1e3 * v for k, v in per_rhs.items()},
            "field_gen_s": gen_s, "m0_fingerprints_match": fp_ok}


def fine_roofline(mg, dev, peaks, peak_kind, Lb=2048, launches=20, warm=3):
    """HBM roofline of the FP32 fine Wilson apply on a lattice larger than L2.

    At 256^2 one fine apply moves 3.1 MB and stays in L2, so the kernel's
    bandwidth bound shows only on a larger lattice: 2048^2 (48 B per site, 201 MB
    per apply), with L2 flushed (a 256 MB write) before every timed launch.
    Seeded random U(1) links and a Gaussian spinor; the arithmetic does not
    depend on the values.
    """
    import numpy as np
    import torch
    gen = torch.Generator(device=dev).manual_seed(1912)
    th = torch.rand((Lb, Lb, 2), generator=gen, device=dev) * (2 * np.pi)
    U = torch.polar(torch.ones_like(th), th).contiguous()
    x = torch.complex(torch.randn((Lb, Lb, 2), generator=gen, device=dev),
                      torch.randn((Lb, Lb, 2), generator=gen, device=dev)).contiguous()
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ms = []
    for i in range(warm + launches):
        flush.fill_(i & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mg.mg_wilson_apply(U, Lb, Lb, 0.1, x, y, precision=mg.MG_F32)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warm:
            ms.append(e0.elapsed_time(e1))
    avg_s = float(np.mean(ms)) / 1e3
    nbytes = 48 * Lb * Lb
    ach = nbytes / avg_s / 1e9
    del U, x, y, flush
    return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "kernel": f"k_wilson<float> (fine Wilson-Dirac apply, {Lb}^2 x 2)",
            "bytes_per_launch": nbytes, "avg_launch_us": avg_s * 1e6, "launches": launches,
            "l2": "flushed before every launch", "peak_source": peak_kind}


def l2_copy_rate(torch, dev, mb=24, reps=50):
    """Aggregate L2-resident copy rate (GB/s, bytes read + written): a 24 MB
    tensor copied into another, both held in L2 (126 MB) across the timed
    copies."""
    x = torch.empty(mb << 20, dtype=torch.uint8, device=dev).fill_(1)
    y = torch.empty_like(x)
    for _ in range(5):
        y.copy_(x)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        y.copy_(x)
    e1.record(stream)
    torch.cuda.synchronize()
    return 2 * (mb << 20) * reps / (e0.elapsed_time(e1) / 1e3) / 1e9


def timed_launches(torch, dev, fn, launches=10, warm=3):
    """Mean CUDA-event time (s) of fn() on the current stream, L2 flushed (a 256 MB
    write) before every launch."""
    import numpy as np
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ms = []
    for i in range(warm + launches):
        flush.fill_(i & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warm:
            ms.append(e0.elapsed_time(e1))
    del flush
    return float(np.mean(ms)) / 1e3


def timed_level_applies(mg, torch, dev, h, level, fn, launches=10, warm=3):
    """Mean kernel time (s) of the level applies fn() makes, from the handle's own
    CUDA events around each apply (mg_timing_enable), L2 flushed before every call.
    (The level-apply entry synchronizes before it returns, so events recorded
    around the call would also count the host's return.)"""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for i in range(warm):
        flush.fill_(i & 0xFF)
        fn()
    mg.mg_timing_enable(h, level, True)
    for i in range(launches):
        flush.fill_((warm + i) & 0xFF)
        fn()
    torch.cuda.synchronize()
    ms, n = mg.mg_timing_read(h, level)
    mg.mg_timing_enable(h, level, False)
    del flush
    return ms / 1e3 / max(n, 1)


def run_scale(mg, torch, np, dev, peaks, peak_kind, nrhs=16, Ls=1024):
    """The scale-up workload: one 1024^2 configuration (2000 sweeps, tuned m0),
    hierarchy 1024^2 x 2 -> 256^2 x 24 -> 64^2 x 24, GMRES-DR(40,16) on the
    first right-hand side, then 16 right-hand sides in one lockstep block solve
    with FP16 tensor-core block products, FP64 outer residual to 1e-8.  Beside
    it, the HBM fractions of the fine Wilson apply (FP32) and of the 24-dof
    block stencil of the intermediate grid (256^2 x 24) at this size, each timed
    alone with L2 flushed: the FP32 single-vector kernel and the FP16 tensor-core
    kernel on the 16 right-hand sides."""
    import synth
    t0 = time.perf_counter()
    U = synth.gauge_field(Ls, 0, gpu=True)
    gen_s = time.perf_counter() - t0
    fp_ok = synth.check_fingerprint(Ls, 0, U)
    m0 = synth.m0_for(Ls, 0)
    Ud = torch.from_numpy(U).to(dev)
    t0 = time.perf_counter()
    h = mg.mg_setup(Ud, Ls, Ls, m0, params=mg.default_params(precision=mg.MG_MIXED_FP16, dr_m=40, dr_k=16),
                    starts0=torch.from_numpy(synth.nullvec_starts(Ls, 0, 0, 12, Ls * Ls * 2)).to(dev),
                    starts1=torch.from_numpy(synth.nullvec_starts(Ls, 0, 1, 12, (Ls // 4) ** 2 * 24)).to(dev))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    try:
        B = torch.from_numpy(synth.rhs(Ls, 0, 200, nrhs=1 + 2 * nrhs)).to(dev)
        X = torch.zeros_like(B)
        t0 = time.perf_counter()
        _, it0, rr0, _ = mg.mg_solve(h, B[0], X[0], 1, TOL)  # GMRES-DR: builds the deflation space
        dr_s = time.perf_counter() - t0
        mg.mg_solve(h, B[1:1 + nrhs], X[1:1 + nrhs], nrhs, TOL)  # warm: graphs, block workspaces
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = mg.mg_kernel_launches()
        e0.record(stream)
        _, its, rrs, sd = mg.mg_solve(h, B[1 + nrhs:], X[1 + nrhs:], nrhs, TOL)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = mg.mg_kernel_launches() - l0
        ms = e0.elapsed_time(e1)
        assert max(rrs) <= TOL and rr0[0] <= TOL
        # K3 at this size: the intermediate-grid block stencil, 256^2 x 24
        n1 = (Ls // 4) ** 2 * 24
        s1 = (Ls // 4) ** 2
        x1 = torch.complex(torch.randn((nrhs, n1), device=dev), torch.randn((nrhs, n1), device=dev))
        y1 = torch.empty_like(x1)
        t_mma = timed_launches(torch, dev, lambda: mg.mg_apply_block(h, 1, x1, y1, nrhs, mg.MG_F16))
        b_mma = 5 * 576 * 4 * s1 + 2 * nrhs * n1 * 8  # FP16 operator once, 16 vectors in and out (complex64)
        t_f32 = timed_level_applies(mg, torch, dev, h, 1, lambda: mg.mg_apply(h, 1, x1[0], y1[0], precision=mg.MG_F32))
        b_f32 = (LR_SITE + 2 * 24) * 8 * s1
        # K1 at this size through the handle's fine apply, every launch shape (L2 flushed)
        try:
            k1_shapes = k1_by_shape(mg, torch, dev, h, Ls, peaks["hbm_gbs"])
        except Exception as e:  # reported, not fatal: the solve figures above stand
            k1_shapes = {"error": str(e)}
    finally:
        h.close()
    fine = fine_roofline(mg, dev, peaks, peak_kind, Lb=Ls)
    hb = peaks["hbm_gbs"]
    return {"metric": "MG-FGMRES solves/s to true rel-res 1e-8", "value": nrhs / (ms / 1e3), "unit": "solves/s",
            "workload": f"{Ls}^2 config 0 x {nrhs} RHS in one lockstep block solve, GMRES-DR(40,16)/"
                        "GMRES-Proj(40,16), FP16 tensor-core block products, FP32 V-cycle, FP64 outer",
            "ms": ms, "outer_iters_mean": float(np.mean(its)), "outer_iters_max": int(max(its)),
            "coarse_iters": sd["coarse_iters"], "max_relres": float(max(rrs)), "gpu_launches": int(launches),
            "first_rhs_gmres_dr_s": dr_s, "setup_s": setup_s, "field_gen_s": gen_s,
            "field": "GPU heatbath, bit-identical to the host generator", "m0_fingerprint_match": fp_ok,
            "k1_wilson_roofline": fine,
            "k1_wilson_by_shape": {"what": "FP32 fine apply of the 1024^2 handle pinned to each launch shape: 0 "
                                           "built-in (256 threads, one site each), 64/128/256 threads, 1004/1008 "
                                           "tiles of 32 x 4 / 32 x 8 sites staged in shared memory, 2002/2004 "
                                           "columns of 2 / 4 sites a lane with x neighbours by warp shuffles; "
                                           "48 B a site, L2 flushed before every apply", "shapes": k1_shapes},
            "k3_block_stencil_roofline": {
                "bound": "hbm", "kernel": f"k_bstencil_mma<fp16> (256^2 x 24, {nrhs} RHS)",
                "achieved": b_mma / t_mma / 1e9, "peak": hb, "unit": "GB/s", "frac": b_mma / t_mma / 1e9 / hb,
                "bytes_per_launch": b_mma, "avg_launch_us": t_mma * 1e6, "l2": "flushed before every launch",
                "peak_source": peak_kind},
            "k3_stencil_f32_roofline": {
                "bound": "hbm", "kernel": "k_stencil_lr<float> (256^2 x 24, one vector, rank-4 hop factors)",
                "achieved": b_f32 / t_f32 / 1e9, "peak": hb, "unit": "GB/s", "frac": b_f32 / t_f32 / 1e9 / hb,
                "bytes_per_launch": b_f32, "avg_launch_us": t_f32 * 1e6, "l2": "flushed before every launch",
                "peak_source": peak_kind}}


def dist_env():
    from paper_1912_02868_gb300 import replicas
    return replicas.rank_env()


def profile_of(name):
    """Figures of a committed ncu summary (profiles/*.json), {} when absent."""
    path = os.path.join(ROOT, "profiles", name)
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def workload_inputs(nconf):
    import synth
    Us, m0s, fps = [], [], []
    for c in range(nconf):
        U = synth.gauge_field(L, c)
        Us.append(U)
        m0s.append(synth.m0_for(L, c))
        fps.append(synth.check_fingerprint(L, c, U))
    return Us, m0s, all(fps)


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, dev):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(dev)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r[4].isdigit() and int(r[4]) > 10] or rows
        sm = [float(r[1]) for r in load if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(load)}


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(U, m0, nsolves, conf=0, seed_base=5000):
    """The FP64 oracle on one configuration: hierarchy (untimed), then nsolves
    right-hand sides; the first builds the deflation space (untimed warm-up)."""
    import synth
    from oracle import hierarchy, mg as omg
    t0 = time.perf_counter()
    h = hierarchy.build(U, m0, synth.nullvec_starts(L, conf, 0, 12, L * L * 2),
                        synth.nullvec_starts(L, conf, 1, 12, (L // 4) ** 2 * 24))
    setup_s = time.perf_counter() - t0
    s = omg.MGSolver(h)
    s.solve(synth.rhs(L, conf, seed_base)[0], TOL)  # builds the deflation space
    times = []
    for i in range(nsolves):
        b = synth.rhs(L, conf, seed_base + 1 + i)[0]
        t0 = time.perf_counter()
        x, info = s.solve(b, TOL)
        times.append(time.perf_counter() - t0)
        assert info.converged
    return times, setup_s


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synth
    U = synth.gauge_field(L, 0)
    m0 = synth.m0_for(L, 0)
    times, setup_s = oracle_sample(U, m0, args.warmup + args.steps)
    timed = times[args.warmup:]
    value = len(timed) / sum(timed)
    sample = (f"oracle (numpy FP64) deflated MG-FGMRES, 256^2 config 0, {len(timed)} right-hand sides to 1e-8 "
              f"after {args.warmup} warm-up solves; hierarchy set-up {setup_s:.1f}s untimed")
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(timed) / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": L, "configs": NCONF, "beta": 6.0, "tol": TOL,
                       "precision": "f64 (the oracle)",
                       "sample": "per right-hand side, configuration 0 only: each further configuration's "
                                 "hierarchy set-up costs about 25 s on the host; the rate is solves/s, the same "
                                 "unit as the native arm's ten configurations per step"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_native(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import paper_1912_02868_gb300 as mg
    import synth
    if rank == 0:
        mg.build()
    if world > 1:
        torch.distributed.barrier()
    mg.build()

    nconf = args.configs
    Us, m0s, fp_ok = workload_inputs(nconf)
    K, W = args.steps, args.warmup
    n0 = L * L * 2
    stream = torch.cuda.current_stream(dev)

    def make_handles(precision, **over):
        hs = []
        t0 = time.perf_counter()
        for c in range(nconf):
            hs.append(mg.mg_setup(torch.from_numpy(Us[c]).to(dev), L, L, m0s[c],
                                  params=mg.default_params(precision=precision, **over),
                                  starts0=torch.from_numpy(synth.nullvec_starts(L, c, 0, 12, n0)).to(dev),
                                  starts1=torch.from_numpy(
                                      synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24)).to(dev)))
        torch.cuda.synchronize()
        return hs, time.perf_counter() - t0

    # right-hand sides: step s, config c, rank r -> seed (L, c, rhs_index(r, s)); resident in HBM
    from paper_1912_02868_gb300 import replicas
    B = torch.stack([torch.stack([torch.from_numpy(synth.rhs(L, c, replicas.rhs_index(rank, s))[0])
                                  for c in range(nconf)])
                     for s in range(W + K)]).to(dev)
    X = torch.zeros((nconf,) + B.shape[2:], dtype=torch.complex128, device=dev)

    # one host thread and one CUDA stream per configuration: the ten independent
    # solves of a step run concurrently on the GPU (handles are independent)
    streams = [torch.cuda.Stream(dev) for _ in range(nconf)]
    pool = ThreadPoolExecutor(max_workers=nconf)

    def solve_config(h, c, steps, Bsrc, Xdst):
        out = []
        for s in steps:
            t0 = time.perf_counter()
            st, iters, relres, sd = mg.mg_solve(h, Bsrc[s, c], Xdst[c], 1, TOL, stream=streams[c])
            out.append((time.perf_counter() - t0, iters[0], relres[0], sd))
        return out

    def run_steps(hs, steps, timed, timer_levels=(), Bsrc=None, Xdst=None):
        Bsrc = B if Bsrc is None else Bsrc
        Xdst = X if Xdst is None else Xdst
        for lev in timer_levels:
            for h in hs:
                mg.mg_timing_enable(h, lev, True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = mg.mg_kernel_launches()
        e0.record(stream)
        futs = [pool.submit(solve_config, h, c, list(steps), Bsrc, Xdst) for c, h in enumerate(hs)]
        res = [r for f in futs for r in f.result()]
        torch.cuda.synchronize()
        e1.record(stream)
        torch.cuda.synchronize()
        lat = [r[0] for r in res]
        iters_all = [r[1] for r in res]
        worst = max(r[2] for r in res)
        launches = mg.mg_kernel_launches() - l0
        if world > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1)
        kt = {}
        for lev in timer_levels:
            tot, cnt = 0.0, 0
            for h in hs:
                a, b = mg.mg_timing_read(h, lev)
                tot += a
                cnt += b
                mg.mg_timing_enable(h, lev, False)
            kt[lev] = (tot, cnt)
        kt["wall_ms"] = ms
        kt["coarse_iters"] = sum(r[3]["coarse_iters"] for r in res)
        kt["coarse_solves"] = sum(r[3]["coarse_solves"] for r in res)
        kt["dr_solves"] = sum(r[3]["dr_solves"] for r in res)
        return ms, lat, iters_all, worst, launches, kt

    def max_over_ranks(v):
        return replicas.max_over_ranks(v, device=dev)

    # ---------------- mixed precision (headline) ----------------
    hs, setup_s = make_handles(mg.MG_MIXED, coarse_mma=args.coarse_mma)
    # launch shapes the set-up's autotuner chose (the same for every handle of this size)
    shapes = {}
    for lvl in range(3):
        sh, t_c, t_b = mg.mg_launch_shape(hs[0], lvl, mg.MG_F32)
        shapes[f"level{lvl}_f32"] = {"shape": sh, "us": t_c, "builtin_us": t_b}
    run_steps(hs, range(W), False)
    clk = Clocks(local)
    ms, lat, iters, worst, launches, _ = run_steps(hs, range(W, W + K), True)
    clocks = clk.stop()
    ms = max_over_ranks(ms)
    solves = replicas.total_units(world, K, nconf)
    value = solves / (ms / 1e3)
    assert worst <= TOL, f"a solve missed the tolerance: {worst}"

    # per-launch kernel times for the rooflines: the same steps again with CUDA events around every
    # grid-1 apply and coarse solve (not part of the headline; the V-cycle graph is off while timing)
    _, _, _, _, _, kt = run_steps(hs, range(W, W + K), False, timer_levels=(1, 2))

    # e2e: the same solves through the C ABI with pinned host buffers (H2D + D2H inside the timed region)
    Bh = B.cpu().pin_memory()
    Xh = torch.zeros(X.shape, dtype=torch.complex128).pin_memory()
    e2e_ms, _, _, worst_e2e, _, _ = run_steps(hs, range(W, W + K), True, Bsrc=Bh, Xdst=Xh)
    e2e_value = solves / (max_over_ranks(e2e_ms) / 1e3)
    assert worst_e2e <= TOL

    # Roofline of the dominant kernel: the coarsest-grid GMRES-Proj solve (one cluster
    # kernel per coarse solve, ~90% of the solve time).  Algorithmic bytes of one of
    # its Krylov steps: the 16^2 x 5 x 24 x 24 stencil read once (its FP16 copy, 4 bytes
    # an entry, as the mixed default streams it), v_j read and v_{j+1} written once
    # (complex64); steps per launch from the solve counters.
    peaks, peak_kind = measured_peaks()
    s2 = (L // 16) ** 2
    step_bytes = (5 * 576 * 4 + 2 * 24 * 8) * s2
    c_ms, c_n = kt[2]
    steps_per_launch = kt["coarse_iters"] / max(kt["coarse_solves"] - kt["dr_solves"], 1)
    c_avg = c_ms / 1e3 / max(c_n, 1)
    c_bytes = steps_per_launch * step_bytes
    c_ach = c_bytes / c_avg / 1e9

    # share of the steady-state GPU time from the committed ncu launch list (cold,
    # serialised launches: the share, not the absolute times, carries over)
    share = profile_of("coarse_proj_f32_256.json").get("share_of_steady_state_gpu_time")
    roofline = {"bound": "hbm", "achieved": c_ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": c_ach / peaks["hbm_gbs"],
                "traffic": profile_of("coarse_proj_f32_256.json").get("dram_bytes_per_launch"),
                "kernel": "k_coarse_proj<float> (whole coarse GMRES-Proj solve, 16^2 x 24, FP16 operator"
                          + (" applied on tensor cores" if args.coarse_mma else "") + ", cluster of 16 CTAs)",
                "bytes_per_launch": c_bytes, "steps_per_launch": steps_per_launch,
                "us_per_step": 1e6 * c_avg / max(steps_per_launch, 1), "avg_launch_us": c_avg * 1e6,
                "launches": c_n, "share_of_timed_gpu_time": share, "peak_source": peak_kind,
                "note": "latency-bound: each Krylov step is two DSMEM reductions and a neighbour exchange, "
                        "counted on mbarriers; the stencil operand (5.9 MB) is L2-resident, so HBM is not the "
                        "binding limit"}
    # second bound: per Arnoldi step each of the 16 CTAs reads its two L2-streamed
    # FP16 operator directions (16 sites x 2 x 576 x 4 B) from L2, and from shared
    # memory the three held directions plus the basis rows of the two CGS2 passes
    # (2 x (ms + 1) / 2 rows of 16 x 24 complex64 on average over a cycle)
    l2_total = l2_copy_rate(torch, dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    l2_sm = l2_total / sms
    smem_sm = 128 * 2.07  # GB/s per SM: 128 B per cycle at the maximum SM clock (nominal)
    ms_c = max(H_DR_M - 10, 1)
    l2_b = 16 * 2 * 576 * 4
    sm_b = 16 * 3 * 576 * 4 + (ms_c + 1) * 16 * 24 * 8
    t_floor = max(l2_b / (l2_sm * 1e9), sm_b / (smem_sm * 1e9))
    roofline["second_bound"] = {
        "what": "per-SM L2 and shared-memory rates; step floor = max(L2 bytes / L2 rate, SMEM bytes / SMEM rate)",
        "l2_bytes_per_cta_step": l2_b, "smem_bytes_per_cta_step": sm_b,
        "l2_gbs_per_sm": l2_sm, "l2_source": f"L2-resident copy over all {sms} SMs (torch), divided by the SM count",
        "smem_gbs_per_sm": smem_sm, "smem_source": "nominal 128 B/cycle at 2.07 GHz",
        "floor_us_per_step": t_floor * 1e6, "frac": t_floor * 1e6 / roofline["us_per_step"]}
    # the bandwidth-bound kernel of the V-cycle: the intermediate-grid 24x24 block stencil (FP32),
    # self block dense and the four hop blocks as rank-4 factors (lowrank_hops, the default)
    s1 = (L // 4) ** 2
    bytes_per_launch = (LR_SITE + 2 * 24) * 8 * s1  # self block + factors + input + output, complex64
    kt_ms, kt_n = kt[1]
    avg_s = kt_ms / 1e3 / max(kt_n, 1)
    achieved = bytes_per_launch / avg_s / 1e9
    stencil_roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved / peaks["hbm_gbs"],
                        "traffic": profile_of("stencil_lr_f32_256.json").get("dram_bytes_per_launch"),
                        "kernel": "k_stencil_lr<float> (intermediate grid, 64^2 x 24, rank-4 hop factors)",
                        "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_s * 1e6, "launches": kt_n,
                        "peak_source": peak_kind}

    for h in hs:
        h.close()
    fine = fine_roofline(mg, dev, peaks, peak_kind)

    # ---------------- plain FP64 path on the same work ----------------
    fp64 = None
    if not args.no_fp64:
        hs64, setup64 = make_handles(mg.MG_FP64)
        run_steps(hs64, range(min(W, 1)), False)
        ms64, lat64, it64, worst64, _, _ = run_steps(hs64, range(W, W + K), True)
        ms64 = max_over_ranks(ms64)
        fp64 = {"value": solves / (ms64 / 1e3), "unit": "solves/s", "ms_per_step": ms64 / K,
                "p50_ms": 1e3 * float(np.percentile(lat64, 50)), "p99_ms": 1e3 * float(np.percentile(lat64, 99)),
                "outer_iters_mean": float(np.mean(it64)), "setup_s": setup64}
        for h in hs64:
            h.close()

    # ---------- the paper's partial intermediate solve (Section 2 variant), mixed ----------
    partial = None
    if not args.no_partial:
        hsp, setupp = make_handles(mg.MG_MIXED, partial_tol=0.2, coarse_mma=args.coarse_mma)
        run_steps(hsp, range(W), False)
        msp, latp, itp, worstp, _, _ = run_steps(hsp, range(W, W + K), True)
        msp = max_over_ranks(msp)
        assert worstp <= TOL, f"a partial-solve run missed the tolerance: {worstp}"
        partial = {"value": solves / (msp / 1e3), "unit": "solves/s", "ms_per_step": msp / K,
                   "p50_ms": 1e3 * float(np.percentile(latp, 50)), "p99_ms": 1e3 * float(np.percentile(latp, 99)),
                   "outer_iters_mean": float(np.mean(itp)), "setup_s": setupp,
                   "what": "same workload; intermediate grid solved to 0.2 by FGMRES with the two-grid cycle, "
                           "coarse solves to 1e-8 in each right-hand side's first outer iteration, 1e-2 after"}
        for h in hsp:
            h.close()

    pool.shutdown(wait=True)  # the per-configuration solve threads end here, not at interpreter exit

    # ---------- batching: 64 right-hand sides of one 256^2 configuration ----------
    batching = None
    block_roofline = None
    if not args.no_batching:
        batching = {"rhs": 64, "config": 0}
        B64 = torch.stack([torch.from_numpy(synth.rhs(L, 0, 50000 + i)[0]) for i in range(64)]).to(dev)
        n2 = (L // 16) ** 2 * 24
        for mode, prec, over in (("block_bf16", mg.MG_MIXED_BF16, {}), ("block_fp16", mg.MG_MIXED_FP16, {}),
                                 ("contexts_fp32", mg.MG_MIXED, dict(parallel=7))):
            h = mg.mg_setup(torch.from_numpy(Us[0]).to(dev), L, L, m0s[0],
                            params=mg.default_params(precision=prec, **over),
                            starts0=torch.from_numpy(synth.nullvec_starts(L, 0, 0, 12, n0)).to(dev),
                            starts1=torch.from_numpy(synth.nullvec_starts(L, 0, 1, 12, (L // 4) ** 2 * 24)).to(dev))
            X64 = torch.zeros_like(B64)
            mg.mg_solve(h, B64[0], X64[0], 1, TOL)  # builds the deflation space
            mg.mg_solve(h, B64[1:15], X64[1:15], 14, TOL)  # graphs captured, contexts created, warm
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, it64, rr64, sd64 = mg.mg_solve(h, B64, X64, 64, TOL)
            e1.record(stream)
            torch.cuda.synchronize()
            assert max(rr64) <= TOL
            ms_b = max_over_ranks(e0.elapsed_time(e1))
            batching[mode] = {"solves_per_s": 64 / (ms_b / 1e3), "ms": ms_b, "outer_iters_mean": float(np.mean(it64)),
                              "coarse_iters": sd64["coarse_iters"]}
            if mode == "block_bf16":
                # the dominant kernel of the block solve: the batched coarse GMRES-Proj (one
                # cooperative kernel per GMRES cycle), timed alone on 64 coarse right-hand sides
                Bc = torch.stack([torch.from_numpy(synth.complex_gaussian((n2,), 77, r)) for r in range(64)]
                                 ).to(torch.complex64).to(dev)
                Xc = torch.zeros_like(Bc)
                mg.mg_coarse_solve(h, Bc, Xc, TOL, mg.MG_BF16, nrhs=64)
                torch.cuda.synchronize()
                e0.record(stream)
                _, itc, _, _ = mg.mg_coarse_solve(h, Bc, Xc, TOL, mg.MG_BF16, nrhs=64)
                e1.record(stream)
                torch.cuda.synchronize()
                cms = e0.elapsed_time(e1)
                steps = max(itc)  # lockstep: the block takes as many steps as its slowest right-hand side
                ms_cyc = max(H_DR_M - 10, 1)
                # algorithmic bytes of one lockstep step: the BF16 operator once (4 bytes an entry),
                # and per right-hand side v_j in, w out, and the two CGS2 passes over V_0..V_j
                # ((ms + 1) / 2 vectors each on average over a cycle of ms steps), complex64
                step_bytes = (5 * 576 * 4) * (L // 16) ** 2 + 64 * (2 + ms_cyc + 1) * n2 * 8
                ach = step_bytes * steps / (cms / 1e3) / 1e9
                block_roofline = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                  "frac": ach / peaks["hbm_gbs"],
                                  "traffic": profile_of("cb_cycle_bf16_256_64rhs.json").get("dram_bytes_per_step"),
                                  "traffic_unit": "bytes per lockstep step",
                                  "kernel": "k_cb_cycle<bf16> (batched coarse GMRES-Proj, 16^2 x 24, 64 RHS, "
                                            "one cooperative kernel per GMRES cycle)",
                                  "us_per_step": 1e3 * cms / steps, "steps": steps, "bytes_per_step": step_bytes,
                                  "ms": cms, "peak_source": peak_kind,
                                  "note": "the Krylov bases of the 64 right-hand sides (65 MB) stay in L2; each "
                                          "step is three tile barriers apart"}
            h.close()
        batching["what"] = ("64 right-hand sides of one 256^2 configuration in one mg_solve: lockstep block "
                            "solve with the 24x24 block products of the intermediate and coarsest grids on tensor "
                            "cores (BF16 or FP16 operator, FP32 vectors split into two 16-bit parts, FP32 "
                            "accumulation), against 7 concurrent FP32 solve contexts")

    # ---------------- comparison arms of the 256^2 study (Section 2) ----------------
    arms = None
    if not args.no_arms:
        arms = {}
        narm = min(2, nconf)
        for name, over in (("deflated_mg", {}),
                           ("undeflated_mg_cgne", {"coarse_solver": mg.MG_COARSE_CGNE}),
                           ("fine_gmres_dr", {"method": mg.MG_METHOD_FINE_DEFLATION})):
            t0 = time.perf_counter()
            tot = 0.0
            fe = []
            for c in range(narm):
                h = mg.mg_setup(torch.from_numpy(Us[c]).to(dev), L, L, m0s[c],
                                params=mg.default_params(precision=mg.MG_FP64, **over),
                                starts0=torch.from_numpy(synth.nullvec_starts(L, c, 0, 12, n0)).to(dev),
                                starts1=torch.from_numpy(
                                    synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24)).to(dev))
                torch.cuda.synchronize()
                ts = time.perf_counter()
                st, it_, rr, sd = mg.mg_solve(h, B[0, c], X[c], 1, TOL, stream=stream, allow_notconv=True)
                tot += time.perf_counter() - ts
                fe.append(sd["fine_equiv_mvps"])
                h.close()
            arms[name] = {"solves_per_s": narm / tot, "fine_equiv_mvps_mean": float(np.mean(fe)),
                          "first_rhs": True, "configs": narm, "precision": "f64",
                          "wall_s": time.perf_counter() - t0}

    # ---------------- scale-up: 1024^2, 16 right-hand sides, FP16 tensor cores ----------------
    scale = None
    if not args.no_scale:
        scale = run_scale(mg, torch, np, dev, peaks, peak_kind)

    # ---------------- served stream (continuous batching over many operators) ----------------
    serving = None
    if not args.no_serving:
        serving = run_serving(mg, torch, np, dev, rank)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        times, osetup = oracle_sample(Us[0], m0s[0], 1)
        cpu = {"value": 1.0 / times[0], "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"1 right-hand side of 256^2 config 0 to 1e-8 by the numpy FP64 oracle after its "
                         f"deflation-building warm-up solve ({times[0]:.1f}s); oracle set-up {osetup:.1f}s untimed"}
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "lattice": L, "configs": nconf, "beta": 6.0, "tol": TOL, "precision": "mixed",
                   "l2": "working set > L2: 10 resident hierarchies (~3.8 GB) cycled every step",
                   "parallelism": f"replicas x{world}", "m0_fingerprints_match": fp_ok},
        "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
        "outer_iters_mean": float(np.mean(iters)), "setup_s": setup_s,
        "launch_shapes": shapes,
        "fp64": fp64,
        "partial_solve": partial,
        "batching_64rhs": batching,
        "scale_1024": scale,
        "arms_256": arms,
        "serving": serving,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": nconf * n0 * 16,
                "d2h_bytes_per_step": nconf * n0 * 16 + nconf * 8},
        "roofline": roofline,
        "block_roofline": block_roofline,
        "stencil_roofline": stencil_roofline,
        "fine_roofline": fine,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)


def study_methods(mg):
    """mg_params overrides of the six methods of the paper's Table 1."""
    return {
        "deflated_mg_partial": dict(partial_tol=0.2),
        "deflated_mg": dict(),
        # GMRES-DR(30,10) on the fine grid near criticality needs far more cycles than
        # the coarse grid's limits allow (the paper used m = 200 there for that reason)
        "gmres_dr": dict(method=mg.MG_METHOD_FINE_DEFLATION, dr_max_cycles=20000, dr_stall_cycles=1000),
        "nondeflated_mg_partial": dict(coarse_solver=mg.MG_COARSE_CGNE, partial_tol=0.2),
        "cgne": dict(method=mg.MG_METHOD_FINE_CGNE),
        "nondeflated_mg": dict(coarse_solver=mg.MG_COARSE_CGNE),
    }


def fit_power(sizes, mvps):
    """The power alpha of Table 1 (Section 3): least squares of log Mvps against
    log size, size = L^2 sites, for lattice sizes L.  Returns (alpha, its
    standard error from the residuals, with at least one degree of freedom)."""
    import numpy as np
    xv = np.log(np.array(sizes, dtype=float) ** 2)
    yv = np.log(np.array(mvps, dtype=float))
    A = np.stack([xv, np.ones_like(xv)], axis=1)
    coef = np.linalg.lstsq(A, yv, rcond=None)[0]
    dof = max(len(sizes) - 2, 1)
    s2 = float(np.sum((yv - A @ coef) ** 2)) / dof
    return float(coef[0]), float(np.sqrt(s2 * np.linalg.inv(A.T @ A)[0, 0]))


def run_study(args):
    """Counter studies of the paper's Section 3 on the synthetic configurations,
    FP64, one Z(4) right-hand side (the paper's noise) per configuration and
    method, first solve of a fresh handle (the deflated methods build their
    space in it), tol 1e-8.  The mass gap g sets m0 = g - Re lambda_min(D(0)) from
    the tuned table; only configurations whose leftmost eigenvalue is real are
    used, so min |lambda(D)| = g.
      table1: fine-equivalent Mvps (Eq. 1) against lattice size at g = 1e-4 for
              the six methods of Table 1, and the fitted power alpha in
              Mvps = size^alpha (least squares on log-log, size = L^2 sites;
              alpha per L is twice that);
      massgap: at 64^2, 128^2, 256^2 and g = 1e-1 .. 1e-4: fine Mvps and the
              average coarse and intermediate Mvps per outer iteration (Figs. 1
              and 4), deflated and non-deflated, with and without the partial
              intermediate solve."""
    import numpy as np
    import torch
    import paper_1912_02868_gb300 as mg
    import synth
    dev = torch.device("cuda:0")
    table = synth.m0_table()["entries"]
    methods = study_methods(mg)

    def real_configs(L, count):
        out = []
        for c in range(SERVE_CONFIGS):
            e = table.get(f"{L}:{c}")
            if e is not None and abs(e.get("lambda_min_im", 1.0)) < 1e-6:
                out.append((c, e["lambda_min_re"]))
            if len(out) == count:
                break
        return out

    def solve_once(L, c, lam, gap, over):
        U = torch.from_numpy(synth.gauge_field(L, c, gpu=True)).to(dev)
        p = mg.default_params(precision=mg.MG_FP64, cgne_max_iters=400000, **over)
        h = mg.mg_setup(U, L, L, gap - lam, params=p,
                        starts0=torch.from_numpy(synth.nullvec_starts(L, c, 0, 12, L * L * 2)).to(dev),
                        starts1=torch.from_numpy(synth.nullvec_starts(L, c, 1, 12, (L // 4) ** 2 * 24)).to(dev))
        try:
            b = torch.from_numpy(synth.z4_noise((L, L, 2), 0x5A34, L, c)).to(dev)
            x = torch.zeros_like(b)
            t0 = time.perf_counter()
            st, it, rr, sd = mg.mg_solve(h, b, x, 1, TOL, allow_notconv=True)
            torch.cuda.synchronize()
            return {"L": L, "config": c, "gap": gap, "outer": it[0], "relres": rr[0],
                    "fine_equiv_mvps": sd["fine_equiv_mvps"], "mvps": list(sd["mvps"]),
                    "coarse_iters": sd["coarse_iters"], "s": time.perf_counter() - t0}
        finally:
            h.close()

    out = {"study": args.study, "precision": "f64", "rhs": "Z(4) noise, one per configuration", "tol": TOL}
    if args.study == "table1":
        sizes = [int(v) for v in args.study_sizes.split(",")]
        runs, fits = [], {}
        for name, over in methods.items():
            per_size, conv = [], {}
            for L in sizes:
                rs = [solve_once(L, c, lam, 1e-4, over) for c, lam in real_configs(L, args.study_configs)]
                runs += [dict(r, method=name) for r in rs]
                # the mean over the runs that met the tolerance (CG stops on its recursive
                # residual, so its true residual may sit a rounding above)
                ok = [r for r in rs if r["relres"] <= 2 * TOL]
                conv[str(L)] = f"{len(ok)}/{len(rs)}"
                per_size.append(float(np.mean([r["fine_equiv_mvps"] for r in ok])) if ok else None)
            fit = {"mean_fine_equiv_mvps": dict(zip(map(str, sizes), per_size)), "converged": conv}
            if all(v is not None for v in per_size):
                alpha, se = fit_power(sizes, per_size)
                fit.update({"alpha_volume": alpha, "alpha_volume_se": se, "alpha_per_L": 2 * alpha})
            else:
                fit["alpha_volume"] = None  # some size had no converged run
            fits[name] = fit
        out.update({"gap": 1e-4, "sizes": sizes, "fits": fits, "runs": runs})
    else:
        sizes = [int(v) for v in args.study_sizes.split(",")]
        gaps = [float(v) for v in args.study_gaps.split(",")]
        runs = []
        for name in ("deflated_mg", "nondeflated_mg", "deflated_mg_partial", "nondeflated_mg_partial"):
            for L in sizes:
                for gap in gaps:
                    for c, lam in real_configs(L, args.study_configs):
                        r = solve_once(L, c, lam, gap, methods[name])
                        r["method"] = name
                        r["coarse_mvps_per_outer"] = r["mvps"][2] / max(r["outer"], 1)
                        r["intermediate_mvps_per_outer"] = r["mvps"][1] / max(r["outer"], 1)
                        runs.append(r)
        out.update({"sizes": sizes, "gaps": gaps, "runs": runs})
    print(json.dumps(out), flush=True)


K1_SHAPES = (0, 64, 128, 256, 1004, 1008, 2002, 2004)  # fine-apply shapes: 0 built-in, threads a block,
#                                                        1000 + shared-memory tile rows, 2000 + sites a lane


def k1_by_shape(mg, torch, dev, h, Lf, hbm, launches=10):
    """The FP32 fine Wilson-Dirac apply of handle h (an Lf^2 lattice) pinned to each
    launch shape in turn, L2 flushed before every apply, timed by the handle's own
    events: {shape: {us, GB_per_s, frac}} at 48 B a site.  The handle's shape is
    put back afterwards."""
    n0 = Lf * Lf * 2
    x = torch.complex(torch.randn(n0, device=dev), torch.randn(n0, device=dev))
    y = torch.empty_like(x)
    kept = mg.mg_launch_shape(h, 0, mg.MG_F32)[0]
    out = {}
    try:
        for shp in K1_SHAPES:
            mg.mg_set_launch_shape(h, 0, mg.MG_F32, shp)
            t = timed_level_applies(mg, torch, dev, h, 0, lambda: mg.mg_apply(h, 0, x, y, precision=mg.MG_F32),
                                    launches=launches, warm=2)
            gbs = 48 * Lf * Lf / t / 1e9
            out[str(shp)] = {"us": t * 1e6, "GB_per_s": gbs, "frac": gbs / hbm}
    finally:
        mg.mg_set_launch_shape(h, 0, mg.MG_F32, kept)
    return out


def run_micro_wilson(args):
    """The FP32 fine Wilson-Dirac apply alone on an L^2 lattice (--micro-lattice),
    every launch shape, L2 flushed before every apply: the one-thread-per-site
    kernel at 64/128/256 threads a block, the shared-memory tiles of 32 x 4 and
    32 x 8 sites, and the register columns of 2 and 4 sites a lane.  The hierarchy around it is built from random vectors with
    seeded random U(1) links (the apply's cost does not depend on the values)."""
    import numpy as np
    import torch
    import paper_1912_02868_gb300 as mg
    dev = torch.device("cuda:0")
    Lm = args.micro_lattice
    gen = torch.Generator(device=dev).manual_seed(1912)
    th = torch.rand((Lm, Lm, 2), generator=gen, device=dev, dtype=torch.float64) * (2 * np.pi)
    U = torch.polar(torch.ones_like(th), th).contiguous()
    v0 = torch.complex(torch.randn((12, Lm * Lm * 2), generator=gen, device=dev, dtype=torch.float64),
                       torch.randn((12, Lm * Lm * 2), generator=gen, device=dev, dtype=torch.float64))
    n1 = (Lm // 4) ** 2 * 24
    v1 = torch.complex(torch.randn((12, n1), generator=gen, device=dev, dtype=torch.float64),
                       torch.randn((12, n1), generator=gen, device=dev, dtype=torch.float64))
    h = mg.mg_setup_from_vectors(U, Lm, Lm, 0.1, v0, v1, params=mg.default_params(precision=mg.MG_MIXED))
    del v0, v1
    try:
        peaks, kind = measured_peaks()
        res = k1_by_shape(mg, torch, dev, h, Lm, peaks["hbm_gbs"], launches=args.micro_reps)
        tuned = mg.mg_launch_shape(h, 0, mg.MG_F32)
    finally:
        h.close()
    print(json.dumps({"kernel": "k_wilson<float> / k_wilson_tile<float> / k_wilson_col<float>", "lattice": Lm, "bytes": 48 * Lm * Lm,
                      "by_shape": res, "autotuner_choice": {"shape": tuned[0], "us": tuned[1], "builtin_us": tuned[2],
                                                            "l2": "not flushed (set-up timing)"},
                      "peak_gbs": peaks["hbm_gbs"], "peak_source": kind}), flush=True)


def run_micro(args):
    """One kernel alone, one JSON line per block size.  bstencil: the tensor-core
    block stencil of grid 1 or 2 (L2 flushed before every launch; algorithmic
    bytes and flops per launch as in the kernel table).  coarse_block: one batched
    coarse GMRES-Proj solve of nrhs right-hand sides to 1e-8 on the coarsest grid
    (the cycle kernel), after the deflation-building first solve; time per
    lockstep Arnoldi step."""
    import numpy as np
    import torch
    import paper_1912_02868_gb300 as mg
    import synth
    dev = torch.device("cuda:0")
    Lm = args.micro_lattice
    prec = mg.MG_MIXED_FP16 if args.micro_fp16 else mg.MG_MIXED_BF16
    op = mg.MG_F16 if args.micro_fp16 else mg.MG_BF16
    U = synth.gauge_field(Lm, 0, gpu=True)
    h = mg.mg_setup(torch.from_numpy(U).to(dev), Lm, Lm, synth.m0_for(Lm, 0),
                    params=mg.default_params(precision=prec, lowrank_hops=0 if args.micro_dense else 1),
                    starts0=torch.from_numpy(synth.nullvec_starts(Lm, 0, 0, 12, Lm * Lm * 2)).to(dev),
                    starts1=torch.from_numpy(synth.nullvec_starts(Lm, 0, 1, 12, (Lm // 4) ** 2 * 24)).to(dev))
    try:
        for nb in [int(v) for v in args.micro_nrhs.split(",")]:
            if args.micro == "stencil":
                # the FP32 intermediate-grid stencil of one vector as the V-cycle applies it
                nx, nt, dof = mg.mg_level_shape(h, 1)
                n1, s1 = nx * nt * dof, nx * nt
                x = torch.complex(torch.randn(n1, device=dev), torch.randn(n1, device=dev))
                if args.micro_f64:
                    x = x.to(torch.complex128)
                y = torch.empty_like(x)
                pa = mg.MG_F64 if args.micro_f64 else mg.MG_F32
                t = timed_level_applies(mg, torch, dev, h, 1, lambda: mg.mg_apply(h, 1, x, y, precision=pa),
                                        launches=args.micro_reps, warm=1)
                fac, err = mg.mg_stencil_info(h, 1)
                esz = 16 if args.micro_f64 else 8
                nbytes = ((LR_SITE if fac else 5 * 576) + 2 * 24) * esz * s1
                tn = "double" if args.micro_f64 else "float"
                out = {"kernel": f"k_stencil_lr<{tn}>" if fac else ("k_stencil<double,24>" if args.micro_f64
                                                                      else "k_stencil_f32"),
                       "sites": s1, "us": t * 1e6, "GB_per_s": nbytes / t / 1e9, "bytes": nbytes,
                       "factor_rel_err": err}
            elif args.micro == "bstencil":
                nx, nt, dof = mg.mg_level_shape(h, args.micro_level)
                n1, s1 = nx * nt * dof, nx * nt
                x = torch.complex(torch.randn((nb, n1), device=dev), torch.randn((nb, n1), device=dev))
                y = torch.empty_like(x)
                t = timed_launches(torch, dev, lambda: mg.mg_apply_block(h, args.micro_level, x, y, nb, op),
                                   launches=args.micro_reps, warm=1)
                nbytes = 5 * 576 * 4 * s1 + 2 * nb * n1 * 8
                out = {"kernel": "k_bstencil_mma", "level": args.micro_level, "sites": s1, "nrhs": nb,
                       "us": t * 1e6, "GB_per_s": nbytes / t / 1e9, "TFLOP_per_s": 46080 * nb * s1 / t / 1e12,
                       "bytes": nbytes}
            else:
                b = synth.rhs(Lm, 0, 0)[0]
                mg.mg_solve(h, torch.from_numpy(b).to(dev), torch.zeros(b.shape, dtype=torch.complex128, device=dev),
                            1, TOL)
                n2 = (Lm // 16) ** 2 * 24
                Bc = torch.from_numpy(np.stack([synth.complex_gaussian((n2,), 77, r) for r in range(nb)])).to(
                    torch.complex64).to(dev)
                Xc = torch.zeros_like(Bc)
                ms = []
                for i in range(1 + args.micro_reps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    _, it, _, _ = mg.mg_coarse_solve(h, Bc, Xc, TOL, op, nrhs=nb)
                    torch.cuda.synchronize()
                    if i:
                        ms.append(time.perf_counter() - t0)
                t = float(np.mean(ms))
                out = {"kernel": "k_cb_cycle", "coarse_sites": (Lm // 16) ** 2, "nrhs": nb, "ms": t * 1e3,
                       "steps": int(max(it)), "us_per_step": t * 1e6 / max(it)}
            print(json.dumps(out), flush=True)
    finally:
        h.close()


def main():
    args = parse()
    if args.micro == "wilson":
        run_micro_wilson(args)
        return
    if args.micro:
        run_micro(args)
        return
    if args.study:
        run_study(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
