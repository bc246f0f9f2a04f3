#!/usr/bin/env python
"""Benchmark: rank-structured FP64 control solves per second on GB300.

Workload: the control equation (A^-alpha + beta A^alpha) u = y_Omega on the
n^3 grid, n = 2048 interior points per axis, coefficients
a_l(x) = 1 + 0.5 sin(pi x + phi_l) (seeded phases), design function of
canonical rank 5 (seeded sine factors), eps_trunc = 1e-6, F2 as a fitted
separable exponential sum (target 1e-8; the sinc form is a measured variant),
solved by rank-truncated PCG (Algorithm 1) in the eigenbasis with FP64
scalars, Grams and orthonormalisation and the Hadamard-product contractions
as 6-digit (42-bit) BF16 digit-split tensor-core GEMMs. One step solves the
3 x 3 grid alpha in {0.25, 0.5, 0.75} x
beta in {1e-4, 1e-2, 1} (nine seeded problems) concurrently: one context,
one CUDA stream and one host thread per problem. Each context (1D
eigendecompositions, exp-sums) is built once per coefficient set; its time is
reported as setup_ms, and the end-to-end number (e2e) includes it.

A solve counts only if its relative L2 error against the FP64 oracle's exact
solution is <= 1e-6 (checked after timing, by the slab-streamed oracle).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 run under torch.distributed.run: every rank solves its own seeded
problems (independent problems, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_DEFAULT, ALPHA, BETA, RANK, EPS = 2048, 0.5, 1e-2, 5, 1e-6
ALPHAS, BETAS = (0.25, 0.5, 0.75), (1e-4, 1e-2, 1.0)
CONFIG_ID = 1
METRIC = "control solves/s at rel.err<=1e-6 vs FP64 oracle"
# FP64 pipe of GB300: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop at the max SM clock
# (2070 MHz): 1.26 TFLOP/s, consistent with the nominal 1.25 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--batch", type=int, default=9, help="concurrent solves per step (<= 9)")
    ap.add_argument("--no-check", action="store_true", help="skip the oracle error check")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--batch-count", type=int, default=256,
                    help="problems of the uneven batch section (0 = skip)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP64-sinc / FP64-fitted / learned-preconditioner comparison")
    ap.add_argument("--all-variants", action="store_true",
                    help="also the set-up-fitted r = 12 preconditioner and the paper's case (A)")
    ap.add_argument("--fullgrid-n", type=int, default=512,
                    help="grid of the full-grid mode-product measurement (0: skip)")
    ap.add_argument("--fullgrid-only", action="store_true",
                    help="run only the full-grid mode-product measurement")
    ap.add_argument("--no-scale", action="store_true",
                    help="skip the rank-structured solves at n = 256, 512, 1024")
    ap.add_argument("--tune", action="store_true",
                    help="--single only: the tensor-core GEMM autotuner instead of fixed chunks")
    ap.add_argument("--op-tol", type=float, default=None,
                    help="target of the fitted F2 exponential sum (default: the library's 1e-8)")
    ap.add_argument("--single", action="store_true",
                    help="one context and one solve per step (alpha = 0.5, beta = 1e-2), for "
                         "profiler captures: one problem's memory, no checks")
    return ap.parse_args()


# ---------------------------------------------------------------- oracle side
def _oracle_slab(args):
    from oracle import fullgrid as fg
    l1, l2, l3c, Y1, Y2, w3, alpha, beta = args
    S = l1[:, None] + l2[None, :] + l3c
    u = (Y1 * w3[None, :]) @ Y2.T / fg.F2(S, alpha, beta)
    return float(u[0, 0])


def _pool(ncores):
    import multiprocessing as mp
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    return mp.get_context("spawn").Pool(ncores)


def oracle_sample_rate(pr, n_slabs, pool):
    """Oracle exact solve of the same problem, timed on a bounded sample.

    The oracle solves by full-grid diagonalization: three LAPACK (stemr)
    eigendecompositions, the forward mode products of the canonical y_Omega,
    then u_hat = y_hat ./ F2(S) one i3-slab at a time (the n^3 grid does not
    fit host memory at n = 2048). `n_slabs` evenly spaced slabs are timed and
    the slab time is extrapolated to all n slabs. Returns solves/s and detail.
    """
    from oracle import operator as op
    n = pr.n
    t0 = time.perf_counter()
    lams, Vs = [], []
    for l in range(3):
        lam, V = op.eig(*op.assemble(pr.coeffs[l]))
        lams.append(lam)
        Vs.append(V)
    yh = [Vs[l].T @ pr.yU[l] for l in range(3)]
    t1 = time.perf_counter()
    idx = np.linspace(0, n - 1, n_slabs).astype(int)
    jobs = [(lams[0], lams[1], lams[2][c], yh[0], yh[1], pr.yw * yh[2][c, :], pr.alpha, pr.beta)
            for c in idx]
    t2 = time.perf_counter()
    list(pool.map(_oracle_slab, jobs, chunksize=1))
    t3 = time.perf_counter()
    per_slab_wall = (t3 - t2) / n_slabs  # wall time per slab with the pool's parallelism
    total = (t1 - t0) + per_slab_wall * n
    return 1.0 / total, dict(setup_s=t1 - t0, slab_s=per_slab_wall, slabs=n_slabs, total_s=total)


def oracle_errors(pr, sols, pool):
    """Relative L2 errors of several GPU solutions (list of (uw, uU)) of problem pr
    against its exact solution (oracle), in one streamed pass."""
    from oracle import fullgrid as fg
    from oracle import operator as op
    lams, Vs = [], []
    for l in range(3):
        lam, V = op.eig(*op.assemble(pr.coeffs[l]))
        lams.append(lam)
        Vs.append(V)
    yh = [Vs[l].T @ pr.yU[l] for l in range(3)]
    hs = [(uw, [Vs[l].T @ uU[l] for l in range(3)]) for uw, uU in sols]
    return fg.streamed_rel_errors(lams, pr.yw, yh, hs, pr.alpha, pr.beta, pool=pool)


def oracle_error(pr, uw, uU, pool):
    """Relative L2 error of the GPU solution against the exact solution (oracle)."""
    from oracle import fullgrid as fg
    from oracle import operator as op
    lams, Vs = [], []
    for l in range(3):
        lam, V = op.eig(*op.assemble(pr.coeffs[l]))
        lams.append(lam)
        Vs.append(V)
    yh = [Vs[l].T @ pr.yU[l] for l in range(3)]
    uh = [Vs[l].T @ uU[l] for l in range(3)]
    return fg.streamed_rel_error(lams, pr.yw, yh, uw, uh, pr.alpha, pr.beta, pool=pool)


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None
        # the raw samples go to $TCTL_CLOCKS_DIR (default: the temp directory)
        out = os.environ.get("TCTL_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_rank{dev}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- arms
def reference_arm(args, rank):
    if rank != 0:
        return
    ncores = len(os.sched_getaffinity(0))
    probs = _problems(args.n, 0, args.batch)
    with _pool(ncores) as pool:
        for _ in range(args.warmup):
            oracle_sample_rate(probs[0], 4, pool)
        totals, walls = [], []
        for _ in range(args.steps):
            w0 = time.perf_counter()
            totals.append(sum(oracle_sample_rate(p, 8, pool)[1]["total_s"] for p in probs))
            walls.append(time.perf_counter() - w0)
    value = len(probs) / statistics.mean(totals)
    sample = (f"exact eigenbasis solve of each of the {len(probs)} n={args.n} problems: 3 LAPACK "
              f"stemr eigendecompositions + 8 of {args.n} i3-slabs of u_hat = y_hat/F2 per "
              "problem and step, slab time extrapolated to all slabs")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(totals), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (f"rank-structured control solves, n={args.n}, the "
                                    f"{len(ALPHAS)}x{len(BETAS)} (alpha, beta) grid, design rank "
                                    f"{RANK}, eps={EPS}; one step = {len(probs)} solves"),
                       "n": args.n, "batch": len(probs)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": ncores, "kind": "oracle",
                             "sample": sample},
            "sample_wall_ms_per_step": 1000.0 * statistics.mean(walls),
            "note": ("ms_per_step is one full step of the workload (9 exact solves) extrapolated "
                     "from the timed sample; sample_wall_ms_per_step is the wall time the sample "
                     "took"),
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(value, world, device):
    """The largest value over the ranks (the job takes as long as its slowest rank)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _problems(n, rank, batch):
    """The (alpha, beta) grid of the n-point rank-structured configuration, seeded per problem."""
    from paper_2006_09314_gb300.inputs import make_problem, problem_seed
    grid = [(a, b) for a in ALPHAS for b in BETAS][:batch]
    return [make_problem(n, a, b, RANK, problem_seed(CONFIG_ID, rank * len(grid) + i))
            for i, (a, b) in enumerate(grid)]


def ours_arm(args, rank, world):
    import threading

    import torch
    import torch.distributed as dist
    from paper_2006_09314_gb300 import tensorctl as T

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    n = args.n
    probs = _problems(n, rank, args.batch)
    B = len(probs)
    pool = None
    if rank == 0 and (not args.no_check or not args.no_cpu):
        pool = _pool(len(os.sched_getaffinity(0)))  # spawn: safe after CUDA init
    master = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in range(B)]
    main_opts = T.tctl_default_opts(op_tol=args.op_tol) if args.op_tol else None
    ctxs = [T.Context(p.coeffs, n, p.alpha, p.beta, EPS, opts=main_opts, stream=s.cuda_stream)
            for p, s in zip(probs, streams)]
    setup_ms = [c.stats()["t_setup_ms"] for c in ctxs]
    bs = []
    for p, s in zip(probs, streams):
        with torch.cuda.stream(s):
            bs.append(T.CP.from_numpy(p.yw, p.yU))
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    results = [None] * B

    def worker(i, start_evt, end_evt):
        with torch.cuda.stream(streams[i]):
            streams[i].wait_event(start_evt)
            results[i] = ctxs[i].pcg_solve(bs[i])
            end_evt.record(streams[i])

    def batch_step():
        """All B solves concurrently (one host thread and stream each), device-timed."""
        start = torch.cuda.Event(enable_timing=True)
        final = torch.cuda.Event(enable_timing=True)
        ends = [torch.cuda.Event() for _ in range(B)]
        start.record(master)
        th = [threading.Thread(target=worker, args=(i, start, ends[i])) for i in range(B)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for e in ends:
            master.wait_event(e)
        final.record(master)
        final.synchronize()
        return start.elapsed_time(final)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def batch_runner(cs, steps, warmup, rhs=None):
        """Concurrent solves of the problems on contexts cs: (ms per step list, results)."""
        rhs = bs if rhs is None else rhs
        out = [None] * B

        def wk(i, start_evt, end_evt):
            with torch.cuda.stream(streams[i]):
                streams[i].wait_event(start_evt)
                try:
                    out[i] = cs[i].pcg_solve(rhs[i])
                except T.TctlError as ex:  # a failed solve is reported, not fatal
                    out[i] = None
                    print(f"solve {i} failed: {ex}", file=sys.stderr)
                end_evt.record(streams[i])

        def step():
            start = torch.cuda.Event(enable_timing=True)
            final = torch.cuda.Event(enable_timing=True)
            ends = [torch.cuda.Event() for _ in range(B)]
            start.record(master)
            th = [threading.Thread(target=wk, args=(i, start, ends[i])) for i in range(B)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            for e in ends:
                master.wait_event(e)
            final.record(master)
            final.synchronize()
            return start.elapsed_time(final)
        for _ in range(warmup):
            step()
        ts = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            ts.append(step())
        return ts, out

    for _ in range(args.warmup):
        batch_step()
    barrier()
    clocks = Clocks(dev)
    clocks.start()
    l0 = sum(c.launch_count() for c in ctxs)
    times = []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        times.append(batch_step())
        barrier()
    launches = sum(c.launch_count() for c in ctxs) - l0
    clk = clocks.stop()
    total_ms_max = max_over_ranks(sum(times), world, "cuda")
    sols = [r[0] for r in results]
    stats = [r[1] for r in results]

    # live per-kernel timing (events around every launch) on one more batch step
    for c in ctxs:
        c.profile(True)
    batch_step()
    prof = {}
    for c in ctxs:
        for k, v in c.profile_report().items():
            a = prof.setdefault(k, {"launches": 0, "ms": 0.0, "flops": 0.0})
            a["launches"] += v["launches"]
            a["ms"] += v["ms"]
            a["flops"] += v["flops"]
        c.profile(False)

    # end to end through the host-buffer entry point (setup + copies + solve), concurrently
    pinned = [(torch.from_numpy(p.yw).pin_memory(), torch.from_numpy(np.stack(p.yU)).pin_memory())
              for p in probs]
    e2e_rank = [0] * B

    def e2e_worker(i):
        p = probs[i]
        uw, uU, _ = T.tctl_solve_host(p.coeffs, n, p.alpha, p.beta, EPS, pinned[i][0].numpy(),
                                      [pinned[i][1][l].numpy() for l in range(3)])
        e2e_rank[i] = len(uw)

    e2e_times = []
    for _ in range(max(2, args.steps // 2)):
        barrier()
        t0 = time.perf_counter()
        th = [threading.Thread(target=e2e_worker, args=(i,)) for i in range(B)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    h2d = sum(8 * (3 * (n + 1) + RANK + 3 * n * RANK) for _ in probs)
    d2h = sum(8 * (r + 3 * n * r) for r in e2e_rank)

    variants, variant_sols = None, {}
    if not args.no_variants:
        variants, variant_sols = variants_section(args, T, probs, streams, bs, master, sols,
                                                  batch_runner)

    scalesec = None
    if rank == 0 and not args.no_scale:
        scalesec = scale_section(args, T, pool, streams, master, batch_runner, flush)
    if rank != 0:
        return
    fgsec = fullgrid_section(args, check=not args.no_check) if args.fullgrid_n > 0 else None
    batchsec = batch_section(args, T, pool) if args.batch_count > 0 else None
    errs = []
    direct = {f: [None] * B for f in variant_sols}
    t_chk = time.perf_counter()
    if not args.no_check:
        # every solve of the main run and of the directly checked forms (DIRECT_FORMS)
        # against the oracle, one pass per problem
        for i, (p, x) in enumerate(zip(probs, sols)):
            forms = list(variant_sols)
            e = oracle_errors(p, [x.to_numpy()] + [variant_sols[f][i] for f in forms], pool)
            errs.append(e[0])
            for f, ef in zip(forms, e[1:]):
                direct[f][i] = ef
    t_chk = time.perf_counter() - t_chk
    passing = B if args.no_check else sum(e <= 1e-6 for e in errs)
    value = (world * passing * args.steps) / (total_ms_max / 1000.0)
    if variants and errs:
        verify_variants(variants, direct, errs)
    e2e_value = world * B / statistics.mean(e2e_times)

    # the same kernels traced on one solve alone (alpha = 0.5, beta = 1e-2): per-launch
    # durations without the other streams' kernels interleaved; the roofline comes
    # from this trace
    iso, roofline = None, None
    if rank == 0:
        k_iso = min(range(B), key=lambda i: abs(probs[i].alpha - 0.5) + abs(math.log10(probs[i].beta) + 2))
        ctxs[k_iso].profile(True)
        with torch.cuda.stream(streams[k_iso]):
            ctxs[k_iso].pcg_solve(bs[k_iso])
        rep = ctxs[k_iso].profile_report()
        ctxs[k_iso].profile(False)
        iso, roofline = roofline_from_trace(rep)
        iso["problem"] = {"alpha": probs[k_iso].alpha, "beta": probs[k_iso].beta, "n": n}
        roofline["note"] = (f"kernel with the largest share ({roofline['share']:.3f}) of one solve "
                            f"traced alone (alpha={probs[k_iso].alpha}, beta={probs[k_iso].beta}), "
                            "CUDA events around every launch on the solve's stream; "
                            "achieved = algorithmic work per launch / mean launch time")

    cpu = None
    if not args.no_cpu:
        rate, det = oracle_sample_rate(probs[0], 64, pool)
        cpu = {"value": rate, "unit": "solves/s", "cores": len(os.sched_getaffinity(0)),
               "kind": "oracle",
               "sample": (f"one of the {B} problems: 3 LAPACK stemr eigendecompositions + 64 of {n} "
                          "i3-slabs of the exact eigenbasis solve u_hat = y_hat/F2, slab time "
                          f"extrapolated to {n} slabs")}
    if pool is not None:
        pool.close()
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": (f"rank-structured FP64 PCG control solves, n={n}, the "
                                f"{len(ALPHAS)}x{len(BETAS)} (alpha, beta) grid "
                                f"alpha in {ALPHAS}, beta in {BETAS}, design rank {RANK}, "
                                f"eps={EPS}, fitted exp-sum F2 to 1e-8, tensor-core contractions; "
                                f"one step = {B} concurrent solves"),
                   "n": n, "batch": B, "rank": RANK, "eps_trunc": EPS,
                   "contractions": ("sketch and core-projection GEMMs of the truncated Hadamard "
                                    "products: 6 signed 7-bit BF16 digits per operand (42-bit "
                                    "fixed point under one exponent per row / column), 21 digit "
                                    "products on tcgen05 with FP32 accumulators, exact low levels, "
                                    "FP64 K-chunk sums; the same split for the boundary basis "
                                    "changes V_l^T U, V_l Q; Gram, QR, Jacobi, the triple core "
                                    "products, PCG scalars and residual updates in FP64"),
                   "l2": "flushed between timed steps (256 MB write)",
                   "setup_ms_mean": statistics.mean(setup_ms),
                   "iters": [s["iters"] for s in stats],
                   "rank_x": [s["rank_x"] for s in stats],
                   "op_rank": [c.stats()["op_rank"] for c in ctxs],
                   "op_basis": [c.stats()["op_basis"] for c in ctxs],
                   "workspace_peak_mb": [round(c.stats()["ws_peak_mb"], 1) for c in ctxs],
                   "workspace_mb": ctxs[0].stats()["ws_size_mb"],
                   "rel_err_vs_oracle": errs or None, "solves_passing": passing,
                   "oracle_check_s": round(t_chk, 1),
                   "parallelism": f"replicas x{world}, {B} concurrent streams per GPU"},
        "roofline": roofline,
        "roofline_isolated": iso,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "note": f"tctl_solve_host x{B} concurrently: setup + H2D (pinned) + PCG + D2H"},
        "mode_products": fgsec,
        "rank_structured_sizes": scalesec,
        "variants": variants,
        "uneven_batch": batchsec,
        "autotuner": T.tctl_tune_report(),
        "gpu_launches": launches,
        "clocks": clk,
        "kernels_concurrent": {
            "note": (f"one traced step of the {B} concurrent solves: event pairs also cover "
                     "the other streams' kernels, so these times overlap and add up to more "
                     "than the step"),
            **{k: {"launches": v["launches"], "ms": round(v["ms"], 4)} for k, v in
               sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]}},
    }
    print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()


def _pipe_peaks():
    """Denominators: FP64 pipe (unit counts x max clock), BF16 tensor pipe and HBM (measured)."""
    return {"alu": (FP64_PEAK_TFLOPS, "TFLOP/s",
                    "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (no measured FP64 peak; "
                    "an FP64 FMA probe reached 1.256 TFLOP/s)"),
            "tensor": (_peak("bf16_tflops", 1900.0), "TFLOP/s",
                       "measured: MEASURED_PEAKS.json bf16_tflops (cuBLAS burst; kernel timed alone)"
                       if _peak("bf16_tflops", None) else "fallback 1.9 PFLOP/s bf16 burst"),
            "hbm": (_peak("hbm_gbs", 6800.0), "GB/s",
                    "measured: MEASURED_PEAKS.json hbm_gbs (copy)" if _peak("hbm_gbs", None)
                    else "fallback 6.8 TB/s")}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, bytes)
# of one n = 2048 solve traced alone (profiles/dram_rank_structured_n2048_single_solve.md),
# keyed by kernel; a kernel missing here has no capture of its current code
TRAFFIC_PER_LAUNCH = {
    "dgemm_group_kernel": 1250863,
    "tcg_group_kernel": 69086451,
    "split_group_kernel": 13568216,
    "split_kernel": 7716070,
    "row_exp_group_kernel": 2323766,
    "row_exp_kernel": 5858475,
    "rowdot_group_kernel": 48150699,
    "contract_b_kernel": 18570169,
    "core_proj_kernel": 631808,
    "ttm3_kernel": 219968,
    "tcg_reduce_group_kernel": 13552423,
    "trsm_rows_multi_kernel": 1116879,
    "splitk_reduce_group": 239608,
}


def roofline_from_trace(rep):
    """Per-kernel roofline of a traced solve and the roofline object of its largest kernel.

    Each kernel is held against the pipe its work runs on: the digit-split
    tensor-core GEMMs against the BF16 tensor peak (counting the BF16 digit
    products, 2 MNK each), the FP64 GEMMs against the FP64 pipe, and kernels
    with a byte model (digit splits, reductions, row contractions) against HBM.
    """
    peaks = _pipe_peaks()
    tot = sum(v["ms"] for v in rep.values())
    kern = {}
    for name, v in rep.items():
        e = {"launches": v["launches"], "ms": round(v["ms"], 4), "share": round(v["ms"] / tot, 4)}
        sec = v["ms"] / 1000.0
        if v.get("mma_flops", 0) > 0:
            e["bound"], e["achieved"] = "tensor", v["mma_flops"] / sec / 1e12
            e["fp64_class_tflops"] = v["flops"] / sec / 1e12
        elif v.get("flops", 0) > 0:
            e["bound"], e["achieved"] = "alu", v["flops"] / sec / 1e12
        elif v.get("bytes", 0) > 0:
            e["bound"], e["achieved"] = "hbm", v["bytes"] / sec / 1e9
        if "bound" in e:
            e["frac"] = round(e["achieved"] / peaks[e["bound"]][0], 4)
            e["achieved"] = round(e["achieved"], 4)
        if name in TRAFFIC_PER_LAUNCH:
            # measured DRAM bytes of the capture over this trace's launch time
            gbs = TRAFFIC_PER_LAUNCH[name] * v["launches"] / sec / 1e9
            e["dram_gbs"] = round(gbs, 1)
            e["dram_frac_of_hbm"] = round(gbs / peaks["hbm"][0], 4)
        kern[name] = e
    iso = {"solve_kernel_ms": tot,
           "kernels": dict(sorted(kern.items(), key=lambda kv: -kv[1]["ms"])[:12])}
    modeled = [(k, e) for k, e in kern.items() if "bound" in e]
    name, e = max(modeled, key=lambda kv: kv[1]["ms"])
    v = rep[name]
    peak, unit, src = peaks[e["bound"]]
    per_launch = ((v["mma_flops"] if e["bound"] == "tensor" else v["flops"] if e["bound"] == "alu"
                   else v["bytes"]) / v["launches"])
    roofline = {"bound": e["bound"], "kernel": name, "achieved": e["achieved"], "peak": peak,
                "unit": unit, "frac": e["achieved"] / peak,
                "traffic": TRAFFIC_PER_LAUNCH.get(name), "share": e["share"],
                "work_per_launch": per_launch, "launches": v["launches"],
                "ms_per_launch": v["ms"] / v["launches"],
                "peak_source": src + (" (of derived)" if e["bound"] == "alu" else
                                      " (of measured)" if src.startswith("measured") else
                                      " (of fallback)")}
    if v.get("bytes", 0) > 0:
        roofline["algorithmic_bytes_per_launch"] = v["bytes"] / v["launches"]
    return iso, roofline


def verify_variants(variants, direct, errs):
    """Oracle-error status of the variant solves (adds keys to each variant).

    Forms in `direct` (the plain FP64 sinc form, the learned preconditioner and
    the three-term split forms)
    were checked against the oracle solve by solve. For the others a solve's
    oracle error is at most the main solve's (checked) plus their distance
    (exact canonical inner products), and it counts as verified when that
    bound is <= 1e-6.
    """
    for name, v in variants.items():
        if not isinstance(v, dict) or "rel_diff_to_main" not in v:
            continue
        if name in direct and all(e is not None for e in direct[name]):
            v["rel_err_vs_oracle"] = direct[name]
            ok = [e <= 1e-6 for e in direct[name]]
        else:
            bnd = [e + d for e, d in zip(errs, v["rel_diff_to_main"])]
            v["err_bound_vs_oracle"] = bnd
            ok = [b <= 1e-6 for b in bnd]
        v["verified_le_1e-6"] = sum(ok)
        v["verified_solves_per_s"] = v["solves_per_s"] * sum(ok) / len(ok)


def variants_section(args, T, probs, streams, bs, master, ref_sols, batch_runner):
    """The same step with other forms of the method, on the same problems.

    fp64_sinc: sinc-quadrature F2 (Section 3.4) and FP64 FMA contractions (the
    plain method); fp64_fitted: fitted exponential sums, FP64; learned_pre: the
    default (fitted sums, tensor-core contractions) with an r = 12 preconditioner
    predicted by a network trained here on the library's own fitted sums;
    bf16x3: the contractions in the three-term BF16 split (21 bits, six
    products, FP32 accumulation); bf16x3_refined: the same inner solves inside
    up to two steps of FP64 outer residual refinement;
    fitted_pre: the same with the r = 12 sum fitted at set-up (what a perfect
    network would give); aniso_pre: the paper's case (A) preconditioner, 1/F2
    of the anisotropic constant-coefficient Laplacian in its sine basis.
    Error bound of each solve: the main run's oracle error (checked) plus the
    canonical-format distance to the main run's solution (exact inner products).
    """
    import torch
    from oracle import formats as Fm
    n = args.n
    out = {}
    t0 = time.perf_counter()
    r = 12
    X, Y, dl = T.tctl_expsum_dataset(1, r, LEARN_SAMPLES, seed=2024)
    t1 = time.perf_counter()
    model, loss = T.tctl_mlp_train(r, X, Y, steps=6000, batch=512, lr=3e-3, seed=7)
    t2 = time.perf_counter()
    forms = [("fp64_sinc", dict(expsum_src=0, tc_gemm=0)),
             ("fp64_fitted", dict(expsum_src=1, tc_gemm=0)),
             ("learned_pre", dict(pre_src=2, pre_r=r, pre_model=model.ctypes.data, pre_delta_max=0.25)),
             ("bf16x3", dict(tc_digits=3)),
             ("bf16x3_refined", dict(tc_digits=3, refine=2)),
             ("fitted_pre", dict(pre_src=1, pre_r=r, pre_delta_max=0.25)),
             ("aniso_pre", dict(pre_src=3))]
    if not args.all_variants:
        forms = forms[:5]
    ref = [x.to_numpy() for x in ref_sols]
    keep_sols = {}  # solutions of the directly checked forms
    for name, kw in forms:
        cs = [T.Context(p.coeffs, n, p.alpha, p.beta, EPS, opts=T.tctl_default_opts(**kw),
                        stream=s.cuda_stream) for p, s in zip(probs, streams)]
        steps = max(1, min(2, args.steps))
        ts, res = batch_runner(cs, steps, 1)
        diffs = []
        for (w0, U0), r_i in zip(ref, res):
            if r_i is None:
                # the solve raised (e.g. not converged): counted as a failed,
                # unverified solve (a zero solution: oracle error 1)
                w1, U1 = np.zeros(0), [np.zeros((n, 0)) for _ in range(3)]
                diffs.append(float("inf"))
            else:
                w1, U1 = r_i[0].to_numpy()
                d2 = (Fm.cp_inner(w0, U0, w0, U0) - 2 * Fm.cp_inner(w0, U0, w1, U1)
                      + Fm.cp_inner(w1, U1, w1, U1))
                diffs.append(float(np.sqrt(max(d2, 0.0)) / np.sqrt(Fm.cp_inner(w0, U0, w0, U0))))
            if name in DIRECT_FORMS:
                keep_sols.setdefault(name, []).append((w1, U1))
        out[name] = {"solves_per_s": len(probs) * steps / (sum(ts) / 1000.0),
                     "ms_per_step": sum(ts) / steps,
                     "rel_diff_to_main": diffs,
                     "failed": sum(r_i is None for r_i in res),
                     "iters": [x[1]["iters"] if x else -1 for x in res],
                     "refines": [x[1]["refines"] if x else -1 for x in res],
                     "op_rank": [c.stats()["op_rank"] for c in cs],
                     "pre_rank": [c.stats()["pre_rank"] for c in cs],
                     "pre_used": [c.stats()["pre_used"] for c in cs],
                     "pre_delta": [c.stats()["pre_delta"] for c in cs]}
        for c in cs:
            c.close()
        torch.cuda.synchronize()
    out["learned_pre"]["training"] = {
        "r": r, "samples": int(X.shape[0]), "fit_s": t1 - t0, "train_s": t2 - t1,
        "fitted_delta_median": float(np.median(dl)),
        "mse_before": float(loss[0]), "mse_after": float(loss[1]),
        "net": f"4 -> 64 -> 64 -> {2 * r} FP32 tanh, Adam 6000 steps x 512, GPU kernels + CUDA graph"}
    out["learned_operator"] = learned_operator_section(T, probs, n)
    return out, keep_sols


LEARN_SAMPLES = 20000
# variant forms whose every solve is checked against the oracle itself
DIRECT_FORMS = ("fp64_sinc", "learned_pre", "bf16x3", "bf16x3_refined")


def learned_operator_section(T, probs, n, r=16):
    """Operator head: a network trained on LEARN_SAMPLES r-term sums of F2(s)/s from
    the library's fitter predicts the nodes of F2 for each problem's spectrum; the
    set-up measures the resulting relative error of F2 and uses the sum only if it
    is <= 1e-7 (op_judge), else the sinc quadrature; the sinc sum with 24 terms per
    function is measured beside it. An r-term sum of F2/s over the n = 2048
    spectra (s_max / s_min ~ 2.6e6) is far from 1e-7 for r <= 16."""
    t0 = time.perf_counter()
    X, Y, e = T.tctl_expsum_dataset(0, r, LEARN_SAMPLES, seed=4048)
    t1 = time.perf_counter()
    model, loss = T.tctl_mlp_train(r, X, Y, steps=6000, batch=512, lr=3e-3, seed=9)
    t2 = time.perf_counter()
    rows = []
    for p in probs:
        o = T.tctl_default_opts(expsum_src=2, op_model=model.ctypes.data, op_r=r)
        with T.Context(p.coeffs, n, p.alpha, p.beta, EPS, opts=o) as c:
            st = c.stats()
        rows.append({"alpha": p.alpha, "beta": p.beta, "learned_err": st["op_learned_err"],
                     "sinc24_err": st["sinc24_err"], "expsum_used": st["expsum_used"],
                     "op_rank_in_use": st["op_rank"], "op_rel_err_in_use": st["op_rel_err"]})
    return {"r": r, "samples": int(X.shape[0]), "fit_s": t1 - t0, "train_s": t2 - t1,
            "fitted_err_median": float(np.median(e)), "fitted_err_min": float(np.min(e)),
            "mse_before": float(loss[0]), "mse_after": float(loss[1]), "judge": 1e-7,
            "accepted": sum(x["expsum_used"] == 2 for x in rows), "problems": rows}


SCALE_SIZES = (256, 512, 1024)


def scale_section(args, T, pool, streams, master, batch_runner, flush):
    """The rank-structured configuration at its other grid sizes (n = 256, 512,
    1024): the same 3 x 3 (alpha, beta) grid, nine concurrent solves per step,
    3 timed steps after one warm-up (L2 flushed before each), every solve
    checked against the oracle (streamed exact solve)."""
    import torch
    out = {}
    for n in SCALE_SIZES:
        probs = _problems(n, 0, len(streams))
        cs = [T.Context(p.coeffs, n, p.alpha, p.beta, EPS, stream=st.cuda_stream)
              for p, st in zip(probs, streams)]
        rhs = []
        for p, st in zip(probs, streams):
            with torch.cuda.stream(st):
                rhs.append(T.CP.from_numpy(p.yw, p.yU))
        torch.cuda.synchronize()
        flush.zero_()
        ts, res = batch_runner(cs, 3, 1, rhs)
        errs = []
        if pool is not None and not args.no_check:
            for p, (x, st, _) in zip(probs, res):
                xw, xU = x.to_numpy()
                errs.append(oracle_error(p, xw, xU, pool))
        passing = len(probs) if not errs else sum(e <= 1e-6 for e in errs)
        out[str(n)] = {"solves_per_s": passing * 3 / (sum(ts) / 1000.0),
                       "ms_per_step": sum(ts) / 3, "solves_passing": passing,
                       "setup_ms_mean": statistics.mean(c.stats()["t_setup_ms"] for c in cs),
                       "iters": [x[1]["iters"] for x in res],
                       "max_rel_err_vs_oracle": max(errs) if errs else None}
        for c in cs:
            c.close()
        torch.cuda.synchronize()
    return out


def batch_section(args, T, pool):
    """Uneven batch: `batch_count` problems (n in {64, 96, ..., 512}, design rank 1-8,
    alpha ~ U[0.2, 0.8], log10 beta ~ U[-4, 0]) through tctl_solve_batch (host buffers,
    16 worker threads, each problem set up, solved and torn down); per-problem latency
    percentiles. Four problems (the smallest n) are checked against the oracle."""
    from paper_2006_09314_gb300.inputs import batch_problems
    probs = batch_problems(args.batch_count, 4000)
    items = [dict(coeffs=p.coeffs, n=p.n, alpha=p.alpha, beta=p.beta, yw=p.yw, yU=p.yU) for p in probs]
    T.tctl_solve_batch(items[:8], EPS, workers=8)  # warm-up (module load, first allocations)
    t0 = time.perf_counter()
    res = T.tctl_solve_batch(items, EPS, workers=16)
    wall = time.perf_counter() - t0
    lat = np.array([r["latency_ms"] for r in res])
    ws = max(r["stats"]["ws_peak_mb"] / r["stats"]["ws_size_mb"] for r in res)
    ok = [r["status"] == 0 for r in res]
    errs = []
    if pool is not None and not args.no_check:
        for i in np.argsort([p.n for p in probs])[:4]:
            errs.append(oracle_error(probs[i], res[i]["uw"], res[i]["uU"], pool))
    return {"problems": len(probs), "workers": 16, "wall_s": wall,
            "problems_per_s": len(probs) / wall, "all_ok": bool(all(ok)),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "n_range": [min(p.n for p in probs), max(p.n for p in probs)],
            "workspace_peak_frac_max": ws,
            "rel_err_sample": errs or None,
            "note": "latency = set-up (eigendecomposition, exp-sum fits) + H2D + PCG + D2H + teardown"}


def fullgrid_section(args, check=True, only_main=False):
    """Full-grid spectral solve (six mode products + divide), n = 128, 256, 512.

    The n^3 design function (expanded from the canonical y_Omega of the
    precision configuration: alpha = 0.5, beta = 1e-2) is solved with the BF16
    digit-split tcgen05 GEMMs (precision 1) and with the FP64 FMA GEMMs
    (precision 0); both results are compared with the oracle's exact
    full-grid solve. The mode-product figures of the largest n (args.fullgrid_n)
    are the section's top-level keys.
    """
    from oracle import fullgrid as fg
    from oracle import operator as op
    from paper_2006_09314_gb300.inputs import make_problem, problem_seed

    main_n = args.fullgrid_n
    sizes = [main_n] if only_main else sorted({n for n in (128, 256) if n < main_n} | {main_n})
    per_n = {}
    out = None
    for n in sizes:
        pr = make_problem(n, 0.5, 1e-2, RANK, problem_seed(2, 0))
        Y = np.einsum("j,ij,kj,lj->ikl", pr.yw, pr.yU[0], pr.yU[1], pr.yU[2], optimize=True)
        ustar = None
        if check:
            lams, Vs = [], []
            for l in range(3):
                lam, V = op.eig(*op.assemble(pr.coeffs[l]))
                lams.append(lam)
                Vs.append(V)
            ustar = fg.solve_exact(Y, lams, Vs, 0.5, 1e-2)
        r = _fullgrid_one(args, pr, Y, ustar, n)
        per_n[str(n)] = {k: r[k] for k in ("ms_per_solve", "solves_per_s", "mode_product_ms",
                                            "frac_of_bf16_peak", "fp64_ms_per_solve",
                                            "rel_err_vs_oracle", "fp64_rel_err_vs_oracle") if k in r}
        if n == main_n:
            out = r
        del Y, ustar
    out["sizes"] = per_n
    return out


def _fullgrid_one(args, pr, Y, ustar, n):
    import torch
    from paper_2006_09314_gb300 import tensorctl as T
    yd = torch.from_numpy(np.asfortranarray(Y).reshape(-1, order="F")).cuda()
    out = {"workload": (f"full-grid spectral solve n={n} (6 mode products n x n by n x n^2 and the "
                        "spectral divide), alpha=0.5, beta=1e-2, design rank 5")}
    with T.Context(pr.coeffs, n, 0.5, 1e-2, EPS, opts=T.tctl_default_opts(precision=1)) as ctx:
        for _ in range(max(2, args.warmup)):
            u = ctx.fullgrid_solve(yd)
        times = []
        for _ in range(max(3, args.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            u = ctx.fullgrid_solve(yd)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ctx.profile(True)
        ctx.fullgrid_solve(yd)
        prof = ctx.profile_report()
        ctx.profile(False)
    tc = prof.get("tc_modeprod_kernel", {"ms": float("nan"), "launches": 0})
    ms = statistics.median(times)
    bf16_flops = 15 * 2.0 * n ** 4 * 6  # 15 digit products per mode product, 6 products
    out.update({"precision": "BF16 digit split (5 x 7-bit digits, 15 products, exact low levels) "
                             "on tcgen05, FP32 storage",
                "ms_per_solve": ms, "solves_per_s": 1000.0 / ms,
                "mode_product_ms": tc["ms"] / max(tc["launches"], 1),
                "bf16_tflops_effective": bf16_flops / (tc["ms"] / 1000.0) / 1e12,
                "bf16_peak_tflops": _peak("bf16_tflops", 1900.0),
                "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3)}
                            for k, v in prof.items()}})
    out["frac_of_bf16_peak"] = out["bf16_tflops_effective"] / out["bf16_peak_tflops"]
    if ustar is not None:
        ug = u.cpu().numpy().reshape((n, n, n), order="F")
        out["rel_err_vs_oracle"] = float(np.linalg.norm(ug - ustar) / np.linalg.norm(ustar))
        del ug
    del u
    with T.Context(pr.coeffs, n, 0.5, 1e-2, EPS, opts=T.tctl_default_opts(precision=0)) as ctx:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.fullgrid_solve(yd)
        e0.record()
        u = ctx.fullgrid_solve(yd)
        e1.record()
        torch.cuda.synchronize()
        out["fp64_ms_per_solve"] = e0.elapsed_time(e1)
    if ustar is not None:
        ug = u.cpu().numpy().reshape((n, n, n), order="F")
        out["fp64_rel_err_vs_oracle"] = float(np.linalg.norm(ug - ustar) / np.linalg.norm(ustar))
    del u, yd
    torch.cuda.empty_cache()
    return out


def _peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except Exception:
        return fallback


def single_arm(args):
    """One n-point problem (alpha = 0.5, beta = 1e-2) solved W + K times on one stream."""
    import torch
    from paper_2006_09314_gb300 import tensorctl as T
    from paper_2006_09314_gb300.inputs import make_problem, problem_seed
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    p = make_problem(args.n, ALPHA, BETA, RANK, problem_seed(CONFIG_ID, 4))
    st = torch.cuda.Stream()
    opts = T.tctl_default_opts(tune=1 if args.tune else 0)
    with torch.cuda.stream(st), T.Context(p.coeffs, args.n, p.alpha, p.beta, EPS, opts=opts,
                                          stream=st.cuda_stream) as ctx:
        b = T.CP.from_numpy(p.yw, p.yU)
        for _ in range(args.warmup):
            ctx.pcg_solve(b)
        times = []
        l0 = ctx.launch_count()
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            x, stats, _ = ctx.pcg_solve(b)
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        launches = (ctx.launch_count() - l0) / max(1, args.steps)
        print(json.dumps({"single": {"n": args.n, "alpha": p.alpha, "beta": p.beta,
                                     "ms_per_solve": times, "launches_per_solve": launches,
                                     "iters": stats["iters"],
                                     "rank_x": list(stats["rank_x"]),
                                     "setup_ms": ctx.stats()["t_setup_ms"],
                                     "tune": T.tctl_tune_report()}}), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
    if args.single:
        if rank == 0:
            single_arm(args)
        return
    if args.fullgrid_only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        if rank == 0:
            print(json.dumps({"mode_products": fullgrid_section(args, check=not args.no_check,
                                                                only_main=True)}), flush=True)
        return
    if args.impl == "reference":
        reference_arm(args, rank)
    else:
        ours_arm(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
