"""Benchmark: random-walk factor construction + PCG on one GB300.

Default workload (5), the configuration the headline metric is quoted on:
3D 27-point grid 128^3 (n = 2,097,152, 55.7 M stored entries), conductances
log-uniform in [0.1, 10], diagonal excess 1e-4 * row sum, seeded random
symmetric ordering, drop tolerance 1e-3, one right-hand side ~ N(0,1), PCG to
1e-6 true relative residual.  Synthetic, seeded inputs.  Two forms of the
same step (build the factor, solve) are timed on the same matrix:
  learned  the walk budget predicted by the network (12 -> 64 -> 64 -> 1,
           trained untimed beforehand on pilot-walk labels of 50 seeded 64^3
           instances of the same distribution, mean 300 walks per row, at
           least 20), factor build, FP32 PCG (FP64 dots / alpha / beta / x,
           residual replacement every 50 iterations) on the batched engine;
  plain    300 walks on every row, FP64 PCG.
value = seconds of the learned form (build + solve); the plain form's
seconds, both forms' walk-hops/s, build and PCG seconds, iterations and
factor sizes are reported beside it.  A third arm sets the walk counts by the
adaptive rule of Sec. 5.1 (--adapt-delta; 0 skips it).  `e2e` times the
learned form through the C ABI with host buffers: the copy of A and b from
pinned host memory to the GPU and the copy of x back are inside each step.

Other workloads (--workload N):
  2  3D 7-point grid 64^3 (n = 262,144), conductances log-uniform in
     [0.1, 10], excess U[0, 1e-3] * row sum, 500 walks per row, 4 right-hand
     sides, FP64 PCG to 1e-6; value = walk-hops per second of step time.
  3  2D 1000^2 grid + 2 long-range edges per row (n = 1e6), 200 walks, factor
     stored FP32, PCG FP32 (FP64 dots / alpha / beta / x, residual replacement
     every 50 iterations) to 1e-6; the FP32 solution's error against the FP64
     solve of the same factor is stated.
  4  256 random geometric graph Laplacians (n log-uniform in [1e3, 2e5]),
     16 right-hand sides each, 200 walks: one walk launch for all matrices
     (rw_build_factor_batched), one block-diagonal PCG with the iteration
     replayed from a CUDA graph (rw_batch_create + pcg_solve_batch).
  6  the paper's Table 1 grids: 7-point Dirichlet Laplacians 50^3 .. 100^3,
     random order, b = 1, walk reuse (Sec. 5.3), no dropping (as the paper's
     implementation), the walks per row of each grid set so that the factor
     size C is Table 1's; value = seconds for the six builds and solves, with
     C, I, M2 per matrix beside the paper's.
  7  a nonsymmetric 64^3 7-point grid (skewed conductances, dominant by rows
     and columns): GPU transpose, the factors of the walk games on A and on
     A^T (Sec. 7.1), BiCGSTAB with the two-game preconditioner to 1e-6; beside
     it the factor of A alone as the preconditioner.

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the
library's stream, with an L2 flush (a 512 MB write) between steps outside
the timed events, and a barrier + synchronize on both sides of the timed
region.  Under torchrun each rank runs its own replica (the factor build and
the solves of independent matrices do not exchange data); value = all ranks'
work / max-over-ranks time.

--impl reference times the CPU oracle on a bounded sample of the same
workload (the oracle is the baseline: a plain C program; its factor build
runs on all host cores).  For workload 5 it reports the estimated seconds of
the plain form (uniform 300 walks, FP64 PCG) on the full matrix: build time
from a row sample stratified by row index, PCG time from the oracle's
per-iteration cost on the full matrix and its iteration count on a 32^3
instance of the same distribution.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "walk-hops/s, factor-build s; PCG s to 1e-6 rel. residual (learned+FP32 vs plain)"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _dist():
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if os.environ.get("RW_BACKEND") != "gloo" else "gloo")
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def aggregate(units, ms, ws):
    """Whole-job figures of a replicated run: the units every rank processed
    (sum) and the slowest rank's time (max).  Single process: unchanged."""
    if ws <= 1:
        return float(units), float(ms)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded samples)
# ---------------------------------------------------------------------------

def cpu_oracle_sample(A, walks, seed, drop, label, target_s=12.0, rng_seed=2024):
    """Time the oracle (single thread) on a random sample of walk rows of the
    matrix with the same walks, until about target_s seconds of CPU work."""
    import oracle
    rng = np.random.default_rng(rng_seed)
    wr = oracle.walk_rows(A)
    order = rng.permutation(wr)
    done_rows, hops, t_used = 0, 0, 0.0
    chunk = 256
    while t_used < target_s and done_rows < order.size:
        rows = np.sort(order[done_rows:done_rows + chunk])
        t0 = time.perf_counter()
        F = oracle.build_factor(A, walks, seed, drop, rows=rows)
        t_used += time.perf_counter() - t0
        hops += int(F["hops"].sum())
        done_rows += rows.size
        chunk = min(chunk * 2, 8192)
    return {"value": hops / t_used, "unit": "hops/s", "cores": 1, "kind": "oracle",
            "sample": f"{done_rows} random walk rows of {label} x {walks} walks "
                      f"({hops} hops) in {t_used:.1f} s, single thread, factor rows only",
            "seconds": t_used}


def _oracle_sample_for(workload, cfg, target_s, rng_seed):
    if workload == 4:
        A = cfg["A"][int(np.argmax([a.n for a in cfg["A"]]))]
        return cpu_oracle_sample(A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"],
                                 "the largest matrix of the 256-RGG batch", target_s, rng_seed)
    if workload == 6:
        return cpu_oracle_sample(cfg["A"][0], cfg["walks"], cfg["walk_seed"], 1e-3,
                                 "the 50^3 Dirichlet grid (m1)", target_s, rng_seed)
    return cpu_oracle_sample(cfg["A"], cfg["walks"], cfg["walk_seed"], cfg["drop_tol"],
                             f"the {W.CONFIGS[workload]['name']} workload", target_s, rng_seed)


class OracleEstimate:
    """Seconds the CPU oracle needs for the plain form of workload 5 (uniform
    walks, FP64 PCG to tol) on the full matrix, estimated from bounded samples.

    Build: rows are independent (Sec. 4), and a row's cost falls steeply with
    its index (rows early in the order have few homes, so their walks are
    long), so rows are sampled uniformly within strata of the row index
    [0, 64), [64, 256), ... (factor 4), the sample is built by the oracle on
    all host cores, and each stratum's hops and factor entries are scaled by
    its size over its sample size.  Estimated build seconds = the oracle's
    fixed cost (validation and tables, timed with no rows) + the sample's
    remaining time x estimated hops / sample hops.
    PCG: seconds per iteration = the oracle's time for two extra iterations on
    the full matrix with a one-walk-per-row factor, per multiplication of the
    paper's count M1 = 2C + E + 4N (Sec. 6), times the estimated M1 of the
    full factor; iterations = the oracle's count to tol on a 32^3 instance of
    the same distribution (full factor, same walks)."""

    def __init__(self, A, b, walks, seed, drop, tol, small, threads=None):
        import oracle
        self.oracle = oracle
        self.A, self.b, self.walks, self.seed, self.drop, self.tol = A, b, walks, seed, drop, tol
        self.threads = threads or os.cpu_count() or 1
        self.m = 16
        n = A.n
        edges = [0]
        e = 64
        while e < n:
            edges.append(e)
            e *= 4
        edges.append(n)
        self.strata = [(a, b_) for a, b_ in zip(edges[:-1], edges[1:]) if b_ > a]
        t0 = time.perf_counter()
        oracle.build_factor(A, walks, seed, drop, rows=np.zeros(0, np.int32), threads=self.threads)
        self.t_fixed = time.perf_counter() - t0
        # PCG: per-iteration cost on the full matrix, iterations on the small instance
        F1 = oracle.build_factor(A, 1, seed, drop, threads=self.threads)
        t0 = time.perf_counter()
        oracle.pcg(A, F1, b, 0.0, 1)
        t1 = time.perf_counter()
        oracle.pcg(A, F1, b, 0.0, 3)
        t2 = time.perf_counter()
        m1_one = 2 * (F1["nnz"] + n) + A.nnz + 4 * n
        self.sec_per_mult = max(0.0, (t2 - t1) - (t1 - t0)) / 2.0 / m1_one
        As, bs = small
        Fs = oracle.build_factor(As, walks, seed, drop, threads=self.threads)
        _, self.iters_small, _, _ = oracle.pcg(As, Fs, bs, tol, 3000)

    def step(self, rng, target_s):
        """One sample; returns (estimated seconds, details)."""
        oracle = self.oracle
        A = self.A
        picks = []
        sizes = []
        for a, b_ in self.strata:
            k = min(b_ - a, self.m)
            picks.append(np.sort(rng.choice(np.arange(a, b_), size=k, replace=False)))
            sizes.append((b_ - a, k))
        rows = np.concatenate(picks).astype(np.int32)
        t0 = time.perf_counter()
        F = oracle.build_factor(A, self.walks, self.seed, self.drop, rows=rows, threads=self.threads)
        t_s = time.perf_counter() - t0
        rownnz = np.diff(F["rowptr"])
        H_est = C_est = 0.0
        H_s = 0
        for (N, k), pk in zip(sizes, picks):
            h = int(F["hops"][pk].sum())
            H_s += h
            H_est += N / k * h
            C_est += N / k * float(rownnz[pk].sum())
        t_walk = max(t_s - self.t_fixed, 1e-9)
        build_s = self.t_fixed + t_walk * (H_est / max(H_s, 1))
        m1 = 2 * (C_est + A.n) + A.nnz + 4 * A.n
        pcg_s = self.iters_small * self.sec_per_mult * m1
        # the next sample sized for about target_s of walk time
        self.m = int(min(4096, max(4, round(self.m * target_s / t_walk))))
        return build_s + pcg_s, dict(build_s=build_s, pcg_s=pcg_s, rows=int(rows.size), hops=H_s,
                                     hops_est=H_est, factor_entries_est=C_est, sample_s=t_s)

    def describe(self, d):
        return (f"{d['rows']} rows stratified by row index ({len(self.strata)} strata, factor 4), "
                f"{self.walks} walks each ({d['hops']} hops) built by the oracle on {self.threads} host "
                f"threads in {d['sample_s']:.1f} s; scaled to {d['hops_est']:.3e} hops (build "
                f"{d['build_s']:.0f} s) and {d['factor_entries_est']:.3e} factor entries; PCG "
                f"{self.iters_small} iterations (oracle, 32^3 instance) x "
                f"{self.sec_per_mult * 1e9:.3f} ns per multiplication of M1 on the full matrix "
                f"({d['pcg_s']:.1f} s)")


def _small_instance():
    cfg = W.make_config(5, scale=0.25)
    return cfg["A"], cfg["b"][:, 0]


def oracle_baseline_c5(cfg, target_s=10.0, seed=2024):
    """The oracle's estimated seconds for workload 5's plain form (one bounded
    sample after calibration), as the bench line's cpu_baseline."""
    est = OracleEstimate(cfg["A"], cfg["b"][:, 0], cfg["walks"], cfg["walk_seed"], cfg["drop_tol"],
                         cfg["tol"], _small_instance())
    rng = np.random.default_rng(seed)
    est.step(rng, target_s)            # sizes the sample
    v, d = est.step(rng, target_s)
    return {"value": v, "unit": "s to 1e-6 (build + solve)", "cores": est.threads, "kind": "oracle",
            "form": "plain: uniform 300 walks + FP64 PCG", "sample": est.describe(d)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    if args.workload == 5:
        cfg = W.make_config(5, scale=args.scale)
        est = OracleEstimate(cfg["A"], cfg["b"][:, 0], cfg["walks"], cfg["walk_seed"], cfg["drop_tol"],
                             cfg["tol"], _small_instance())
        target = max(2.0, 60.0 / max(1, args.warmup + args.steps))
        rng = np.random.default_rng(100)
        vals = []
        for i in range(args.warmup + args.steps):
            v, d = est.step(rng, target)
            if i >= args.warmup:
                vals.append((v, d))
        v = statistics.mean(x for x, _ in vals)
        unit = "s to 1e-6 (build + solve)"
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": unit,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * statistics.mean(d["sample_s"] for _, d in vals),
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": W.CONFIGS[5]["name"], "form": "plain: uniform 300 walks + FP64 PCG"},
                "cpu_baseline": {"value": v, "unit": unit, "cores": est.threads, "kind": "oracle",
                                 "sample": est.describe(vals[-1][1])},
                "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    cfg = W.make_config(args.workload)
    vals = []
    for i in range(args.warmup + args.steps):
        r = _oracle_sample_for(args.workload, cfg, max(2.0, 60.0 / max(1, args.warmup + args.steps)),
                               100 + i)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.mean(r["value"] for r in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "hops/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(r["seconds"] for r in vals),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W.CONFIGS[args.workload]["name"]},
            "cpu_baseline": {"value": v, "unit": "hops/s", "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "hops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class Timer:
    """Per-step CUDA-event timing with an L2 flush between steps."""

    def __init__(self, torch, dev, stream):
        self.torch, self.stream = torch, stream
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run(self, fn, steps, warmup, ws, local):
        torch = self.torch
        for _ in range(warmup):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        infos = []
        clocks = ClockSampler(local)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks.start()
        for i in range(steps):
            self.flush.fill_(float(i))
            torch.cuda.nvtx.range_push("bench_step")  # profilers select the timed steps by this range
            ev[i][0].record(self.stream)
            infos.append(fn())
            ev[i][1].record(self.stream)
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clk = clocks.stop()
        if ws > 1:
            torch.distributed.barrier()
        ms = statistics.mean(a.elapsed_time(b_) for a, b_ in ev)
        return ms, infos, clk


def _tables_bytes(A):
    """Bytes of the walk tables of A (group sectors plus summary sectors)."""
    deg = np.diff(A.rowptr).astype(np.int64) - 1
    ng = (deg + 4) // 4
    return int(((ng + (ng > 2)) * 32).sum())


def _walk_roofline(P, ctx, peaks, peak_kind, As, hops, walk_ms, l2_bytes, tag):
    """Roofline of the walk kernel: algorithmic bytes per hop (stationary-
    weighted over the matrices) x hops / kernel time, against the measured
    HBM copy peak, or against the L2 random-sector gather peak (measured live)
    when the tables fit in three quarters of the L2.  Traffic comes from the
    profile of this workload while the walk sources are unchanged."""
    As = As if isinstance(As, list) else [As]
    num = den = 0.0
    for A in As:
        deg = np.diff(A.rowptr).astype(np.int64) - 1
        rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
        diag = A.val[A.col == rows]
        num += float((diag * 32.0 * (2 + np.ceil(4.0 * (deg + 1) / 32.0))).sum())
        den += float(diag.sum())
    bph = num / den
    tb = sum(_tables_bytes(A) for A in As)
    achieved = bph * hops / (walk_ms * 1e-3) / 1e9 if walk_ms > 0 else 0.0
    gather_l2 = P.rw_probe_gather(ctx, 32 << 20, 32)
    gather_tab = P.rw_probe_gather(ctx, max(tb, 1 << 20), 32)
    tph, tsrc = _walk_traffic_per_hop(tag)
    if tb * 4 <= l2_bytes * 3:
        bound, peak, pk = "l2", gather_l2, "measured live: random 32-byte gathers over an L2-resident buffer"
    else:
        bound, peak, pk = "hbm", peaks["hbm_gbs"], peak_kind
    return {"kernel": "k_walk", "bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if peak else None, "traffic": tph * hops if tph else None,
            "traffic_source": tsrc, "bytes_per_hop": bph, "hops_per_launch": hops, "ms_per_launch": walk_ms,
            "peak_kind": pk, "tables_bytes": tb,
            "gather": {"tables_random_sector_gbs": gather_tab, "l2_random_sector_gbs": gather_l2,
                       "dram_gbs": (tph * hops / (walk_ms * 1e-3) / 1e9) if tph else None}}


def _solve_kernels(opt):
    """Names of the triangular-solve kernels the tuned options run."""
    def one(mode):
        free = "k_syncfree_vec" if opt.get("wide_slices") == -1 else "k_syncfree"
        return free if mode == 1 else f"k_thin/{free}" if mode == 2 else "k_thin/k_wide"
    fwd = one(opt.get("solve_mode", 0))
    bwd = one(opt.get("solve_mode_bwd", -1) if opt.get("solve_mode_bwd", -1) >= 0 else opt.get("solve_mode", 0))
    return f"{fwd} (forward) + {bwd} (backward)"


def _solve_roofline(peaks, napply, nnz_y, n, nrhs, tri_ms, vbytes, ybytes, kernels="triangular solves"):
    # per application of the preconditioner the factor (Y and Y^T) and the
    # vectors (read and written per solve) must be touched once
    tri_bytes = napply * (2 * ybytes * nnz_y + 2 * 3 * vbytes * nrhs * n)
    achieved = tri_bytes / (tri_ms * 1e-3) / 1e9 if tri_ms > 0 else 0.0
    return {"kernel": kernels, "bound": "hbm", "achieved": achieved,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
            "traffic": None, "ms_per_step": tri_ms,
            "note": "latency-bound: dependency DAG depth x dependent memory round trips"}


def _base_line(args, ws, ms, dtype, config):
    return {"metric": METRIC, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": config}


def run_gpu_single(args, P, torch, dev, stream, ws, rank, local):
    """Workloads 2 and 3: one matrix, build + PCG per step."""
    cfg = W.make_config(args.workload)
    A, b = cfg["A"], cfg["b"]
    walks, seed, drop, tol = cfg["walks"], cfg["walk_seed"], cfg["drop_tol"], cfg["tol"]
    mixed = cfg["precision"] == "fp32"
    prec = P.RW_FP32_MIXED if mixed else P.RW_FP64
    nrhs = b.shape[1]
    ctx = P.Context(stream=stream)
    dA = P.CSR.from_host(A, device=dev)
    db = torch.as_tensor(b, device=dev)
    dx = torch.zeros_like(db)

    # schedule autotuning on this matrix's factor (untimed)
    F0 = P.rw_build_factor(ctx, dA, walks, seed, drop)
    tuned, tuned_ms = P.rw_autotune(ctx, dA, F0, nrhs, prec)
    F0.destroy()

    def step():
        F = P.rw_build_factor(ctx, dA, walks, seed, drop)
        rc, st, its, rel = P.pcg_solve(ctx, dA, F, db, dx, tol, 3000, prec)
        d = F.desc
        info = dict(hops=int(d.total_hops), walks=int(d.total_walks), nnz=int(d.nnz),
                    phase=list(d.phase_ms), fwd=d.fwd_levels, bwd=d.bwd_levels,
                    iters=its.tolist(), rel=rel.tolist(), rc=rc, solve_ms=st.solve_ms,
                    spmv_ms=st.spmv_ms, bwd_ms=st.bwd_ms, fwd_ms=st.fwd_ms,
                    launches=int(d.kernel_launches) + int(st.kernel_launches))
        F.destroy()
        return info

    timer = Timer(torch, dev, stream)
    ms, infos, clk = timer.run(step, args.steps, args.warmup, ws, local)
    hops = statistics.mean(i["hops"] for i in infos)
    all_hops, ms = aggregate(hops, ms, ws)
    walk_ms = statistics.mean(i["phase"][1] for i in infos)
    build_ms = statistics.mean(i["phase"][7] for i in infos)
    solve_ms = statistics.mean(i["solve_ms"] for i in infos)

    # end to end through the C ABI with host buffers: H2D of A and b from
    # pinned memory, build, solve, D2H of x, every step
    hA = [torch.as_tensor(a).pin_memory() for a in (A.rowptr, A.col, A.val)]
    hb = torch.as_tensor(b).pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    dA2 = [torch.empty_like(t, device=dev) for t in hA]
    db2 = torch.empty_like(hb, device=dev)
    dx2 = torch.empty_like(hb, device=dev)
    A2 = P.CSR(*dA2)
    h2d = sum(t.numel() * t.element_size() for t in hA) + hb.numel() * hb.element_size()
    d2h = hx.numel() * hx.element_size()
    e2e_ms = []
    for i in range(max(1, args.steps)):
        timer.flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d_, h_ in zip(dA2, hA):
            d_.copy_(h_, non_blocking=True)
        db2.copy_(hb, non_blocking=True)
        F = P.rw_build_factor(ctx, A2, walks, seed, drop)
        P.pcg_solve(ctx, A2, F, db2, dx2, tol, 3000, prec)
        hx.copy_(dx2, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        F.destroy()
    e2e = statistics.mean(e2e_ms)

    # the two latencies that bound the solves' dependency chains (untimed)
    handoff_ns, l2_ns = P.rw_probe_latency(ctx, 20000)
    extra = {}
    if mixed:
        # the same factor solved in FP64 (untimed comparison run): error of the
        # FP32 solution, iteration counts and solve times of both
        F = P.rw_build_factor(ctx, dA, walks, seed, drop)
        x32 = torch.zeros_like(db)
        x64 = torch.zeros_like(db)
        _, st32, it32, rel32 = P.pcg_solve(ctx, dA, F, db, x32, tol, 3000, P.RW_FP32_MIXED)
        _, st64, it64, rel64 = P.pcg_solve(ctx, dA, F, db, x64, tol, 3000, P.RW_FP64)
        err = float(torch.linalg.norm(x32 - x64) / torch.linalg.norm(x64))
        extra["fp32_vs_fp64"] = {"rel_error_x": err, "iters_fp32": it32.tolist(), "iters_fp64": it64.tolist(),
                                 "rel_residual_fp32": rel32.tolist(), "rel_residual_fp64": rel64.tolist(),
                                 "pcg_s_fp32": st32.solve_ms * 1e-3, "pcg_s_fp64": st64.solve_ms * 1e-3}
        F.destroy()
    peaks, peak_kind = _peaks()
    walk_roof = _walk_roofline(P, ctx, peaks, peak_kind, A, hops, walk_ms,
                               torch.cuda.get_device_properties(dev).L2_cache_size,
                               {2: "grid3d7pt_64cube", 3: "grid2d_1000sq_longrange"}[args.workload])
    ctx.close()
    if rank != 0:
        return
    napply = statistics.mean(max(i["iters"]) for i in infos)
    tri_ms = statistics.mean(i["bwd_ms"] + i["fwd_ms"] for i in infos)
    solve_roof = _solve_roofline(peaks, napply, infos[-1]["nnz"], A.n, nrhs, tri_ms,
                                 4.0 if mixed else 8.0, 8.0 if mixed else 12.0,
                                 _solve_kernels(tuned))
    # latency view of the solves: each level of a solve waits for at least one
    # value stored by another SM, so one SM-to-SM hand-off per level is a floor
    nlev = infos[-1]["fwd"] + infos[-1]["bwd"]
    per_level_us = tri_ms * 1e3 / (napply * nlev) if napply and nlev else 0.0
    solve_roof["latency"] = {"per_level_us": per_level_us, "handoff_us": handoff_ns * 1e-3,
                             "l2_load_us": l2_ns * 1e-3, "levels_per_application": nlev,
                             "applications": napply,
                             "frac": handoff_ns * 1e-3 / per_level_us if per_level_us > 0 else None}
    dominant = solve_roof if tri_ms > walk_ms else walk_roof
    line = _base_line(args, ws, ms, "f32-mixed" if mixed else "f64",
                      {"workload": W.CONFIGS[args.workload]["name"], "n": A.n, "nnz": A.nnz,
                       "walks_per_row": walks, "drop_tol": drop, "nrhs": nrhs, "pcg_tol": tol,
                       "precision": cfg["precision"], "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{ws}"})
    line.update({
        "value": all_hops / (ms * 1e-3), "unit": "hops/s", "higher_is_better": True,
        "factor_build_s": build_ms * 1e-3, "pcg_s": solve_ms * 1e-3,
        "walk_kernel_hops_per_s": hops / (walk_ms * 1e-3),
        "pcg_iterations": infos[-1]["iters"], "pcg_rel_residual": infos[-1]["rel"],
        "factor_nnz": infos[-1]["nnz"], "levels": [infos[-1]["fwd"], infos[-1]["bwd"]],
        "phase_ms": {k: round(v, 3) for k, v in zip(
            ["tables", "walk", "merge", "emit", "transpose", "levels", "fp32", "build_total"],
            infos[-1]["phase"])},
        "roofline": dominant if dominant is walk_roof else dict(dominant, peak_kind=peak_kind),
        "roofline_walk": walk_roof,
        "solve_phase_ms": {"spmv": infos[-1]["spmv_ms"], "bwd": infos[-1]["bwd_ms"],
                           "fwd": infos[-1]["fwd_ms"]},
        "clocks": clk,
        "e2e": {"value": aggregate(hops, e2e, ws)[0] / (aggregate(0, e2e, ws)[1] * 1e-3), "unit": "hops/s",
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e},
        "gpu_launches": infos[-1]["launches"],
        "autotuned": {"options": tuned, "precond_ms": tuned_ms[0], "spmv_ms": tuned_ms[1]},
    })
    line.update(extra)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_oracle_sample(A, walks, seed, drop,
                                                 f"the {W.CONFIGS[args.workload]['name']} workload")
    print(json.dumps(line), flush=True)


def run_gpu_batched(args, P, torch, dev, stream, ws, rank, local):
    """Workload 4: 256 matrices, one walk launch, one block-diagonal PCG."""
    cfg = W.make_config(4, nmat=args.nmat)
    As, bs = cfg["A"], cfg["b"]
    walks, drop, tol = cfg["walks"], cfg["drop_tol"], cfg["tol"]
    nmat = len(As)
    seeds = [cfg["walk_seed"] + 7919 * m for m in range(nmat)]
    nrhs = bs[0].shape[1]
    ctx = P.Context(stream=stream)
    dAs = [P.CSR.from_host(A, device=dev) for A in As]
    dbs = [torch.as_tensor(b, device=dev) for b in bs]
    dxs = [torch.zeros_like(b) for b in dbs]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    # schedule autotuning on the combined system (untimed)
    Fs0 = P.rw_build_factor_batched(ctx, dAs, walks, seeds, drop)
    B0 = P.Batch(ctx, dAs, Fs0)
    tuned, tuned_ms = P.rw_batch_autotune(ctx, B0, nrhs, P.RW_FP64)
    B0.destroy()
    for F in Fs0:
        F.destroy()

    def step():
        ev[0].record(stream)
        Fs = P.rw_build_factor_batched(ctx, dAs, walks, seeds, drop)
        ev[1].record(stream)
        B = P.Batch(ctx, dAs, Fs)
        ev[2].record(stream)
        rc, st, its, rel = P.pcg_solve_batch(ctx, B, dbs, dxs, tol, 3000)
        ev[3].record(stream)
        torch.cuda.synchronize()
        d0 = Fs[0].desc
        info = dict(hops=sum(int(F.desc.total_hops) for F in Fs), walks=sum(int(F.desc.total_walks) for F in Fs),
                    nnz=sum(int(F.desc.nnz) for F in Fs), walk_ms=d0.phase_ms[1],
                    build_ms=ev[0].elapsed_time(ev[1]), batch_ms=ev[1].elapsed_time(ev[2]),
                    pcg_ms=ev[2].elapsed_time(ev[3]), iters=its, rel=float(rel.max()), rc=rc,
                    info=B.info(), launches=int(d0.kernel_launches) + int(st[0].kernel_launches))
        B.destroy()
        for F in Fs:
            F.destroy()
        return info

    timer = Timer(torch, dev, stream)
    ms, infos, clk = timer.run(step, args.steps, args.warmup, ws, local)
    hops = statistics.mean(i["hops"] for i in infos)
    all_hops, ms = aggregate(hops, ms, ws)
    last = infos[-1]
    peaks, peak_kind = _peaks()
    walk_roof = _walk_roofline(P, ctx, peaks, peak_kind, As, hops, last["walk_ms"],
                               torch.cuda.get_device_properties(dev).L2_cache_size, "rgg256")
    ctx.close()
    if rank != 0:
        return
    line = _base_line(args, ws, ms, "f64",
                      {"workload": W.CONFIGS[4]["name"], "nmat": nmat, "n_total": sum(A.n for A in As),
                       "nnz_total": sum(A.nnz for A in As), "walks_per_row": walks, "drop_tol": drop,
                       "nrhs": nrhs, "pcg_tol": tol, "precision": "fp64", "graphs": True,
                       "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{ws}"})
    its = last["iters"]
    line.update({
        "value": all_hops / (ms * 1e-3), "unit": "hops/s", "higher_is_better": True,
        "factor_build_s": statistics.mean(i["build_ms"] for i in infos) * 1e-3,
        "batch_create_s": statistics.mean(i["batch_ms"] for i in infos) * 1e-3,
        "pcg_s": statistics.mean(i["pcg_ms"] for i in infos) * 1e-3,
        "walk_kernel_hops_per_s": hops / (last["walk_ms"] * 1e-3) if last["walk_ms"] > 0 else None,
        "pcg_iterations": {"max": int(its.max()), "median": float(np.median(its)), "min": int(its.min())},
        "pcg_rel_residual_max": last["rel"], "factor_nnz_total": last["nnz"], "batch": last["info"],
        "roofline": walk_roof,
        "clocks": clk,
        "gpu_launches": last["launches"],
        "autotuned": {"options": tuned, "precond_ms": tuned_ms[0], "spmv_ms": tuned_ms[1]},
    })
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = _oracle_sample_for(4, cfg, 12.0, 2024)
    print(json.dumps(line), flush=True)


def train_budget_model(P, torch, ctx, dev, ninst, edge, epochs, pilot_walks=64, quantity=0):
    """Features and pilot-walk labels (quantity 0: walk lengths, 1: visits to
    the start row, 2: visits per unit walk cost) of `ninst` training instances
    (seeds 100 + j), then Adam training; returns the model and a summary."""
    feats, labels, masks = [], [], []
    t0 = time.time()
    for j in range(ninst):
        A = W.training_instance(j, edge=edge)
        dA = P.CSR.from_host(A, device=dev)
        f = torch.zeros((A.n, 16), device=dev)
        P.rw_row_features(ctx, dA, f)
        out = [torch.zeros(A.n, device=dev) for _ in range(4)]
        P.rw_pilot_stats(ctx, dA, pilot_walks, 1000 + j, *out, quantity=quantity)
        feats.append(f)
        labels.append(out[2])
        masks.append(out[3])
    F = torch.cat(feats)
    Y = torch.cat(labels)
    Mk = torch.cat(masks)
    t_data = time.time() - t0
    M = P.Mlp(ctx, seed=0)
    t0 = time.time()
    losses = P.rw_mlp_train(ctx, M, F, Y, Mk, epochs=epochs, batch=4096, lr=2e-3, seed=1)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    yv = Y[Mk > 0]
    return M, {"instances": ninst, "edge": edge, "seeds": f"{100}..{100 + ninst - 1}", "rows": int(yv.numel()),
               "epochs": epochs, "batch": 4096, "lr": 2e-3, "train_seed": 1, "init_seed": 0,
               "pilot_walks": pilot_walks, "pilot_seeds": f"{1000}..{1000 + ninst - 1}",
               "label": ["walk length", "visits to the start row", "visits per unit walk cost"][quantity],
               "data_s": t_data, "train_s": t_train,
               "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
               "label_var": float(yv.var()), "r2": 1.0 - float(losses[-1]) / float(yv.var())}


def walk_bytes_per_hop(A):
    """Algorithmic bytes of one hop (SURVEY-style count, per node l): a row
    header sector, the threshold sectors the sampling rule must see
    (ceil(4 (deg_l + 1) / 32)) and one successor sector, 32 bytes each --
    96 B for 5- and 7-point nodes, 192 B for interior 27-point nodes, 128 B at
    degree 8.  Averaged with the stationary weights of the walk (proportional
    to A_ll for a chain with transition probabilities -A_lj / A_ll on an
    undirected graph)."""
    deg = np.diff(A.rowptr).astype(np.int64) - 1
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag = A.val[A.col == rows]
    b = 32.0 * (2 + np.ceil(4.0 * (deg + 1) / 32.0))
    return float((diag * b).sum() / diag.sum())


def _source_digest(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# Walk-kernel DRAM traffic per hop from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch divided by its hops), and the digest of
# the sources the kernel was built from when it was taken; the line reports
# traffic only while the sources are unchanged.
WALK_SOURCES = ["paper_math_0609672_gb300/csrc/rw_walk.cu", "paper_math_0609672_gb300/csrc/rw_tables.cu",
                "paper_math_0609672_gb300/csrc/rw_common.cuh"]


def _walk_traffic_per_hop(tag):
    """(DRAM bytes per hop, profile file) from profiles/k_walk_<tag>.md when
    its source digest matches the current walk sources, else (None, None)."""
    import re
    path = os.path.join(ROOT, "profiles", f"k_walk_{tag}.md")
    if not os.path.exists(path):
        return None, None
    txt = open(path).read()
    m = re.search(r"source digest:\s*([0-9a-f]{16})", txt)
    t = re.search(r"DRAM bytes per hop:\s*([0-9.]+)", txt)
    if m and t and m.group(1) == _source_digest(WALK_SOURCES):
        return float(t.group(1)), os.path.relpath(path, ROOT)
    return None, None


def run_gpu_learned(args, P, torch, dev, stream, ws, rank, local):
    """Workload 5: learned budget + FP32 on the batched engine vs plain."""
    cfg = W.make_config(5, scale=args.scale)
    A, b = cfg["A"], cfg["b"]
    drop, tol, seed = cfg["drop_tol"], cfg["tol"], cfg["walk_seed"]
    ctx = P.Context(stream=stream)      # learned + FP32 path
    ctxp = P.Context(stream=stream)     # plain path
    M, train = train_budget_model(P, torch, ctx, dev, args.train_instances, args.train_edge, args.epochs,
                                  quantity=args.label)
    dA = P.CSR.from_host(A, device=dev)
    db = torch.as_tensor(b, device=dev)
    dx = torch.zeros_like(db)
    budget = torch.zeros(A.n, dtype=torch.int32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    # schedule autotuning of each path on its own factor (untimed)
    P.rw_budget_predict(ctx, dA, M, 300.0, 20, budget)
    F0 = P.rw_build_factor_budget(ctx, dA, budget, seed, drop)
    B0 = P.Batch(ctx, [dA], [F0])
    tuned_l, _ = P.rw_batch_autotune(ctx, B0, 1, P.RW_FP32_MIXED)
    B0.destroy()
    F0.destroy()
    F0 = P.rw_build_factor(ctxp, dA, 300, seed, drop)
    tuned_p, _ = P.rw_autotune(ctxp, dA, F0, 1, P.RW_FP64)
    F0.destroy()

    def learned():
        ev[0].record(stream)
        P.rw_budget_predict(ctx, dA, M, 300.0, 20, budget)
        F = P.rw_build_factor_budget(ctx, dA, budget, seed, drop)
        ev[1].record(stream)
        B = P.Batch(ctx, [dA], [F])
        rc, st, its, rel = P.pcg_solve_batch(ctx, B, [db], [dx], tol, 3000, P.RW_FP32_MIXED)
        ev[2].record(stream)
        torch.cuda.synchronize()
        d = F.desc
        info = dict(hops=int(d.total_hops), walks=int(d.total_walks), nnz=int(d.nnz),
                    build_ms=ev[0].elapsed_time(ev[1]), pcg_ms=ev[1].elapsed_time(ev[2]),
                    iters=int(its.max()), rel=float(rel.max()), rc=rc, walk_ms=d.phase_ms[1],
                    phase=list(d.phase_ms), levels=[d.fwd_levels, d.bwd_levels],
                    launches=int(d.kernel_launches) + int(st[0].kernel_launches))
        B.destroy()
        F.destroy()
        return info

    z99 = 2.5758293035489004           # Q^-1((1 - 0.99) / 2): alpha = 99 %

    def adaptive():
        ev[0].record(stream)
        rounds = P.rw_adaptive_budget(ctx, dA, seed, args.adapt_delta, z99, 20, 65535, 12, budget)
        ev[3].record(stream)
        F = P.rw_build_factor_budget(ctx, dA, budget, seed, drop)
        ev[1].record(stream)
        B = P.Batch(ctx, [dA], [F])
        rc, st, its, rel = P.pcg_solve_batch(ctx, B, [db], [dx], tol, 3000, P.RW_FP32_MIXED)
        ev[2].record(stream)
        torch.cuda.synchronize()
        d = F.desc
        info = dict(hops=int(d.total_hops), walks=int(d.total_walks), nnz=int(d.nnz),
                    build_ms=ev[0].elapsed_time(ev[1]), pcg_ms=ev[1].elapsed_time(ev[2]),
                    count_ms=ev[0].elapsed_time(ev[3]), iters=int(its.max()), rel=float(rel.max()), rc=rc,
                    rounds=rounds)
        B.destroy()
        F.destroy()
        return info

    def plain():
        ev[0].record(stream)
        F = P.rw_build_factor(ctxp, dA, 300, seed, drop)
        ev[1].record(stream)
        rc, st, its, rel = P.pcg_solve(ctxp, dA, F, db, dx, tol, 3000, P.RW_FP64)
        ev[2].record(stream)
        torch.cuda.synchronize()
        d = F.desc
        info = dict(hops=int(d.total_hops), walks=int(d.total_walks), nnz=int(d.nnz),
                    build_ms=ev[0].elapsed_time(ev[1]), pcg_ms=ev[1].elapsed_time(ev[2]),
                    iters=int(its.max()), rel=float(rel.max()), rc=rc, walk_ms=d.phase_ms[1],
                    launches=int(d.kernel_launches) + int(st.kernel_launches))
        F.destroy()
        return info

    timer = Timer(torch, dev, stream)
    ms_l, inf_l, clk = timer.run(learned, args.steps, args.warmup, ws, local)
    ms_p, inf_p, clk_p = timer.run(plain, args.steps, args.warmup, ws, local)
    _, ms_l = aggregate(0, ms_l, ws)
    _, ms_p = aggregate(0, ms_p, ws)
    adapt = None
    if args.adapt_delta > 0:
        ms_a, inf_a, _ = timer.run(adaptive, args.steps, args.warmup, ws, local)
        _, ms_a = aggregate(0, ms_a, ws)
        Ad = inf_a[-1]
        adapt = {"delta": args.adapt_delta, "alpha": 0.99, "min_walks": 20, "s": ms_a * 1e-3,
                 "build_s": statistics.mean(i["build_ms"] for i in inf_a) * 1e-3,
                 "count_s": statistics.mean(i["count_ms"] for i in inf_a) * 1e-3,
                 "pcg_s": statistics.mean(i["pcg_ms"] for i in inf_a) * 1e-3, "iterations": Ad["iters"],
                 "rel_residual": Ad["rel"], "factor_nnz": Ad["nnz"], "walks": Ad["walks"], "hops": Ad["hops"],
                 "rounds": Ad["rounds"],
                 "form": "Sec. 5.1 counts (walks run twice: rounds, then build) + FP32 PCG (batched engine)"}

    # end to end through the C ABI with host buffers: the learned form with the
    # H2D copy of A and b from pinned memory and the D2H copy of x in every step
    hA = [torch.as_tensor(a).pin_memory() for a in (A.rowptr, A.col, A.val)]
    hb = torch.as_tensor(b).pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    dA2 = [torch.empty_like(t, device=dev) for t in hA]
    db2 = torch.empty_like(hb, device=dev)
    dx2 = torch.empty_like(hb, device=dev)
    A2 = P.CSR(*dA2)
    h2d = sum(t.numel() * t.element_size() for t in hA) + hb.numel() * hb.element_size()
    d2h = hx.numel() * hx.element_size()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        timer.flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d_, h_ in zip(dA2, hA):
            d_.copy_(h_, non_blocking=True)
        db2.copy_(hb, non_blocking=True)
        P.rw_budget_predict(ctx, A2, M, 300.0, 20, budget)
        F = P.rw_build_factor_budget(ctx, A2, budget, seed, drop)
        B = P.Batch(ctx, [A2], [F])
        P.pcg_solve_batch(ctx, B, [db2], [dx2], tol, 3000, P.RW_FP32_MIXED)
        hx.copy_(dx2, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        B.destroy()
        F.destroy()
    e2e = statistics.mean(e2e_ms)
    _, e2e = aggregate(0, e2e, ws)
    peaks, peak_kind = _peaks()
    L, Pn = inf_l[-1], inf_p[-1]
    walk_ms = statistics.mean(i["walk_ms"] for i in inf_l)
    walk_roof = _walk_roofline(P, ctx, peaks, peak_kind, A, L["hops"], walk_ms,
                               torch.cuda.get_device_properties(dev).L2_cache_size, "grid3d27pt_128cube")
    M.destroy()
    ctx.close()
    ctxp.close()
    if rank != 0:
        return
    name = W.CONFIGS[5]["name"] + ("" if args.scale == 1.0 else f" (edge scale {args.scale})")
    line = _base_line(args, ws, ms_l, "f32-mixed",
                      {"workload": name, "n": A.n, "nnz": A.nnz, "mean_budget": 300, "min_budget": 20,
                       "drop_tol": drop, "nrhs": 1, "pcg_tol": tol,
                       "learned": "predict + build + FP32 PCG (batched engine, graphs)",
                       "plain": "uniform 300 + FP64 PCG", "training": "untimed, before the timed steps",
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{ws}"})

    def arm(infos, last):
        b_s = statistics.mean(i["build_ms"] for i in infos) * 1e-3
        w_ms = statistics.mean(i["walk_ms"] for i in infos)
        return {"build_s": b_s, "pcg_s": statistics.mean(i["pcg_ms"] for i in infos) * 1e-3,
                "walk_kernel_ms": w_ms, "walk_hops_per_s": last["hops"] / (w_ms * 1e-3),
                "build_hops_per_s": last["hops"] / b_s, "iterations": last["iters"],
                "rel_residual": last["rel"], "factor_nnz": last["nnz"], "walks": last["walks"],
                "hops": last["hops"]}

    line.update({
        "value": ms_l * 1e-3, "unit": "s to 1e-6 (build + solve)", "higher_is_better": False,
        "plain_s": ms_p * 1e-3, "speedup_vs_plain": ms_p / ms_l,
        "learned": dict(arm(inf_l, L), phase_ms={k: round(v, 3) for k, v in zip(
            ["tables", "walk", "merge", "emit", "transpose", "levels", "fp32", "build_total"], L["phase"])},
            levels=L["levels"]),
        "plain": arm(inf_p, Pn),
        "adaptive": adapt,
        "training": train,
        "autotuned": {"learned": tuned_l, "plain": tuned_p},
        "roofline": walk_roof,
        "clocks": clk, "clocks_plain": clk_p,
        "e2e": {"value": e2e * 1e-3, "unit": "s to 1e-6 (build + solve)", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e,
                "form": "learned, through the C ABI from pinned host buffers"},
        "gpu_launches": L["launches"],
    })
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = oracle_baseline_c5(cfg)
    print(json.dumps(line), flush=True)


# Table 1 of the paper, hybrid-solver columns for m1..m6 (the 50^3 .. 100^3
# Dirichlet grids): factor size C (entries of the Cholesky-like factor,
# diagonal included), iterations I to 1e-6, total multiplications M2; and
# Table 4: preconditioning time T1 and solve time T2 (s, one 2.8 GHz CPU).
PAPER_TABLE1 = {
    "C": [1.6e6, 2.8e6, 4.4e6, 6.7e6, 9.6e6, 1.3e7],
    "I": [18, 19, 19, 19, 20, 20],
    "M2": [8.1e7, 1.5e8, 2.4e8, 3.6e8, 5.5e8, 7.5e8],
    "T1": [5.38, 10.39, 17.97, 28.78, 44.01, 71.57],
    "T2": [2.52, 5.80, 10.59, 17.50, 28.61, 41.07],
}


def run_gpu_table1(args, P, torch, dev, stream, ws, rank, local):
    """Workload 6: the paper's Table 1 grids, regenerated.  Each matrix is put in
    random order on the GPU (Sec. 5.4).  As in the paper's implementation no
    entry is dropped (footnote of Sec. 4): the factor size is set by the walks,
    so the walks per row of each matrix are the integer (bisection, untimed
    builds) whose factor size C is nearest the paper's (scaled by N when the
    grids are scaled).  A step builds all six factors (walk reuse of Sec. 5.3
    unless --no-reuse) and solves b = 1 to 1e-6 in FP64."""
    cfg = W.make_config(6, scale=args.scale)
    seed, tol = cfg["walk_seed"], cfg["tol"]
    reuse = 0 if args.no_reuse else 1
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    mats = []
    for j, (m, A, b) in enumerate(zip(cfg["edges"], cfg["A"], cfg["b"])):
        ctx = P.Context(stream=stream, options=P.rw_options_default(reuse=reuse))
        dA0 = P.CSR.from_host(A, device=dev)
        perm = torch.empty(A.n, dtype=torch.int32, device=dev)
        P.rw_random_permutation(ctx, A.n, seed + j, perm)
        dA = P.rw_permute_csr(ctx, dA0, perm)
        m_paper = W.CONFIGS[6]["edges"][j]
        c_target = PAPER_TABLE1["C"][j] * A.n / m_paper ** 3
        sizes = {}

        def size(walks):
            if walks not in sizes:
                F = P.rw_build_factor(ctx, dA, walks, seed, 0.0)
                sizes[walks] = int(F.desc.nnz) + A.n
                F.destroy()
            return sizes[walks]

        if args.walks:
            walks = args.walks
        else:
            lo, hi = 1, 512                       # smallest walks with C >= target, then the nearer neighbour
            while lo < hi:
                mid = (lo + hi) // 2
                if size(mid) >= c_target:
                    hi = mid
                else:
                    lo = mid + 1
            walks = lo
            if walks > 1 and abs(size(walks - 1) - c_target) < abs(size(walks) - c_target):
                walks -= 1
        F1 = P.rw_build_factor(ctx, dA, walks, seed, 0.0)
        tuned, _ = P.rw_autotune(ctx, dA, F1, 1, P.RW_FP64)
        F1.destroy()
        db = torch.as_tensor(b, device=dev)
        mats.append(dict(m=m, n=A.n, E=A.nnz, ctx=ctx, dA=dA, db=db, dx=torch.zeros_like(db), walks=walks,
                         c_target=c_target, tuned=tuned, probes=len(sizes)))

    def step():
        out = []
        launches = 0
        for M in mats:
            ev[0].record(stream)
            F = P.rw_build_factor(M["ctx"], M["dA"], M["walks"], seed, 0.0)
            ev[1].record(stream)
            rc, st, its, rel = P.pcg_solve(M["ctx"], M["dA"], F, M["db"], M["dx"], tol, 3000, P.RW_FP64)
            ev[2].record(stream)
            torch.cuda.synchronize()
            d = F.desc
            out.append(dict(T1=ev[0].elapsed_time(ev[1]) * 1e-3, T2=ev[1].elapsed_time(ev[2]) * 1e-3,
                            I=int(its.max()), rel=float(rel.max()), C=int(d.nnz) + M["n"], hops=int(d.total_hops),
                            walks=int(d.total_walks), extra=int(d.extra_walks), walk_ms=d.phase_ms[1], rc=rc))
            launches += int(d.kernel_launches) + int(st.kernel_launches)
            F.destroy()
        return dict(rows=out, launches=launches)

    timer = Timer(torch, dev, stream)
    ms, infos, clk = timer.run(step, args.steps, args.warmup, ws, local)
    _, ms = aggregate(0, ms, ws)
    for M in mats:
        M["ctx"].close()
    if rank != 0:
        return
    rows = []
    for j, M in enumerate(mats):
        r = infos[-1]["rows"][j]
        M1 = 2 * r["C"] + M["E"] + 4 * M["n"]
        rows.append({"matrix": f"m{j + 1}", "edge": M["m"], "N": M["n"], "E": M["E"], "walks_per_row": M["walks"],
                     "C": r["C"], "C_paper_scaled": round(M["c_target"]), "M1": M1, "I": r["I"],
                     "M2": M1 * r["I"], "rel_residual": r["rel"],
                     "T1_s": statistics.mean(i["rows"][j]["T1"] for i in infos),
                     "T2_s": statistics.mean(i["rows"][j]["T2"] for i in infos),
                     "walks": r["walks"], "extra_walks": r["extra"], "hops": r["hops"],
                     "walk_kernel_ms": r["walk_ms"], "size_probes": M["probes"],
                     "paper": {k: PAPER_TABLE1[k][j] for k in PAPER_TABLE1}})
    name = W.CONFIGS[6]["name"] + ("" if args.scale == 1.0 else f" (edge scale {args.scale})")
    line = _base_line(args, ws, ms, "f64",
                      {"workload": name, "reuse": bool(reuse), "ordering": "random (GPU)",
                       "walks_per_row": "per matrix: factor size C of Table 1" if not args.walks else args.walks,
                       "drop_tol": 0.0, "rhs": "b = 1", "pcg_tol": tol,
                       "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{ws}"})
    line.update({
        "value": ms * 1e-3, "unit": "s (build + solve, m1-m6)", "higher_is_better": False,
        "paper_s": sum(PAPER_TABLE1["T1"]) + sum(PAPER_TABLE1["T2"]),
        "matrices": rows, "clocks": clk, "gpu_launches": infos[-1]["launches"],
        "autotuned": [M["tuned"] for M in mats],
    })
    print(json.dumps(line), flush=True)


def run_gpu_asym(args, P, torch, dev, stream, ws, rank, local):
    """Workload 7: a nonsymmetric matrix (Sec. 7.1).  A step transposes A on the
    GPU, builds the factors of the games on A and on A^T and solves A x = b by
    BiCGSTAB with the two-game preconditioner to 1e-6.  The one-game arm uses
    the factor of A alone (Y_A^T D Y_A) as the preconditioner."""
    cfg = W.make_config(7, scale=args.scale)
    A, b = cfg["A"], cfg["b"]
    walks, seed, drop, tol = cfg["walks"], cfg["walk_seed"], cfg["drop_tol"], cfg["tol"]
    ctx = P.Context(stream=stream)
    dA = P.CSR.from_host(A, device=dev)
    db = torch.as_tensor(b, device=dev)
    dx = torch.zeros_like(db)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    F0 = P.rw_build_factor(ctx, dA, walks, seed, drop)
    tuned, _ = P.rw_autotune(ctx, dA, F0, 1, P.RW_FP64)
    F0.destroy()

    def step(two=True):
        ev[0].record(stream)
        FA = P.rw_build_factor(ctx, dA, walks, seed, drop)
        FAT = FA
        if two:
            dAT = P.rw_csr_transpose(ctx, dA)
            FAT = P.rw_build_factor(ctx, dAT, walks, seed + 1, drop)
        ev[1].record(stream)
        rc, st = P.bicgstab_solve(ctx, dA, FA, FAT, db, dx, tol, 2000)
        ev[2].record(stream)
        torch.cuda.synchronize()
        info = dict(build_ms=ev[0].elapsed_time(ev[1]), solve_ms=ev[1].elapsed_time(ev[2]), iters=int(st.iterations),
                    rel=float(st.rel_residual), rc=rc, hops=int(FA.desc.total_hops) + (int(FAT.desc.total_hops) if two else 0),
                    nnz=int(FA.desc.nnz) + (int(FAT.desc.nnz) if two else 0),
                    launches=int(FA.desc.kernel_launches) + (int(FAT.desc.kernel_launches) if two else 0)
                    + int(st.kernel_launches))
        if two:
            FAT.destroy()
        FA.destroy()
        return info

    timer = Timer(torch, dev, stream)
    ms, infos, clk = timer.run(step, args.steps, args.warmup, ws, local)
    ms1, infos1, _ = timer.run(lambda: step(False), args.steps, args.warmup, ws, local)
    _, ms = aggregate(0, ms, ws)
    _, ms1 = aggregate(0, ms1, ws)
    ctx.close()
    if rank != 0:
        return
    I, I1 = infos[-1], infos1[-1]
    name = W.CONFIGS[7]["name"] + ("" if args.scale == 1.0 else f" (edge scale {args.scale})")
    line = _base_line(args, ws, ms, "f64",
                      {"workload": name, "n": A.n, "nnz": A.nnz, "walks_per_row": walks, "drop_tol": drop,
                       "nrhs": 1, "tol": tol, "solver": "BiCGSTAB, right preconditioner Y_AT^T D Y_A",
                       "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{ws}"})
    line.update({
        "value": ms * 1e-3, "unit": "s to 1e-6 (transpose + two builds + BiCGSTAB)", "higher_is_better": False,
        "two_games": {"build_s": statistics.mean(i["build_ms"] for i in infos) * 1e-3,
                      "solve_s": statistics.mean(i["solve_ms"] for i in infos) * 1e-3, "iterations": I["iters"],
                      "rel_residual": I["rel"], "factor_nnz": I["nnz"], "hops": I["hops"]},
        "one_game": {"s": ms1 * 1e-3, "build_s": statistics.mean(i["build_ms"] for i in infos1) * 1e-3,
                     "solve_s": statistics.mean(i["solve_ms"] for i in infos1) * 1e-3, "iterations": I1["iters"],
                     "rel_residual": I1["rel"], "form": "factor of A only: Y_A^T D Y_A"},
        "clocks": clk, "gpu_launches": I["launches"], "autotuned": tuned,
    })
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import paper_math_0609672_gb300 as P
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.workload in (2, 3):
        run_gpu_single(args, P, torch, dev, stream, ws, rank, local)
    elif args.workload == 4:
        run_gpu_batched(args, P, torch, dev, stream, ws, rank, local)
    elif args.workload == 6:
        run_gpu_table1(args, P, torch, dev, stream, ws, rank, local)
    elif args.workload == 7:
        run_gpu_asym(args, P, torch, dev, stream, ws, rank, local)
    else:
        run_gpu_learned(args, P, torch, dev, stream, ws, rank, local)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", type=int, default=5, choices=[2, 3, 4, 5, 6, 7])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nmat", type=int, default=None, help="workload 4: number of matrices (default 256)")
    ap.add_argument("--scale", type=float, default=1.0, help="workloads 5, 6, 7: grid edge scale (default 1)")
    ap.add_argument("--walks", type=int, default=0,
                    help="workload 6: walks per row (default: the count that gives Table 1's factor size)")
    ap.add_argument("--no-reuse", action="store_true", help="workload 6: no walk reuse")
    ap.add_argument("--train-instances", type=int, default=50, help="workload 5: training instances")
    ap.add_argument("--train-edge", type=int, default=64, help="workload 5: training grid edge")
    ap.add_argument("--epochs", type=int, default=10, help="workload 5: training epochs")
    ap.add_argument("--label", type=int, default=2, choices=[0, 1, 2],
                    help="workload 5: pilot label (0 walk length, 1 visits, 2 visits per unit walk cost)")
    ap.add_argument("--adapt-delta", type=float, default=0.25,
                    help="workload 5: relative margin of the Sec. 5.1 adaptive-count arm (0 skips it)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
