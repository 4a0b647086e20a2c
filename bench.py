"""Benchmark: random-walk factor construction + PCG on one GB300.

Workload: 3D 7-point grid 64^3 (n = 262,144), conductances log-uniform in
[0.1, 10], diagonal excess U[0, 1e-3] * row sum, seeded random symmetric
ordering, 500 walks per row, drop tolerance 1e-3, 4 right-hand sides ~ N(0,1),
PCG to 1e-6 true relative residual in FP64.  Synthetic, seeded inputs.

One step = the whole hot path on one batch: build the factor
(rw_build_factor: tables, walks, merge, emission, transpose, levels) and solve
the 4 right-hand sides (pcg_solve), then release the factor.  The headline
value is walk-hops per second of step time (hops of the build / step time);
factor-build seconds and PCG seconds are reported beside it.

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the
library's stream, with an L2 flush (a 512 MB write) between steps outside
the timed events, and a barrier + synchronize on both sides of the timed
region.  Under torchrun each rank runs its own replica (the factor build and
the solves of independent matrices do not exchange data); value = all ranks'
hops / max-over-ranks time.

--impl reference times the CPU oracle on a bounded row sample of the same
workload (the oracle is the baseline: a plain single-threaded C program).
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

WORKLOAD = 2
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


def make_inputs():
    cfg = W.make_config(WORKLOAD)
    return cfg


def cpu_oracle_sample(cfg, target_s=12.0, seed=2024):
    """Time the oracle (single thread) on a random sample of rows of the same
    matrix with the same walks, until about target_s seconds of CPU work."""
    import oracle
    A = cfg["A"]
    rng = np.random.default_rng(seed)
    wr = oracle.walk_rows(A)
    order = rng.permutation(wr)
    done_rows, hops, t_used = 0, 0, 0.0
    chunk = 256
    while t_used < target_s and done_rows < order.size:
        rows = np.sort(order[done_rows:done_rows + chunk])
        t0 = time.perf_counter()
        F = oracle.build_factor(A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"], rows=rows)
        t_used += time.perf_counter() - t0
        hops += int(F["hops"].sum())
        done_rows += rows.size
        chunk = min(chunk * 2, 8192)
    return {"value": hops / t_used, "unit": "hops/s", "cores": 1, "kind": "oracle",
            "sample": f"{done_rows} random walk rows of the 64^3 workload x {cfg['walks']} walks "
                      f"({hops} hops) in {t_used:.1f} s, single thread, factor rows only"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    cfg = make_inputs()
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_sample(cfg, target_s=max(2.0, 60.0 / max(1, args.warmup + args.steps)),
                              seed=100 + i)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.mean(r["value"] for r in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "hops/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W.CONFIGS[WORKLOAD]["name"], "n": cfg["A"].n,
                       "walks_per_row": cfg["walks"], "drop_tol": cfg["drop_tol"],
                       "nrhs": cfg["nrhs"]},
            "cpu_baseline": {"value": v, "unit": "hops/s", "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "hops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import paper_math_0609672_gb300 as P
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = make_inputs()
    A, b = cfg["A"], cfg["b"]
    walks, seed, drop, tol = cfg["walks"], cfg["walk_seed"], cfg["drop_tol"], cfg["tol"]
    nrhs = b.shape[1]
    stream = torch.cuda.current_stream(dev)
    ctx = P.Context(stream=stream)
    dA = P.CSR.from_host(A, device=dev)
    db = torch.as_tensor(b, device=dev)
    dx = torch.zeros_like(db)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        F = P.rw_build_factor(ctx, dA, walks, seed, drop)
        rc, st, its, rel = P.pcg_solve(ctx, dA, F, db, dx, tol, 2000)
        d = F.desc
        info = dict(hops=int(d.total_hops), walks=int(d.total_walks), nnz=int(d.nnz),
                    phase=list(d.phase_ms), fwd=d.fwd_levels, bwd=d.bwd_levels,
                    iters=its.tolist(), rel=rel.tolist(), rc=rc, solve_ms=st.solve_ms,
                    spmv_ms=st.spmv_ms, bwd_ms=st.bwd_ms, fwd_ms=st.fwd_ms,
                    launches=int(d.kernel_launches) + int(st.kernel_launches))
        F.destroy()
        return info

    for _ in range(args.warmup):
        step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    infos = []
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        infos.append(step())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b_) for a, b_ in ev]
    ms = statistics.mean(step_ms)
    hops = statistics.mean(i["hops"] for i in infos)
    walk_ms = statistics.mean(i["phase"][1] for i in infos)
    build_ms = statistics.mean(i["phase"][7] for i in infos)
    solve_ms = statistics.mean(i["solve_ms"] for i in infos)
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())

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
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d_, h_ in zip(dA2, hA):
            d_.copy_(h_, non_blocking=True)
        db2.copy_(hb, non_blocking=True)
        F = P.rw_build_factor(ctx, A2, walks, seed, drop)
        P.pcg_solve(ctx, A2, F, db2, dx2, tol, 2000)
        hx.copy_(dx2, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        F.destroy()
    e2e = statistics.mean(e2e_ms)

    if rank != 0:
        return
    peaks, peak_kind = _peaks()
    walks_total = infos[-1]["walks"]
    nnz_y = infos[-1]["nnz"]
    # algorithmic bytes of the walk kernel: per hop one 32-byte sector of
    # thresholds (degree <= 6 here) + one sector for the chosen successor; per
    # walk one 8-byte record
    alg_bytes = 64.0 * hops + 8.0 * walks_total
    achieved = alg_bytes / (walk_ms * 1e-3) / 1e9
    walk_roof = {"kernel": "k_walk", "bound": "hbm", "achieved": achieved,
                 "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                 "traffic": None, "ms_per_launch": walk_ms}
    # triangular solves: per application of the preconditioner the factor
    # (12 B per stored entry, twice: Y and Y^T) and the vectors (8 B x nrhs x
    # n read and written per solve) must be touched once
    napply = statistics.mean(len(i["iters"]) and max(i["iters"]) for i in infos)
    tri_ms = statistics.mean(i["bwd_ms"] + i["fwd_ms"] for i in infos)
    applies = napply  # one application per iteration (the first before the loop, none after the last)
    tri_bytes = applies * (2 * 12.0 * nnz_y + 2 * 3 * 8.0 * nrhs * A.n)
    tri_achieved = tri_bytes / (tri_ms * 1e-3) / 1e9 if tri_ms > 0 else 0.0
    solve_roof = {"kernel": "k_thin/k_wide (triangular solves)", "bound": "hbm",
                  "achieved": tri_achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "frac": tri_achieved / peaks["hbm_gbs"], "traffic": None,
                  "ms_per_step": tri_ms,
                  "note": "latency-bound: dependency DAG depth x dependent memory round trips"}
    dominant = solve_roof if tri_ms > walk_ms else walk_roof
    line = {
        "metric": METRIC, "value": hops * ws / (ms * 1e-3), "unit": "hops/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": W.CONFIGS[WORKLOAD]["name"], "n": A.n, "nnz": A.nnz,
                   "walks_per_row": walks, "drop_tol": drop, "nrhs": nrhs, "pcg_tol": tol,
                   "precision": "fp64", "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas x{ws}"},
        "factor_build_s": build_ms * 1e-3, "pcg_s": solve_ms * 1e-3,
        "walk_kernel_hops_per_s": hops / (walk_ms * 1e-3),
        "pcg_iterations": infos[-1]["iters"], "pcg_rel_residual": infos[-1]["rel"],
        "factor_nnz": infos[-1]["nnz"], "levels": [infos[-1]["fwd"], infos[-1]["bwd"]],
        "phase_ms": {k: round(v, 3) for k, v in zip(
            ["tables", "walk", "merge", "emit", "transpose", "levels", "fp32", "build_total"],
            infos[-1]["phase"])},
        "roofline": dict(dominant, peak_kind=peak_kind),
        "roofline_walk": dict(walk_roof, peak_kind=peak_kind),
        "solve_phase_ms": {"spmv": infos[-1]["spmv_ms"], "bwd": infos[-1]["bwd_ms"],
                           "fwd": infos[-1]["fwd_ms"]},
        "clocks": clk,
        "e2e": {"value": hops * ws / (e2e * 1e-3), "unit": "hops/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e},
        "gpu_launches": infos[-1]["launches"],
    }
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_oracle_sample(cfg)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
