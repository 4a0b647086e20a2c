"""Full-size solve parity and the learned budget's gain, on the GPU.

* The 64^3 7-point workload at full size: the GPU factor equals the oracle's
  full factor bit for bit, and PCG (autotuned schedule, four right-hand sides
  at once) matches the oracle's PCG on every right-hand side: equal
  iteration counts, solutions within 1e-10 relative (FP64, Algorithm 1).
* The FP32 mode against the oracle's FP32 mode (the same mixed-precision
  algorithm, rounded in a different order), element by element at equal
  iteration counts, within a bound derived from FP32 rounding; its error
  against the FP64 oracle solution is computed as well.
* The learned walk budget (Sec. 5.1's per-row accuracy target, learned from
  pilot walks) trained by the library's own kernels over several epochs,
  against the uniform budget at equal total walks, on a 32^3 27-point grid of
  the 128^3 workload's distribution.
* The 256-matrix random geometric graph batch at full size: sampled rows of
  sampled matrices bit for bit against the oracle.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_math_0609672_gb300 as P
    from paper_math_0609672_gb300 import _build
    _build.build()
    return P


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_full_size_c2_pcg_matches_oracle(P):
    cfg = W.make_config(2)
    A, b = cfg["A"], cfg["b"]
    walks, seed, drop, tol = cfg["walks"], cfg["walk_seed"], cfg["drop_tol"], cfg["tol"]
    ref = oracle.build_factor(A, walks, seed, drop, threads=THREADS)
    ctx = P.Context()
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, walks, seed, drop)
    t = {k: v.cpu().numpy() for k, v in F.tensors().items()}
    assert np.array_equal(t["y_row_ptr"], ref["rowptr"])
    assert np.array_equal(t["y_col"], ref["col"])
    assert np.array_equal(t["y_val"].view(np.int64), ref["val"].view(np.int64))
    assert np.array_equal(t["d"].view(np.int64), ref["D"].view(np.int64))
    P.rw_autotune(ctx, dA, F, b.shape[1], P.RW_FP64)
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve(ctx, dA, F, _dev(b), x, tol, 3000)
    assert rc == 0 and np.all(rel < tol)
    xg = x.cpu().numpy()
    for j in range(b.shape[1]):
        xr, itr, rr, rcr = oracle.pcg(A, ref, b[:, j], tol, 3000)
        assert rcr == 0 and its[j] == itr, (j, its[j], itr)
        assert np.linalg.norm(xg[:, j] - xr) / np.linalg.norm(xr) < 1e-10, j
        assert abs(rel[j] - rr) <= 1e-6 * rr
    F.destroy()
    ctx.close()


# FP32 mode: both sides run the same algorithm (FP32 vectors, SpMV, factor and
# solves; FP64 dots, alpha, beta and x; FP64 residual replacement every 50
# iterations) and differ only in the order of the FP32 roundings inside the
# SpMV and the two triangular solves.  One FP32 sum of m terms rounded in two
# orders differs by about sqrt(m) u relative to the terms' size under the
# usual random-rounding model (u = 2^-24); the handful of other FP32 roundings
# per iteration add a small multiple of u, and CG damps the differences of
# earlier iterations as it converges instead of accumulating them.  The bound
# is therefore 8 sqrt(m) u max|x| element-wise at every iteration count, with
# m the longest row of A, Y and Y^T (measured: at most 1.7 sqrt(m) u, after
# the first iteration; below 0.4 sqrt(m) u from the third on).
U32 = 2.0 ** -24


def fp32_bound(m):
    return 8.0 * np.sqrt(m) * U32


@pytest.mark.parametrize("case", ["grid2d_longrange", "grid3d27"])
def test_fp32_mixed_matches_oracle_mixed(P, case):
    if case == "grid2d_longrange":
        cfg = W.make_config(3, scale=0.1)
        walks, seed = cfg["walks"], cfg["walk_seed"]
    else:
        cfg = W.make_config(5, scale=0.25)
        walks, seed = 300, cfg["walk_seed"]
    A, b = cfg["A"], cfg["b"][:, 0]
    ctx = P.Context()
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, walks, seed, cfg["drop_tol"])
    ref = oracle.build_factor(A, walks, seed, cfg["drop_tol"], threads=THREADS)
    ytr = np.bincount(ref["col"], minlength=A.n) if ref["nnz"] else np.zeros(1)
    m = int(max(np.diff(A.rowptr).max(), np.diff(ref["rowptr"]).max(), ytr.max()))
    x64, it64, _, _ = oracle.pcg(A, ref, b, cfg["tol"], 3000)
    xm_conv, itm, rrm, _ = oracle.pcg(A, ref, b, cfg["tol"], 3000, mixed=True)
    db = _dev(b[:, None])
    for K in sorted({1, 3, itm // 2, itm}):
        xm, _, _, _ = oracle.pcg(A, ref, b, 0.0, K, mixed=True)
        x = _dev(np.zeros((A.n, 1)))
        rc, st, its, rel = P.pcg_solve(ctx, dA, F, db, x, 0.0, K, P.RW_FP32_MIXED)
        assert its[0] == K
        d = np.abs(x.cpu().numpy()[:, 0] - xm)
        bound = fp32_bound(m) * np.abs(xm).max()
        assert d.max() <= bound, (K, d.max() / np.abs(xm).max(), fp32_bound(m))
    # to tolerance: equal iteration counts; the error against the FP64 oracle
    x = _dev(np.zeros((A.n, 1)))
    rc, st, its, rel = P.pcg_solve(ctx, dA, F, db, x, cfg["tol"], 3000, P.RW_FP32_MIXED)
    xg = x.cpu().numpy()[:, 0]
    assert rc == 0 and rel[0] < cfg["tol"]
    assert abs(int(its[0]) - itm) <= 1, (its[0], itm)
    err64 = np.linalg.norm(xg - x64) / np.linalg.norm(x64)
    errm = np.linalg.norm(xm_conv - x64) / np.linalg.norm(x64)
    # both FP32 solutions reach the tolerance; their distance to the FP64
    # solution is of the same size (kappa * tol at most)
    assert err64 <= max(4.0 * errm, 1e-9), (err64, errm)
    print(f"{case}: FP32 vs FP64 oracle {err64:.2e} (oracle FP32 {errm:.2e}), iterations {its[0]} / {itm} / {it64}")
    F.destroy()
    ctx.close()


def test_learned_budget_gain_over_uniform(P):
    """Train the budget network on pilot-walk labels of eight 32^3 training
    instances (the library's pilot statistics, forward/backward and Adam
    kernels, 12 epochs), predict budgets at mean 300 on a 32^3 test grid of
    the same distribution, and compare with 300 walks on every row (the same
    total walks).  The label is the relative variance of the visits to the
    start row per unit walk cost, so the trained network moves walks away from
    rows whose walks are long: the build must need clearly fewer hops, and the
    total work -- hops plus PCG iterations x the paper's per-iteration
    multiplication count M1 = 2C + E + 4N (Sec. 6) -- must be smaller."""
    import torch
    ctx = P.Context()
    feats, labels, masks = [], [], []
    for j in range(8):
        At = W.training_instance(j, edge=32)
        dAt = P.CSR.from_host(At)
        f = torch.zeros((At.n, 16), device="cuda")
        P.rw_row_features(ctx, dAt, f)
        out = [torch.zeros(At.n, device="cuda") for _ in range(4)]
        P.rw_pilot_stats(ctx, dAt, 64, 1000 + j, *out, quantity=2)
        feats.append(f)
        labels.append(out[2])
        masks.append(out[3])
    Fe, Y, Mk = torch.cat(feats), torch.cat(labels), torch.cat(masks)
    M = P.Mlp(ctx, seed=0)
    losses = P.rw_mlp_train(ctx, M, Fe, Y, Mk, epochs=12, batch=2048, lr=2e-3, seed=1)
    assert losses[-1] < 0.9 * losses[0], losses
    assert np.all(np.diff(losses[2:]) < 0.05 * losses[0]), losses
    yv = Y[Mk > 0]
    r2 = 1.0 - float(losses[-1]) / float(yv.var())
    assert r2 > 0.2, r2
    cfg = W.make_config(5, scale=0.25)
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    budget = torch.zeros(A.n, dtype=torch.int32, device="cuda")
    P.rw_budget_predict(ctx, dA, M, 300.0, 20, budget)
    wr = oracle.walk_rows(A)
    bud = budget.cpu().numpy().view(np.uint32)
    assert int(bud[wr].sum()) == 300 * wr.size and bud[wr].min() >= 20
    res = {}
    for arm in ("learned", "uniform"):
        if arm == "learned":
            F = P.rw_build_factor_budget(ctx, dA, budget, cfg["walk_seed"], cfg["drop_tol"])
        else:
            F = P.rw_build_factor(ctx, dA, 300, cfg["walk_seed"], cfg["drop_tol"])
        x = _dev(np.zeros_like(b))
        rc, st, its, rel = P.pcg_solve(ctx, dA, F, _dev(b), x, cfg["tol"], 3000, P.RW_FP32_MIXED)
        assert rc == 0 and rel[0] < cfg["tol"]
        C = int(F.desc.nnz) + A.n
        m1 = 2 * C + A.nnz + 4 * A.n
        res[arm] = dict(walks=int(F.desc.total_walks), hops=int(F.desc.total_hops), iters=int(its[0]),
                        work=int(F.desc.total_hops) + int(its[0]) * m1)
        F.destroy()
    L, U = res["learned"], res["uniform"]
    print("learned", L, "uniform", U, "r2", r2)
    assert L["walks"] == U["walks"]
    assert L["hops"] < 0.8 * U["hops"], (L, U)
    assert L["work"] < 0.9 * U["work"], (L, U)
    M.destroy()
    ctx.close()


def test_full_batch_sampled_matrices(P):
    """All 256 random geometric graphs of the batched workload (sum n about
    10^7) built in one walk launch; 12 sampled matrices, 40 sampled rows each
    (plus their first and last rows), recomputed by the oracle with the same
    matrix index and seed: Y rows, D and the counters bit for bit."""
    cfg = W.make_config(4)
    As = cfg["A"]
    nmat = len(As)
    seeds = [cfg["walk_seed"] + 7919 * m for m in range(nmat)]
    ctx = P.Context()
    dAs = [P.CSR.from_host(A) for A in As]
    Fs = P.rw_build_factor_batched(ctx, dAs, cfg["walks"], seeds, cfg["drop_tol"])
    rng = np.random.default_rng(44)
    pick = np.unique(np.concatenate([rng.choice(nmat, 10, replace=False),
                                     [int(np.argmax([A.n for A in As])), nmat - 1]]))
    for mi in pick:
        A = As[mi]
        t = {k: v.cpu().numpy() for k, v in Fs[mi].tensors().items()}
        rows = np.unique(np.concatenate([rng.choice(A.n, min(40, A.n), replace=False), [0, A.n - 1]]))
        ref = oracle.build_factor(A, cfg["walks"], seeds[mi], cfg["drop_tol"], matrix_index=int(mi),
                                  rows=rows, threads=THREADS)
        for k in rows:
            a, b_ = t["y_row_ptr"][k], t["y_row_ptr"][k + 1]
            c, d = ref["rowptr"][k], ref["rowptr"][k + 1]
            assert np.array_equal(t["y_col"][a:b_], ref["col"][c:d]), (mi, k)
            assert np.array_equal(t["y_val"][a:b_].view(np.int64), ref["val"][c:d].view(np.int64)), (mi, k)
            assert t["d"][k].view(np.int64) == ref["D"][k].view(np.int64), (mi, k)
            assert t["walks"][k] == ref["M"][k] and t["visits"][k] == ref["J"][k], (mi, k)
            assert t["ground"][k] == ref["G"][k], (mi, k)
    for F in Fs:
        F.destroy()
    ctx.close()
