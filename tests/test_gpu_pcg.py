"""GPU solve path vs the CPU oracle: SpMV, the preconditioner application
z = (Y^T D Y)^-1 r, and PCG (Algorithm 1) in FP64 (1e-10 relative at an equal
iteration count) and in FP32 mixed precision (reaches the tolerance; error
against the FP64 oracle solution reported and bounded)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_math_0609672_gb300 as P
    from paper_math_0609672_gb300 import _build
    _build.build()
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context()
    yield c
    c.close()


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_spmv_matches_reference(P, ctx):
    rng = np.random.default_rng(1)
    A = W.make_config(2, scale=0.25)["A"]
    x = rng.standard_normal((A.n, 4))
    y = _dev(np.zeros_like(x))
    P.rw_spmv(ctx, P.CSR.from_host(A), _dev(x), y)
    ref = A.to_scipy() @ x
    assert np.allclose(y.cpu().numpy(), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("nrhs", [1, 3, 4, 16])
def test_precond_matches_oracle(P, ctx, nrhs):
    rng = np.random.default_rng(nrhs)
    A = W.make_config(2, scale=0.25)["A"]
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, 100, 7, 1e-3)
    ref = oracle.build_factor(A, 100, 7, 1e-3)
    r = rng.standard_normal((A.n, nrhs))
    z = _dev(np.zeros_like(r))
    P.rw_precond_apply(ctx, F, _dev(r), z)
    zg = z.cpu().numpy()
    for j in range(nrhs):
        zr = oracle.precond_apply(ref, r[:, j])
        assert np.linalg.norm(zg[:, j] - zr) / np.linalg.norm(zr) < 1e-12
    F.destroy()


def test_pcg_fp64_equal_iterations_c1(P, ctx):
    cfg = W.make_config(1)
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    ref = oracle.build_factor(A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    for K in (1, 5, 12):
        x = _dev(np.zeros_like(b))
        rc, st, its, rel = P.pcg_solve(ctx, dA, F, _dev(b), x, 0.0, K)
        xr, itr, rr, rcr = oracle.pcg(A, ref, b[:, 0], 0.0, K)
        assert its[0] == K == itr
        xg = x.cpu().numpy()[:, 0]
        assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) < 1e-10, K
        assert abs(rel[0] - rr) <= 1e-8 * max(rr, 1e-30) + 1e-15
    F.destroy()


def test_pcg_fp64_converges_like_oracle_c1(P, ctx):
    cfg = W.make_config(1)
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    ref = oracle.build_factor(A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve(ctx, dA, F, _dev(b), x, cfg["tol"], 500)
    xr, itr, rr, rcr = oracle.pcg(A, ref, b[:, 0], cfg["tol"], 500)
    assert rc == 0 and rcr == 0 and rel[0] < cfg["tol"]
    assert its[0] == itr
    xg = x.cpu().numpy()[:, 0]
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) < 1e-10
    F.destroy()


def test_pcg_multi_rhs_c2_scaled(P, ctx):
    cfg = W.make_config(2, scale=0.25)
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    ref = oracle.build_factor(A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve(ctx, dA, F, _dev(b), x, cfg["tol"], 500)
    assert rc == 0 and np.all(rel < cfg["tol"])
    xg = x.cpu().numpy()
    true = np.linalg.norm(b - A.to_scipy() @ xg, axis=0) / np.linalg.norm(b, axis=0)
    assert np.all(true < cfg["tol"])
    for j in range(b.shape[1]):
        xr, itr, rr, rcr = oracle.pcg(A, ref, b[:, j], cfg["tol"], 500)
        assert its[j] == itr
        assert np.linalg.norm(xg[:, j] - xr) / np.linalg.norm(xr) < 1e-10
    F.destroy()


def test_pcg_fp32_mixed_reaches_tolerance(P, ctx):
    cfg = W.make_config(3, scale=0.1)          # 100^2 grid + long-range edges
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    ref = oracle.build_factor(A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve(ctx, dA, F, _dev(b), x, cfg["tol"], 1000, P.RW_FP32_MIXED)
    assert rc == 0 and rel[0] < cfg["tol"]
    xg = x.cpu().numpy()[:, 0]
    true = np.linalg.norm(b[:, 0] - A.to_scipy() @ xg) / np.linalg.norm(b[:, 0])
    assert true < cfg["tol"]
    x64, it64, rr64, _ = oracle.pcg(A, ref, b[:, 0], cfg["tol"], 1000)
    xm, itm, rrm, _ = oracle.pcg(A, ref, b[:, 0], cfg["tol"], 1000, mixed=True)
    # the oracle's FP32 mode is the same algorithm rounded in another order:
    # equal iteration counts and x within 8 sqrt(m) u max|x| element-wise (the
    # bound of tests/test_gpu_fullsize.py, m the longest row of A, Y and Y^T)
    m = int(max(np.diff(A.rowptr).max(), np.diff(ref["rowptr"]).max(),
                np.bincount(ref["col"], minlength=A.n).max()))
    assert int(its[0]) == itm, (its[0], itm)
    assert np.abs(xg - xm).max() <= 8.0 * np.sqrt(m) * 2.0 ** -24 * np.abs(xm).max()
    # the error against the FP64 solution is that of the oracle's FP32 mode
    err = np.linalg.norm(xg - x64) / np.linalg.norm(x64)
    errm = np.linalg.norm(xm - x64) / np.linalg.norm(x64)
    assert err <= max(2.0 * errm, 1e-9), (err, errm)
    F.destroy()


def test_pcg_zero_rhs_and_nonfinite(P, ctx):
    A = W.grid2d_5pt(8, 8)
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, 10, 1, 0.0)
    b = np.zeros((A.n, 2))
    b[:, 1] = 1.0
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve(ctx, dA, F, _dev(b), x, 1e-8, 100)
    assert rc == 0 and its[0] == 0 and not x.cpu().numpy()[:, 0].any() and rel[1] < 1e-8
    b[3, 1] = np.nan
    with pytest.raises(P.RwError) as e:
        P.pcg_solve(ctx, dA, F, _dev(b), x, 1e-8, 100)
    assert e.value.code == -1
    F.destroy()


def test_pcg_reports_no_convergence(P, ctx):
    cfg = W.make_config(1)
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, 20, 0, 1e-2)
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve(ctx, dA, F, _dev(b), x, 1e-14, 2)
    assert rc == -5 and its[0] == 2 and rel[0] > 1e-14
    F.destroy()


def test_batched_pcg_matches_single(P, ctx):
    """Batched factor build + batched PCG on matrices of uneven size: each
    solution equals the oracle PCG on the oracle factor with that matrix index."""
    rng = np.random.default_rng(9)
    mats = [W.rgg(int(n), rng) for n in (500, 2500, 1200)]
    seeds = [11, 22, 33]
    dAs = [P.CSR.from_host(A) for A in mats]
    Fs = P.rw_build_factor_batched(ctx, dAs, 60, seeds, 1e-3)
    bs = [rng.standard_normal((A.n, 3)) for A in mats]
    xs = [_dev(np.zeros_like(b)) for b in bs]
    rc, st, its, rel = P.pcg_solve_batched(ctx, dAs, Fs, [_dev(b) for b in bs], xs, 1e-8, 500)
    assert rc == 0 and np.all(rel < 1e-8)
    for m, A in enumerate(mats):
        ref = oracle.build_factor(A, 60, seeds[m], 1e-3, matrix_index=m)
        xg = xs[m].cpu().numpy()
        for j in range(3):
            xr, itr, rr, _ = oracle.pcg(A, ref, bs[m][:, j], 1e-8, 500)
            assert its[m, j] == itr
            assert np.linalg.norm(xg[:, j] - xr) / np.linalg.norm(xr) < 1e-10
    for F in Fs:
        F.destroy()


def test_batch_graphs_match_direct_launches_and_oracle(P):
    """The combined block-diagonal solve: 16 right-hand sides over matrices of
    uneven size (rows of several reduction chunks and a ragged tail); replaying
    the captured iteration gives the same bits as launching it directly, and
    every system matches the oracle PCG on its own matrix."""
    import torch
    rng = np.random.default_rng(12)
    mats = [W.rgg(int(n), rng) for n in (3000, 700, 5000, 1)] + [W.grid2d_5pt(30, 20)]
    seeds = [5, 6, 7, 8, 9]
    out = {}
    for graphs in (1, 0):
        ctx = P.Context(options=P.rw_options_default(graphs=graphs))
        dAs = [P.CSR.from_host(A) for A in mats]
        Fs = P.rw_build_factor_batched(ctx, dAs, 40, seeds, 1e-3)
        bs = [np.random.default_rng(100 + m).standard_normal((A.n, 16)) for m, A in enumerate(mats)]
        xs = [_dev(np.zeros_like(b)) for b in bs]
        B = P.Batch(ctx, dAs, Fs)
        info = B.info()
        assert info["n"] == sum(A.n for A in mats)
        rc, st, its, rel = P.pcg_solve_batch(ctx, B, [_dev(b) for b in bs], xs, 1e-9, 400)
        assert rc == 0 and np.all(rel < 1e-9), rel.max()
        out[graphs] = ([x.cpu().numpy() for x in xs], its, bs)
        B.destroy()
        for F in Fs:
            F.destroy()
        ctx.close()
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1], out[1][1])
    xs, its, bs = out[1]
    for m, A in enumerate(mats):
        ref = oracle.build_factor(A, 40, seeds[m], 1e-3, matrix_index=m)
        for j in (0, 7, 15):
            xr, itr, rr, _ = oracle.pcg(A, ref, bs[m][:, j], 1e-9, 400)
            assert its[m, j] == itr, (m, j, its[m, j], itr)
            assert np.linalg.norm(xs[m][:, j] - xr) <= 1e-10 * max(1e-300, np.linalg.norm(xr))
    del torch


def test_batch_fp32_mixed(P, ctx):
    rng = np.random.default_rng(13)
    mats = [W.rgg(int(n), rng) for n in (4000, 900, 2500)]
    dAs = [P.CSR.from_host(A) for A in mats]
    Fs = P.rw_build_factor_batched(ctx, dAs, 60, [1, 2, 3], 1e-3)
    bs = [rng.standard_normal((A.n, 4)) for A in mats]
    xs = [_dev(np.zeros_like(b)) for b in bs]
    rc, st, its, rel = P.pcg_solve_batched(ctx, dAs, Fs, [_dev(b) for b in bs], xs, 1e-6, 1000,
                                           P.RW_FP32_MIXED)
    assert rc == 0 and np.all(rel < 1e-6)
    for m, A in enumerate(mats):
        xg = xs[m].cpu().numpy()
        true = np.linalg.norm(bs[m] - A.to_scipy() @ xg, axis=0) / np.linalg.norm(bs[m], axis=0)
        assert np.all(true < 1e-6)
        ref = oracle.build_factor(A, 60, m + 1, 1e-3, matrix_index=m)
        mm = int(max(np.diff(A.rowptr).max(), np.diff(ref["rowptr"]).max(),
                     np.bincount(ref["col"], minlength=A.n).max() if ref["nnz"] else 1))
        for j in range(bs[m].shape[1]):
            xr, itr, rr, _ = oracle.pcg(A, ref, bs[m][:, j], 1e-6, 1000, mixed=True)
            # the batched engine's per-system sums run in another order than
            # the single solve's: iteration counts within one, x within the
            # FP32 bound once both stopped at the same count
            assert abs(int(its[m, j]) - itr) <= 1, (m, j, its[m, j], itr)
            if int(its[m, j]) == itr:
                assert np.abs(xg[:, j] - xr).max() <= 8.0 * np.sqrt(mm) * 2.0 ** -24 * np.abs(xr).max()
    for F in Fs:
        F.destroy()


def test_batch_on_a_fresh_context(P, ctx):
    """A batch made on a context other than the factors' (that has run
    nothing yet) builds and solves."""
    A = W.grid2d_5pt(20, 20)
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, 30, 1, 1e-3)
    c2 = P.Context()
    B = P.Batch(c2, [dA], [F])
    b = np.ones((A.n, 1))
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve_batch(c2, B, [_dev(b)], [x], 1e-8, 200)
    assert rc == 0 and rel[0, 0] < 1e-8
    B.destroy()
    c2.close()
    F.destroy()


def test_batch_of_one_uses_the_factor_in_place(P, ctx):
    cfg = W.make_config(2, scale=0.2)
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, 80, 3, 1e-3)
    ref = oracle.build_factor(A, 80, 3, 1e-3)
    B = P.Batch(ctx, [dA], [F])
    assert B.info()["fwd_levels"] == F.desc.fwd_levels
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve_batch(ctx, B, [_dev(b)], [x], 1e-8, 500)
    assert rc == 0 and np.all(rel < 1e-8)
    xg = x.cpu().numpy()
    for j in range(b.shape[1]):
        xr, itr, rr, _ = oracle.pcg(A, ref, b[:, j], 1e-8, 500)
        assert its[0, j] == itr
        assert np.linalg.norm(xg[:, j] - xr) / np.linalg.norm(xr) < 1e-10
    x32 = _dev(np.zeros_like(b))
    rc, st, its32, rel32 = P.pcg_solve_batch(ctx, B, [_dev(b)], [x32], 1e-6, 500, P.RW_FP32_MIXED)
    assert rc == 0 and np.all(rel32 < 1e-6)
    B.destroy()
    F.destroy()


def test_autotune_installs_options_and_caches(P, ctx, tmp_path):
    cfg = W.make_config(2, scale=0.25)
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    c2 = P.Context()
    F = P.rw_build_factor(c2, dA, 60, 2, 1e-3)
    cache = str(tmp_path / "tune.jsonl")
    chosen, ms = P.rw_autotune(c2, dA, F, b.shape[1], P.RW_FP64, cache)
    assert ms[0] > 0 and ms[1] > 0
    assert (chosen["wide_slices"] >= 1 or chosen["wide_slices"] == -1) and chosen["spmv_slices"] >= 1
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and '"key":' in lines[0]
    again, ms2 = P.rw_autotune(c2, dA, F, b.shape[1], P.RW_FP64, cache)
    assert again == chosen and ms2 == (0.0, 0.0)
    assert len(open(cache).read().strip().splitlines()) == 1
    # the tuned context solves like the oracle
    ref = oracle.build_factor(A, 60, 2, 1e-3)
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve(c2, dA, F, _dev(b), x, 1e-8, 500)
    xg = x.cpu().numpy()
    for j in range(b.shape[1]):
        xr, itr, rr, _ = oracle.pcg(A, ref, b[:, j], 1e-8, 500)
        assert its[j] == itr and np.linalg.norm(xg[:, j] - xr) / np.linalg.norm(xr) < 1e-10
    # batch tuning (FP32)
    B = P.Batch(c2, [dA], [F])
    chosen32, ms32 = P.rw_batch_autotune(c2, B, b.shape[1], P.RW_FP32_MIXED, cache)
    assert ms32[0] > 0 and len(open(cache).read().strip().splitlines()) == 2
    B.destroy()
    F.destroy()
    c2.close()


@pytest.mark.parametrize("mode,cw,ws,bwd,tc,bps,tf,tl", [(1, 0, 0, -1, 0, 1, 0, 0), (0, 256, 0, -1, 0, 1, 0, 0),
                                                         (0, 0, -1, -1, 0, 1, 0, 0), (0, 256, -1, -1, 0, 1, 0, 0),
                                                         (1, 0, -1, -1, 0, 1, 0, 0), (1, 0, -1, 0, 0, 1, 0, 0),
                                                         (0, 0, -1, 1, 0, 1, 0, 0), (2, 0, -1, -1, 0, 1, 0, 0),
                                                         (2, 0, 0, -1, 0, 1, 0, 0), (1, 0, -1, 2, 0, 1, 0, 0),
                                                         (2, 0, -1, -1, 8, 1, 0, 0), (0, 0, 8, -1, 4, 1, 0, 0),
                                                         (2, 0, -1, -1, 0, 2, 0, 0), (1, 0, -1, -1, 0, 2, 0, 0),
                                                         (2, 0, -1, -1, 0, 1, 1, 0), (0, 0, 8, -1, 0, 1, 1, 0),
                                                         (2, 0, -1, -1, 0, 1, 0, 8), (2, 0, -1, -1, 0, 1, 1, 8),
                                                         (0, 0, 8, -1, 0, 1, 0, 16), (2, 0, -1, -1, 0, 2, 1, 16)])
def test_precond_modes_match_oracle(P, mode, cw, ws, bwd, tc, bps, tf, tl):
    """The sync-free solve, the cluster runs and the vector rows (wide_slices
    -1: every lane reads all right-hand sides of its entries; level-scheduled,
    sync-free or hybrid, also with the backward solve in another mode, thin
    runs on one block or on a cluster, sync-free parts with one or two blocks
    per SM, thin runs with ready flags, thin runs with 8 or 16 lanes per row)
    give the oracle's z (1e-12)."""
    rng = np.random.default_rng(30 + mode)
    A = W.make_config(2, scale=0.25)["A"]
    c2 = P.Context(options=P.rw_options_default(solve_mode=mode, cluster_width=cw, wide_slices=ws,
                                                solve_mode_bwd=bwd, thin_cluster=tc, solve_blocks_per_sm=bps,
                                                thin_flags=tf, thin_lanes=tl))
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(c2, dA, 100, 7, 1e-3)
    ref = oracle.build_factor(A, 100, 7, 1e-3)
    for nrhs in (1, 3, 4, 16):
        r = rng.standard_normal((A.n, nrhs))
        z = _dev(np.zeros_like(r))
        P.rw_precond_apply(c2, F, _dev(r), z)
        zg = z.cpu().numpy()
        for j in (0, nrhs - 1):
            zr = oracle.precond_apply(ref, r[:, j])
            assert np.linalg.norm(zg[:, j] - zr) / np.linalg.norm(zr) < 1e-12
    b = rng.standard_normal((A.n, 2))
    x = _dev(np.zeros_like(b))
    rc, st, its, rel = P.pcg_solve(c2, dA, F, _dev(b), x, 1e-8, 500)
    xr, itr, rr, _ = oracle.pcg(A, ref, b[:, 0], 1e-8, 500)
    assert its[0] == itr and np.linalg.norm(x.cpu().numpy()[:, 0] - xr) / np.linalg.norm(xr) < 1e-10
    # FP32 mixed solve on the same schedule reaches the tolerance
    x32 = _dev(np.zeros_like(b))
    rc, st, its32, rel32 = P.pcg_solve(c2, dA, F, _dev(b), x32, 1e-6, 500, P.RW_FP32_MIXED)
    assert rc == 0 and np.all(rel32 < 1e-6)
    F.destroy()
    c2.close()


def test_vector_rows_with_long_dependency_lists(P):
    """Rows with more than the 128 prefetched entries (here rows of Y^T, up to
    several hundred) take the batched remainder loop of the vector rows; in
    the backward solve column 0 is computed last, so a padding slot that read
    its x would poison the sum.  Every mode must give the oracle's z."""
    rng = np.random.default_rng(41)
    A = W.make_config(2, scale=0.5)["A"]
    ref = oracle.build_factor(A, 100, 7, 1e-3)
    assert np.bincount(ref["col"], minlength=A.n).max() > 128
    dA = P.CSR.from_host(A)
    r = rng.standard_normal((A.n, 4))
    zr = [oracle.precond_apply(ref, r[:, j]) for j in (0, 3)]
    for mode, bwd, tc, tl in ((0, -1, 0, 0), (1, -1, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (2, -1, 0, 0), (1, 2, 0, 0),
                              (2, -1, 8, 0), (2, -1, 0, 8), (0, -1, 0, 16)):
        c2 = P.Context(options=P.rw_options_default(solve_mode=mode, solve_mode_bwd=bwd, wide_slices=-1,
                                                    thin_cluster=tc, thin_lanes=tl))
        F = P.rw_build_factor(c2, dA, 100, 7, 1e-3)
        z = _dev(np.zeros_like(r))
        P.rw_precond_apply(c2, F, _dev(r), z)
        zg = z.cpu().numpy()
        for zj, j in zip(zr, (0, 3)):
            assert np.linalg.norm(zg[:, j] - zj) / np.linalg.norm(zj) < 1e-12, (mode, bwd, j)
        F.destroy()
        c2.close()


def test_latency_probe(P, ctx):
    """The hand-off and L2-load latencies come back positive and in a plausible
    range; bad arguments are rejected."""
    h, l2 = P.rw_probe_latency(ctx, 2000)
    assert 20.0 < l2 < 5000.0 and 50.0 < h < 20000.0, (h, l2)
    with pytest.raises(P.RwError) as e:
        P.rw_probe_latency(ctx, 0)
    assert e.value.code == -1
