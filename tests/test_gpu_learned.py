"""GPU learned-budget path vs the CPU oracle (oracle/learned.py): row
features, pilot-walk statistics, the network's forward pass and gradient
(BF16 tensor-core products against the FP64 oracle that rounds at the same
points), one Adam step, the integer budget normaliser (bit-exact), and the
end-to-end predicted budgets.

Tolerances.  Features and pilot statistics are computed in FP64 on both sides
and stored as FP32: 2 FP32 ulps (rtol 2.5e-7 ... 1e-6).  The network
accumulates in FP32 on the tensor cores where the oracle sums in FP64; a
layer-1 activation whose FP32 and FP64 values round to different BF16
neighbours (probability about 12 * 2^-24 / 2^-9 per unit) moves the output by
at most 2^-8 of that unit's contribution, so the bulk of the rows agree to
1e-5 of the output scale and every row to 2e-2 of it."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import learned as L

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


def _zeros(shape, dtype="float32"):
    import torch
    return torch.zeros(shape, dtype=getattr(torch, dtype), device="cuda")


def _matrices():
    rng = np.random.default_rng(21)
    return [W.grid2d_5pt(17, 13), W.rgg(700, rng), W.grid3d(7, 6, 5, 27, rng, excess_frac=1e-4),
            W.random_rmatrix(40, rng), W.tridiag(3)]


def _features(P, ctx, A):
    f = _zeros((A.n, 16))
    P.rw_row_features(ctx, P.CSR.from_host(A), f)
    return f


def test_features_match_oracle(P, ctx):
    for A in _matrices():
        got = _features(P, ctx, A).cpu().numpy()
        ref = L.row_features(A)
        assert np.allclose(got, ref, rtol=1e-6, atol=1e-6), np.abs(got - ref).max()
        assert not got[:, 12:].any()


def test_pilot_stats_match_oracle(P, ctx):
    for A, walks, seed in [(W.grid3d(6, 6, 6, 27, np.random.default_rng(3), excess_frac=1e-4), 64, 5),
                           (W.rgg(500, np.random.default_rng(4)), 17, 9), (W.grid2d_5pt(9, 9), 2, 1)]:
        dA = P.CSR.from_host(A)
        out = [_zeros(A.n) for _ in range(4)]
        P.rw_pilot_stats(ctx, dA, walks, seed, *out)
        mean, sd, label, has = [t.cpu().numpy() for t in out]
        ref = L.pilot_stats(A, walks, seed)
        assert np.array_equal(has, ref["has"])
        # the walks are bit-identical, so the mean (exact integer sum / walks) is too
        assert np.array_equal(mean, ref["mean"])
        assert np.allclose(sd, ref["sd"], rtol=1e-6, atol=0)
        assert np.allclose(label, ref["label"], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("quantity", [1, 2])
def test_pilot_returns_match_oracle(P, ctx, quantity):
    A = W.grid3d(6, 6, 6, 27, np.random.default_rng(3), excess_frac=1e-4)
    dA = P.CSR.from_host(A)
    out = [_zeros(A.n) for _ in range(4)]
    P.rw_pilot_stats(ctx, dA, 64, 5, *out, quantity=quantity)
    mean, sd, label, has = [t.cpu().numpy() for t in out]
    ref = L.pilot_stats(A, 64, 5, quantity=quantity)
    assert np.array_equal(has, ref["has"]) and np.array_equal(mean, ref["mean"])
    assert np.all(mean[has > 0] >= 1.0)
    assert np.allclose(sd, ref["sd"], rtol=1e-6, atol=0)
    assert np.allclose(label, ref["label"], rtol=1e-6, atol=1e-6)


def _random_model(rng, feat):
    params = (rng.standard_normal(L.NUM_PARAMS) * 0.25).astype(np.float32)
    params[L.OFF_W1:L.OFF_B1] *= 1.5
    params[L.OFF_B1:L.OFF_W2] = rng.standard_normal(64) * 0.1
    mu = feat[:, :12].mean(axis=0)
    sd = feat[:, :12].std(axis=0)
    norm = np.zeros(32, np.float32)
    norm[:12] = mu
    norm[16:28] = 1.0 / np.where(sd > 1e-6, sd, 1.0)
    return params, norm


def _feature_rows(P, ctx):
    rng = np.random.default_rng(8)
    A = W.grid3d(12, 12, 12, 27, rng, excess_frac=1e-4)
    f = _features(P, ctx, A)
    return A, f, L.row_features(A)


def test_mlp_predict_matches_oracle(P, ctx):
    A, f, fref = _feature_rows(P, ctx)
    rng = np.random.default_rng(0)
    params, norm = _random_model(rng, fref)
    M = P.Mlp(ctx, seed=1)
    M.set_params(params, norm)
    got_p, got_n = M.params()
    assert np.array_equal(got_p, params) and np.array_equal(got_n, norm)
    # ragged tail: 16-row warp tiles over 1000 + 7 rows
    for rows in (A.n, 1007, 5):
        y = _zeros(rows)
        P.rw_mlp_predict(ctx, M, f[:rows].contiguous(), y)
        yg = y.cpu().numpy().astype(np.float64)
        yr, _ = L.forward(params, norm, fref[:rows])
        scale = max(1e-3, float(np.sqrt(np.mean(yr * yr))))
        err = np.abs(yg - yr) / scale
        assert np.quantile(err, 0.99) < 1e-5 and err.max() < 2e-2, (np.quantile(err, 0.99), err.max())
    M.destroy()


def test_mlp_gradient_matches_oracle(P, ctx):
    import torch
    A, f, fref = _feature_rows(P, ctx)
    rng = np.random.default_rng(1)
    params, norm = _random_model(rng, fref)
    label = rng.standard_normal(A.n).astype(np.float32)
    M = P.Mlp(ctx, seed=2)
    M.set_params(params, norm)
    for rows in (np.arange(A.n), rng.choice(A.n, 777, replace=False)):
        g, loss = P.rw_mlp_gradient(ctx, M, f, _dev(label), _dev(rows.astype(np.int32)))
        gr, lr_ = L.gradient(params, norm, fref[rows], label[rows])
        assert abs(loss - lr_) <= 1e-4 * lr_
        blocks = [(L.OFF_W1, L.OFF_B1), (L.OFF_B1, L.OFF_W2), (L.OFF_W2, L.OFF_B2),
                  (L.OFF_B2, L.OFF_W3), (L.OFF_W3, L.OFF_B3), (L.OFF_B3, L.NUM_PARAMS)]
        for a, b in blocks:
            rel = np.linalg.norm(g[a:b] - gr[a:b]) / max(1e-30, np.linalg.norm(gr[a:b]))
            assert rel < 2e-3, (a, b, rel)
    del torch
    M.destroy()


def test_adam_step_matches_oracle(P, ctx):
    A, f, fref = _feature_rows(P, ctx)
    rng = np.random.default_rng(2)
    params, norm = _random_model(rng, fref)
    label = rng.standard_normal(A.n).astype(np.float32)
    M = P.Mlp(ctx, seed=3)
    M.set_params(params, norm)
    lr = 1e-3
    # one epoch of one full batch = one Adam step on the whole set
    P.rw_mlp_train(ctx, M, f, _dev(label), _dev(np.ones(A.n, np.float32)), epochs=1, batch=A.n,
                   lr=lr, seed=0, set_norm=False)
    after, n2 = M.params()
    assert np.array_equal(n2, norm)
    gr, _ = L.gradient(params, norm, fref, label)
    ref, _, _ = L.adam_step(params.astype(np.float64), 0.0, 0.0, gr, 1, lr)
    firm = np.abs(gr) > 1e-2 * np.sqrt(np.mean(gr * gr))
    assert np.all(np.abs(after - ref)[firm] < 1e-3 * lr + 1e-6)
    assert np.all(np.abs(after - params) <= lr * (1 + 1e-4) + 1e-6)
    M.destroy()


def _norm_cases():
    rng = np.random.default_rng(77)
    g = W.grid3d(40, 40, 40, 7, rng, excess_frac=1e-3)
    r = W.rgg(3000, rng)
    t = W.grid2d_5pt(50, 30)
    n1, n2, n3 = g.n, r.n, t.n
    return [
        (g, rng.lognormal(0, 2, n1), 300.0, 20),
        (g, np.ones(n1), 300.0, 20),
        (g, np.where(rng.random(n1) < 0.3, 0.0, rng.lognormal(0, 1, n1)), 123.4, 20),
        (r, rng.integers(1, 5, n2).astype(float), 77.7, 20),
        (r, rng.lognormal(0, 8, n2), 300.0, 50),
        (t, rng.random(n3), 20.0, 20),
        (t, np.zeros(n3), 31.0, 3),
        (t, rng.lognormal(0, 1, n3) * 1e-30, 500.0, 1),
    ]


def test_normalize_bit_exact(P, ctx):
    for A, w, mean, mn in _norm_cases():
        w = w.astype(np.float32)
        b = _zeros(A.n, "int32")
        P.rw_budget_normalize(ctx, P.CSR.from_host(A), _dev(w), mean, mn, b)
        got = b.cpu().numpy().view(np.uint32)
        ref = L.budget_normalize(A, w, mean, mn)
        assert np.array_equal(got, ref), (mean, mn, np.flatnonzero(got != ref)[:10])


def test_normalize_rejects_bad_input(P, ctx):
    A = W.grid2d_5pt(8, 8)
    dA = P.CSR.from_host(A)
    b = _zeros(A.n, "int32")
    w = np.ones(A.n, np.float32)
    for bad in (np.nan, -1.0, np.inf):
        w2 = w.copy()
        w2[5] = bad
        with pytest.raises(P.RwError) as e:
            P.rw_budget_normalize(ctx, dA, _dev(w2), 100.0, 20, b)
        assert e.value.code == -1
    # a bad weight on a row without walks (the last row) is ignored
    w2 = w.copy()
    w2[-1] = np.nan
    P.rw_budget_normalize(ctx, dA, _dev(w2), 100.0, 20, b)
    for mean, mn in ((10.0, 20), (100.0, 0), (2.0 ** 32, 20)):
        with pytest.raises(P.RwError):
            P.rw_budget_normalize(ctx, dA, _dev(w), mean, mn, b)


def test_budget_predict_end_to_end(P, ctx):
    rng = np.random.default_rng(5)
    A = W.grid3d(14, 14, 14, 27, rng, excess_frac=1e-4)
    fref = L.row_features(A)
    params, norm = _random_model(np.random.default_rng(6), fref)
    params *= 0.5
    M = P.Mlp(ctx, seed=4)
    M.set_params(params, norm)
    b = _zeros(A.n, "int32")
    P.rw_budget_predict(ctx, P.CSR.from_host(A), M, 300.0, 20, b)
    got = b.cpu().numpy().view(np.uint32).astype(np.int64)
    y, _ = L.forward(params, norm, fref)
    w = np.exp(np.clip(y.astype(np.float32), -60, 60)).astype(np.float32)
    ref = L.budget_normalize(A, w, 300.0, 20).astype(np.int64)
    assert got.sum() == ref.sum()
    assert got[oracle.walk_rows(A)].min() >= 20
    d = np.abs(got - ref)
    assert np.mean(d == 0) > 0.95 and np.all(d <= np.maximum(2, 2e-2 * ref)), (np.mean(d == 0), d.max())
    # and the budgets drive a factor build
    F = P.rw_build_factor_budget(ctx, P.CSR.from_host(A), b, 7, 1e-3)
    assert F.desc.total_walks == ref.sum()
    F.destroy()
    M.destroy()
