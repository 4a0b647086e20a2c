"""Pins of the learned-budget oracle (CPU only): features against closed forms
on a grid, pilot-walk length moments against the exact absorbing-chain
moments, the BF16 rounding against torch's conversion, the FP64 network
gradient against central differences, the first Adam step against its closed
form, and the budget normaliser against hand-worked apportionments."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import learned as L


def test_bf16_round_matches_reference_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.standard_normal(20000).astype(np.float32) * np.float32(10.0) ** rng.integers(-6, 6, 20000),
        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.5, 0.0, -0.0,
                  3.0e38, 1e-40], dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    got = L.bf16_round(x)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    # ties go to the even neighbour
    assert L.bf16_round(np.float32(1 + 2 ** -8)) == np.float32(1.0)
    assert L.bf16_round(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)


def test_features_closed_form_grid_interior():
    A = W.grid2d_5pt(6, 6)
    F = L.row_features(A)
    k = 2 * 6 + 2                      # interior node whose neighbours are interior too
    ref = [math.log(5), 0.5, 0.5, 0.0, 0.5, math.log(4), 0.25, k / 35, 0.0, math.log(5),
           math.log(6), math.log(4)]
    assert np.allclose(F[k, :12], np.array(ref, dtype=np.float32), rtol=1e-6, atol=1e-7)
    assert not F[:, 12:].any()


def test_features_closed_form_path():
    A = W.tridiag(5, diag=3.0, off=-1.0)
    F = L.row_features(A)
    # row 0: one (upper) neighbour, excess 2 of 3, entropy 0, row sum of row 1 is 1
    assert np.allclose(F[0, :12], np.array([math.log(2), 1, 0, 2 / 3, 1 / 3, 0, 1, 0,
                                            1 / 3, math.log(3), math.log(2), math.log(3)],
                                           dtype=np.float32), rtol=1e-6, atol=1e-7)
    # row 2: neighbours 1 and 3 (row sums 1 each), upper neighbour 3 has one column > 2 (4)
    assert np.allclose(F[2, :12], np.array([math.log(3), 0.5, 0.5, 1 / 3, 1 / 3, math.log(2), 0.5,
                                            0.5, 1 / 3, math.log(3), math.log(2), math.log(3)],
                                           dtype=np.float32), rtol=1e-6, atol=1e-7)


def test_pilot_length_moments_match_absorbing_chain():
    rng = np.random.default_rng(5)
    A = W.random_rmatrix(7, rng)
    walks = 20000
    S = L.pilot_stats(A, walks, seed=3)
    assert set(np.flatnonzero(S["has"])) == set(oracle.walk_rows(A))
    for k in oracle.walk_rows(A):
        m, v = L.exact_length_moments(A, int(k))
        assert abs(S["mean64"][k] - m) < 4 * math.sqrt(v / walks), (k, S["mean64"][k], m)
        assert abs(S["var64"][k] - v) < 0.1 * v + 1e-12, (k, S["var64"][k], v)


def test_pilot_visits_of_a_forced_row():
    # the path of the length pin: every walk from row 1 comes back at least
    # once, and after each return ends (at 0) with p = 1/4, so the returns are
    # geometric on 1, 2, ... and J = 1 + returns has mean 1 + 1/p
    from workloads import assemble
    A = assemble(3, np.array([0, 1]), np.array([1, 2]), np.array([1.0, 3.0]),
                 np.array([1.0, 0.0, 0.0]))
    S = L.pilot_stats(A, 40000, seed=11, quantity=1)
    vis = S["lengths"][40000:80000]
    p = 0.25
    assert vis.min() == 2.0
    assert abs(vis.mean() - (1 + 1 / p)) < 4 * math.sqrt((1 - p) / p ** 2 / 40000)
    # visits and lengths of the same walks: length = 2 J - 1 here
    S0 = L.pilot_stats(A, 40000, seed=11)
    assert np.array_equal(S0["lengths"][40000:80000], 2 * vis - 1)


def test_cost_label_combines_visits_and_lengths():
    rng = np.random.default_rng(5)
    A = W.random_rmatrix(9, rng)
    S1 = L.pilot_stats(A, 500, seed=2, quantity=1)
    S0 = L.pilot_stats(A, 500, seed=2, quantity=0)
    S2 = L.pilot_stats(A, 500, seed=2, quantity=2)
    h = S2["has"] > 0
    # exp(label) = sqrt(relative variance of the visits / mean walk length)
    want = np.sqrt((np.exp(S1["label"][h].astype(np.float64))) / S0["mean"][h].astype(np.float64))
    assert np.allclose(np.exp(S2["label"][h].astype(np.float64)), want, rtol=1e-6)
    assert np.array_equal(S2["mean"], S1["mean"])


def test_pilot_lengths_of_a_forced_row():
    # Path 0-1-2 without excess at nodes 1 and 2: a walk from 1 steps to 2 (its
    # only upper neighbour), comes back to 1 (every time), and from 1 ends at 0
    # or goes to 2 again -> lengths 3, 5, 7 ... with P(len = 1 + 2j) =
    # p (1-p)^(j-1), p = A_10 / (A_10 + A_12).
    from workloads import assemble
    A = assemble(3, np.array([0, 1]), np.array([1, 2]), np.array([1.0, 3.0]),
                 np.array([1.0, 0.0, 0.0]))
    S = L.pilot_stats(A, 40000, seed=11)
    lens = S["lengths"][40000:80000]      # the walks of row 1 (row 0 comes first)
    assert np.all(lens % 2 == 1) and lens.min() == 3
    p = 1.0 / 4.0
    mean = 1 + 2 / p
    var = 4 * (1 - p) / p ** 2
    assert abs(lens.mean() - mean) < 4 * math.sqrt(var / 40000)


def _rand_model(rng, n=300):
    params = rng.standard_normal(L.NUM_PARAMS) * 0.3
    norm = np.concatenate([rng.standard_normal(16) * 0.1, 1 + rng.random(16)]).astype(np.float32)
    feat = rng.standard_normal((n, 16)).astype(np.float32)
    label = rng.standard_normal(n)
    return params, norm, feat, label


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    params, norm, feat, label = _rand_model(rng)
    g, loss = L.gradient(params, norm, feat, label, emulate=False)
    idx = np.concatenate([rng.choice(np.arange(L.OFF_W1, L.OFF_B1).reshape(64, 16)[:, :12].ravel(), 15),
                          rng.integers(L.OFF_B1, L.NUM_PARAMS, 45), [L.NUM_PARAMS - 1]])
    h = 1e-6
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        l1 = L.gradient(p1, norm, feat, label, emulate=False)[1]
        l2 = L.gradient(p2, norm, feat, label, emulate=False)[1]
        fd = (l1 - l2) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
    # padding inputs 12..15 carry no gradient
    assert not g[L.OFF_W1:L.OFF_B1].reshape(64, 16)[:, 12:].any()


def test_emulated_network_is_exact_on_bf16_representable_values():
    rng = np.random.default_rng(2)
    params = np.zeros(L.NUM_PARAMS)
    params[L.OFF_W1:L.OFF_B1] = rng.integers(-2, 3, 64 * 16) * 0.25
    params[L.OFF_W2:L.OFF_B2] = rng.integers(-1, 2, 64 * 64) * 0.125
    params[L.OFF_W3:L.OFF_B3] = rng.integers(-2, 3, 64) * 0.5
    norm = np.concatenate([np.zeros(16), np.ones(16)]).astype(np.float32)
    feat = rng.integers(-3, 4, (50, 16)).astype(np.float32)
    y1, _ = L.forward(params, norm, feat, emulate=True)
    y0, _ = L.forward(params, norm, feat, emulate=False)
    assert np.array_equal(y1, y0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p = rng.standard_normal(100)
    g = rng.standard_normal(100)
    g[:5] = 0.0
    q, m1, m2 = L.adam_step(p, np.zeros(100), np.zeros(100), g, 1, 1e-2)
    assert np.allclose(q - p, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.array_equal(q[:5], p[:5])


def _path(n):
    return W.tridiag(n)


def test_normalize_hand_examples():
    A = _path(4)                               # walk rows 0, 1, 2
    w = np.array([1, 2, 3, 7], np.float32)
    assert L.budget_normalize(A, w, 2.0, 1).tolist() == [1, 2, 3, 0]
    # quota of row 0 clamps at the minimum 5; the others split 25 -> 12.5 each,
    # the tie goes to the lower row
    w = np.array([0.001, 1, 1, 1], np.float32)
    assert L.budget_normalize(A, w, 10.0, 5).tolist() == [5, 13, 12, 0]
    # 8 walks over three equal rows: 3, 3, 2
    w = np.ones(4, np.float32)
    assert L.budget_normalize(A, w, 2.5, 1).tolist() == [3, 3, 2, 0]
    # all weights zero: every row at its quota of mean walks
    assert L.budget_normalize(A, np.zeros(4, np.float32), 7.0, 2).tolist() == [7, 7, 7, 0]


@pytest.mark.parametrize("case", range(6))
def test_normalize_properties(case):
    rng = np.random.default_rng(40 + case)
    A = W.rgg(400, rng) if case % 2 else W.grid2d_5pt(20, 20)
    n = A.n
    w = [rng.lognormal(0, 2, n), rng.random(n), np.ones(n),
         np.where(rng.random(n) < 0.5, 0.0, rng.lognormal(0, 1, n)),
         rng.integers(1, 4, n).astype(float), rng.lognormal(0, 6, n)][case].astype(np.float32)
    mean, mn = [300.0, 37.5, 20.0, 100.0, 300.0, 50.0][case], 20
    b = L.budget_normalize(A, w, mean, mn)
    wr = oracle.walk_rows(A)
    T = int(math.floor(mean * len(wr) + 0.5))
    assert int(b.sum(dtype=np.int64)) == T
    assert b[wr].min() >= mn
    mask = np.ones(n, bool)
    mask[wr] = False
    assert not b[mask].any()
    # rows with a larger weight get no fewer walks (up to the one-walk rounding)
    order = np.argsort(w[wr], kind="stable")
    bw = b[wr][order].astype(np.int64)
    assert np.all(np.diff(bw) >= -1), "budgets not monotone in the weights"
    # unclamped rows get walks in proportion to their weight (within one walk)
    free = (b[wr] > mn + 1)
    if free.sum() > 2:
        c = b[wr][free].sum() / w[wr][free].astype(np.float64).sum()
        assert np.all(np.abs(b[wr][free] - c * w[wr][free]) <= 1.0 + 1e-6 * c * w[wr][free])
