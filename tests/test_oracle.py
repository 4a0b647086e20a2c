"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: published Philox
known-answer vectors, the hand-derived closed form of a 3x3 game, the dense
exact reverse-order LDL^T factor (numpy Cholesky of rev(A)), exact end-point
probabilities of the absorbing Markov chain (dense fundamental matrix), the
paper's worked example of walk reuse, the reachable-set lemma checked by BFS,
and a direct sparse solve for PCG.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_Y(F, n):
    Y = np.zeros((n, n))
    for k in range(n):
        s, e = F["rowptr"][k], F["rowptr"][k + 1]
        Y[k, F["col"][s:e]] = F["val"][s:e]
    return Y


def row_sigmas(A, F, records=True):
    """4-sigma envelopes of Y and D from the walk counts (binomial for the end
    points, delta method on the sample variance of visits for D)."""
    n = A.n
    Ad = A.to_dense()
    dg = np.diag(Ad)
    S = np.array([Ad[k, k + 1:].sum() for k in range(n)])
    a = S / dg
    M = F["M"].astype(float)
    sig_y = np.zeros((n, n))
    sig_d = np.zeros(n)
    start = 0
    rec_ret = F.get("rec_ret")
    for k in range(n):
        if M[k] == 0:
            continue
        m = int(M[k])
        ends = F["rec_end"][start:start + m]
        vis = 1.0 + F["rec_ret"][start:start + m].astype(float)
        start += m
        for i in range(k):
            p = np.count_nonzero(ends == i) / m
            sig_y[k, i] = abs(a[k]) * math.sqrt(p * (1 - p) / m)
        q = vis.mean()
        sq = vis.std(ddof=1) / math.sqrt(m) if m > 1 else 0.0
        den = 1.0 + a[k] * (1.0 - q)
        sig_d[k] = abs(dg[k] * a[k] / den ** 2) * sq
    return sig_y, sig_d, a


# ---------------------------------------------------------------------------
# Philox-4x32-10 (counter-based generator of the walk draws)
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_draw_keying():
    seed = 0x0123456789ABCDEF
    for (mi, tag, k, w, s) in [(0, 0, 5, 7, 0), (3, 1, 9, 2, 6), (1, 2, 0, 0, 13)]:
        out = oracle.philox4x32_10([s // 4, w, k, (mi << 2) | tag],
                                   [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.draw(seed, mi, tag, k, w, s) == out[s % 4]


# ---------------------------------------------------------------------------
# Sampling rule (Sec. 2.1, Eq. map): integer thresholds of the cumulative
# transition probabilities.
# ---------------------------------------------------------------------------

def test_thresholds_bound_and_monotone():
    rng = np.random.default_rng(5)
    A = W.random_rmatrix(30, rng, p_edge=0.4)
    for l in range(A.n):
        t = oracle.row_thresholds(A, l)
        s, e = A.rowptr[l], A.rowptr[l + 1]
        cols, vals = A.col[s:e], A.val[s:e]
        all_ = Fraction(float(vals[cols == l][0]))
        w = [Fraction(-float(v)) for c, v in zip(cols, vals) if c != l]
        assert len(t) == len(w)
        assert np.all(np.diff(t.astype(np.int64)) >= 0)
        c = Fraction(0)
        for m, wm in enumerate(w):
            c += wm
            exact = c / all_ * 2**32
            # cumulative sum and division each round once per term
            slack = 1 + float(exact) * (m + 2) * 2.0**-52
            assert abs(float(t[m]) - float(exact)) <= slack


# ---------------------------------------------------------------------------
# Closed form: A = tridiag(-1, 2, -1), n = 3, worked by hand from the game.
# Row 3 has no upper neighbour and is exact (Sec. 5.2).  Row 2: first step to 3,
# from 3 ground w.p. 1/2 or back to 2; from 2 home 1 w.p. 1/2 or to 3:
# P(end at 1) = 1/3, E[visits to 2] = 5/3, so Y_21 = -1/2 + (-1/2)(1/3) = -2/3
# and D_22 = 2 / (1 + 1/3) = 3/2.  Row 1: E[visits] = 2, D_11 = 4/3.
# ---------------------------------------------------------------------------

def test_closed_form_3x3():
    A = W.tridiag(3)
    F = oracle.build_factor(A, 10**6, seed=11, drop_tol=0.0, records=True)
    sy, sd, _ = row_sigmas(A, F)
    Y = dense_Y(F, 3)
    assert Y[2, 1] == -0.5 and F["D"][2] == 2.0 and F["M"][2] == 0   # exact row, no walks
    assert abs(Y[1, 0] - (-2.0 / 3.0)) <= 4 * sy[1, 0]
    assert abs(F["D"][1] - 1.5) <= 4 * sd[1]
    assert abs(F["D"][0] - 4.0 / 3.0) <= 4 * sd[0]
    assert F["col"].tolist() == [0, 1] and F["rowptr"].tolist() == [0, 0, 1, 2]


# ---------------------------------------------------------------------------
# Walk semantics against the absorbing Markov chain (Sec. 3.1: homes 1..k-1,
# ground absorbs; Sec. 5.2: first step among the upper neighbours).
# ---------------------------------------------------------------------------

def test_endpoint_frequencies_match_absorbing_chain():
    rng = np.random.default_rng(21)
    A = W.random_rmatrix(10, rng, p_edge=0.35)
    M = 200000
    F = oracle.build_factor(A, M, seed=3, drop_tol=0.0, records=True)
    ends, ground, visits = oracle.exact_walk_probabilities(A)
    start = 0
    for k in range(A.n):
        m = int(F["M"][k])
        if m == 0:
            continue
        assert m == M
        e = F["rec_end"][start:start + m]
        v = 1.0 + F["rec_ret"][start:start + m]
        start += m
        for i in range(k):
            p = ends[k, i]
            ph = np.count_nonzero(e == i) / m
            assert abs(ph - p) <= 4 * math.sqrt(max(p * (1 - p), 0.0) / m) + 1e-12
            if p == 0.0:
                assert ph == 0.0
        pg = ground[k]
        assert abs(np.count_nonzero(e == -1) / m - pg) <= 4 * math.sqrt(max(pg * (1 - pg), 0.0) / m) + 1e-12
        assert abs(v.mean() - visits[k]) <= 4 * v.std(ddof=1) / math.sqrt(m)
        assert np.all(e < k)


# ---------------------------------------------------------------------------
# The factor converges to the exact reverse-order LDL^T (Sec. 3, Eqs. y, d;
# estimator of Sec. 5.2): every Y and D entry within 4 sigma.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["tridiag12", "grid4x4", "rand14", "rand16"])
def test_factor_converges_to_exact(case):
    rng = np.random.default_rng(hash(case) % 2**32)
    if case == "tridiag12":
        A = W.tridiag(12)
    elif case == "grid4x4":
        A = W.grid2d_5pt(4, 4)
    elif case == "rand14":
        A = W.random_rmatrix(14, rng, p_edge=0.3)
    else:
        A = W.random_rmatrix(16, rng, p_edge=0.5, p_ground=0.1, excess_hi=0.05)
    walks = 10**6 if case == "grid4x4" else 250000
    F = oracle.build_factor(A, walks, seed=17, drop_tol=0.0, records=True)
    Yx, Dx = oracle.exact_factor(A)
    Y = dense_Y(F, A.n)
    sy, sd, _ = row_sigmas(A, F)
    lower = np.tril(np.ones((A.n, A.n), bool), -1)
    err = np.abs(Y - Yx)[lower]
    tol = (4 * sy + 1e-12)[lower]
    assert np.all(err <= tol), (err - tol).max()
    assert np.all(np.abs(F["D"] - Dx) <= 4 * sd + 1e-12 * Dx)


def test_exact_rows_need_no_walks():
    # rows without an upper neighbour use no walks and are the exact factor
    # (Sec. 5.2, closing remarks on one-step walks)
    rng = np.random.default_rng(8)
    A = W.random_rmatrix(20, rng, p_edge=0.25)
    F = oracle.build_factor(A, 1000, seed=1, drop_tol=0.0)
    Yx, Dx = oracle.exact_factor(A)
    Y = dense_Y(F, A.n)
    Ad = A.to_dense()
    exact_rows = [k for k in range(A.n) if not np.any(Ad[k, k + 1:] != 0)]
    assert exact_rows, "case must contain exact rows"
    for k in exact_rows:
        assert F["M"][k] == 0 and F["hops"][k] == 0
        assert np.allclose(Y[k, :k], Yx[k, :k], rtol=1e-13, atol=1e-15)
        assert abs(F["D"][k] - Dx[k]) <= 1e-13 * Dx[k]


def test_diagonal_matrix_is_exact():
    A = W.assemble(5, np.array([], np.int64), np.array([], np.int64), np.array([]),
                   np.array([1.0, 2.0, 3.0, 4.0, 5.0]))
    F = oracle.build_factor(A, 10, seed=0, drop_tol=0.0)
    assert F["nnz"] == 0 and F["D"].tolist() == [1.0, 2.0, 3.0, 4.0, 5.0]
    b = np.arange(1.0, 6.0)
    x, it, rr, rc = oracle.pcg(A, F, b, 1e-12, 10)
    assert rc == 0 and it == 1 and np.allclose(x, 1.0)


# ---------------------------------------------------------------------------
# Invariants: reachable-set pattern lemma (Sec. 3.2), counters, row sums,
# bounds on D (Sec. 3.3).
# ---------------------------------------------------------------------------

def _reachable_through_higher(A, k):
    """Nodes i < k reachable from k through nodes > k (Definition of the
    reachable set, Sec. 3.2), by breadth-first search."""
    seen = {k}
    frontier = [k]
    out = set()
    while frontier:
        nxt = []
        for u in frontier:
            for p in range(A.rowptr[u], A.rowptr[u + 1]):
                v = int(A.col[p])
                if v in seen:
                    continue
                seen.add(v)
                if v < k:
                    out.add(v)
                elif v > k:
                    nxt.append(v)
        frontier = nxt
    return out


def test_pattern_within_reachable_set_and_exact_pattern():
    A = W.grid2d_5pt(12, 12)
    F = oracle.build_factor(A, 400, seed=5, drop_tol=0.0)
    Yx, _ = oracle.exact_factor(A)
    for k in range(A.n):
        cols = set(F["col"][F["rowptr"][k]:F["rowptr"][k + 1]].tolist())
        assert cols <= _reachable_through_higher(A, k)
        assert all(abs(Yx[k, i]) > 0 for i in cols)


def test_counter_invariants_and_row_sums():
    rng = np.random.default_rng(2)
    A = W.random_rmatrix(40, rng, p_edge=0.15)
    F = oracle.build_factor(A, 3000, seed=9, drop_tol=0.0, records=True)
    Ad = A.to_dense()
    dg = np.diag(Ad)
    excess = Ad.sum(axis=1)
    Y = dense_Y(F, A.n)
    start = 0
    for k in range(A.n):
        m = int(F["M"][k])
        assert 0 < F["D"][k] <= dg[k]
        if m == 0:
            assert F["J"][k] == 0 and F["G"][k] == 0
            continue
        e = F["rec_end"][start:start + m]
        r = F["rec_ret"][start:start + m]
        ln = F["rec_len"][start:start + m]
        start += m
        assert F["G"][k] == np.count_nonzero(e == -1)
        assert F["J"][k] == m + int(r.sum()) and F["J"][k] >= m
        assert F["hops"][k] == int(ln.sum()) and np.all(ln >= 2)
        a = Ad[k, k + 1:].sum() / dg[k]
        # H'_ki recovered from Y (drop_tol = 0) equals the end counts of the records
        H_rec = np.bincount(e[e >= 0], minlength=k)[:k]
        H_y = np.rint((Y[k, :k] - Ad[k, :k] / dg[k]) / a * m)
        assert np.array_equal(H_y, H_rec)
        s = 1.0 + Y[k, :k].sum()
        assert -1e-12 <= s <= 1 + 1e-12
        assert abs(s - (excess[k] / dg[k] + (-a) * F["G"][k] / m)) <= 1e-12


def test_drop_rule_filters_exactly():
    A = W.grid2d_5pt(10, 10)
    F0 = oracle.build_factor(A, 300, seed=4, drop_tol=0.0)
    F1 = oracle.build_factor(A, 300, seed=4, drop_tol=2e-2)
    keep = np.abs(F0["val"]) >= 2e-2
    assert F1["nnz"] == int(keep.sum()) and F1["nnz"] < F0["nnz"]
    assert np.array_equal(F1["col"], F0["col"][keep])
    assert np.array_equal(F1["val"], F0["val"][keep])
    assert np.array_equal(F1["D"], F0["D"])
    rows = np.repeat(np.arange(A.n), np.diff(F0["rowptr"]))
    assert np.array_equal(np.diff(F1["rowptr"]), np.bincount(rows[keep], minlength=A.n))


def test_row_subset_matches_full_build():
    A = W.make_config(2, scale=0.25)["A"]
    full = oracle.build_factor(A, 50, seed=1, drop_tol=1e-3, records=True)
    rows = np.array([3, 100, 2000, A.n - 1])
    sub = oracle.build_factor(A, 50, seed=1, drop_tol=1e-3, rows=rows, records=True)
    for k in rows:
        a, b = full["rowptr"][k], full["rowptr"][k + 1]
        c, d = sub["rowptr"][k], sub["rowptr"][k + 1]
        assert np.array_equal(full["col"][a:b], sub["col"][c:d])
        assert np.array_equal(full["val"][a:b], sub["val"][c:d])
        assert full["D"][k] == sub["D"][k] and full["M"][k] == sub["M"][k]


# ---------------------------------------------------------------------------
# Algorithm 2 (walk reuse, Sec. 5.3) against the paper's worked example.
# ---------------------------------------------------------------------------

def test_reuse_worked_example():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "reuse_figure_sequence.txt"))
             if l.strip() and not l.startswith("#")]
    walk = [int(x) for x in lines[0][1:]]
    extras = [[int(x) for x in l[1:]] for l in lines[1:]]
    dM, dJ, H = oracle.reuse_trace(walk, 8)
    # the paper's three extra walks plus the simulated walk itself
    expect = sorted([(e[0], e[-1]) for e in extras] + [(walk[0], walk[-1])])
    assert sorted(H) == expect
    M_exp = np.zeros(9, np.int64)
    J_exp = np.zeros(9, np.int64)
    for seq in extras + [walk]:
        M_exp[seq[0]] += 1
    # J: visits of each extracted walk (and of the simulated walk) to its start
    for seq in extras + [walk]:
        J_exp[seq[0]] += seq[:-1].count(seq[0])
    assert dM.tolist() == M_exp.tolist()
    assert dJ.tolist() == J_exp.tolist()
    assert dM[2] == 1 and dM[4] == 1 and dM[5] == 2 and dJ[2] == 2 and dJ[4] == 2 and dJ[5] == 2


def test_reuse_estimator_converges_to_exact():
    A = W.grid2d_5pt(4, 4)
    F = oracle.build_factor(A, 200000, seed=23, drop_tol=0.0, reuse=True)
    F0 = oracle.build_factor(A, 200000, seed=23, drop_tol=0.0)
    Yx, Dx = oracle.exact_factor(A)
    Y = dense_Y(F, A.n)
    assert np.all(F["M"] >= F0["M"]) and F["M"].sum() > F0["M"].sum()
    Ad = A.to_dense()
    dg = np.diag(Ad)
    for k in range(A.n):
        m = F["M"][k]
        if m == 0:
            continue
        a = Ad[k, k + 1:].sum() / dg[k]
        for i in range(k):
            p = (Yx[k, i] - Ad[k, i] / dg[k]) / a
            sig = abs(a) * math.sqrt(max(p * (1 - p), 1e-300) / m)
            assert abs(Y[k, i] - Yx[k, i]) <= 4 * sig + 1e-12
    assert np.allclose(F["D"], Dx, rtol=2e-2)


# ---------------------------------------------------------------------------
# PCG (Algorithm 1) against a direct solve; exact preconditioner => 1 iteration.
# ---------------------------------------------------------------------------

def _csr_from_dense_lower(Yd):
    n = Yd.shape[0]
    rp = [0]
    cols, vals = [], []
    for k in range(n):
        nz = np.flatnonzero(np.abs(Yd[k, :k]) > 0)
        cols += nz.tolist()
        vals += Yd[k, nz].tolist()
        rp.append(len(cols))
    return dict(rowptr=np.array(rp, np.int64), col=np.array(cols, np.int32),
                val=np.array(vals))


def test_pcg_exact_preconditioner_one_iteration():
    rng = np.random.default_rng(4)
    A = W.random_rmatrix(25, rng, p_edge=0.2)
    Yx, Dx = oracle.exact_factor(A)
    F = _csr_from_dense_lower(np.tril(Yx, -1))
    F["D"] = Dx
    b = rng.standard_normal(A.n)
    x, it, rr, rc = oracle.pcg(A, F, b, 1e-10, 5)
    assert rc == 0 and it == 1 and rr < 1e-10


def test_pcg_matches_direct_solve_c1():
    import scipy.sparse.linalg as sla
    cfg = W.make_config(1)
    A, b = cfg["A"], cfg["b"][:, 0]
    F = oracle.build_factor(A, cfg["walks"], seed=cfg["walk_seed"], drop_tol=cfg["drop_tol"])
    x, it, rr, rc = oracle.pcg(A, F, b, cfg["tol"], 500)
    xs = sla.spsolve(A.to_scipy().tocsc(), b)
    assert rc == 0 and rr < cfg["tol"]
    ev = np.linalg.eigvalsh(A.to_dense())
    kappa = ev[-1] / ev[0]
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * cfg["tol"]
    # the preconditioner helps: plain CG needs far more iterations
    I = dict(rowptr=np.zeros(A.n + 1, np.int64), col=np.zeros(0, np.int32), val=np.zeros(0),
             D=np.ones(A.n))
    _, it_plain, _, _ = oracle.pcg(A, I, b, cfg["tol"], 2000)
    assert it < 0.6 * it_plain


def test_pcg_mixed_precision_reaches_tolerance():
    import scipy.sparse.linalg as sla
    A = W.grid2d_longrange(40, 40, np.random.default_rng(3))
    b = np.random.default_rng(4).standard_normal(A.n)
    F = oracle.build_factor(A, 200, seed=2, drop_tol=1e-3)
    x, it, rr, rc = oracle.pcg(A, F, b, 1e-6, 1000, mixed=True, refine_every=50)
    x64, it64, rr64, _ = oracle.pcg(A, F, b, 1e-6, 1000)
    xs = sla.spsolve(A.to_scipy().tocsc(), b)
    assert rc == 0 and rr < 1e-6
    assert abs(it - it64) <= max(3, it64 // 5)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-3


def test_pcg_zero_rhs():
    A = W.grid2d_5pt(5, 5)
    F = oracle.build_factor(A, 20, seed=1, drop_tol=0.0)
    x, it, rr, rc = oracle.pcg(A, F, np.zeros(A.n), 1e-8, 10)
    assert rc == 0 and it == 0 and not x.any()


# ---------------------------------------------------------------------------
# Argument and matrix validation, step cap.
# ---------------------------------------------------------------------------

def test_rejects_non_rmatrices_and_bad_args():
    A = W.grid2d_5pt(4, 4)
    bad = W.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.val[1] = 0.5  # positive off-diagonal
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_factor(bad, 10, 0, 0.0)
    assert e.value.code == -2
    bad = W.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.val[0] = 1.0  # not diagonally dominant
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_factor(bad, 10, 0, 0.0)
    assert e.value.code == -2
    bad = W.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.col[[0, 1]] = bad.col[[1, 0]]  # unsorted columns
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_factor(bad, 10, 0, 0.0)
    assert e.value.code == -2
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_factor(A, 0, 0, 0.0)
    assert e.value.code == -1


def test_step_cap():
    A = W.make_config(2, scale=0.1)["A"]
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_factor(A, 5, 0, 0.0, max_steps=3)
    assert e.value.code == -3
    F = oracle.build_factor(A, 5, 0, 0.0, max_steps=1 << 20, records=True)
    assert F["rec_len"].max() < (1 << 20)


# ---------------------------------------------------------------------------
# Input generators: sizes of the benchmark families.
# ---------------------------------------------------------------------------

def test_workload_sizes():
    c1 = W.make_config(1)["A"]
    assert (c1.n, c1.nnz) == (1024, 4992) and oracle.validate(c1) == 0
    c2 = W.make_config(2)["A"]
    assert (c2.n, c2.nnz) == (262144, 1810432) and oracle.validate(c2) == 0
    # Table 1 of the paper: the 50^3 SPARSKIT Laplacian has N = 1.25e5, E = 8.6e5
    t1 = W.grid3d(50, 50, 50, 7, np.random.default_rng(0), excess_frac=0.0, permute=False)
    assert t1.n == 125000 and round(t1.nnz / 1e4) == 86


def test_table1_grids():
    # Table 1: N and E (matrix entries, diagonal included) of m1..m6, printed
    # to two digits; every row of the Dirichlet Laplacian has diagonal 6 and
    # the exact factor of the smallest grid gives a PCG solve in one step
    N = [1.3e5, 2.2e5, 3.4e5, 5.1e5, 7.3e5, 1.0e6]
    E = [8.6e5, 1.5e6, 2.4e6, 3.5e6, 5.1e6, 6.9e6]
    for j, m in enumerate((50, 60, 70, 80, 90, 100)):
        n = m ** 3
        e = 7 * n - 6 * m * m          # 6 neighbours per node minus the missing boundary ones
        for got, printed in ((n, N[j]), (e, E[j])):
            half_unit = 0.5 * 10 ** (math.floor(math.log10(printed)) - 1)
            assert abs(got - printed) <= half_unit * (1 + 1e-12), (m, got, printed)
    A = W.laplace3d_dirichlet(6)
    assert A.n == 216 and A.nnz == 7 * 216 - 6 * 36 and oracle.validate(A) == 0
    d = A.to_dense()
    assert np.all(np.diag(d) == 6.0) and set(np.unique(d[d != np.diag(np.diag(d))])) <= {-1.0, 0.0}
    assert np.allclose(d, d.T) and np.all(np.linalg.eigvalsh(d) > 0)
    cfg = W.make_config(6, scale=0.1)
    assert [a.n for a in cfg["A"]] == [e ** 3 for e in cfg["edges"]] and cfg["edges"] == (5, 6, 7, 8, 9, 10)


def test_multithreaded_build_equals_single_thread():
    """Rows are independent (Sec. 4): the oracle's build on several host
    threads gives the single-thread factor bit for bit, for every thread
    count, for uniform and per-row budgets and for a subset of rows."""
    rng = np.random.default_rng(11)
    cases = [(W.make_config(1)["A"], 200), (W.make_config(2, scale=0.2)["A"], 60),
             (W.random_rmatrix(70, rng), 40)]
    for A, walks in cases:
        budget = rng.integers(1, walks, A.n).astype(np.uint32)
        for wk in (walks, budget):
            ref = oracle.build_factor(A, wk, 9, 1e-3)
            for threads in (2, 3, 8):
                got = oracle.build_factor(A, wk, 9, 1e-3, threads=threads)
                for key in ("rowptr", "col", "val", "D", "M", "J", "G", "hops"):
                    assert np.array_equal(ref[key], got[key]), (A.n, threads, key)
    A = W.make_config(1)["A"]
    rows = np.array([0, 5, 31, 500, 1000, 1023])
    ref = oracle.build_factor(A, 100, 3, 1e-3, rows=rows)
    got = oracle.build_factor(A, 100, 3, 1e-3, rows=rows, threads=4)
    for key in ("rowptr", "col", "val", "D", "M", "J", "G", "hops"):
        assert np.array_equal(ref[key], got[key]), key
