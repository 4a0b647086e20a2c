"""GPU factor construction vs the CPU oracle (bit-exact).

Walk records, counters (M', J', G'), hop totals, Y (CSR pattern and FP64
values) and D must be identical to the oracle's on the same seeded inputs:
the walk game, keying, sampling rule and the FP64 operation order of
Eqs. newy/newz are fixed on both sides.
"""
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
    c = P.Context(options=P.rw_options_default(keep_records=1))
    yield c
    c.close()


def gpu_factor(P, ctx, A, walks, seed, drop, budget=None):
    import torch
    dA = P.CSR.from_host(A)
    if budget is None:
        F = P.rw_build_factor(ctx, dA, walks, seed, drop)
    else:
        F = P.rw_build_factor_budget(ctx, dA, torch.as_tensor(budget.astype(np.int32)).cuda(),
                                     seed, drop)
    t = {k: v.cpu().numpy() for k, v in F.tensors().items()}
    t["total_hops"] = int(F.desc.total_hops)
    t["fwd_levels"], t["bwd_levels"] = F.desc.fwd_levels, F.desc.bwd_levels
    t["phase_ms"] = list(F.desc.phase_ms)
    F.destroy()
    return t


def assert_factor_equal(t, ref, records=True):
    n = len(ref["D"])
    assert np.array_equal(t["y_row_ptr"], ref["rowptr"])
    assert np.array_equal(t["y_col"], ref["col"])
    assert np.array_equal(t["y_val"].view(np.int64), ref["val"].view(np.int64))
    assert np.array_equal(t["d"].view(np.int64), ref["D"].view(np.int64))
    assert np.array_equal(t["walks"].astype(np.uint64), ref["M"])
    assert np.array_equal(t["visits"].astype(np.uint64), ref["J"])
    assert np.array_equal(t["ground"].astype(np.uint64), ref["G"])
    assert t["total_hops"] == int(ref["hops"].sum())
    if records and "rec_end" in ref:
        rec = t["records"].reshape(-1, 2)
        assert np.array_equal(rec[:, 0], ref["rec_end"])
        assert np.array_equal(rec[:, 1].astype(np.uint32), ref["rec_ret"])
        assert np.array_equal(t["walk_rows"], ref["walk_rows"])


def levels_of(n, rp, col):
    lev = np.zeros(n, np.int64)
    for k in range(n):
        s, e = rp[k], rp[k + 1]
        if e > s:
            lev[k] = 1 + lev[col[s:e]].max()
    return lev


def test_c1_bit_exact(P, ctx):
    cfg = W.make_config(1)
    A = cfg["A"]
    t = gpu_factor(P, ctx, A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    ref = oracle.build_factor(A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"], records=True)
    assert_factor_equal(t, ref)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_rmatrices_bit_exact(P, ctx, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 400))
    A = W.random_rmatrix(n, rng, p_edge=float(rng.uniform(0.005, 0.2)),
                         excess_hi=float(rng.uniform(0.001, 0.5)))
    walks = int(rng.integers(1, 80))
    drop = [0.0, 1e-3, 2e-2, 0.2][seed]
    wseed = int(rng.integers(0, 2**63))
    t = gpu_factor(P, ctx, A, walks, wseed, drop)
    ref = oracle.build_factor(A, walks, wseed, drop, records=True)
    assert_factor_equal(t, ref)


def test_per_row_budgets_bit_exact(P, ctx):
    rng = np.random.default_rng(7)
    A = W.grid3d(9, 9, 9, 27, rng, excess_frac=1e-3)
    budget = rng.integers(1, 120, size=A.n).astype(np.uint32)
    t = gpu_factor(P, ctx, A, 0, 99, 1e-3, budget=budget)
    ref = oracle.build_factor(A, budget, 99, 1e-3, records=True)
    assert_factor_equal(t, ref)


def test_large_row_budgets_use_block_merge(P, ctx):
    # rows with more than 768 possible end points (min(walks + lower
    # neighbours, k)) go to the block-level merge; both paths must agree with
    # the oracle.  Rows below 768 stay on the warp tables whatever their budget.
    rng = np.random.default_rng(8)
    A = W.grid2d_5pt(40, 40)
    budget = np.where(rng.random(A.n) < 0.3, 3000, 40).astype(np.uint32)
    t = gpu_factor(P, ctx, A, 0, 5, 0.0, budget=budget)
    ref = oracle.build_factor(A, budget, 5, 0.0, records=True)
    assert_factor_equal(t, ref)


def test_huge_row_budgets_use_global_tables(P, ctx):
    # rows with more than 12288 possible end points merge in global-memory
    # tables; a low row with a huge budget stays on the block tables (k bounds it)
    A = W.grid2d_5pt(120, 115)
    budget = np.full(A.n, 2, np.uint32)
    budget[[A.n - 200, A.n - 150, A.n - 121, A.n - 2]] = [14000, 30000, 13000, 20000]
    budget[[5, 900]] = [40000, 20000]
    t = gpu_factor(P, ctx, A, 0, 12, 0.0, budget=budget)
    ref = oracle.build_factor(A, budget, 12, 0.0, records=True)
    assert_factor_equal(t, ref)


@pytest.mark.parametrize("family", ["grid7", "grid27", "rgg", "longrange"])
def test_families_bit_exact(P, ctx, family):
    rng = np.random.default_rng(11)
    if family == "grid7":
        A = W.make_config(2, scale=0.25)["A"]      # 16^3, weak grounding
        walks, drop = 200, 1e-3
    elif family == "grid27":
        A = W.make_config(5, scale=0.125)["A"]     # 16^3, degree 26: multi-sector rows
        walks, drop = 60, 1e-3
    elif family == "rgg":
        A = W.rgg(3000, rng)
        walks, drop = 100, 1e-3
    else:
        A = W.make_config(3, scale=0.06)["A"]      # 60^2 + long-range edges
        walks, drop = 100, 1e-3
    t = gpu_factor(P, ctx, A, walks, 12345, drop)
    ref = oracle.build_factor(A, walks, 12345, drop, records=True)
    assert_factor_equal(t, ref)


def test_full_size_c2_sampled_rows(P, ctx):
    """Workload 2 at full size (n = 262144, 500 walks/row) on the GPU; the
    oracle recomputes a seeded sample of rows (rows are independent)."""
    cfg = W.make_config(2)
    A = cfg["A"]
    t = gpu_factor(P, ctx, A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    rng = np.random.default_rng(2024)
    rows = np.unique(np.concatenate([rng.choice(A.n, 120, replace=False), [0, 1, A.n - 1]]))
    ref = oracle.build_factor(A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"], rows=rows)
    for k in rows:
        a, b = t["y_row_ptr"][k], t["y_row_ptr"][k + 1]
        c, d = ref["rowptr"][k], ref["rowptr"][k + 1]
        assert np.array_equal(t["y_col"][a:b], ref["col"][c:d]), k
        assert np.array_equal(t["y_val"][a:b].view(np.int64), ref["val"][c:d].view(np.int64)), k
        assert t["d"][k].view(np.int64) == ref["D"][k].view(np.int64), k
        assert t["walks"][k] == ref["M"][k] and t["visits"][k] == ref["J"][k]
        assert t["ground"][k] == ref["G"][k]
    # properties that hold at any size
    n = A.n
    assert np.all(t["d"] > 0) and np.all(np.diff(t["y_row_ptr"]) >= 0)
    assert np.all(np.abs(t["y_val"]) >= cfg["drop_tol"])
    wr = oracle.walk_rows(A)
    assert np.all(t["walks"][wr] == cfg["walks"])
    assert t["total_hops"] > 0


@pytest.mark.parametrize("workload,nsample", [(3, 60), (5, 40)])
def test_full_size_sampled_rows(P, ctx, workload, nsample):
    """Workloads 3 (n = 10^6, 200 walks/row) and 5 (128^3 27-point grid,
    uniform 300 walks/row: the plain arm's build) at full size on the GPU;
    the oracle recomputes a seeded sample of rows bit for bit."""
    cfg = W.make_config(workload)
    A = cfg["A"]
    t = gpu_factor(P, ctx, A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"])
    rng = np.random.default_rng(7 + workload)
    rows = np.unique(np.concatenate([rng.choice(A.n, nsample, replace=False), [0, A.n - 1]]))
    ref = oracle.build_factor(A, cfg["walks"], cfg["walk_seed"], cfg["drop_tol"], rows=rows)
    for k in rows:
        a, b = t["y_row_ptr"][k], t["y_row_ptr"][k + 1]
        c, d = ref["rowptr"][k], ref["rowptr"][k + 1]
        assert np.array_equal(t["y_col"][a:b], ref["col"][c:d]), k
        assert np.array_equal(t["y_val"][a:b].view(np.int64), ref["val"][c:d].view(np.int64)), k
        assert t["d"][k].view(np.int64) == ref["D"][k].view(np.int64), k
        assert t["walks"][k] == ref["M"][k] and t["visits"][k] == ref["J"][k] and t["ground"][k] == ref["G"][k]
    assert np.all(t["d"] > 0) and np.all(np.abs(t["y_val"]) >= cfg["drop_tol"])
    assert np.all(t["walks"][oracle.walk_rows(A)] == cfg["walks"])


def test_transpose_and_levels(P, ctx):
    import scipy.sparse as sp
    A = W.make_config(2, scale=0.25)["A"]
    t = gpu_factor(P, ctx, A, 100, 3, 1e-3)
    n = A.n
    Y = sp.csr_matrix((t["y_val"], t["y_col"], t["y_row_ptr"]), shape=(n, n))
    Yt = Y.T.tocsr()
    Yt.sort_indices()
    assert np.array_equal(t["yt_row_ptr"], Yt.indptr)
    assert np.array_equal(t["yt_col"], Yt.indices)
    assert np.array_equal(t["yt_val"], Yt.data)
    assert t["fwd_levels"] == levels_of(n, t["y_row_ptr"], t["y_col"]).max() + 1
    rev = levels_of(n, *(lambda M: (M.indptr, M.indices))(
        sp.csr_matrix((Yt.data, (n - 1 - np.repeat(np.arange(n), np.diff(Yt.indptr)),
                                 n - 1 - Yt.indices)), shape=(n, n))))
    assert t["bwd_levels"] == rev.max() + 1
    assert np.allclose(t["y_val32"], t["y_val"].astype(np.float32), rtol=0, atol=0)
    # every row's level, not only the depth: the rows of level l are fwd_order[ptr[l] .. ptr[l+1])
    check_level_order(t["fwd_order"], t["fwd_level_ptr"], levels_of(n, t["y_row_ptr"], t["y_col"]))
    check_level_order(t["bwd_order"], t["bwd_level_ptr"], rev[::-1])


def check_level_order(order, ptr, lev):
    """order lists every row once, grouped by level as ptr says, and each row's
    group is its longest-path level lev."""
    n = lev.size
    assert ptr.size == lev.max() + 2 and ptr[0] == 0 and ptr[-1] == n
    assert np.all(np.diff(ptr) > 0)
    assert np.array_equal(np.sort(order), np.arange(n))
    got = np.repeat(np.arange(ptr.size - 1), np.diff(ptr))
    assert np.array_equal(lev[order], got)


def test_levels_wide_and_deep(P, ctx):
    """Level order of the 27-point grid (wide levels, several frontier
    rounds with thousands of rows) and of a 2D grid with long-range edges."""
    import scipy.sparse as sp
    for A in (W.make_config(5, scale=0.125)["A"], W.make_config(3, scale=0.05)["A"]):
        t = gpu_factor(P, ctx, A, 40, 7, 1e-3)
        n = A.n
        lf = levels_of(n, t["y_row_ptr"], t["y_col"])
        check_level_order(t["fwd_order"], t["fwd_level_ptr"], lf)
        Y = sp.csr_matrix((t["y_val"], t["y_col"], t["y_row_ptr"]), shape=(n, n))
        # backward DAG in reversed numbering: row n-1-c depends on n-1-k for every Y_kc
        R = sp.csr_matrix((np.ones(Y.nnz), (n - 1 - Y.indices, n - 1 - np.repeat(np.arange(n), np.diff(Y.indptr)))),
                          shape=(n, n))
        R.sort_indices()
        lb = levels_of(n, R.indptr, R.indices)[::-1]
        check_level_order(t["bwd_order"], t["bwd_level_ptr"], lb)


def test_edge_cases(P, ctx):
    # one node; a diagonal matrix (no walks at all); rows without upper neighbours
    one = W.assemble(1, np.array([], np.int64), np.array([], np.int64), np.array([]), [2.0])
    t = gpu_factor(P, ctx, one, 10, 0, 0.0)
    assert t["d"].tolist() == [2.0] and t["y_col"].size == 0
    diag = W.assemble(5, np.array([], np.int64), np.array([], np.int64), np.array([]),
                      np.arange(1.0, 6.0))
    t = gpu_factor(P, ctx, diag, 7, 0, 0.0)
    assert t["d"].tolist() == [1, 2, 3, 4, 5] and t["total_hops"] == 0
    A = W.tridiag(2)
    t = gpu_factor(P, ctx, A, 1, 0, 0.0)
    ref = oracle.build_factor(A, 1, 0, 0.0, records=True)
    assert_factor_equal(t, ref)


def test_rejects_bad_inputs(P, ctx):
    A = W.grid2d_5pt(4, 4)
    bad = W.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.val[1] = 0.5
    with pytest.raises(P.RwError) as e:
        gpu_factor(P, ctx, bad, 5, 0, 0.0)
    assert e.value.code == -2
    bad = W.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.col[[0, 1]] = bad.col[[1, 0]]
    with pytest.raises(P.RwError) as e:
        gpu_factor(P, ctx, bad, 5, 0, 0.0)
    assert e.value.code == -2
    with pytest.raises(P.RwError) as e:
        gpu_factor(P, ctx, A, 0, 0, 0.0)
    assert e.value.code == -1
    with pytest.raises(P.RwError) as e:
        gpu_factor(P, ctx, A, 0, 0, 0.0, budget=np.zeros(A.n, np.uint32))
    assert e.value.code == -1
    with pytest.raises(P.RwError) as e:
        gpu_factor(P, ctx, A, 5, 0, -1.0)
    assert e.value.code == -1


def test_step_cap_reported(P):
    # walks longer than max_steps are stopped and reported; nothing hangs
    c = P.Context(options=P.rw_options_default(max_steps=3))
    A = W.make_config(2, scale=0.1)["A"]
    with pytest.raises(P.RwError) as e:
        gpu_factor(P, c, A, 5, 0, 0.0)
    assert e.value.code == -3
    c.close()


def test_torch_allocator_context(P):
    c = P.Context(torch_allocator=True)
    A = W.make_config(1)["A"]
    t = gpu_factor(P, c, A, 20, 4, 1e-3)
    ref = oracle.build_factor(A, 20, 4, 1e-3)
    assert np.array_equal(t["y_val"], ref["val"]) and np.array_equal(t["d"], ref["D"])
    c.close()


def test_batched_build_matches_per_matrix_oracle(P, ctx):
    """One walk launch over several matrices of uneven size and family; matrix
    m draws with matrix index m and must equal the oracle with that index."""
    import torch
    rng = np.random.default_rng(31)
    mats = [W.rgg(int(n), rng) for n in (300, 1700, 40, 5000)]
    mats.append(W.make_config(2, scale=0.2)["A"])
    mats.append(W.tridiag(2))
    seeds = [int(x) for x in rng.integers(0, 2**62, size=len(mats))]
    dAs = [P.CSR.from_host(A) for A in mats]
    budgets = [None] * len(mats)
    budgets[1] = torch.as_tensor(rng.integers(1, 60, size=mats[1].n).astype(np.int32)).cuda()
    Fs = P.rw_build_factor_batched(ctx, dAs, 37, seeds, 1e-3, budgets=budgets)
    for m, (A, F) in enumerate(zip(mats, Fs)):
        t = {k: v.cpu().numpy() for k, v in F.tensors().items()}
        t["total_hops"] = int(F.desc.total_hops)
        walks = np.asarray(budgets[m].cpu().numpy(), np.uint32) if budgets[m] is not None else 37
        ref = oracle.build_factor(A, walks, seeds[m], 1e-3, matrix_index=m)
        assert_factor_equal(t, ref, records=False)
        F.destroy()


# ---------------------------------------------------------------------------
# Walk reuse (Algorithm 2 of Sec. 5.3): the simulated walks are the plain
# build's; every legal sub-walk they contain counts for its start row.  Y, D
# and the counters must equal the oracle's reuse build bit for bit.

@pytest.fixture(scope="module")
def ctx_reuse(P):
    c = P.Context(options=P.rw_options_default(keep_records=1, reuse=1))
    yield c
    c.close()


def _reuse_cases():
    rng = np.random.default_rng(301)
    yield "grid2d", W.grid2d_5pt(23, 19), 30, 1e-3
    yield "grid7", W.make_config(2, scale=0.25)["A"], 40, 1e-3
    yield "grid27", W.make_config(5, scale=0.125)["A"], 12, 1e-3
    yield "rgg", W.rgg(3000, rng), 25, 0.0
    yield "longrange", W.make_config(3, scale=0.04)["A"], 20, 2e-2
    for j in range(3):
        n = int(rng.integers(2, 300))
        A = W.random_rmatrix(n, rng, p_edge=float(rng.uniform(0.01, 0.2)),
                             excess_hi=float(rng.uniform(0.001, 0.5)))
        yield f"random{j}", A, int(rng.integers(1, 50)), [0.0, 1e-3, 0.1][j]


def _degree_classes_matrix(seed):
    """Random R-matrix whose nodes span every transition-table layout: at most
    two groups of four slots (degree <= 7), three to eight groups (8..31) and
    more than eight (32 and up), so every path of a hop is taken."""
    rng = np.random.default_rng(seed)
    n = 3000
    perm = rng.permutation(n)
    ei, ej = [perm[:-1]], [perm[1:]]
    extra = rng.choice([0, 1, 4, 8, 13, 18, 24, 30, 45, 150], size=n,
                       p=[0.45, 0.2, 0.1, 0.07, 0.06, 0.05, 0.04, 0.02, 0.008, 0.002])
    for i in range(n):
        nb = rng.choice(n, size=int(extra[i]), replace=False)
        nb = nb[nb != i]
        ei.append(np.minimum(nb, i))
        ej.append(np.maximum(nb, i))
    ei, ej = np.concatenate(ei), np.concatenate(ej)
    g = np.exp(rng.uniform(np.log(0.1), np.log(10.0), ei.size))
    ei, ej, g = W._dedup_edges(ei, ej, g)
    rs = W.conductance_sums(n, ei, ej, g)
    excess = np.where(rng.random(n) < 0.3, rng.uniform(0.0, 0.05, n) * rs, 0.0)
    excess[rng.integers(n)] = 0.1 * rs.max()
    A = W.assemble(n, ei, ej, g, excess)
    deg = np.diff(A.rowptr) - 1
    ng = (deg + 4) // 4
    assert (ng <= 2).any() and ((ng > 2) & (ng <= 8)).any() and (ng > 8).any()
    assert len(set(ng[(ng > 2) & (ng <= 8)].tolist())) == 6   # every class 3..8
    return A


@pytest.mark.parametrize("reuse", [False, True])
def test_degree_classes_bit_exact(P, ctx, ctx_reuse, reuse):
    A = _degree_classes_matrix(21)
    c = ctx_reuse if reuse else ctx
    t = gpu_factor(P, c, A, 40, 4242, 1e-3)
    ref = oracle.build_factor(A, 40, 4242, 1e-3, reuse=reuse, records=True)
    assert_factor_equal(t, ref)


@pytest.mark.parametrize("case", list(range(8)))
def test_reuse_bit_exact(P, ctx_reuse, case):
    name, A, walks, drop = list(_reuse_cases())[case]
    t = gpu_factor(P, ctx_reuse, A, walks, 17 + case, drop)
    ref = oracle.build_factor(A, walks, 17 + case, drop, reuse=True, records=True)
    assert_factor_equal(t, ref)
    wr = ref["walk_rows"]
    assert int(ref["M"].sum()) > len(wr) * walks or A.n < 4   # sub-walks were counted


def test_reuse_per_row_budgets_and_big_rows(P, ctx_reuse):
    # large budgets push the later rows (which collect most sub-walks) onto the
    # block merge tables
    rng = np.random.default_rng(9)
    A = W.grid2d_5pt(60, 50)
    budget = np.where(rng.random(A.n) < 0.2, 800, 6).astype(np.uint32)
    t = gpu_factor(P, ctx_reuse, A, 0, 3, 0.0, budget=budget)
    ref = oracle.build_factor(A, budget, 3, 0.0, reuse=True, records=True)
    assert_factor_equal(t, ref)
    assert ref["M"].max() > 768


def test_reuse_extra_walks_reported(P):
    c = P.Context(options=P.rw_options_default(reuse=1))
    try:
        A = W.grid2d_5pt(30, 30)
        F = P.rw_build_factor(c, P.CSR.from_host(A), 20, 5, 1e-3)
        ref = oracle.build_factor(A, 20, 5, 1e-3, reuse=True)
        assert F.desc.total_walks == 20 * len(ref["walk_rows"])
        assert F.desc.extra_walks == int(ref["M"].sum()) - F.desc.total_walks > 0
        F.destroy()
        # reuse is single-matrix only
        with pytest.raises(P.RwError) as e:
            P.rw_build_factor_batched(c, [P.CSR.from_host(A), P.CSR.from_host(A)], 4, [1, 2], 0.0)
        assert e.value.code == -1
    finally:
        c.close()
