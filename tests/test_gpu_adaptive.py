"""GPU adaptive walk counts (Sec. 5.1, Eq. lengthdelta) against the oracle:
bit-exact counts and round numbers (exact integer length sums, the FP64 test
rounded once per operation on both sides), the factor built from them
bit-identical to the oracle's, the degenerate cases, and bad arguments."""
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


def _budget(P, ctx, A, seed, delta, z, mn, mx, rounds):
    import torch
    b = torch.zeros(max(1, A.n), dtype=torch.int32, device="cuda")
    r = P.rw_adaptive_budget(ctx, P.CSR.from_host(A), seed, delta, z, mn, mx, rounds, b)
    return b.cpu().numpy().view(np.uint32)[:A.n], r


def _cases():
    rng = np.random.default_rng(31)
    return [(W.grid2d_5pt(17, 13), 0.1, 1.96, 20, 4000, 8),
            (W.rgg(700, rng), 0.2, 1.645, 10, 2000, 6),
            (W.grid3d(7, 6, 5, 27, rng, excess_frac=1e-4), 0.15, 2.576, 16, 65535, 10),
            (W.random_rmatrix(40, rng), 0.05, 1.96, 2, 500, 3),
            (W.tridiag(3), 0.1, 1.96, 20, 100, 4)]


def test_counts_bit_exact(P, ctx):
    for i, (A, delta, z, mn, mx, rounds) in enumerate(_cases()):
        got, r = _budget(P, ctx, A, 40 + i, delta, z, mn, mx, rounds)
        ref, rr = oracle.adaptive_budget(A, 40 + i, delta, z, min_walks=mn, max_walks=mx, max_rounds=rounds)
        assert r == rr, (i, r, rr)
        assert np.array_equal(got, ref), (i, np.flatnonzero(got != ref)[:10])


def test_factor_from_adaptive_counts(P, ctx):
    A = W.grid2d_5pt(24, 20)
    seed = 9
    b, _ = _budget(P, ctx, A, seed, 0.1, 1.96, 20, 3000, 8)
    import torch
    F = P.rw_build_factor_budget(ctx, P.CSR.from_host(A), torch.as_tensor(b.view(np.int32), device="cuda"),
                                 seed, 1e-3)
    ref = oracle.build_factor(A, b, seed, 1e-3)
    got = {k: v.cpu().numpy() for k, v in F.tensors().items()}
    F.destroy()
    assert np.array_equal(got["walks"].astype(np.uint64), ref["M"])
    assert np.array_equal(got["y_row_ptr"], ref["rowptr"])
    assert np.array_equal(got["y_col"], ref["col"])
    assert np.array_equal(got["y_val"].view(np.uint64), ref["val"].view(np.uint64))
    assert np.array_equal(got["d"].view(np.uint64), ref["D"].view(np.uint64))


def test_degenerate_cases(P, ctx):
    A = W.grid2d_5pt(6, 5)
    wr = oracle.walk_rows(A)
    got, r = _budget(P, ctx, A, 3, 0.01, 3.0, 17, 4000, 1)
    assert r == 1 and np.all(got[wr] == 17) and np.all(np.delete(got, wr) == 0)
    got, r = _budget(P, ctx, A, 3, 1e-4, 3.0, 5, 40, 8)
    ref, rr = oracle.adaptive_budget(A, 3, 1e-4, 3.0, min_walks=5, max_walks=40, max_rounds=8)
    assert r == rr == 2 and np.array_equal(got, ref)
    # a diagonal matrix has no walk rows: all zero, no rounds
    D = W.assemble(4, np.array([], np.int64), np.array([], np.int64), np.array([]), np.ones(4))
    got, r = _budget(P, ctx, D, 1, 0.1, 2.0, 4, 10, 3)
    assert r == 0 and np.all(got == 0)


def test_rejects_bad_arguments(P, ctx):
    A = W.grid2d_5pt(4, 4)
    for delta, z, mn, mx, rounds in ((0.0, 2.0, 4, 100, 4), (0.1, -1.0, 4, 100, 4), (0.1, 2.0, 1, 100, 4),
                                     (0.1, 2.0, 4, 3, 4), (0.1, 2.0, 4, 70000, 4), (0.1, 2.0, 4, 100, 0)):
        with pytest.raises(P.RwError) as e:
            _budget(P, ctx, A, 1, delta, z, mn, mx, rounds)
        assert e.value.code == -1


@pytest.mark.parametrize("ahead", [0, 25, 400])
def test_run_ahead_changes_no_count(P, ahead):
    """How far the launch rounds run past a row's next decision point
    (rw_options.adapt_ahead) changes the time only: counts and the decision
    count stay the oracle's."""
    c = P.Context(options=P.rw_options_default(adapt_ahead=ahead))
    try:
        for i, (A, delta, z, mn, mx, rounds) in enumerate(_cases()[:3]):
            got, r = _budget(P, c, A, 60 + i, delta, z, mn, mx, rounds)
            ref, rr = oracle.adaptive_budget(A, 60 + i, delta, z, min_walks=mn, max_walks=mx, max_rounds=rounds)
            assert r == rr and np.array_equal(got, ref), (ahead, i)
    finally:
        c.close()
