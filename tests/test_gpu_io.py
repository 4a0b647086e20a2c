"""Factor files (save / load with SHA-256) and seeded orderings, on the GPU."""
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


def test_factor_save_load_round_trip(P, ctx, tmp_path):
    cfg = W.make_config(2, scale=0.2)
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, 50, 9, 1e-3)
    path = tmp_path / "f.rwf"
    P.rw_factor_save(F, path)
    G = P.rw_factor_load(ctx, path)
    t0 = {k: v.cpu().numpy() for k, v in F.tensors().items()}
    t1 = {k: v.cpu().numpy() for k, v in G.tensors().items()}
    for k in ("y_row_ptr", "y_col", "y_val", "d", "yt_row_ptr", "yt_col", "yt_val", "walks", "visits", "ground",
              "y_val32", "yt_val32", "d32"):
        assert np.array_equal(t0[k].view(np.uint8), t1[k].view(np.uint8)), k
    assert (G.desc.total_hops, G.desc.total_walks, G.desc.fwd_levels) == \
        (F.desc.total_hops, F.desc.total_walks, F.desc.fwd_levels)
    x0, x1 = _dev(np.zeros_like(b)), _dev(np.zeros_like(b))
    _, _, i0, _ = P.pcg_solve(ctx, dA, F, _dev(b), x0, 1e-8, 500)
    _, _, i1, _ = P.pcg_solve(ctx, dA, G, _dev(b), x1, 1e-8, 500)
    assert np.array_equal(i0, i1) and np.array_equal(x0.cpu().numpy(), x1.cpu().numpy())
    # a flipped payload byte, a truncated file and a foreign file are refused
    raw = bytearray(path.read_bytes())
    raw[100] ^= 1
    bad = tmp_path / "bad.rwf"
    bad.write_bytes(bytes(raw))
    for p, data in ((bad, None), (tmp_path / "short.rwf", path.read_bytes()[:-40]),
                    (tmp_path / "foreign.rwf", b"not a factor" * 10)):
        if data is not None:
            p.write_bytes(data)
        with pytest.raises(P.RwError) as e:
            P.rw_factor_load(ctx, p)
        assert e.value.code == -1
    G.destroy()
    F.destroy()


def test_random_permutation_matches_philox_keys(P, ctx):
    import torch
    for n, seed in ((1, 3), (1000, 7), (70000, 2 ** 40 + 5)):
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        P.rw_random_permutation(ctx, n, seed, perm)
        got = perm.cpu().numpy()
        keys = np.array([oracle.philox4x32_10([i & 0xFFFFFFFF, i >> 32, 0, 2],
                                              [seed & 0xFFFFFFFF, seed >> 32])[0] for i in range(n)],
                        dtype=np.uint64)
        order = np.argsort(keys, kind="stable")
        want = np.empty(n, np.int64)
        want[order] = np.arange(n)
        assert np.array_equal(got, want)


def test_permute_csr_is_p_a_pt(P, ctx):
    import torch
    rng = np.random.default_rng(4)
    A = W.rgg(3000, rng)
    dA = P.CSR.from_host(A)
    perm = torch.empty(A.n, dtype=torch.int32, device="cuda")
    P.rw_random_permutation(ctx, A.n, 11, perm)
    B = P.rw_permute_csr(ctx, dA, perm)
    p = perm.cpu().numpy()
    S = A.to_scipy().tocoo()
    import scipy.sparse as sp
    ref = sp.csr_matrix((S.data, (p[S.row], p[S.col])), shape=S.shape)
    ref.sort_indices()
    assert np.array_equal(B.rowptr.cpu().numpy(), ref.indptr)
    assert np.array_equal(B.col.cpu().numpy(), ref.indices)
    assert np.array_equal(B.val.cpu().numpy(), ref.data)
    # the permuted matrix is still an R-matrix the library accepts
    F = P.rw_build_factor(ctx, B, 20, 1, 1e-3)
    F.destroy()
    bad = torch.zeros(A.n, dtype=torch.int32, device="cuda")
    with pytest.raises(P.RwError):
        P.rw_permute_csr(ctx, dA, bad)
