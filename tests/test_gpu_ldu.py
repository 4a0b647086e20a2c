"""Nonsymmetric matrices on the GPU (Sec. 7.1) against the oracle: the CSR
transpose (bit-exact), the factor of the game on A^T (bit-exact, like any
factor), the preconditioner of the two games (1e-12 relative, FP64) and
BiCGSTAB (the direct solution to 1e-8, the oracle's iteration count within
one, the true residual below the tolerance)."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import ldu as L

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


def _cases():
    rng = np.random.default_rng(50)
    return [W.asym_grid((9, 7), rng), W.asym_grid((10, 8, 6), rng, skew=0.9), W.grid2d_5pt(8, 6),
            W.random_rmatrix(40, rng)]


def test_transpose_bit_exact(P, ctx):
    for A in _cases():
        T = P.rw_csr_transpose(ctx, P.CSR.from_host(A))
        R = W.transpose(A)
        assert np.array_equal(T.rowptr.cpu().numpy(), R.rowptr)
        assert np.array_equal(T.col.cpu().numpy(), R.col)
        assert np.array_equal(T.val.cpu().numpy().view(np.uint64), R.val.view(np.uint64))


def test_game_on_transpose_bit_exact(P, ctx):
    A = _cases()[1]
    AT = P.rw_csr_transpose(ctx, P.CSR.from_host(A))
    F = P.rw_build_factor(ctx, AT, 60, 11, 1e-3)
    ref = oracle.build_factor(W.transpose(A), 60, 11, 1e-3)
    t = {k: v.cpu().numpy() for k, v in F.tensors().items()}
    F.destroy()
    assert np.array_equal(t["y_row_ptr"], ref["rowptr"]) and np.array_equal(t["y_col"], ref["col"])
    assert np.array_equal(t["y_val"].view(np.uint64), ref["val"].view(np.uint64))
    assert np.array_equal(t["d"].view(np.uint64), ref["D"].view(np.uint64))


@pytest.mark.parametrize("mode", [0, 2])
def test_ldu_preconditioner_and_bicgstab(P, mode):
    import torch
    c = P.Context(options=P.rw_options_default(solve_mode=mode, wide_slices=-1))
    try:
        rng = np.random.default_rng(60 + mode)
        A = W.asym_grid((12, 10, 8), rng, skew=0.7)
        dA = P.CSR.from_host(A)
        dAT = P.rw_csr_transpose(c, dA)
        FA = P.rw_build_factor(c, dA, 120, 3, 1e-3)
        FAT = P.rw_build_factor(c, dAT, 120, 4, 1e-3)
        ra = oracle.build_factor(A, 120, 3, 1e-3)
        rat = oracle.build_factor(W.transpose(A), 120, 4, 1e-3)
        r = rng.standard_normal((A.n, 3))
        z = torch.zeros_like(_dev(r))
        P.rw_precond_apply_ldu(c, FA, FAT, _dev(r), z)
        zg = z.cpu().numpy()
        for j in range(3):
            zr = L.ldu_apply(ra, rat, r[:, j])
            assert np.linalg.norm(zg[:, j] - zr) / np.linalg.norm(zr) < 1e-12
        b = rng.standard_normal(A.n)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        rc, st = P.bicgstab_solve(c, dA, FA, FAT, _dev(b), x, 1e-10, 500)
        assert rc == 0 and st.rel_residual < 1e-10
        xd = np.linalg.solve(A.to_dense(), b)
        assert np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd) < 1e-8
        xo, ito, relo = L.bicgstab(A, lambda v: L.ldu_apply(ra, rat, v), b, 1e-10, 500)
        assert abs(st.iterations - ito) <= 1, (st.iterations, ito)
        FA.destroy()
        FAT.destroy()
    finally:
        c.close()


def test_bad_arguments(P, ctx):
    import torch
    A = _cases()[0]
    B = W.asym_grid((5, 5), np.random.default_rng(2))
    dA, dB = P.CSR.from_host(A), P.CSR.from_host(B)
    FA = P.rw_build_factor(ctx, dA, 20, 1, 0.0)
    FB = P.rw_build_factor(ctx, dB, 20, 1, 0.0)
    r = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.RwError) as e:
        P.rw_precond_apply_ldu(ctx, FA, FB, r, r.clone())
    assert e.value.code == -1
    with pytest.raises(P.RwError) as e:
        P.bicgstab_solve(ctx, dB, FA, FA, r, r.clone(), 1e-8, 10)
    assert e.value.code == -1
    FA.destroy()
    FB.destroy()
