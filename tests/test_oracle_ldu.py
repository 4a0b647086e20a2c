"""Pins of the nonsymmetric oracle (Sec. 7.1), CPU only: the exact LDU of
rev(A) reconstructs A and reduces to the Cholesky form for a symmetric A; the
game on A converges to its U part (Eq. y2) and the game on A^T to its L part
(Eq. y3), every entry within 4 sigma, D from either game within 4 sigma of the
exact one; BiCGSTAB with the exact factors converges in one iteration and with
the walk factors to the direct solution."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import ldu as L
from test_oracle import dense_Y, row_sigmas


def test_exact_ldu_reconstructs_and_reduces_to_cholesky():
    rng = np.random.default_rng(3)
    A = W.asym_grid((5, 4), rng)
    Q, P, D = L.exact_ldu(A)
    assert np.allclose(np.diag(Q), 1) and np.allclose(np.diag(P), 1)
    assert np.all(np.triu(Q, 1) == 0) and np.all(np.tril(P, -1) == 0) and np.all(D > 0)
    assert np.abs(P @ np.diag(D) @ Q - A.to_dense()).max() < 1e-12 * np.abs(A.to_dense()).max()
    S = W.grid2d_5pt(5, 4)
    Qs, Ps, Ds = L.exact_ldu(S)
    Y, Dy = oracle.exact_factor(S)
    assert np.allclose(Qs, Y, atol=1e-14) and np.allclose(Ps, Y.T, atol=1e-14) and np.allclose(Ds, Dy, rtol=1e-14)


def test_generator_is_dominant_both_ways():
    A = W.asym_grid((4, 3, 3), np.random.default_rng(5))
    d = A.to_dense()
    off = d - np.diag(np.diag(d))
    assert np.all(off <= 0) and np.abs(d - d.T).max() > 0
    assert np.all(np.diag(d) + off.sum(1) >= 0) and np.all(np.diag(d) + off.sum(0) >= 0)
    assert oracle.validate(A) == 0 and oracle.validate(W.transpose(A)) == 0
    assert np.array_equal(W.transpose(A).to_dense(), d.T)


@pytest.mark.parametrize("case", [0, 1])
def test_two_games_converge_to_the_exact_ldu(case):
    rng = np.random.default_rng(20 + case)
    A = W.asym_grid((4, 4) if case == 0 else (3, 3, 2), rng, skew=0.8)
    AT = W.transpose(A)
    Q, P, D = L.exact_ldu(A)
    walks = 400000
    FA = oracle.build_factor(A, walks, seed=5, drop_tol=0.0, records=True)
    FAT = oracle.build_factor(AT, walks, seed=6, drop_tol=0.0, records=True)
    lower = np.tril(np.ones((A.n, A.n), bool), -1)
    for F, M, Exact in ((FA, A, Q), (FAT, AT, P.T)):
        Y = dense_Y(F, A.n)
        sy, sd, _ = row_sigmas(M, F)
        err = np.abs(Y - Exact)[lower]
        assert np.all(err <= (4 * sy + 1e-12)[lower]), (err - 4 * sy[lower]).max()
        assert np.all(np.abs(F["D"] - D) <= 4 * sd + 1e-12 * D)


def test_bicgstab_exact_and_walk_factors():
    rng = np.random.default_rng(9)
    A = W.asym_grid((7, 6), rng)
    b = rng.standard_normal(A.n)
    xd = np.linalg.solve(A.to_dense(), b)
    Q, P, D = L.exact_ldu(A)
    M = P @ np.diag(D) @ Q
    x, it, rel = L.bicgstab(A, lambda r: np.linalg.solve(M, r), b, 1e-12, 50)
    assert it == 1 and rel < 1e-12
    FA = oracle.build_factor(A, 300, 7, 0.0)
    FAT = oracle.build_factor(W.transpose(A), 300, 8, 0.0)
    x, it, rel = L.bicgstab(A, lambda r: L.ldu_apply(FA, FAT, r), b, 1e-10, 200)
    assert rel < 1e-10 and np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
    x0, it0, rel0 = L.bicgstab(A, lambda r: r, b, 1e-10, 2000)   # no preconditioner
    assert rel0 < 1e-10 and it0 > it
