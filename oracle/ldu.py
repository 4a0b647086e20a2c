"""CPU oracle for nonsymmetric matrices (Sec. 7.1): the exact LDU factors of
rev(A), the preconditioner built from the two walk games (on A and on A^T),
and BiCGSTAB.  Test infrastructure: only the tests, smoke() and the bench's
CPU legs use it.

Convention (the library's): A ~= P diag(D) Q with P unit upper and Q unit
lower triangular.  The paper factors rev(A) = L D U (Lemma 1 and its LDU form
in Sec. 7.1); reversing rows and columns turns this into A = rev(L) rev(D)
rev(U), so P = rev(L), D = rev(D), Q = rev(U).  By Eq. y2 the game on A
estimates Q (its Y), by Eq. y3 the game on A^T estimates P^T (its Y).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular


def exact_ldu(A):
    """Exact (Q, P, D): Q unit lower, P unit upper, A = P diag(D) Q (dense).

    Doolittle elimination without pivoting on rev(A), written out: for every
    pivot k the multipliers of the rows below are stored in L and the rows are
    reduced; what remains is upper triangular, split into D (its diagonal) and
    the unit upper U.  No pivoting is needed: rev(A) is diagonally dominant by
    rows (an R-matrix), so every pivot stays positive.
    """
    Ad = A.to_dense() if hasattr(A, "to_dense") else np.asarray(A, dtype=float)
    R = Ad[::-1, ::-1].copy()
    n = R.shape[0]
    L = np.eye(n)
    for k in range(n):
        piv = R[k, k]
        for i in range(k + 1, n):
            if R[i, k] != 0.0:
                m = R[i, k] / piv
                L[i, k] = m
                R[i, k:] -= m * R[k, k:]
    Dr = np.diag(R).copy()
    U = np.triu(R) / Dr[:, None]  # the eliminated entries are zero by construction
    Q = U[::-1, ::-1].copy()
    P = L[::-1, ::-1].copy()
    return Q, P, Dr[::-1].copy()


def _unit_lower(F, n):
    strict = sp.csr_matrix((F["val"], F["col"], F["rowptr"]), shape=(n, n))
    return (strict + sp.identity(n, format="csr")).tocsr()


def ldu_apply(FA, FAT, r):
    """z = (Y_AT^T diag(D) Y_A)^-1 r: backward substitution with the unit upper
    Y_AT^T, division by D (the game on A), forward substitution with the unit
    lower Y_A (factor dicts of build_factor on A and on A^T)."""
    n = len(FA["D"])
    upper = _unit_lower(FAT, n).T.tocsr()
    w = spsolve_triangular(upper, np.asarray(r, dtype=float), lower=False, unit_diagonal=True)
    return spsolve_triangular(_unit_lower(FA, n), w / FA["D"], lower=True, unit_diagonal=True)


def bicgstab(A, apply_m, b, tol, max_iter):
    """BiCGSTAB with right preconditioning (van der Vorst's recurrences), from
    x = 0; stops when the true residual ||b - A x|| < tol ||b|| (checked when
    the recursive residual passes).  Returns (x, iterations, relative true
    residual)."""
    Am = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
    b = np.asarray(b, dtype=float)
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = b.copy()
    rh = r.copy()
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho_old = alpha = omega = 1.0
    relres = 1.0
    for it in range(1, max_iter + 1):
        rho = rh @ r
        if rho == 0.0:
            return x, it, relres
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = apply_m(p)
        v = Am @ ph
        alpha = rho / (rh @ v)
        s = r - alpha * v
        if np.linalg.norm(s) < tol * bnorm:
            x = x + alpha * ph
            relres = np.linalg.norm(b - Am @ x) / bnorm
            if relres < tol:
                return x, it, relres
            r = b - Am @ x
            rho_old, omega = rho, 1.0
            continue
        sh = apply_m(s)
        t = Am @ sh
        omega = (t @ s) / (t @ t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        relres = np.linalg.norm(r) / bnorm
        if relres < tol:
            relres = np.linalg.norm(b - Am @ x) / bnorm
            if relres < tol:
                return x, it, relres
        rho_old = rho
    return x, max_iter, np.linalg.norm(b - Am @ x) / bnorm
