"""CPU oracle for the random-walk incomplete LDL^T preconditioner.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_math_0609672_gb300``); both are fed from the
separate input generators in ``workloads``.

The walk game, its counters and the factor are plain C (``rw_oracle.c``),
written step by step from the paper (Qian & Sapatnekar, "Stochastic
Preconditioning for Iterative Linear Equation Solvers"):

* walk game: Sec. 2.1 (Eq. map), homes created by the ordering: Sec. 2.2.1;
* journey record M, H, J and the factor: Sec. 3.1 (Eq. yzdetail), Sec. 3.3 (Eq. d);
* one-step-exact estimator: Sec. 5.2 (Eqs. newy, newz);
* walk reuse: Sec. 5.3, Algorithm 2;
* PCG with (Y^T D Y)^-1: Algorithm 1.

This module adds the dense exact factor (reverse-order elimination, Lemma 1
and Eqs. y/d) used to pin the estimator.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rw_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

ERRORS = {0: "ok", -1: "bad argument", -2: "not an R-matrix", -3: "walk step cap",
          -4: "out of memory", -5: "no convergence", -6: "breakdown"}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({code})")
        self.code = code


def build(force=False):
    """Compile the C oracle with gcc (no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "rw_oracle.h"))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    u32p, i32p, i64p = P(ctypes.c_uint32), P(ctypes.c_int32), P(ctypes.c_int64)
    u64p, f64p = P(ctypes.c_uint64), P(ctypes.c_double)
    lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.orc_philox4x32_10.restype = None
    lib.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                             ctypes.c_uint32, ctypes.c_uint64]
    lib.orc_draw.restype = ctypes.c_uint32
    lib.orc_row_thresholds.argtypes = [i32p, i32p, f64p, ctypes.c_int32, u32p]
    lib.orc_row_thresholds.restype = ctypes.c_int32
    lib.orc_validate.argtypes = [ctypes.c_int32, i32p, i32p, f64p]
    lib.orc_validate.restype = ctypes.c_int
    lib.orc_factor_build.argtypes = [ctypes.c_int32, i32p, i32p, f64p, u32p, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                     ctypes.c_uint64, ctypes.c_int32, i32p, ctypes.c_int32,
                                     i32p, u32p, u32p, ctypes.c_int64, P(ctypes.c_void_p)]
    lib.orc_factor_build.restype = ctypes.c_int
    lib.orc_factor_build_mt.argtypes = [ctypes.c_int32, i32p, i32p, f64p, u32p, ctypes.c_uint64,
                                        ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                        ctypes.c_uint64, i32p, ctypes.c_int32, ctypes.c_int32,
                                        P(ctypes.c_void_p)]
    lib.orc_factor_build_mt.restype = ctypes.c_int
    lib.orc_factor_nnz.argtypes = [ctypes.c_void_p]
    lib.orc_factor_nnz.restype = ctypes.c_int64
    lib.orc_factor_get.argtypes = [ctypes.c_void_p, i64p, i32p, f64p, f64p, u64p, u64p, u64p, u64p]
    lib.orc_factor_get.restype = None
    lib.orc_factor_free.argtypes = [ctypes.c_void_p]
    lib.orc_factor_free.restype = None
    lib.orc_reuse_trace.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, i64p, i64p, i32p, i32p,
                                    ctypes.c_int32]
    lib.orc_reuse_trace.restype = ctypes.c_int32
    lib.orc_pcg.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i64p, i32p, f64p, f64p, f64p, f64p,
                            ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                            i32p, f64p]
    lib.orc_pcg.restype = ctypes.c_int
    lib.orc_precond_apply.argtypes = [ctypes.c_int32, i64p, i32p, f64p, f64p, f64p, f64p]
    lib.orc_precond_apply.restype = ctypes.c_int
    lib.orc_adaptive_budget.argtypes = [ctypes.c_int32, i32p, i32p, f64p, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_int32, ctypes.c_uint64, u32p, i32p]
    lib.orc_adaptive_budget.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                          _ptr(o, ctypes.c_uint32))
    return o


def draw(seed, matrix_index, tag, k, w, s):
    return int(_load().orc_draw(seed, matrix_index, tag, k, w, s))


def row_thresholds(A, l):
    lib = _load()
    out = np.zeros(max(1, int(A.rowptr[l + 1] - A.rowptr[l])), dtype=np.uint32)
    m = lib.orc_row_thresholds(_ptr(A.rowptr, ctypes.c_int32), _ptr(A.col, ctypes.c_int32),
                               _ptr(A.val, ctypes.c_double), l, _ptr(out, ctypes.c_uint32))
    return out[:m]


def validate(A):
    return int(_load().orc_validate(A.n, _ptr(A.rowptr, ctypes.c_int32),
                                    _ptr(A.col, ctypes.c_int32), _ptr(A.val, ctypes.c_double)))


def walk_rows(A):
    """Rows with at least one upper neighbour (the rows that run walks)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return np.unique(rows[A.col > rows])


def build_factor(A, walks, seed, drop_tol, matrix_index=0, tag=0, max_steps=1 << 24,
                 reuse=False, records=False, rows=None, threads=1):
    """Factor A ~= Y^T diag(D) Y from walks.

    walks: int (uniform budget) or uint32 array [n] of per-row budgets.
    Returns dict with Y CSR (rowptr int64, col, val), D, per-row counters
    M, J, G (walks, visits to the start row, ground ends) and hops, and with
    ``records=True`` the per-walk records (end, returns, length) in walk order.
    ``rows``: optional subset of rows to compute (the rows are independent);
    the other rows come back empty with D = 0.  ``threads`` > 1 runs the rows
    of the plain build (no reuse, no records) on that many host threads
    (``orc_factor_build_mt``; the same factor bit for bit).
    """
    lib = _load()
    n = A.n
    if np.isscalar(walks):
        budget = np.full(n, int(walks), dtype=np.uint32)
    else:
        budget = np.ascontiguousarray(walks, dtype=np.uint32)
    wr = walk_rows(A)
    sel = None
    if rows is not None:
        sel = np.unique(np.asarray(rows, dtype=np.int32))
        wr = np.intersect1d(wr, sel)
    total = int(budget[wr].sum()) if wr.size else 0
    rec_end = rec_ret = rec_len = None
    cap = 0
    if records:
        cap = total
        rec_end = np.zeros(max(1, cap), dtype=np.int32)
        rec_ret = np.zeros(max(1, cap), dtype=np.uint32)
        rec_len = np.zeros(max(1, cap), dtype=np.uint32)
    h = ctypes.c_void_p()
    if threads > 1:
        if reuse or records:
            raise ValueError("the multi-threaded build has no reuse and no records")
        rc = lib.orc_factor_build_mt(
            n, _ptr(A.rowptr, ctypes.c_int32), _ptr(A.col, ctypes.c_int32),
            _ptr(A.val, ctypes.c_double), _ptr(budget, ctypes.c_uint32), seed, matrix_index, tag,
            float(drop_tol), int(max_steps), _ptr(sel, ctypes.c_int32) if sel is not None else None,
            0 if sel is None else int(sel.size), int(threads), ctypes.byref(h))
    else:
        rc = lib.orc_factor_build(
            n, _ptr(A.rowptr, ctypes.c_int32), _ptr(A.col, ctypes.c_int32),
            _ptr(A.val, ctypes.c_double), _ptr(budget, ctypes.c_uint32), seed, matrix_index, tag,
            float(drop_tol), int(max_steps), 1 if reuse else 0,
            _ptr(sel, ctypes.c_int32) if sel is not None else None,
            0 if sel is None else int(sel.size),
            _ptr(rec_end, ctypes.c_int32) if records else None,
            _ptr(rec_ret, ctypes.c_uint32) if records else None,
            _ptr(rec_len, ctypes.c_uint32) if records else None, cap, ctypes.byref(h))
    if rc:
        raise OracleError(rc, "oracle factor build")
    try:
        nnz = lib.orc_factor_nnz(h)
        out = dict(rowptr=np.zeros(n + 1, np.int64), col=np.zeros(max(1, nnz), np.int32),
                   val=np.zeros(max(1, nnz)), D=np.zeros(max(1, n)), M=np.zeros(max(1, n), np.uint64),
                   J=np.zeros(max(1, n), np.uint64), G=np.zeros(max(1, n), np.uint64),
                   hops=np.zeros(max(1, n), np.uint64))
        lib.orc_factor_get(h, _ptr(out["rowptr"], ctypes.c_int64), _ptr(out["col"], ctypes.c_int32),
                           _ptr(out["val"], ctypes.c_double), _ptr(out["D"], ctypes.c_double),
                           _ptr(out["M"], ctypes.c_uint64), _ptr(out["J"], ctypes.c_uint64),
                           _ptr(out["G"], ctypes.c_uint64), _ptr(out["hops"], ctypes.c_uint64))
    finally:
        lib.orc_factor_free(h)
    for key in ("col", "val"):
        out[key] = out[key][:nnz]
    for key in ("D", "M", "J", "G", "hops"):
        out[key] = out[key][:n]
    out["nnz"] = int(nnz)
    out["walk_rows"] = wr
    out["budget"] = budget
    if records:
        out["rec_end"], out["rec_ret"], out["rec_len"] = rec_end[:cap], rec_ret[:cap], rec_len[:cap]
    return out


def adaptive_budget(A, seed, delta, z, min_walks=20, max_walks=4096, max_rounds=8, max_steps=1 << 24,
                    matrix_index=0):
    """Adaptive walk counts of Sec. 5.1 (rounds; see orc_adaptive_budget).
    Returns (budget uint32 [n], rounds)."""
    lib = _load()
    budget = np.zeros(max(1, A.n), dtype=np.uint32)
    rounds = ctypes.c_int32()
    rc = lib.orc_adaptive_budget(A.n, _ptr(A.rowptr, ctypes.c_int32), _ptr(A.col, ctypes.c_int32),
                                 _ptr(A.val, ctypes.c_double), ctypes.c_uint64(int(seed)), int(matrix_index),
                                 ctypes.c_double(delta), ctypes.c_double(z), int(min_walks), int(max_walks),
                                 int(max_rounds), ctypes.c_uint64(int(max_steps)), _ptr(budget, ctypes.c_uint32),
                                 ctypes.byref(rounds))
    if rc:
        raise OracleError(rc, "oracle adaptive budget")
    return budget[:A.n], rounds.value


def reuse_trace(seq, nlabels):
    """Algorithm 2 on one explicit walk; returns (dM, dJ, list of (start, end))."""
    lib = _load()
    s = np.ascontiguousarray(seq, dtype=np.int32)
    dM = np.zeros(nlabels + 1, np.int64)
    dJ = np.zeros(nlabels + 1, np.int64)
    hs = np.zeros(len(s), np.int32)
    he = np.zeros(len(s), np.int32)
    m = lib.orc_reuse_trace(_ptr(s, ctypes.c_int32), len(s), nlabels, _ptr(dM, ctypes.c_int64),
                            _ptr(dJ, ctypes.c_int64), _ptr(hs, ctypes.c_int32),
                            _ptr(he, ctypes.c_int32), len(s))
    if m < 0:
        raise OracleError(m, "reuse trace")
    return dM, dJ, list(zip(hs[:m].tolist(), he[:m].tolist()))


def precond_apply(F, r):
    """z = (Y^T diag(D) Y)^-1 r for one vector (FP64)."""
    lib = _load()
    n = len(F["D"])
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.zeros(n)
    yrp = np.ascontiguousarray(F["rowptr"], dtype=np.int64)
    ycol = np.ascontiguousarray(F["col"], dtype=np.int32)
    yval = np.ascontiguousarray(F["val"], dtype=np.float64)
    if ycol.size == 0:
        ycol, yval = np.zeros(1, np.int32), np.zeros(1)
    D = np.ascontiguousarray(F["D"], dtype=np.float64)
    rc = lib.orc_precond_apply(n, _ptr(yrp, ctypes.c_int64), _ptr(ycol, ctypes.c_int32),
                               _ptr(yval, ctypes.c_double), _ptr(D, ctypes.c_double),
                               _ptr(r, ctypes.c_double), _ptr(z, ctypes.c_double))
    if rc:
        raise OracleError(rc, "oracle precond")
    return z


def pcg(A, F, b, tol, max_iter, mixed=False, refine_every=50):
    """PCG with M = Y^T diag(D) Y on one right-hand side (Algorithm 1).

    Returns (x, iterations, true relative residual, status code); status 0 =
    converged, -5 = max_iter reached (always the case for tol = 0).
    """
    lib = _load()
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.n)
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    yrp = np.ascontiguousarray(F["rowptr"], dtype=np.int64)
    ycol = np.ascontiguousarray(F["col"], dtype=np.int32)
    yval = np.ascontiguousarray(F["val"], dtype=np.float64)
    if ycol.size == 0:
        ycol = np.zeros(1, np.int32)
        yval = np.zeros(1)
    D = np.ascontiguousarray(F["D"], dtype=np.float64)
    rc = lib.orc_pcg(A.n, _ptr(A.rowptr, ctypes.c_int32), _ptr(A.col, ctypes.c_int32),
                     _ptr(A.val, ctypes.c_double), _ptr(yrp, ctypes.c_int64),
                     _ptr(ycol, ctypes.c_int32), _ptr(yval, ctypes.c_double),
                     _ptr(D, ctypes.c_double), _ptr(b, ctypes.c_double), _ptr(x, ctypes.c_double),
                     float(tol), int(max_iter), 1 if mixed else 0, int(refine_every),
                     ctypes.byref(it), ctypes.byref(rr))
    if rc not in (0, -5):
        raise OracleError(rc, "oracle pcg")
    return x, int(it.value), float(rr.value), rc


# ----------------------------------------------------------------------------
# Dense exact factor (pins the estimator; small matrices only)
# ----------------------------------------------------------------------------

def exact_factor(A):
    """Exact Y (unit lower, dense) and D with A = Y^T diag(D) Y.

    The paper's exact reference is the LDL^T factorization of rev(A)
    (Lemma 1, Eqs. y and d): rev(A) = L diag(D') L^T gives
    Y = rev(L)^T and D = rev(D').  rev(L) is computed here by a textbook
    Cholesky of the reversed dense matrix (numpy), not by any method code.
    """
    Ad = A.to_dense() if hasattr(A, "to_dense") else np.asarray(A, dtype=float)
    R = Ad[::-1, ::-1]
    C = np.linalg.cholesky(R)
    d = np.diag(C).copy()
    L = C / d[None, :]
    Dp = d * d
    Y = L[::-1, ::-1].T.copy()
    D = Dp[::-1].copy()
    return Y, D


def exact_walk_probabilities(A):
    """Exact end-point probabilities and expected returns of the one-step-exact
    walks, from the absorbing Markov chain (fundamental matrix), for every row.

    For row k the chain runs on the motels {k..n-1}; P[k][i] is the probability
    that a walk whose first step is drawn among the upper neighbours ends at
    home i < k, g[k] the probability it ends at ground, and q[k] = E[J'/M'] the
    expected visits to k counting the start.  Plain dense linear algebra
    (Kemeny-Snell fundamental matrix); used to pin the estimator's expectation.
    """
    Ad = A.to_dense()
    n = Ad.shape[0]
    dg = np.diag(Ad)
    P = -Ad / dg[:, None]
    np.fill_diagonal(P, 0.0)
    ends = np.zeros((n, n))
    ground = np.zeros(n)
    visits = np.ones(n)
    for k in range(n):
        up = np.flatnonzero(Ad[k, k + 1:] != 0) + k + 1
        if up.size == 0:
            continue
        first = -Ad[k, up] / (-Ad[k, up]).sum()
        mot = np.arange(k, n)
        Q = P[np.ix_(mot, mot)]
        N = np.linalg.inv(np.eye(mot.size) - Q)  # expected visits from each motel
        # start distribution after the first step
        s0 = np.zeros(mot.size)
        s0[up - k] = first
        v = s0 @ N                               # expected visits to each motel
        homes = np.arange(k)
        ends[k, homes] = v @ P[np.ix_(mot, homes)]
        exc = 1.0 - P[mot].sum(axis=1)
        ground[k] = v @ exc
        visits[k] = 1.0 + v[0]
    return ends, ground, visits
