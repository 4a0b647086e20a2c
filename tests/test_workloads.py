"""The seeded input recipes (CPU only): sizes as stated for each workload, the
R-matrix form the walk game needs, the recipes' value ranges, and
determinism (the same seed gives the same arrays)."""
import numpy as np
import pytest

import oracle
import workloads as W


def _dense_parts(A):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag = rows == A.col
    d = np.zeros(A.n)
    d[rows[diag]] = A.val[diag]
    off = np.zeros(A.n)
    np.add.at(off, rows[~diag], -A.val[~diag])
    return rows, diag, d, off


def _symmetric(A):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    key = rows.astype(np.int64) * A.n + A.col
    tkey = A.col.astype(np.int64) * A.n + rows
    o, t = np.argsort(key), np.argsort(tkey)
    return np.array_equal(key[o], tkey[t]) and np.array_equal(A.val[o], A.val[t])


def test_small_grid_and_64_cube_sizes():
    A = W.make_config(1)["A"]
    assert (A.n, A.nnz) == (1024, 4992)
    A = W.make_config(2)["A"]
    assert (A.n, A.nnz) == (262144, 1810432)


@pytest.mark.parametrize("scale,m", [(0.125, 16), (0.25, 32)])
def test_27_point_grid_size_formula(scale, m):
    # a 27-point stencil couples i, i' with |i - i'| <= 1 in every dimension:
    # (3m - 2)^3 entries, 55,742,968 for m = 128
    A = W.make_config(5, scale=scale)["A"]
    assert A.n == m ** 3 and A.nnz == (3 * m - 2) ** 3
    assert (3 * 128 - 2) ** 3 == 55742968


def test_table1_grids_have_the_papers_n_and_e():
    # Table 1: N = m^3 and E = nnz(A) = m^3 + 6 m^2 (m - 1): 8.6e5 ... 6.9e6
    mats = W.make_config(6)["A"]
    for A, m, e_paper in zip(mats, (50, 60, 70, 80, 90, 100), (8.6e5, 1.5e6, 2.4e6, 3.5e6, 5.1e6, 6.9e6)):
        assert A.n == m ** 3 and A.nnz == m ** 3 + 6 * m * m * (m - 1)
        assert abs(A.nnz - e_paper) / e_paper < 0.02
        rows, diag, d, off = _dense_parts(A)
        assert np.all(A.val[~diag] == -1.0) and np.all(d == 6.0)


def test_recipes_give_r_matrices_with_the_stated_ranges():
    A = W.make_config(2)["A"]
    assert oracle.validate(A) == 0 and _symmetric(A)
    rows, diag, d, off = _dense_parts(A)
    g = -A.val[~diag]
    assert g.min() >= 0.1 and g.max() <= 10.0
    excess = d - off
    assert excess.min() >= 0.0 and np.all(excess <= 1e-3 * off * (1 + 1e-12))
    A5 = W.make_config(5, scale=0.125)["A"]
    rows, diag, d, off = _dense_parts(A5)
    assert oracle.validate(A5) == 0 and _symmetric(A5)
    assert np.allclose(d - off, 1e-4 * off, rtol=1e-9, atol=0)
    A7 = W.make_config(7, scale=0.25)["A"]
    assert oracle.validate(A7) == 0 and oracle.validate(W.transpose(A7)) == 0 and not _symmetric(A7)


def test_recipes_are_deterministic():
    for i, scale in ((2, 0.25), (3, 0.02), (5, 0.125), (7, 0.25)):
        a, b = W.make_config(i, scale=scale), W.make_config(i, scale=scale)
        for key in ("rowptr", "col", "val"):
            assert np.array_equal(getattr(a["A"], key), getattr(b["A"], key)), (i, key)
        assert np.array_equal(a["b"], b["b"])
    a, b = W.make_config(4, scale=0.01, nmat=3), W.make_config(4, scale=0.01, nmat=3)
    for x, y in zip(a["A"], b["A"]):
        assert np.array_equal(x.val, y.val) and np.array_equal(x.col, y.col)
