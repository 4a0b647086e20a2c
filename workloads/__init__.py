"""Seeded synthetic inputs: R-matrices in CSR form and right-hand sides.

This module only builds inputs.  It holds none of the method's arithmetic (no
transition tables, walks, factors or solves), so both the CPU oracle and the
CUDA library may be fed from it.

An R-matrix (Sec. 1 of the paper) is a symmetric M-matrix that is irreducibly
diagonally dominant.  Every generator here builds one from an undirected
weighted graph: off-diagonal entries are minus the edge conductances, and the
diagonal is the row's conductance sum plus a non-negative "excess" (the
diagonal dominance, which the walk game of Sec. 2.1 turns into absorption at
ground).  Stored off-diagonal entries are strictly negative; columns are sorted
and the diagonal is always stored.

CSR arrays: ``rowptr`` int32[n+1], ``col`` int32[nnz], ``val`` float64[nnz].
Right-hand sides are node-major: ``b[i, r]`` is entry i of right-hand side r,
so one row of ``b`` holds all right-hand sides of one node.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSR", "assemble", "grid2d_5pt", "grid3d", "grid2d_longrange", "rgg",
    "relabel", "rhs", "random_rmatrix", "tridiag", "make_config", "CONFIGS",
]


@dataclasses.dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray     # int32 [nnz]
    val: np.ndarray     # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            a[i, self.col[s:e]] = self.val[s:e]
        return a

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def _dedup_edges(ei, ej, g):
    """Canonicalise undirected edges to i<j and sum the conductances of repeats."""
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    g = np.asarray(g, dtype=np.float64)
    keep = ei != ej
    ei, ej, g = ei[keep], ej[keep], g[keep]
    lo = np.minimum(ei, ej)
    hi = np.maximum(ei, ej)
    key = lo * (int(hi.max(initial=0)) + 1) + hi
    order = np.argsort(key, kind="stable")
    key, lo, hi, g = key[order], lo[order], hi[order], g[order]
    if key.size == 0:
        return lo, hi, g
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    starts = np.flatnonzero(first)
    gsum = np.add.reduceat(g, starts)
    return lo[starts], hi[starts], gsum


def conductance_sums(n, ei, ej, g):
    """Sum of incident conductances per node (the off-diagonal row sum |A_ij|)."""
    return (np.bincount(ei, weights=g, minlength=n)
            + np.bincount(ej, weights=g, minlength=n))


def assemble(n, ei, ej, g, excess) -> CSR:
    """CSR of the R-matrix of an undirected graph with unique edges ei<ej.

    A_ij = A_ji = -g for each edge, A_ii = (sum of incident g) + excess_i.
    """
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    g = np.asarray(g, dtype=np.float64)
    excess = np.broadcast_to(np.asarray(excess, dtype=np.float64), (n,))
    if np.any(g <= 0) or not np.all(np.isfinite(g)):
        raise ValueError("conductances must be finite and positive")
    if np.any(excess < 0):
        raise ValueError("diagonal excess must be non-negative")
    diag = conductance_sums(n, ei, ej, g) + excess
    nodes = np.arange(n, dtype=np.int64)
    rows = np.concatenate([ei, ej, nodes])
    cols = np.concatenate([ej, ei, nodes])
    vals = np.concatenate([-g, -g, diag])
    order = np.argsort(rows * n + cols, kind="stable")
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals)


def relabel(n, ei, ej, perm_new_of_old):
    """Apply a symmetric permutation to an edge list: node v becomes perm[v]."""
    p = np.asarray(perm_new_of_old, dtype=np.int64)
    return p[ei], p[ej]


def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


# ----------------------------------------------------------------------------
# Graph families
# ----------------------------------------------------------------------------

def _grid_edges(shape, offsets):
    """Edges of a structured grid in natural (C-order) numbering."""
    dims = len(shape)
    idx = np.arange(int(np.prod(shape)), dtype=np.int64).reshape(shape)
    eis, ejs = [], []
    for off in offsets:
        src = [slice(None)] * dims
        dst = [slice(None)] * dims
        for d, o in enumerate(off):
            if o > 0:
                src[d] = slice(0, shape[d] - o)
                dst[d] = slice(o, shape[d])
            elif o < 0:
                src[d] = slice(-o, shape[d])
                dst[d] = slice(0, shape[d] + o)
        eis.append(idx[tuple(src)].ravel())
        ejs.append(idx[tuple(dst)].ravel())
    return np.concatenate(eis), np.concatenate(ejs)


def _boundary_mask(shape):
    m = np.zeros(shape, dtype=bool)
    for d in range(len(shape)):
        sl = [slice(None)] * len(shape)
        sl[d] = 0
        m[tuple(sl)] = True
        sl[d] = shape[d] - 1
        m[tuple(sl)] = True
    return m.ravel()


def grid2d_5pt(nx, ny, boundary_excess=1.0, g=1.0):
    """2D 5-point grid Laplacian, unit (or constant) conductance, natural order,
    excess `boundary_excess` on the boundary rows only (Dirichlet ground)."""
    ei, ej = _grid_edges((nx, ny), [(1, 0), (0, 1)])
    n = nx * ny
    excess = np.where(_boundary_mask((nx, ny)), boundary_excess, 0.0)
    return assemble(n, ei, ej, np.full(ei.size, float(g)), excess)


_OFF7 = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
_OFF27 = [o for o in ((a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
          if o > (0, 0, 0)]


def grid3d(nx, ny, nz, stencil, rng, glo=0.1, ghi=10.0, excess_frac_hi=None,
           excess_frac=None, permute=True):
    """3D 7- or 27-point grid with log-uniform conductances in [glo, ghi].

    Excess per row: U[0, excess_frac_hi] * rowsum if `excess_frac_hi` is given,
    else excess_frac * rowsum (rowsum = sum of |off-diagonal| of the row).
    With `permute`, nodes get a seeded random symmetric ordering (the paper's
    implementation uses random ordering, Sec. 5.4).
    """
    offs = _OFF7 if stencil == 7 else _OFF27
    ei, ej = _grid_edges((nx, ny, nz), offs)
    n = nx * ny * nz
    g = _loguniform(rng, glo, ghi, ei.size)
    rs = conductance_sums(n, ei, ej, g)
    if excess_frac_hi is not None:
        excess = rng.uniform(0.0, excess_frac_hi, n) * rs
    else:
        excess = excess_frac * rs
    if permute:
        p = rng.permutation(n)
        ei, ej = relabel(n, ei, ej, p)
        excess_new = np.empty_like(excess)
        excess_new[p] = excess
        excess = excess_new
    return assemble(n, ei, ej, g, excess)


def laplace3d_dirichlet(m):
    """7-point finite-difference Laplacian of an m x m x m grid with Dirichlet
    boundary: every off-diagonal -1 and every diagonal 6, so a boundary node's
    missing neighbours become its excess (ground).  Natural order."""
    ei, ej = _grid_edges((m, m, m), _OFF7)
    n = m * m * m
    deg = np.bincount(ei, minlength=n) + np.bincount(ej, minlength=n)
    return assemble(n, ei, ej, np.ones(ei.size), 6.0 - deg)


def asym_grid(shape, rng, skew=0.6, glo=0.1, ghi=10.0, excess_frac_hi=1e-3, permute=True):
    """Nonsymmetric grid matrix (2D 5-point or 3D 7-point by len(shape)) for
    the two-game factor of Sec. 7.1: edge e = (i, j) with conductance g_e
    log-U[glo, ghi] and skew s_e ~ U[-skew, skew] gives A_ij = -g_e (1 + s_e),
    A_ji = -g_e (1 - s_e); the diagonal is max(row sum, column sum) of the
    off-diagonal magnitudes times (1 + U[0, excess_frac_hi]), so A is
    diagonally dominant by rows (the game on A) and by columns (the game on
    A^T).  With `permute`, a seeded random symmetric ordering."""
    offs = [tuple(1 if d == k else 0 for d in range(len(shape))) for k in range(len(shape))]
    ei, ej = _grid_edges(tuple(shape), offs)
    n = int(np.prod(shape))
    g = _loguniform(rng, glo, ghi, ei.size)
    sk = rng.uniform(-skew, skew, ei.size)
    if permute:
        ei, ej = relabel(n, ei, ej, rng.permutation(n))
    rows = np.concatenate([ei, ej])
    cols = np.concatenate([ej, ei])
    off = np.concatenate([-g * (1.0 + sk), -g * (1.0 - sk)])
    rsum = np.bincount(rows, weights=-off, minlength=n)
    csum = np.bincount(cols, weights=-off, minlength=n)
    dom = np.maximum(rsum, csum)
    diag = dom * (1.0 + rng.uniform(0.0, excess_frac_hi, n))
    r = np.concatenate([rows, np.arange(n)])
    c = np.concatenate([cols, np.arange(n)])
    v = np.concatenate([off, diag])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr.astype(np.int32), c.astype(np.int32), v.astype(np.float64))


def transpose(A):
    """A^T of a host CSR (columns ascending)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    order = np.lexsort((rows, A.col))
    r, c, v = A.col[order], rows[order], A.val[order]
    rowptr = np.zeros(A.n + 1, np.int64)
    np.add.at(rowptr, r + 1, 1)
    return CSR(A.n, np.cumsum(rowptr).astype(np.int32), c.astype(np.int32), v.copy())


def grid2d_longrange(nx, ny, rng, n_long=2, glo=0.01, ghi=1.0, boundary_excess=1.0,
                     permute=True):
    """2D 5-point unit grid plus `n_long` random long-range edges per row.

    Long-range partners are uniform over j != i with log-uniform conductance in
    [glo, ghi]; repeated edges have their conductances summed.  Boundary rows
    of the grid carry excess `boundary_excess`.
    """
    n = nx * ny
    gi, gj = _grid_edges((nx, ny), [(1, 0), (0, 1)])
    src = np.repeat(np.arange(n, dtype=np.int64), n_long)
    dst = rng.integers(0, n - 1, size=src.size)
    dst = dst + (dst >= src)  # uniform over j != i
    gl = _loguniform(rng, glo, ghi, src.size)
    ei = np.concatenate([gi, src])
    ej = np.concatenate([gj, dst])
    g = np.concatenate([np.ones(gi.size), gl])
    ei, ej, g = _dedup_edges(ei, ej, g)
    excess = np.where(_boundary_mask((nx, ny)), boundary_excess, 0.0)
    if permute:
        p = rng.permutation(n)
        ei, ej = relabel(n, ei, ej, p)
        e2 = np.empty_like(excess)
        e2[p] = excess
        excess = e2
        lo, hi = np.minimum(ei, ej), np.maximum(ei, ej)
        ei, ej = lo, hi
    return assemble(n, ei, ej, g, excess)


def rgg(n, rng, mean_degree=8.0, excess_value=1e-2, excess_fraction=0.01, relative=True):
    """Random geometric graph Laplacian in the unit square.

    Points uniform in [0,1]^2, radius r = sqrt(mean_degree / (pi n)),
    conductance 1/distance.  Excess on a random `excess_fraction` of the rows:
    `excess_value` times the row's conductance sum (relative=True), or the
    absolute value `excess_value` (relative=False; with conductances of order
    1/r this grounds so weakly that walks from the first rows run for 1e7+
    hops).  Every connected component without a grounded row gets the excess
    on its lowest-index node so that the matrix is irreducibly dominant per
    component and n is unchanged.
    """
    from scipy.spatial import cKDTree
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    pts = rng.uniform(0.0, 1.0, size=(n, 2))
    r = math.sqrt(mean_degree / (math.pi * n))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray").astype(np.int64)
    ei, ej = pairs[:, 0], pairs[:, 1]
    d = np.sqrt(((pts[ei] - pts[ej]) ** 2).sum(axis=1))
    keep = d > 0
    ei, ej, d = ei[keep], ej[keep], d[keep]
    lo, hi = np.minimum(ei, ej), np.maximum(ei, ej)
    g = 1.0 / d
    scale = conductance_sums(n, lo, hi, g) if relative else np.ones(n)
    scale = np.where(scale > 0, scale, 1.0)  # isolated nodes
    excess = np.zeros(n)
    nground = max(1, int(round(excess_fraction * n)))
    pick = rng.choice(n, size=nground, replace=False)
    excess[pick] = excess_value * scale[pick]
    adj = coo_matrix((np.ones(lo.size), (lo, hi)), shape=(n, n))
    ncomp, lab = connected_components(adj, directed=False)
    grounded = np.zeros(ncomp, dtype=bool)
    grounded[lab[excess > 0]] = True
    first = np.full(ncomp, n, dtype=np.int64)
    np.minimum.at(first, lab, np.arange(n))
    fix = first[~grounded]
    excess[fix] = excess_value * scale[fix]
    return assemble(n, lo, hi, g, excess)


def tridiag(n, diag=2.0, off=-1.0):
    """A = tridiag(off, diag, off): the 1D Dirichlet Laplacian for the defaults."""
    ei = np.arange(n - 1)
    ej = ei + 1
    g = np.full(n - 1, -off)
    rs = conductance_sums(n, ei, ej, g)
    return assemble(n, ei, ej, g, np.full(n, diag) - rs)


def random_rmatrix(n, rng, p_edge=0.3, glo=0.1, ghi=1.0, p_ground=0.3, excess_hi=0.5):
    """Small dense-ish random R-matrix: Erdos-Renyi graph made connected by a
    random spanning path, log-uniform conductances, excess U[0, excess_hi] *
    rowsum on a random subset of rows (at least one)."""
    iu, ju = np.triu_indices(n, 1)
    pick = rng.random(iu.size) < p_edge
    perm = rng.permutation(n)
    ei = np.concatenate([iu[pick], perm[:-1]])
    ej = np.concatenate([ju[pick], perm[1:]])
    g = _loguniform(rng, glo, ghi, ei.size)
    ei, ej, g = _dedup_edges(ei, ej, g)
    rs = conductance_sums(n, ei, ej, g)
    grounded = rng.random(n) < p_ground
    grounded[rng.integers(n)] = True
    excess = np.where(grounded, rng.uniform(0.0, excess_hi, n) * rs, 0.0)
    return assemble(n, ei, ej, g, excess)


def rhs(n, nrhs, rng):
    """Right-hand sides ~ N(0,1), node-major float64 [n, nrhs]."""
    return np.ascontiguousarray(rng.standard_normal((n, nrhs)))


# ----------------------------------------------------------------------------
# The five benchmark workloads
# ----------------------------------------------------------------------------

CONFIGS = {
    1: dict(name="grid2d-5pt-32x32", walks=200, drop_tol=1e-3, tol=1e-8, nrhs=1,
            precision="fp64", gen_seed=0, walk_seed=0),
    2: dict(name="grid3d-7pt-64^3-logU[0.1,10]-excess1e-3", walks=500, drop_tol=1e-3,
            tol=1e-6, nrhs=4, precision="fp64", gen_seed=1, walk_seed=1),
    3: dict(name="grid2d-1000^2+2longrange", walks=200, drop_tol=1e-3, tol=1e-6, nrhs=1,
            precision="fp32", gen_seed=2, walk_seed=2),
    4: dict(name="rgg-256-batched", walks=200, drop_tol=1e-3, tol=1e-6, nrhs=16,
            precision="fp64", gen_seed=3, walk_seed=3, nmat=256),
    5: dict(name="grid3d-27pt-128^3-logU[0.1,10]-excess1e-4", walks=300, drop_tol=1e-3,
            tol=1e-6, nrhs=1, precision="fp32", gen_seed=4, walk_seed=4),
    6: dict(name="laplace3d-7pt-dirichlet-50^3..100^3", walks=20, drop_tol=None, tol=1e-6, nrhs=1,
            precision="fp64", gen_seed=5, walk_seed=5, edges=(50, 60, 70, 80, 90, 100)),
    7: dict(name="asym-grid3d-7pt-64^3-logU[0.1,10]-skew0.6", walks=300, drop_tol=1e-3, tol=1e-6, nrhs=1,
            precision="fp64", gen_seed=6, walk_seed=6),
}


def _rngs(seed):
    ss = np.random.SeedSequence(seed)
    a, b = ss.spawn(2)
    return np.random.default_rng(a), np.random.default_rng(b)


def make_config(i, scale=1.0, nmat=None):
    """Inputs for workload i (1..7).

    Returns dict(A=CSR or list of CSR, b=array or list, plus the settings of
    CONFIGS[i]).  `scale` < 1 shrinks the grid edge lengths (for quick tests);
    `nmat` overrides the number of matrices of workload 4.
    """
    cfg = dict(CONFIGS[i])
    rng_a, rng_b = _rngs(cfg["gen_seed"])
    if i == 1:
        A = grid2d_5pt(32, 32, boundary_excess=1.0)
        b = rhs(A.n, 1, np.random.default_rng(0))
    elif i == 2:
        m = max(4, int(round(64 * scale)))
        A = grid3d(m, m, m, 7, rng_a, excess_frac_hi=1e-3)
        b = rhs(A.n, cfg["nrhs"], rng_b)
    elif i == 3:
        m = max(8, int(round(1000 * scale)))
        A = grid2d_longrange(m, m, rng_a)
        b = rhs(A.n, 1, rng_b)
    elif i == 4:
        k = cfg["nmat"] if nmat is None else nmat
        sizes = np.exp(rng_a.uniform(math.log(1e3), math.log(2e5), k))
        sizes = np.maximum(16, np.round(sizes * scale)).astype(np.int64)
        A, b = [], []
        for j, nj in enumerate(sizes):
            r1, r2 = _rngs((cfg["gen_seed"], j))
            Aj = rgg(int(nj), r1)
            A.append(Aj)
            b.append(rhs(Aj.n, cfg["nrhs"], r2))
    elif i == 5:
        m = max(4, int(round(128 * scale)))
        A = grid3d(m, m, m, 27, rng_a, excess_frac=1e-4)
        b = rhs(A.n, 1, rng_b)
    elif i == 7:
        m = max(4, int(round(64 * scale)))
        A = asym_grid((m, m, m), rng_a, skew=0.6)
        b = rhs(A.n, 1, rng_b)[:, 0]
    elif i == 6:
        cfg["edges"] = tuple(max(4, int(round(e * scale))) for e in cfg["edges"])
        A = [laplace3d_dirichlet(e) for e in cfg["edges"]]
        b = [np.ones(a.n) for a in A]
    else:
        raise ValueError(f"unknown workload {i}")
    cfg["A"] = A
    cfg["b"] = b
    return cfg


def training_instance(j, edge=64):
    """Training matrix j (0..49) of the learned-budget workload: same
    distribution as workload 5 (27-point, log-uniform [0.1,10], excess 1e-4 *
    rowsum) at edge length `edge`, seed 100 + j."""
    rng_a, _ = _rngs(100 + j)
    return grid3d(edge, edge, edge, 27, rng_a, excess_frac=1e-4)
