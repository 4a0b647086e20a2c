"""Random-walk incomplete LDL^T preconditioner and PCG on GB300 (sm_103a).

Python binding of ``librwpc.so``: argument marshalling only.  Every step of the
factor construction and of the solve runs in the library's CUDA kernels; PyTorch
provides device memory (the tensors passed in and out) and streams.  There is no
CPU fallback: if the library is not built, ``load()`` raises.

The functions carry the C ABI's names (see ``include/rwpc.h``):
``rw_context_create``, ``rw_build_factor``, ``rw_build_factor_budget``,
``rw_factor_view``, ``rw_factor_destroy``, ``pcg_solve``, ``rw_precond_apply``,
``rw_spmv``, ``rw_status_string``, ``rw_last_error``.

Method: Qian & Sapatnekar, "Stochastic Preconditioning for Iterative Linear
Equation Solvers" -- walk game of Sec. 2.1, journey record of Sec. 3.1,
one-step-exact estimator of Sec. 5.2, PCG of Algorithm 1.
"""
from __future__ import annotations

import ctypes
import os
import weakref

from . import _build

__all__ = [
    "load", "RwError", "CSR", "Context", "Factor", "rw_options_default", "rw_context_create",
    "rw_build_factor_batched", "pcg_solve_batched",
    "rw_context_destroy", "rw_build_factor", "rw_build_factor_budget", "rw_factor_view",
    "rw_factor_destroy", "pcg_solve", "rw_precond_apply", "rw_precond_apply_static", "rw_spmv",
    "rw_status_string",
    "rw_last_error", "RW_FP64", "RW_FP32_MIXED",
    "Mlp", "rw_row_features", "rw_pilot_stats", "rw_mlp_create", "rw_mlp_predict",
    "rw_mlp_gradient", "rw_mlp_train", "rw_budget_normalize", "rw_budget_predict",
    "rw_adaptive_budget", "rw_csr_transpose", "rw_precond_apply_ldu", "bicgstab_solve",
    "RW_NUM_FEATURES", "RW_FEATURE_STRIDE", "RW_MLP_PARAMS",
    "Batch", "rw_batch_create", "pcg_solve_batch", "rw_autotune", "rw_batch_autotune", "rw_probe_latency",
    "rw_probe_gather",
    "rw_factor_save", "rw_factor_load", "rw_sha256", "rw_random_permutation", "rw_permute_csr",
]

RW_NUM_FEATURES = 12
RW_FEATURE_STRIDE = 16
RW_MLP_PARAMS = 5313

RW_FP64 = 0
RW_FP32_MIXED = 1
RW_OK = 0
STATUS = {0: "RW_OK", -1: "RW_ERR_ARG", -2: "RW_ERR_NOT_RMATRIX", -3: "RW_ERR_WALK_CAP",
          -4: "RW_ERR_ALLOC", -5: "RW_ERR_NO_CONVERGENCE", -6: "RW_ERR_BREAKDOWN",
          -7: "RW_ERR_CUDA", -8: "RW_ERR_TIMEOUT", -9: "RW_ERR_CAPACITY"}

_c_void_p = ctypes.c_void_p
_i32, _i64, _u32, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double


class rw_csr_t(ctypes.Structure):
    _fields_ = [("n", _i32), ("nnz", _i64), ("row_ptr", _c_void_p), ("col", _c_void_p),
                ("val", _c_void_p)]


class rw_options_t(ctypes.Structure):
    _fields_ = [("max_steps", _u64), ("keep_records", _i32), ("record_lengths", _i32),
                ("store_fp32", _i32), ("refine_every", _i32), ("walk_blocks_per_sm", _i32),
                ("timing", _i32), ("solve_blocks_per_sm", _i32), ("graphs", _i32),
                ("wide_slices", _i32), ("spmv_slices", _i32), ("cluster_width", _i32),
                ("cluster_size", _i32), ("solve_mode", _i32), ("reuse", _i32),
                ("solve_mode_bwd", _i32),
                ("thin_levels", _i32), ("thin_cluster", _i32), ("adapt_ahead", _i32),
                ("thin_flags", _i32), ("spin_limit", _i32), ("thin_lanes", _i32)]


class rw_factor_desc_t(ctypes.Structure):
    _fields_ = [("n", _i32), ("nnz", _i64), ("y_row_ptr", _c_void_p), ("y_col", _c_void_p),
                ("y_val", _c_void_p), ("d", _c_void_p), ("yt_row_ptr", _c_void_p),
                ("yt_col", _c_void_p), ("yt_val", _c_void_p), ("y_val32", _c_void_p),
                ("yt_val32", _c_void_p), ("d32", _c_void_p), ("walks", _c_void_p),
                ("visits", _c_void_p), ("ground", _c_void_p), ("walk_rows", _c_void_p),
                ("walk_base", _c_void_p), ("records", _c_void_p), ("n_walk_rows", _i32),
                ("total_walks", _i64), ("total_hops", _u64), ("fwd_levels", _i32),
                ("bwd_levels", _i32), ("phase_ms", ctypes.c_float * 8), ("kernel_launches", _i64),
                ("extra_walks", _i64), ("fwd_order", _c_void_p), ("fwd_level_ptr", _c_void_p),
                ("bwd_order", _c_void_p), ("bwd_level_ptr", _c_void_p)]


class rw_pcg_stats_t(ctypes.Structure):
    _fields_ = [("iterations", _i32), ("rel_residual", _f64), ("solve_ms", ctypes.c_float),
                ("spmv_ms", ctypes.c_float), ("bwd_ms", ctypes.c_float), ("fwd_ms", ctypes.c_float),
                ("kernel_launches", _i64)]


ALLOC_FN = ctypes.CFUNCTYPE(_c_void_p, _c_void_p, ctypes.c_size_t, _c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, _c_void_p, _c_void_p, ctypes.c_size_t, _c_void_p)

_lib = None


class RwError(RuntimeError):
    def __init__(self, code, where):
        msg = rw_last_error() if _lib is not None else ""
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code}): {msg}")
        self.code = code


def load():
    """Load librwpc.so (built by ``_build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library not built ({_build.LIB}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    lib.rw_options_default.argtypes = [P(rw_options_t)]
    lib.rw_options_default.restype = None
    lib.rw_context_create.argtypes = [P(_c_void_p), _c_void_p, ALLOC_FN, FREE_FN, _c_void_p,
                                      P(rw_options_t)]
    lib.rw_context_create.restype = ctypes.c_int
    lib.rw_context_destroy.argtypes = [_c_void_p]
    lib.rw_context_destroy.restype = None
    lib.rw_build_factor.argtypes = [_c_void_p, P(rw_csr_t), _u32, _u64, _f64, P(_c_void_p)]
    lib.rw_build_factor.restype = ctypes.c_int
    lib.rw_build_factor_budget.argtypes = [_c_void_p, P(rw_csr_t), _c_void_p, _u64, _f64,
                                           P(_c_void_p)]
    lib.rw_build_factor_budget.restype = ctypes.c_int
    lib.rw_build_factor_batched.argtypes = [_c_void_p, _i32, P(rw_csr_t), P(_c_void_p), _u32,
                                            P(_u64), _f64, P(_c_void_p)]
    lib.rw_build_factor_batched.restype = ctypes.c_int
    lib.rw_factor_view.argtypes = [_c_void_p, P(rw_factor_desc_t)]
    lib.rw_factor_view.restype = ctypes.c_int
    lib.rw_factor_destroy.argtypes = [_c_void_p]
    lib.rw_factor_destroy.restype = None
    lib.pcg_solve.argtypes = [_c_void_p, P(rw_csr_t), _c_void_p, _c_void_p, _c_void_p, _i32, _f64,
                              _i32, ctypes.c_int, P(rw_pcg_stats_t), _c_void_p, _c_void_p]
    lib.pcg_solve.restype = ctypes.c_int
    lib.pcg_solve_batched.argtypes = [_c_void_p, _i32, P(rw_csr_t), P(_c_void_p), P(_c_void_p),
                                      P(_c_void_p), _i32, _f64, _i32, ctypes.c_int,
                                      P(rw_pcg_stats_t), _c_void_p, _c_void_p]
    lib.pcg_solve_batched.restype = ctypes.c_int
    lib.rw_precond_apply.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i32]
    lib.rw_precond_apply.restype = ctypes.c_int
    lib.rw_precond_apply_static.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i32]
    lib.rw_precond_apply_static.restype = ctypes.c_int
    lib.rw_spmv.argtypes = [_c_void_p, P(rw_csr_t), _c_void_p, _c_void_p, _i32]
    lib.rw_spmv.restype = ctypes.c_int
    lib.rw_status_string.argtypes = [ctypes.c_int]
    lib.rw_status_string.restype = ctypes.c_char_p
    lib.rw_last_error.argtypes = []
    lib.rw_last_error.restype = ctypes.c_char_p
    vp = _c_void_p
    sigs = {
        "rw_row_features": [vp, P(rw_csr_t), vp],
        "rw_pilot_stats": [vp, P(rw_csr_t), _u32, _u64, _i32, vp, vp, vp, vp],
        "rw_mlp_create": [vp, _u64, P(vp)],
        "rw_mlp_params": [vp, vp, vp, vp, vp],
        "rw_mlp_predict": [vp, vp, vp, ctypes.c_int64, vp],
        "rw_mlp_gradient": [vp, vp, vp, vp, vp, ctypes.c_int64, vp, vp],
        "rw_mlp_train": [vp, vp, vp, vp, vp, ctypes.c_int64, _i32, _i32, ctypes.c_float, _u64, _i32, vp],
        "rw_budget_normalize": [vp, P(rw_csr_t), vp, _f64, _u32, vp],
        "rw_budget_predict": [vp, P(rw_csr_t), vp, _f64, _u32, vp],
        "rw_adaptive_budget": [vp, P(rw_csr_t), _u64, _f64, _f64, _u32, _u32, _i32, vp, P(_i32)],
        "rw_csr_transpose": [vp, P(rw_csr_t), vp, vp, vp],
        "rw_precond_apply_ldu": [vp, vp, vp, vp, vp, _i32],
        "bicgstab_solve": [vp, P(rw_csr_t), vp, vp, vp, vp, _f64, _i32, P(rw_pcg_stats_t)],
        "rw_batch_create": [vp, _i32, P(rw_csr_t), P(vp), P(vp)],
        "rw_batch_info": [vp, P(_i32), P(ctypes.c_int64), P(_i32), P(_i32)],
        "pcg_solve_batch": [vp, vp, P(vp), P(vp), _i32, _f64, _i32, ctypes.c_int, P(rw_pcg_stats_t), vp, vp],
        "rw_autotune": [vp, P(rw_csr_t), vp, _i32, ctypes.c_int, ctypes.c_char_p, P(rw_options_t), vp],
        "rw_batch_autotune": [vp, vp, _i32, ctypes.c_int, ctypes.c_char_p, P(rw_options_t), vp],
        "rw_probe_latency": [vp, _i32, P(_f64), P(_f64)],
        "rw_probe_gather": [vp, _u64, _i32, P(_f64)],
        "rw_factor_save": [vp, ctypes.c_char_p],
        "rw_factor_load": [vp, ctypes.c_char_p, P(vp)],
        "rw_random_permutation": [vp, _i32, _u64, vp],
        "rw_permute_csr": [vp, P(rw_csr_t), vp, vp, vp, vp],
    }
    for name, args in sigs.items():
        getattr(lib, name).argtypes = args
        getattr(lib, name).restype = ctypes.c_int
    lib.rw_mlp_destroy.argtypes = [vp]
    lib.rw_mlp_destroy.restype = None
    lib.rw_batch_destroy.argtypes = [vp]
    lib.rw_batch_destroy.restype = None
    lib.rw_sha256.argtypes = [vp, ctypes.c_size_t, vp]
    lib.rw_sha256.restype = None
    _lib = lib
    return lib


def _check(rc, where):
    if rc != RW_OK:
        raise RwError(rc, where)


def rw_status_string(code):
    return load().rw_status_string(code).decode()


def rw_last_error():
    return load().rw_last_error().decode()


def rw_options_default(**overrides):
    o = rw_options_t()
    load().rw_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# Device CSR held by torch tensors
# ---------------------------------------------------------------------------

class CSR:
    """Square CSR on the GPU: rowptr/col int32, val float64 (torch tensors)."""

    def __init__(self, rowptr, col, val):
        import torch
        for t, dt in ((rowptr, torch.int32), (col, torch.int32), (val, torch.float64)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise ValueError("CSR wants contiguous CUDA tensors int32/int32/float64")
        self.rowptr, self.col, self.val = rowptr, col, val
        self.n = rowptr.numel() - 1
        self.nnz = col.numel()
        self._c = rw_csr_t(self.n, self.nnz, rowptr.data_ptr(), col.data_ptr(), val.data_ptr())

    @classmethod
    def from_host(cls, A, device="cuda"):
        import torch
        return cls(torch.as_tensor(A.rowptr, dtype=torch.int32).to(device).contiguous(),
                   torch.as_tensor(A.col, dtype=torch.int32).to(device).contiguous(),
                   torch.as_tensor(A.val, dtype=torch.float64).to(device).contiguous())

    @property
    def c(self):
        return self._c


class _DevArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _dev_tensor(ptr, n, typestr):
    import torch
    dt = {"<i4": torch.int32, "<i8": torch.int64, "<u4": torch.int32, "<u8": torch.int64,
          "<f8": torch.float64, "<f4": torch.float32}[typestr]
    if not ptr or n == 0:
        return torch.empty(0, dtype=dt, device="cuda")
    t = torch.as_tensor(_DevArray(ptr, n, typestr), device="cuda")
    return t.view(dt) if t.dtype != dt else t


# ---------------------------------------------------------------------------
# Context and factor handles
# ---------------------------------------------------------------------------

class Context:
    """A library context bound to the current device and a CUDA stream.

    stream: a torch.cuda.Stream (default: the current stream).  With
    torch_allocator=True the library allocates its storage through PyTorch's
    caching allocator; with allocator=(alloc, free) through the two Python
    callables alloc(nbytes, stream_ptr) -> device pointer (int; 0 or None on
    failure) and free(ptr, nbytes, stream_ptr); otherwise through
    cudaMallocAsync on the stream.
    """

    def __init__(self, stream=None, options=None, torch_allocator=False, allocator=None):
        import torch
        lib = load()
        self.stream = stream or torch.cuda.current_stream()
        self.options = options or rw_options_default()
        self._keep = []
        self._factors = weakref.WeakSet()  # factors free through the context: close them first
        self._mlps = weakref.WeakSet()
        self._batches = weakref.WeakSet()
        if torch_allocator:
            dev = torch.cuda.current_device()

            def _alloc(user, size, stream_ptr):
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), dev, int(stream_ptr or 0))
                except Exception:
                    return None

            def _free(user, ptr, size, stream_ptr):
                torch.cuda.caching_allocator_delete(ptr)

            af, ff = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [af, ff]
        elif allocator is not None:
            user_alloc, user_free = allocator

            def _alloc2(user, size, stream_ptr):
                p = user_alloc(int(size), int(stream_ptr or 0))
                return int(p) if p else None

            def _free2(user, ptr, size, stream_ptr):
                user_free(int(ptr), int(size), int(stream_ptr or 0))

            af, ff = ALLOC_FN(_alloc2), FREE_FN(_free2)
            self._keep += [af, ff]
        else:
            af, ff = ALLOC_FN(), FREE_FN()
        h = _c_void_p()
        _check(lib.rw_context_create(ctypes.byref(h), _c_void_p(self.stream.cuda_stream), af, ff,
                                     None, ctypes.byref(self.options)), "rw_context_create")
        self.handle = h

    def close(self):
        if self.handle:
            for f in list(self._factors):
                f.destroy()
            for m in list(self._mlps):
                m.destroy()
            for b in list(self._batches):
                b.destroy()
            load().rw_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Factor:
    """Handle to a factor built on the GPU: A ~= Y^T diag(D) Y."""

    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.handle = handle
        ctx._factors.add(self)
        self.desc = rw_factor_view(self)

    def tensors(self):
        """Zero-copy torch views of the factor's device arrays (valid while the
        factor lives)."""
        d = self.desc
        n, nnz = d.n, d.nnz
        out = {
            "y_row_ptr": _dev_tensor(d.y_row_ptr, n + 1, "<i8"),
            "y_col": _dev_tensor(d.y_col, nnz, "<i4"),
            "y_val": _dev_tensor(d.y_val, nnz, "<f8"),
            "d": _dev_tensor(d.d, n, "<f8"),
            "yt_row_ptr": _dev_tensor(d.yt_row_ptr, n + 1, "<i8"),
            "yt_col": _dev_tensor(d.yt_col, nnz, "<i4"),
            "yt_val": _dev_tensor(d.yt_val, nnz, "<f8"),
            "walks": _dev_tensor(d.walks, n, "<u4"),
            "visits": _dev_tensor(d.visits, n, "<u8"),
            "ground": _dev_tensor(d.ground, n, "<u4"),
            "fwd_order": _dev_tensor(d.fwd_order, n, "<i4"),
            "fwd_level_ptr": _dev_tensor(d.fwd_level_ptr, d.fwd_levels + 1, "<i8"),
            "bwd_order": _dev_tensor(d.bwd_order, n, "<i4"),
            "bwd_level_ptr": _dev_tensor(d.bwd_level_ptr, d.bwd_levels + 1, "<i8"),
        }
        if d.y_val32:
            out["y_val32"] = _dev_tensor(d.y_val32, nnz, "<f4")
            out["yt_val32"] = _dev_tensor(d.yt_val32, nnz, "<f4")
            out["d32"] = _dev_tensor(d.d32, n, "<f4")
        if d.records:
            out["records"] = _dev_tensor(d.records, 2 * d.total_walks, "<i4")
            out["walk_rows"] = _dev_tensor(d.walk_rows, d.n_walk_rows, "<i4")
            out["walk_base"] = _dev_tensor(d.walk_base, d.n_walk_rows + 1, "<i8")
        return out

    def destroy(self):
        if self.handle and self.ctx.handle:
            rw_factor_destroy(self)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# C ABI entry points (same names)
# ---------------------------------------------------------------------------

def rw_context_create(stream=None, options=None, torch_allocator=False):
    return Context(stream, options, torch_allocator)


def rw_context_destroy(ctx):
    ctx.close()


def rw_build_factor(ctx, A, walks_per_row, seed, drop_tol):
    h = _c_void_p()
    _check(load().rw_build_factor(ctx.handle, ctypes.byref(A.c), int(walks_per_row), int(seed),
                                  float(drop_tol), ctypes.byref(h)), "rw_build_factor")
    return Factor(ctx, h)


def rw_build_factor_budget(ctx, A, budget, seed, drop_tol):
    """budget: CUDA int32/uint32 tensor [n] of walks per row."""
    h = _c_void_p()
    _check(load().rw_build_factor_budget(ctx.handle, ctypes.byref(A.c), _c_void_p(budget.data_ptr()),
                                         int(seed), float(drop_tol), ctypes.byref(h)),
           "rw_build_factor_budget")
    return Factor(ctx, h)


def rw_build_factor_batched(ctx, As, walks_per_row, seeds, drop_tol, budgets=None):
    """Factors of several matrices whose walks run in one launch; matrix m
    draws with matrix index m.  budgets: None or a list of CUDA budget tensors
    (entries may be None).  Returns a list of Factor."""
    nmat = len(As)
    arr = (rw_csr_t * nmat)(*[A.c for A in As])
    sd = (_u64 * nmat)(*[int(x) for x in seeds])
    outs = (_c_void_p * nmat)()
    bud = None
    if budgets is not None:
        bud = (_c_void_p * nmat)(*[(b.data_ptr() if b is not None else None) for b in budgets])
    _check(load().rw_build_factor_batched(ctx.handle, nmat, arr, bud, int(walks_per_row), sd,
                                          float(drop_tol), outs), "rw_build_factor_batched")
    return [Factor(ctx, _c_void_p(outs[m])) for m in range(nmat)]


def rw_factor_view(F):
    d = rw_factor_desc_t()
    _check(load().rw_factor_view(F.handle, ctypes.byref(d)), "rw_factor_view")
    return d


def rw_factor_destroy(F):
    load().rw_factor_destroy(F.handle)
    F.handle = None


def pcg_solve(ctx, A, F, b, x, tol, max_iter, prec=RW_FP64):
    """b, x: CUDA float64 tensors [n] or [n, nrhs] (node-major).  Returns
    (status, stats, iterations per rhs, true relative residual per rhs);
    raises on errors other than RW_ERR_NO_CONVERGENCE."""
    import numpy as np
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    st = rw_pcg_stats_t()
    its = np.zeros(nrhs, np.int32)
    rel = np.zeros(nrhs, np.float64)
    rc = load().pcg_solve(ctx.handle, ctypes.byref(A.c), F.handle, _c_void_p(b.data_ptr()),
                          _c_void_p(x.data_ptr()), nrhs, float(tol), int(max_iter), int(prec),
                          ctypes.byref(st), its.ctypes.data_as(_c_void_p),
                          rel.ctypes.data_as(_c_void_p))
    if rc not in (RW_OK, -5):
        raise RwError(rc, "pcg_solve")
    return rc, st, its, rel


def rw_csr_transpose(ctx, A):
    """A^T of a device CSR as a new device CSR (columns ascending)."""
    import torch
    dev = A.rowptr.device
    rp = torch.empty(A.n + 1, dtype=torch.int32, device=dev)
    col = torch.empty(A.nnz, dtype=torch.int32, device=dev)
    val = torch.empty(A.nnz, dtype=torch.float64, device=dev)
    _check(load().rw_csr_transpose(ctx.handle, ctypes.byref(A.c), _ptr(rp), _ptr(col), _ptr(val)),
           "rw_csr_transpose")
    return CSR(rp, col, val)


def rw_precond_apply_ldu(ctx, F_A, F_AT, r, z):
    """z = (Y_AT^T D Y_A)^-1 r with the factors of the games on A and A^T."""
    nrhs = 1 if r.dim() == 1 else r.shape[1]
    _check(load().rw_precond_apply_ldu(ctx.handle, F_A.handle, F_AT.handle, _c_void_p(r.data_ptr()),
                                       _c_void_p(z.data_ptr()), nrhs), "rw_precond_apply_ldu")


def bicgstab_solve(ctx, A, F_A, F_AT, b, x, tol, max_iter):
    """BiCGSTAB for a nonsymmetric A with the two-game preconditioner; b, x:
    CUDA float64 tensors [n].  Returns (status, stats); raises on errors other
    than RW_ERR_NO_CONVERGENCE."""
    st = rw_pcg_stats_t()
    rc = load().bicgstab_solve(ctx.handle, ctypes.byref(A.c), F_A.handle, F_AT.handle, _c_void_p(b.data_ptr()),
                               _c_void_p(x.data_ptr()), float(tol), int(max_iter), ctypes.byref(st))
    if rc not in (RW_OK, -5):
        raise RwError(rc, "bicgstab_solve")
    return rc, st


def pcg_solve_batched(ctx, As, Fs, bs, xs, tol, max_iter, prec=RW_FP64):
    """pcg_solve over several matrices; bs/xs: lists of CUDA tensors [n_m, nrhs].
    Returns (status, stats list, iterations [nmat, nrhs], relres [nmat, nrhs])."""
    import numpy as np
    nmat = len(As)
    nrhs = 1 if bs[0].dim() == 1 else bs[0].shape[1]
    arr = (rw_csr_t * nmat)(*[A.c for A in As])
    fh = (_c_void_p * nmat)(*[F.handle.value if hasattr(F.handle, "value") else F.handle for F in Fs])
    bp = (_c_void_p * nmat)(*[b.data_ptr() for b in bs])
    xp = (_c_void_p * nmat)(*[x.data_ptr() for x in xs])
    st = (rw_pcg_stats_t * nmat)()
    its = np.zeros((nmat, nrhs), np.int32)
    rel = np.zeros((nmat, nrhs), np.float64)
    rc = load().pcg_solve_batched(ctx.handle, nmat, arr, fh, bp, xp, nrhs, float(tol), int(max_iter),
                                  int(prec), st, its.ctypes.data_as(_c_void_p),
                                  rel.ctypes.data_as(_c_void_p))
    if rc not in (RW_OK, -5):
        raise RwError(rc, "pcg_solve_batched")
    return rc, list(st), its, rel


def rw_precond_apply(ctx, F, r, z):
    nrhs = 1 if r.dim() == 1 else r.shape[1]
    _check(load().rw_precond_apply(ctx.handle, F.handle, _c_void_p(r.data_ptr()),
                                   _c_void_p(z.data_ptr()), nrhs), "rw_precond_apply")


def rw_precond_apply_static(ctx, F, r, z):
    """rw_precond_apply without allocation (scratch in the library's static
    device array; n * nrhs <= 2**20; overlapping calls race)."""
    nrhs = 1 if r.dim() == 1 else r.shape[1]
    _check(load().rw_precond_apply_static(ctx.handle, F.handle, _c_void_p(r.data_ptr()),
                                          _c_void_p(z.data_ptr()), nrhs),
           "rw_precond_apply_static")


def rw_spmv(ctx, A, x, y):
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    _check(load().rw_spmv(ctx.handle, ctypes.byref(A.c), _c_void_p(x.data_ptr()),
                          _c_void_p(y.data_ptr()), nrhs), "rw_spmv")


# ---------------------------------------------------------------------------
# Learned walk budget
# ---------------------------------------------------------------------------

def _ptr(t):
    return _c_void_p(t.data_ptr())


class Mlp:
    """Handle to the budget network (12 -> 64 -> 64 -> 1) on the context's device."""

    def __init__(self, ctx, seed=0):
        self.ctx = ctx
        h = _c_void_p()
        _check(load().rw_mlp_create(ctx.handle, int(seed), ctypes.byref(h)), "rw_mlp_create")
        self.handle = h
        ctx._mlps.add(self)

    def params(self):
        """(parameter vector, standardisation vector) as numpy float32 arrays."""
        import numpy as np
        p = np.zeros(RW_MLP_PARAMS, np.float32)
        nrm = np.zeros(2 * RW_FEATURE_STRIDE, np.float32)
        _check(load().rw_mlp_params(self.handle, p.ctypes.data_as(_c_void_p),
                                    nrm.ctypes.data_as(_c_void_p), None, None), "rw_mlp_params")
        return p, nrm

    def set_params(self, params=None, norm=None):
        import numpy as np
        p = None if params is None else np.ascontiguousarray(params, np.float32)
        nrm = None if norm is None else np.ascontiguousarray(norm, np.float32)
        assert p is None or p.size == RW_MLP_PARAMS
        assert nrm is None or nrm.size == 2 * RW_FEATURE_STRIDE
        _check(load().rw_mlp_params(self.handle, None, None,
                                    None if p is None else p.ctypes.data_as(_c_void_p),
                                    None if nrm is None else nrm.ctypes.data_as(_c_void_p)),
               "rw_mlp_params")

    def save(self, path):
        import numpy as np
        p, nrm = self.params()
        np.savez(path, params=p, norm=nrm)

    def load_file(self, path):
        import numpy as np
        z = np.load(path)
        self.set_params(z["params"], z["norm"])

    def destroy(self):
        if self.handle and self.ctx.handle:
            load().rw_mlp_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def rw_mlp_create(ctx, seed=0):
    return Mlp(ctx, seed)


def rw_row_features(ctx, A, feat):
    """feat: CUDA float32 tensor [n, RW_FEATURE_STRIDE]."""
    _check(load().rw_row_features(ctx.handle, ctypes.byref(A.c), _ptr(feat)), "rw_row_features")


def rw_pilot_stats(ctx, A, pilot_walks, seed, mean, sd, label, has, quantity=0):
    """mean, sd, label, has: CUDA float32 tensors [n]; quantity 0 = walk
    lengths, 1 = visits to the start row (1 + returns)."""
    _check(load().rw_pilot_stats(ctx.handle, ctypes.byref(A.c), int(pilot_walks), int(seed), int(quantity),
                                 _ptr(mean), _ptr(sd), _ptr(label), _ptr(has)), "rw_pilot_stats")


def rw_mlp_predict(ctx, M, feat, out):
    _check(load().rw_mlp_predict(ctx.handle, M.handle, _ptr(feat), int(out.numel()), _ptr(out)),
           "rw_mlp_predict")


def rw_mlp_gradient(ctx, M, feat, label, rows):
    """Gradient (numpy float32 [RW_MLP_PARAMS]) and mean squared error over the
    rows listed in the CUDA int32/uint32 tensor `rows`."""
    import numpy as np
    g = np.zeros(RW_MLP_PARAMS, np.float32)
    loss = ctypes.c_float()
    _check(load().rw_mlp_gradient(ctx.handle, M.handle, _ptr(feat), _ptr(label), _ptr(rows),
                                  int(rows.numel()), g.ctypes.data_as(_c_void_p), ctypes.byref(loss)),
           "rw_mlp_gradient")
    return g, loss.value


def rw_mlp_train(ctx, M, feat, label, mask, epochs, batch, lr, seed=0, set_norm=True):
    """Adam training on the rows with mask > 0.  Returns the per-epoch mean
    squared error (numpy float32 [epochs])."""
    import numpy as np
    losses = np.zeros(max(1, epochs), np.float32)
    _check(load().rw_mlp_train(ctx.handle, M.handle, _ptr(feat), _ptr(label), _ptr(mask),
                               int(label.numel()), int(epochs), int(batch), float(lr), int(seed),
                               1 if set_norm else 0, losses.ctypes.data_as(_c_void_p)), "rw_mlp_train")
    return losses[:epochs]


def rw_budget_normalize(ctx, A, weight, mean_budget, min_budget, budget):
    """weight: CUDA float32 [n]; budget: CUDA int32/uint32 [n] (output)."""
    _check(load().rw_budget_normalize(ctx.handle, ctypes.byref(A.c), _ptr(weight), float(mean_budget),
                                      int(min_budget), _ptr(budget)), "rw_budget_normalize")


def rw_budget_predict(ctx, A, M, mean_budget, min_budget, budget):
    _check(load().rw_budget_predict(ctx.handle, ctypes.byref(A.c), M.handle, float(mean_budget),
                                    int(min_budget), _ptr(budget)), "rw_budget_predict")


def rw_adaptive_budget(ctx, A, seed, delta, z, min_walks, max_walks, max_rounds, budget):
    """Adaptive walk counts of Sec. 5.1 into the device uint32 tensor `budget`;
    returns the number of rounds run."""
    rounds = _i32()
    _check(load().rw_adaptive_budget(ctx.handle, ctypes.byref(A.c), _u64(int(seed)), float(delta), float(z),
                                     int(min_walks), int(max_walks), int(max_rounds), _ptr(budget),
                                     ctypes.byref(rounds)), "rw_adaptive_budget")
    return rounds.value


# ---------------------------------------------------------------------------
# Batched solves
# ---------------------------------------------------------------------------

class Batch:
    """Block-diagonal system of several matrices and their factors."""

    def __init__(self, ctx, As, Fs):
        self.ctx = ctx
        self.nmat = len(As)
        arr = (rw_csr_t * self.nmat)(*[A.c for A in As])
        fh = (_c_void_p * self.nmat)(*[F.handle.value if hasattr(F.handle, "value") else F.handle for F in Fs])
        h = _c_void_p()
        _check(load().rw_batch_create(ctx.handle, self.nmat, arr, fh, ctypes.byref(h)), "rw_batch_create")
        self.handle = h
        ctx._batches.add(self)

    def info(self):
        n, nnz, fl, bl = _i32(), ctypes.c_int64(), _i32(), _i32()
        _check(load().rw_batch_info(self.handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(fl),
                                    ctypes.byref(bl)), "rw_batch_info")
        return dict(n=n.value, nnz_y=nnz.value, fwd_levels=fl.value, bwd_levels=bl.value)

    def destroy(self):
        if self.handle and self.ctx.handle:
            load().rw_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def rw_batch_create(ctx, As, Fs):
    return Batch(ctx, As, Fs)


def pcg_solve_batch(ctx, B, bs, xs, tol, max_iter, prec=RW_FP64):
    """Returns (status, stats list, iterations [nmat, nrhs], relres [nmat, nrhs])."""
    import numpy as np
    nmat = B.nmat
    nrhs = 1 if bs[0].dim() == 1 else bs[0].shape[1]
    bp = (_c_void_p * nmat)(*[b.data_ptr() for b in bs])
    xp = (_c_void_p * nmat)(*[x.data_ptr() for x in xs])
    st = (rw_pcg_stats_t * nmat)()
    its = np.zeros((nmat, nrhs), np.int32)
    rel = np.zeros((nmat, nrhs), np.float64)
    rc = load().pcg_solve_batch(ctx.handle, B.handle, bp, xp, nrhs, float(tol), int(max_iter), int(prec), st,
                                its.ctypes.data_as(_c_void_p), rel.ctypes.data_as(_c_void_p))
    if rc not in (RW_OK, -5):
        raise RwError(rc, "pcg_solve_batch")
    return rc, list(st), its, rel


# ---------------------------------------------------------------------------
# Schedule autotuner
# ---------------------------------------------------------------------------

_TUNED = ("solve_mode", "solve_mode_bwd", "wide_slices", "solve_blocks_per_sm", "cluster_width", "spmv_slices",
          "thin_cluster", "thin_flags", "thin_lanes")


def _tune_result(ctx, opt, ms):
    for k in _TUNED:
        setattr(ctx.options, k, getattr(opt, k))
    return {k: getattr(opt, k) for k in _TUNED}, (float(ms[0]), float(ms[1]))


def rw_autotune(ctx, A, F, nrhs, prec=RW_FP64, cache_path=None):
    """Time the candidate solve / SpMV launch shapes on this factor and install
    the fastest in the context.  Returns (chosen options, (precond ms, spmv ms))
    -- times are 0 when the choice came from the cache file."""
    import numpy as np
    opt = rw_options_t()
    ms = np.zeros(2, np.float32)
    _check(load().rw_autotune(ctx.handle, ctypes.byref(A.c), F.handle, int(nrhs), int(prec),
                              cache_path.encode() if cache_path else None, ctypes.byref(opt),
                              ms.ctypes.data_as(_c_void_p)), "rw_autotune")
    return _tune_result(ctx, opt, ms)


def rw_probe_latency(ctx, iters=20000):
    """(SM-to-SM hand-off through L2 in ns, dependent L2-hit load in ns): the two
    latencies that bound a triangular solve's dependency chain."""
    h, l2 = _f64(0.0), _f64(0.0)
    _check(load().rw_probe_latency(ctx.handle, int(iters), ctypes.byref(h), ctypes.byref(l2)), "rw_probe_latency")
    return float(h.value), float(l2.value)


def rw_probe_gather(ctx, buffer_bytes, access_bytes=32):
    """Random-gather throughput (GB/s of accessed bytes) over a device buffer
    of buffer_bytes, in aligned units of access_bytes (32, 64 or 128)."""
    g = _f64(0.0)
    _check(load().rw_probe_gather(ctx.handle, int(buffer_bytes), int(access_bytes), ctypes.byref(g)),
           "rw_probe_gather")
    return float(g.value)


def rw_batch_autotune(ctx, B, nrhs, prec=RW_FP64, cache_path=None):
    import numpy as np
    opt = rw_options_t()
    ms = np.zeros(2, np.float32)
    _check(load().rw_batch_autotune(ctx.handle, B.handle, int(nrhs), int(prec),
                                    cache_path.encode() if cache_path else None, ctypes.byref(opt),
                                    ms.ctypes.data_as(_c_void_p)), "rw_batch_autotune")
    return _tune_result(ctx, opt, ms)


# ---------------------------------------------------------------------------
# Factor files and orderings
# ---------------------------------------------------------------------------

def rw_factor_save(F, path):
    _check(load().rw_factor_save(F.handle, str(path).encode()), "rw_factor_save")


def rw_factor_load(ctx, path):
    h = _c_void_p()
    _check(load().rw_factor_load(ctx.handle, str(path).encode(), ctypes.byref(h)), "rw_factor_load")
    return Factor(ctx, h)


def rw_sha256(data: bytes) -> bytes:
    out = ctypes.create_string_buffer(32)
    buf = ctypes.create_string_buffer(data, len(data))
    load().rw_sha256(ctypes.cast(buf, _c_void_p), len(data), ctypes.cast(out, _c_void_p))
    return out.raw


def rw_random_permutation(ctx, n, seed, perm):
    """perm: CUDA int32 tensor [n] (new index of each old index)."""
    _check(load().rw_random_permutation(ctx.handle, int(n), int(seed), _ptr(perm)), "rw_random_permutation")


def rw_permute_csr(ctx, A, perm):
    """B = P A P^T as a new device CSR."""
    import torch
    rp = torch.empty(A.n + 1, dtype=torch.int32, device=A.rowptr.device)
    col = torch.empty(A.nnz, dtype=torch.int32, device=A.rowptr.device)
    val = torch.empty(A.nnz, dtype=torch.float64, device=A.rowptr.device)
    _check(load().rw_permute_csr(ctx.handle, ctypes.byref(A.c), _ptr(perm), _ptr(rp), _ptr(col), _ptr(val)),
           "rw_permute_csr")
    return CSR(rp, col, val)
