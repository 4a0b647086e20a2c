"""Failure detection without a GPU fault.

* Bounded device-side waits: with rw_options.spin_limit set to two polls, the
  waits of the level computation (factor build) and of the sync-free solve
  give up almost at once; the call returns RW_ERR_TIMEOUT instead of hanging,
  and the device and the library stay usable (a normal context afterwards
  gets the oracle's results).
* Allocation failures: a context whose allocator fails on its N-th call makes
  every entry point return RW_ERR_ALLOC for every N up to the number of
  allocations a successful call makes, with nothing left allocated, and the
  same context works again once the allocator does.
"""
import time

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

RW_ERR_ALLOC, RW_ERR_TIMEOUT = -4, -8


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_math_0609672_gb300 as P
    from paper_math_0609672_gb300 import _build
    _build.build()
    return P


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_short_wait_limit_returns_timeout(P):
    A = W.tridiag(3000, diag=2.0 + 1e-3)   # a chain: every level waits for the one before
    dA = P.CSR.from_host(A)
    normal = P.Context()
    F = P.rw_build_factor(normal, dA, 20, 3, 0.0)
    assert F.desc.fwd_levels > 1000
    short = P.Context(options=P.rw_options_default(spin_limit=2, solve_mode=1))
    t0 = time.perf_counter()
    with pytest.raises(P.RwError) as e:
        P.rw_build_factor(short, dA, 20, 3, 0.0)
    assert e.value.code == RW_ERR_TIMEOUT
    r = np.random.default_rng(0).standard_normal(A.n)
    z = _dev(np.zeros(A.n))
    with pytest.raises(P.RwError) as e:
        P.rw_precond_apply(short, F, _dev(r), z)
    assert e.value.code == RW_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the device and the library are still usable: the normal context gets the
    # oracle's preconditioner, and the short-limit context still runs calls
    # that do not wait
    P.rw_precond_apply(normal, F, _dev(r), z)
    ref = oracle.build_factor(A, 20, 3, 0.0)
    zr = oracle.precond_apply(ref, r)
    assert np.linalg.norm(z.cpu().numpy() - zr) / np.linalg.norm(zr) < 1e-12
    y = _dev(np.zeros(A.n))
    P.rw_spmv(short, dA, _dev(r), y)
    assert np.allclose(y.cpu().numpy(), A.to_scipy() @ r, rtol=1e-13, atol=1e-13)
    F.destroy()
    short.close()
    normal.close()


class FailingAllocator:
    """Device allocations from PyTorch's caching allocator; the N-th call
    (counting from reset) fails.  Tracks what is outstanding."""

    def __init__(self):
        import torch
        self.torch = torch
        self.dev = torch.cuda.current_device()
        self.fail_at = 0
        self.calls = 0
        self.live = {}

    def reset(self, fail_at=0):
        self.fail_at = fail_at
        self.calls = 0

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.fail_at and self.calls == self.fail_at:
            return 0
        p = self.torch.cuda.caching_allocator_alloc(nbytes, self.dev, stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, nbytes, stream):
        assert ptr in self.live, "free of a pointer the allocator did not hand out"
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)


def _points(count, most=24):
    if count <= most:
        return list(range(1, count + 1))
    return sorted(set(np.linspace(1, count, most).round().astype(int).tolist()))


def test_allocation_failures_are_clean(P):
    import torch
    cfg = W.make_config(2, scale=0.2)
    A, b = cfg["A"], cfg["b"]
    dA = P.CSR.from_host(A)
    db = _dev(b)
    mats = [W.rgg(700, np.random.default_rng(3)), W.rgg(400, np.random.default_rng(4))]
    dms = [P.CSR.from_host(M) for M in mats]
    bms = [_dev(np.random.default_rng(5).standard_normal((M.n, 2))) for M in mats]
    path = "/tmp/rwpc_alloc_test.fac"

    def run(ctx, name, aux):
        if name == "build":
            return [P.rw_build_factor(ctx, dA, 40, 1, 1e-3)]
        if name == "build_budget":
            bud = torch.full((A.n,), 30, dtype=torch.int32, device="cuda")
            return [P.rw_build_factor_budget(ctx, dA, bud, 1, 1e-3)]
        if name == "build_batched":
            return P.rw_build_factor_batched(ctx, dms, 30, [1, 2], 1e-3)
        if name == "pcg_fp64":
            P.pcg_solve(ctx, dA, aux["F"], db, _dev(np.zeros_like(b)), 1e-6, 200)
        elif name == "pcg_fp32":
            P.pcg_solve(ctx, dA, aux["F"], db, _dev(np.zeros_like(b)), 1e-6, 200, P.RW_FP32_MIXED)
        elif name == "precond":
            P.rw_precond_apply(ctx, aux["F"], db, _dev(np.zeros_like(b)))
        elif name == "batch":
            B = P.Batch(ctx, dms, aux["Fm"])
            try:
                P.pcg_solve_batch(ctx, B, bms, [torch.zeros_like(x) for x in bms], 1e-6, 200)
            finally:
                B.destroy()
        elif name == "pilot":
            out = [torch.zeros(A.n, device="cuda") for _ in range(4)]
            P.rw_pilot_stats(ctx, dA, 8, 3, *out, quantity=2)
        elif name == "adaptive":
            bud = torch.zeros(A.n, dtype=torch.int32, device="cuda")
            P.rw_adaptive_budget(ctx, dA, 1, 0.5, 2.576, 20, 200, 4, bud)
        elif name == "features_predict":
            bud = torch.zeros(A.n, dtype=torch.int32, device="cuda")
            P.rw_budget_predict(ctx, dA, aux["M"], 50.0, 20, bud)
        elif name == "train":
            f = torch.zeros((A.n, 16), device="cuda")
            P.rw_row_features(ctx, dA, f)
            y = torch.ones(A.n, device="cuda")
            P.rw_mlp_train(ctx, aux["M"], f, y, torch.ones(A.n, device="cuda"), 1, 256, 1e-3)
        elif name == "load":
            return [P.rw_factor_load(ctx, path)]
        return []

    names = ["build", "build_budget", "build_batched", "pcg_fp64", "pcg_fp32", "precond", "batch", "pilot",
             "adaptive", "features_predict", "train", "load"]
    fa = FailingAllocator()
    ctx = P.Context(allocator=(fa.alloc, fa.free))
    aux = {"F": P.rw_build_factor(ctx, dA, 40, 1, 1e-3), "Fm": P.rw_build_factor_batched(ctx, dms, 30, [1, 2], 1e-3),
           "M": P.Mlp(ctx, seed=0)}
    P.rw_factor_save(aux["F"], path)
    for name in names:
        torch.cuda.synchronize()
        base = dict(fa.live)
        fa.reset()
        made = run(ctx, name, aux)
        count = fa.calls
        for o in made:
            o.destroy()
        assert fa.live == base, name
        assert count >= 1, name
        for nth in _points(count):
            fa.reset(fail_at=nth)
            with pytest.raises(P.RwError) as e:
                run(ctx, name, aux)
            assert e.value.code == RW_ERR_ALLOC, (name, nth, e.value)
            torch.cuda.synchronize()
            assert fa.live == base, (name, nth, len(fa.live) - len(base))
        # the context works again once the allocator does
        fa.reset()
        for o in run(ctx, name, aux):
            o.destroy()
        assert fa.live == base, name
    aux["F"].destroy()
    for F in aux["Fm"]:
        F.destroy()
    aux["M"].destroy()
    ctx.close()
    assert not fa.live
