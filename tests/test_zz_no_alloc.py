"""The allocation-free preconditioner entry point, through the C ABI.

rw_precond_apply_static exists for callers that cannot allocate device memory
when they apply the preconditioner (an outer solver calling it every
iteration, a fixed memory budget, an allocator that must not be re-entered).
Its scratch is a static device array shared by all calls; two calls in a row
must each give the same result as the allocating rw_precond_apply.  This file
is collected last so that a stopping run has already run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_matches_allocating_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_math_0609672_gb300 as P
    from paper_math_0609672_gb300 import _build
    _build.build()
    ctx = P.Context()
    A = W.make_config(2, scale=0.25)["A"]          # n = 4096
    dA = P.CSR.from_host(A)
    F = P.rw_build_factor(ctx, dA, 100, 5, 1e-3)
    rng = np.random.default_rng(3)
    for call, nrhs in enumerate((4, 3)):           # two calls in a row, different shapes
        r = torch.as_tensor(rng.standard_normal((A.n, nrhs)), device="cuda")
        z_ref = torch.zeros_like(r)
        z = torch.full_like(r, 7.0)                 # stale values must not leak through
        P.rw_precond_apply(ctx, F, r, z_ref)
        P.rw_precond_apply_static(ctx, F, r, z)
        zr, zs = z_ref.cpu().numpy(), z.cpu().numpy()
        for j in range(nrhs):
            rel = np.linalg.norm(zs[:, j] - zr[:, j]) / np.linalg.norm(zr[:, j])
            assert rel < 1e-12, (call, j, rel)
    # sizes beyond the static array (2**20 entries) are refused before any device work
    B = W.grid2d_5pt(300, 300)                      # 90000 * 16 > 2**20
    FB = P.rw_build_factor(ctx, P.CSR.from_host(B), 2, 1, 1e-2)
    big = torch.zeros((B.n, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(P.RwError) as e:
        P.rw_precond_apply_static(ctx, FB, big, big.clone())
    assert e.value.code == -9
    FB.destroy()
    F.destroy()
    ctx.close()
