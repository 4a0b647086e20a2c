// rw_levels.cu -- dependency levels of the two triangular systems.
//
// The paper applies the factor by plain forward/backward substitution
// (Sec. 4).  On the GPU the rows are solved in an order where every row comes
// after all rows it depends on: rows sorted by their level in the dependency
// DAG (level 0 = no dependency).  Forward solve Y z = v: row k depends on the
// columns of row k of Y.  Backward solve Y^T w = r: row i depends on the
// columns of row i of Y^T (all larger than i).
#include "rw_internal.h"

namespace rw {

// One warp per row, rows claimed 32 at a time in dependency order (ascending
// for the lower factor, descending for the upper).  A row waits for the levels
// of its dependencies, which belong to earlier claims, so every wait ends;
// each wait is nevertheless bounded.
__global__ void __launch_bounds__(256) k_levels(int32_t n, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, int descending,
                                                int* lev, unsigned* cursor, int* maxlev,
                                                DevStatus* st) {
    const unsigned lane = lane_id();
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(cursor, 32u);
        base = __shfl_sync(kFull, base, 0);
        if (base >= (unsigned)n) break;
        const unsigned cnt = min(32u, (unsigned)n - base);
        for (unsigned j = 0; j < cnt; ++j) {
            const int32_t row = descending ? n - 1 - (int32_t)(base + j) : (int32_t)(base + j);
            const int64_t s = rp[row], e = rp[row + 1];
            int m = -1;
            for (int64_t p = s + lane; p < e; p += 32) {
                const int32_t c = col[p];
                int v;
                unsigned spins = 0;
                while ((v = ld_relaxed(&lev[c])) < 0) {
                    if (wait_gives_up(spins, &st->timeout)) {
                        v = 0;
                        break;
                    }
                }
                m = max(m, v);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
            if (lane == 0) {
                st_relaxed(&lev[row], m + 1);
                atomicMax(maxlev, m + 1);
            }
            __syncwarp();
        }
    }
}

__global__ void k_level_hist(int32_t n, const int* __restrict__ lev, uint32_t* cnt) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&cnt[lev[i]], 1u);
}

__global__ void k_level_scatter(int32_t n, const int* __restrict__ lev,
                                const int64_t* __restrict__ lptr, uint32_t* fill, int32_t* order) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int l = lev[i];
        order[lptr[l] + atomicAdd(&fill[l], 1u)] = i;
    }
}

rw_status compute_levels(rw_context* ctx, int32_t n, const int64_t* rp, const int32_t* col,
                         bool descending, int32_t* order, int32_t* depth, Pool& scratch) {
    cudaStream_t s = ctx->stream;
    *depth = 0;
    if (n == 0) return RW_OK;
    int* lev = alloc_n<int>(scratch, n);
    unsigned* cursor = alloc_n<unsigned>(scratch, 2);
    uint32_t* cnt = alloc_n<uint32_t>(scratch, n + 1);
    int64_t* lptr = alloc_n<int64_t>(scratch, n + 1);
    if (!lev || !cursor || !cnt || !lptr) return RW_ERR_ALLOC;
    rw_status rc;
    if ((rc = check_cuda(cudaMemsetAsync(lev, 0xFF, sizeof(int) * (size_t)n, s), "memset"))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(cursor, 0, 2 * sizeof(unsigned), s), "memset"))) return rc;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels, 256, 0);
    if (per_sm < 1) per_sm = 1;
    const int blocks = grid_for(((int64_t)n + 31) / 32 * 32, 256, ctx->num_sms * per_sm);
    k_levels<<<blocks, 256, 0, s>>>(n, rp, col, descending ? 1 : 0, lev, cursor,
                                     reinterpret_cast<int*>(cursor + 1), ctx->d_status);
    if ((rc = check_launch("levels"))) return rc;
    int* hs = static_cast<int*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(hs, cursor + 1, 4, cudaMemcpyDeviceToHost, s), "copy")))
        return rc;
    if ((rc = read_status(ctx, "levels"))) return rc;
    const int nlev = hs[0] + 1;
    *depth = nlev;
    if ((rc = check_cuda(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(nlev + 1), s),
                         "memset")))
        return rc;
    const int blocks2 = grid_for(n, 256, ctx->num_sms * 8);
    k_level_hist<<<blocks2, 256, 0, s>>>(n, lev, cnt);
    if ((rc = check_launch("level histogram"))) return rc;
    if ((rc = check_cuda(scan_u32_to_i64(cnt, lptr, nlev, s, scratch), "scan"))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(nlev + 1), s),
                         "memset")))
        return rc;
    k_level_scatter<<<blocks2, 256, 0, s>>>(n, lev, lptr, cnt, order);
    return check_launch("level scatter");
}

}  // namespace rw
