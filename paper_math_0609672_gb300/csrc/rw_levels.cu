// rw_levels.cu -- dependency levels of the two triangular systems.
//
// The paper applies the factor by plain forward/backward substitution
// (Sec. 4).  On the GPU a triangular solve visits rows in an order where every
// row comes after the rows it depends on; this file computes each row's level
// in the dependency DAG (level 0 = no dependency; level = 1 + the largest
// level among its dependencies) and the rows sorted by level.  Forward solve
// Y z = v: row k depends on the columns of row k of Y (all < k).  Backward
// solve Y^T w = r: row i depends on the columns of row i of Y^T (all > i).
//
// The levels are computed sync-free in natural order (ascending for Y,
// descending for Y^T, both topological): a co-resident grid, warp w takes rows
// w, w + NW, ...; a row waits (bounded) until the levels of its dependencies
// are published.  With more than a thousand warps in flight the time is close
// to depth x one L2 round trip.
#include "rw_internal.h"

namespace rw {

__global__ void __launch_bounds__(256) k_levels(int32_t n, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, int descending,
                                                int* lev, int* maxlev, DevStatus* st) {
    const int lane = (int)lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int my_max = -1;
    for (int64_t pos = gw; pos < n; pos += nw) {
        const int32_t row = descending ? n - 1 - (int32_t)pos : (int32_t)pos;
        const int64_t s = rp[row], e = rp[row + 1];
        int m = -1;
        for (int64_t p = s + lane; p < e; p += 32) {
            const int32_t c = col[p];
            int v = ld_relaxed(&lev[c]);
            unsigned spins = 0;
            while (v < 0) {
                if (wait_gives_up(spins, &st->timeout)) {
                    v = 0;
                    break;
                }
                __nanosleep(20);
                v = ld_relaxed(&lev[c]);
            }
            m = max(m, v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
        if (lane == 0) st_relaxed(&lev[row], m + 1);
        my_max = max(my_max, m + 1);
    }
    if (lane == 0 && my_max >= 0) atomicMax(maxlev, my_max);
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
                         bool descending, int32_t* order, int32_t* depth, int64_t** lptr_out,
                         Pool& keep, Pool& scratch) {
    cudaStream_t s = ctx->stream;
    *depth = 0;
    *lptr_out = nullptr;
    if (n == 0) return RW_OK;
    int* lev = alloc_n<int>(scratch, n);
    int* maxlev = alloc_n<int>(scratch, 1);
    uint32_t* cnt = alloc_n<uint32_t>(scratch, n + 1);
    int64_t* lptr = alloc_n<int64_t>(keep, n + 1);
    if (!lev || !maxlev || !cnt || !lptr) return RW_ERR_ALLOC;
    rw_status rc;
    if ((rc = check_cuda(cudaMemsetAsync(lev, 0xFF, sizeof(int) * (size_t)n, s), "memset"))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(maxlev, 0, sizeof(int), s), "memset"))) return rc;
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels, 256, 0);
        if (per_sm < 1) per_sm = 1;
    }
    int64_t blocks = (int64_t)per_sm * ctx->num_sms;
    const int64_t need = ((int64_t)n + 7) / 8;
    if (blocks > need) blocks = need;
    int desc = descending ? 1 : 0;
    DevStatus* st = ctx->d_status;
    void* args[] = {(void*)&n, (void*)&rp, (void*)&col, (void*)&desc, (void*)&lev, (void*)&maxlev,
                    (void*)&st};
    RW_COUNT_LAUNCH();
    if ((rc = check_cuda(cudaLaunchCooperativeKernel((const void*)k_levels, dim3((unsigned)blocks),
                                                     dim3(256), args, 0, s),
                         "levels launch")))
        return rc;
    int* hs = static_cast<int*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(hs, maxlev, 4, cudaMemcpyDeviceToHost, s), "copy")))
        return rc;
    if ((rc = read_status(ctx, "levels"))) return rc;
    const int nlev = hs[0] + 1;
    *depth = nlev;
    if ((rc = check_cuda(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(nlev + 1), s),
                         "memset")))
        return rc;
    const int blocks2 = grid_for(n, 256, ctx->num_sms * 8);
    RW_COUNT_LAUNCH();
    k_level_hist<<<blocks2, 256, 0, s>>>(n, lev, cnt);
    if ((rc = check_launch("level histogram"))) return rc;
    if ((rc = check_cuda(scan_u32_to_i64(cnt, lptr, nlev, s, scratch), "scan"))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(nlev + 1), s),
                         "memset")))
        return rc;
    RW_COUNT_LAUNCH();
    k_level_scatter<<<blocks2, 256, 0, s>>>(n, lev, lptr, cnt, order);
    *lptr_out = lptr;
    return check_launch("level scatter");
}

}  // namespace rw
