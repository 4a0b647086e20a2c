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
// are published.  The two DAGs share one launch (even warps on Y, odd warps on
// Y^T), so their depth x L2-round-trip chains overlap instead of adding up.
#include "rw_internal.h"

namespace rw {

// One DAG of a level computation.
struct LevelJob {
    const int64_t* rp;
    const int32_t* col;
    int descending;
    int* lev;
    int* maxlev;
};

// Levels of one or two DAGs in one co-resident launch: with two jobs the even
// warps walk the first DAG and the odd warps the second, each in its own
// topological order, so the two latency chains overlap.
__global__ void __launch_bounds__(256) k_levels(int32_t n, const LevelJob J0, const LevelJob J1, int njobs,
                                                DevStatus* st) {
    const int lane = (int)lane_id();
    const int64_t gw0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw0 = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int job = njobs == 2 ? (int)(gw0 & 1) : 0;
    const int64_t gw = njobs == 2 ? gw0 >> 1 : gw0;
    const int64_t nw = njobs == 2 ? nw0 >> 1 : nw0;
    const LevelJob& J = job ? J1 : J0;
    const int64_t* __restrict__ rp = J.rp;
    const int32_t* __restrict__ col = J.col;
    int* lev = J.lev;
    const unsigned limit = st->spin_limit;
    int my_max = -1;
    for (int64_t pos = gw; pos < n; pos += nw) {
        const int32_t row = J.descending ? n - 1 - (int32_t)pos : (int32_t)pos;
        const int64_t s = rp[row], e = rp[row + 1];
        int m = -1;
        for (int64_t p = s + lane; p < e; p += 32) {
            const int32_t c = col[p];
            int v = ld_relaxed(&lev[c]);
            unsigned spins = 0;
            while (v < 0) {
                if (wait_gives_up(spins, limit, &st->timeout)) {
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
    if (lane == 0 && my_max >= 0) atomicMax(J.maxlev, my_max);
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

// Histogram of the levels, their boundaries and the rows sorted by level.
static rw_status level_order(rw_context* ctx, int32_t n, const int* lev, int nlev, int32_t* order, int64_t* lptr,
                             uint32_t* cnt, Pool& scratch) {
    cudaStream_t s = ctx->stream;
    rw_status rc;
    if ((rc = check_cuda(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(nlev + 1), s), "memset")))
        return rc;
    const int blocks2 = grid_for(n, 256, ctx->num_sms * 8);
    RW_COUNT_LAUNCH();
    k_level_hist<<<blocks2, 256, 0, s>>>(n, lev, cnt);
    if ((rc = check_launch("level histogram"))) return rc;
    if ((rc = check_cuda(scan_u32_to_i64(cnt, lptr, nlev, s, scratch), "scan"))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(nlev + 1), s), "memset")))
        return rc;
    RW_COUNT_LAUNCH();
    k_level_scatter<<<blocks2, 256, 0, s>>>(n, lev, lptr, cnt, order);
    return check_launch("level scatter");
}

rw_status compute_levels_pair(rw_context* ctx, int32_t n, const LevelDag& fwd, const LevelDag& bwd, Pool& keep,
                              Pool& scratch) {
    NvtxRange nvtx_range("rw_levels");
    cudaStream_t s = ctx->stream;
    *fwd.depth = 0;
    *bwd.depth = 0;
    *fwd.lptr_out = nullptr;
    *bwd.lptr_out = nullptr;
    if (n == 0) return RW_OK;
    int* lev = alloc_n<int>(scratch, 2 * (int64_t)n);
    int* maxlev = alloc_n<int>(scratch, 2);
    uint32_t* cnt = alloc_n<uint32_t>(scratch, n + 1);
    int64_t* lptr_f = alloc_n<int64_t>(keep, n + 1);
    int64_t* lptr_b = alloc_n<int64_t>(keep, n + 1);
    if (!lev || !maxlev || !cnt || !lptr_f || !lptr_b) return RW_ERR_ALLOC;
    rw_status rc;
    if ((rc = check_cuda(cudaMemsetAsync(lev, 0xFF, sizeof(int) * 2 * (size_t)n, s), "memset"))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(maxlev, 0, 2 * sizeof(int), s), "memset"))) return rc;
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels, 256, 0);
        if (per_sm < 1) per_sm = 1;
    }
    int64_t blocks = (int64_t)per_sm * ctx->num_sms;
    const int64_t need = ((int64_t)n + 3) / 4;  // two jobs: 8 warps per block, 4 per DAG
    if (blocks > need) blocks = need;
    LevelJob J0{fwd.rp, fwd.col, fwd.descending ? 1 : 0, lev, maxlev};
    LevelJob J1{bwd.rp, bwd.col, bwd.descending ? 1 : 0, lev + n, maxlev + 1};
    int njobs = 2;
    DevStatus* st = ctx->d_status;
    void* args[] = {(void*)&n, (void*)&J0, (void*)&J1, (void*)&njobs, (void*)&st};
    RW_COUNT_LAUNCH();
    if ((rc = check_cuda(cudaLaunchCooperativeKernel((const void*)k_levels, dim3((unsigned)blocks), dim3(256),
                                                     args, 0, s),
                         "levels launch")))
        return rc;
    int* hs = static_cast<int*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(hs, maxlev, 8, cudaMemcpyDeviceToHost, s), "copy"))) return rc;
    if ((rc = read_status(ctx, "levels"))) return rc;
    *fwd.depth = hs[0] + 1;
    *bwd.depth = hs[1] + 1;
    if ((rc = level_order(ctx, n, lev, *fwd.depth, fwd.order, lptr_f, cnt, scratch)) ||
        (rc = level_order(ctx, n, lev + n, *bwd.depth, bwd.order, lptr_b, cnt, scratch)))
        return rc;
    *fwd.lptr_out = lptr_f;
    *bwd.lptr_out = lptr_b;
    return RW_OK;
}

}  // namespace rw
