// rw_adapt.cu -- the adaptive walk count of Sec. 5.1.
//
// The paper runs walks from row k until the mean walk length Xi'_k of its M_k
// walks is within a relative margin Delta of its expectation at confidence
// alpha (Eq. lengthdelta), checked as Delta Xi'_k sqrt(M_k) / sigma_k > z with
// z = Q^-1((1 - alpha)/2), with a lower bound on M_k.  Here all rows advance
// together in rounds: every walk row starts with min_walks walks; after each
// round a row whose walks do not yet meet the criterion gets the number its
// current estimates ask for, z^2 sigma^2 / (Delta^2 Xi'^2) (at least one more,
// at most max_walks in total), and the next round runs walks M, M+1, ... of
// exactly those rows.  A walk is a function of (seed, row, walk index) only, so
// the factor built afterwards with these counts consists of the very walks
// that fixed them.  The sums of lengths and squared lengths are exact
// integers and the test is evaluated in FP64 with every operation rounded
// once, so the counts are reproducible bit for bit.
#include <cmath>
#include <vector>

#include "rw_internal.h"

namespace rw {

// Adds this round's walk lengths to each walk row's M, S1 = sum of lengths and
// S2 = sum of squared lengths (one warp per row).
__global__ void k_adapt_accumulate(int32_t nw, const int64_t* __restrict__ wbase, const int2* __restrict__ rec,
                                   uint32_t* M, unsigned long long* S1, unsigned long long* S2) {
    const int32_t gw = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nwarps = (int32_t)((gridDim.x * blockDim.x) >> 5);
    for (int32_t r = gw; r < nw; r += nwarps) {
        const int64_t b0 = wbase[r], b1 = wbase[r + 1];
        unsigned long long s1 = 0, s2 = 0;
        for (int64_t i = b0 + lane_id(); i < b1; i += 32) {
            const unsigned long long l = (uint32_t)rec[i].y;
            s1 += l;
            s2 += l * l;
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        if (lane_id() == 0 && b1 > b0) {
            M[r] += (uint32_t)(b1 - b0);
            S1[r] += s1;
            S2[r] += s2;
        }
    }
}

// The Sec. 5.1 test for every walk row; rows that need more walks get their
// increment in inc[node] (0 otherwise) and are counted in *pending.
__global__ void k_adapt_decide(int32_t nw, const int4* __restrict__ wrow, const uint32_t* __restrict__ M,
                               const unsigned long long* __restrict__ S1, const unsigned long long* __restrict__ S2,
                               double d2, double z2, uint32_t max_walks, uint32_t* inc, unsigned* pending) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x) {
        const uint32_t m = M[r];
        uint32_t add = 0u;
        if (m > 1u && m < max_walks) {
            const double Md = (double)m;
            const double mean = __ddiv_rn((double)S1[r], Md);
            const double var = __ddiv_rn(__dadd_rn((double)S2[r], -__dmul_rn((double)S1[r], mean)), __dadd_rn(Md, -1.0));
            const double lhs = __dmul_rn(__dmul_rn(d2, __dmul_rn(mean, mean)), Md);
            const double rhs = __dmul_rn(z2, var);
            if (!(lhs > rhs)) {
                const double need = __ddiv_rn(rhs, __dmul_rn(d2, __dmul_rn(mean, mean)));
                uint32_t target = need >= (double)max_walks ? max_walks : (uint32_t)ceil(need);
                if (target < m + 1u) target = m + 1u;
                add = target - m;
            }
        }
        inc[wrow[r].x] = add;
        if (add) atomicAdd(pending, 1u);
    }
}

__global__ void k_adapt_budget(int32_t n, int32_t nw, const int4* __restrict__ wrow, const uint32_t* __restrict__ M,
                               uint32_t* budget) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) budget[k] = 0u;
}
__global__ void k_adapt_budget_rows(int32_t nw, const int4* __restrict__ wrow, const uint32_t* __restrict__ M,
                                    uint32_t* budget) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x)
        budget[wrow[r].x] = M[r];
}
__global__ void k_adapt_first(int32_t nw, const int4* __restrict__ wrow, uint32_t first, uint32_t* inc) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x)
        inc[wrow[r].x] = first;
}

}  // namespace rw

using namespace rw;

extern "C" {

rw_status rw_adaptive_budget(rw_context* ctx, const rw_csr* A, uint64_t seed, double delta, double z,
                             uint32_t min_walks, uint32_t max_walks, int32_t max_rounds, uint32_t* d_budget,
                             int32_t* h_rounds) {
    if (!ctx || !d_budget || !(delta > 0.0) || !(z > 0.0) || min_walks < 2 || max_walks < min_walks ||
        max_walks > 65535u || max_rounds < 1) {
        set_error("rw_adaptive_budget: bad arguments (delta, z > 0; 2 <= min_walks <= max_walks <= 65535; "
                  "max_rounds >= 1)");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr(A);
    if (rc) return rc;
    if (h_rounds) *h_rounds = 0;
    const int32_t n = A->n;
    if (n == 0) return RW_OK;
    cudaStream_t s = ctx->stream;
    Pool sc(ctx);
    Tables T;
    if ((rc = reset_status(ctx)) || (rc = build_tables(ctx, A, T, sc)) || (rc = read_status(ctx, "walk tables")))
        return rc;
    const int32_t nw = T.n_walk_rows;
    const int g = grid_for(n, 256, ctx->num_sms * 8);
    RW_COUNT_LAUNCH();
    k_adapt_budget<<<g, 256, 0, s>>>(n, nw, T.wrow, nullptr, d_budget);
    if ((rc = check_launch("adaptive budget"))) return rc;
    if (nw == 0) return check_cuda(cudaStreamSynchronize(s), "sync");
    uint32_t* M = alloc_n<uint32_t>(sc, nw);
    unsigned long long* S1 = alloc_n<unsigned long long>(sc, nw);
    unsigned long long* S2 = alloc_n<unsigned long long>(sc, nw);
    uint32_t* inc = alloc_n<uint32_t>(sc, n);
    unsigned* pending = alloc_n<unsigned>(sc, 1);
    unsigned long long* hops = alloc_n<unsigned long long>(sc, 1);
    if (!M || !S1 || !S2 || !inc || !pending || !hops) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(M, 0, sizeof(uint32_t) * (size_t)nw, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(S1, 0, sizeof(unsigned long long) * (size_t)nw, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(S2, 0, sizeof(unsigned long long) * (size_t)nw, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(inc, 0, sizeof(uint32_t) * (size_t)n, s), "memset")))
        return rc;
    const int gw = grid_for(nw, 256, ctx->num_sms * 8);
    RW_COUNT_LAUNCH();
    k_adapt_first<<<gw, 256, 0, s>>>(nw, T.wrow, min_walks, inc);
    if ((rc = check_launch("adaptive start"))) return rc;
    const double d2 = delta * delta, z2 = z * z;
    unsigned* hp = static_cast<unsigned*>(ctx->h_small);
    int32_t rounds = 0;
    for (int32_t round = 0; round < max_rounds; ++round) {
        Pool rp(ctx);  // this round's walk space and records
        WalkSpace ws;
        if ((rc = build_walk_space(ctx, T, 0, inc, ws, rp, true))) return rc;
        if (ws.total == 0) break;
        int2* rec = alloc_n<int2>(rp, ws.total);
        if (!rec) return RW_ERR_ALLOC;
        WalkBatch wb;
        wb.m0 = mat_walk(T, seed, 0, 0);  // factor walks: the ones rw_build_factor_budget runs
        wb.table_bytes = table_bytes(T);
    wb.nrows = T.n_walk_rows;
        wb.wrow = T.wrow;
        wb.wbase = ws.wbase;
        wb.wofs = M;  // walks M, M+1, ... of each row
        wb.chunk_row = ws.chunk_row;
        wb.total = ws.total;
        WalkLaunch wl;
        wl.max_steps = ctx->opt.max_steps;
        wl.record_lengths = 1;
        if ((rc = run_walks(ctx, wb, wl, rec, hops, rp, nullptr)) || (rc = read_status(ctx, "adaptive walks")))
            return rc;
        RW_COUNT_LAUNCH();
        k_adapt_accumulate<<<grid_for((int64_t)nw * 32, 256, ctx->num_sms * 8), 256, 0, s>>>(nw, ws.wbase, rec, M,
                                                                                               S1, S2);
        if ((rc = check_cuda(cudaMemsetAsync(pending, 0, sizeof(unsigned), s), "memset"))) return rc;
        RW_COUNT_LAUNCH();
        k_adapt_decide<<<gw, 256, 0, s>>>(nw, T.wrow, M, S1, S2, d2, z2, max_walks, inc, pending);
        if ((rc = check_launch("adaptive decision"))) return rc;
        if ((rc = check_cuda(cudaMemcpyAsync(hp, pending, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "copy")) ||
            (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
            return rc;
        rounds = round + 1;
        if (hp[0] == 0u) break;
    }
    RW_COUNT_LAUNCH();
    k_adapt_budget_rows<<<gw, 256, 0, s>>>(nw, T.wrow, M, d_budget);
    if ((rc = check_launch("adaptive budget"))) return rc;
    if (h_rounds) *h_rounds = rounds;
    return read_status(ctx, "adaptive budget");
}

}  // extern "C"
