// rw_walk.cu -- the random-walk kernel (journey record of Sec. 3.1 with the
// one-step-exact first step of Sec. 5.2).
//
// Persistent kernel, one warp lane per walk.  A warp claims kWalkChunk walk
// indices at a time from a global cursor; a lane whose walk ends takes the next
// index of the warp's pool, so the warp stays full although walk lengths vary
// by orders of magnitude.  A hop reads the 32-byte threshold block of the
// current node (one DRAM sector for degree <= 7) and one 8-byte successor entry
// {column, block offset of the column}, so no row-pointer lookup is needed.
//
// Walk w of row k (rows 0..k-1 are homes, ground absorbs):
//   step 1: draw 0 picks an upper neighbour j > k with probability
//           A_kj / sum_{j>k} A_kj (first-step table);
//   step h: draw h-1 picks the next node by the transition thresholds of the
//           current node; ground if the draw is above every threshold;
//   the walk ends at a node < k (home) or at ground; each visit to k counts a
//   return.  Draw s is word (s mod 4) of Philox(s/4, w, k, tag).
// Output: one record per walk, {end node (-1 ground, -2 step cap), returns or
// length}.
#include "rw_internal.h"

namespace rw {

struct WalkParams {
    const MatWalk* __restrict__ mats;   // per matrix: tables, key, tag
    const int32_t* __restrict__ wmat;   // matrix of each walk row (batched launches)
    const int4* __restrict__ wrow;
    const int64_t* __restrict__ wbase;
    const uint32_t* __restrict__ wofs;  // first walk index of each walk row (NULL: 0)
    const int32_t* __restrict__ chunk_row;
    int64_t total;
    unsigned long long* cursor;
    int2* rec;
    unsigned long long* hops;
    DevStatus* st;
    uint64_t max_steps;
    int record_lengths;
    MatWalk m0;                         // the matrix of a single-matrix launch
};

// Number of thresholds t <= u among the 8 words of a block (padding words are
// 0xFFFFFFFF and are only counted for u = 0xFFFFFFFF, which the callers clamp).
__device__ __forceinline__ uint32_t count_le8(const uint4 a, const uint4 b, uint32_t u) {
    return (uint32_t)(a.x <= u) + (uint32_t)(a.y <= u) + (uint32_t)(a.z <= u) +
           (uint32_t)(a.w <= u) + (uint32_t)(b.x <= u) + (uint32_t)(b.y <= u) +
           (uint32_t)(b.z <= u) + (uint32_t)(b.w <= u);
}

__device__ __forceinline__ uint4 ld_nc4(const uint32_t* p) {
    return __ldg(reinterpret_cast<const uint4*>(p));
}

template <bool MULTI>
__global__ void __launch_bounds__(256) k_walk(const WalkParams P) {
    const unsigned lane = lane_id();
    const unsigned lt = lanemask_lt();

    int64_t pool_next = 0, pool_end = 0;
    int32_t pool_row = 0;
    bool exhausted = false;

    bool active = false;
    int64_t widx = 0;
    uint32_t k = 0, w = 0, coff = 0, ret = 0;
    // the walking lane's matrix (fixed for a single-matrix launch)
    const uint32_t* thr = P.m0.thr;
    const uint2* nxt = P.m0.nxt;
    uint32_t key0 = P.m0.key0, key1 = P.m0.key1, tag = P.m0.tag;
    uint64_t h = 0;
    Philox4 rnd{0u, 0u, 0u, 0u};
    unsigned long long my_hops = 0;
    int32_t my_m = 0;  // matrix whose hops my_hops holds

    for (;;) {
        // ---- refill idle lanes from the warp's pool of walk indices ----
        unsigned idle = __ballot_sync(kFull, !active);
        while (idle != 0u && !exhausted) {
            if (pool_next >= pool_end) {
                unsigned long long base = 0;
                if (lane == 0)
                    base = ld_relaxed_u32(&P.st->walk_cap) != 0u
                               ? (unsigned long long)P.total
                               : atomicAdd(P.cursor, (unsigned long long)kWalkChunk);
                base = __shfl_sync(kFull, base, 0);
                if ((int64_t)base >= P.total) {
                    exhausted = true;
                    break;
                }
                pool_next = (int64_t)base;
                pool_end = min((int64_t)base + kWalkChunk, P.total);
                pool_row = P.chunk_row[base / kWalkChunk];
            }
            const int avail = (int)(pool_end - pool_next);
            const int rank = __popc(idle & lt);
            const bool take = !active && rank < avail;
            int32_t r = pool_row;
            if (take) {
                widx = pool_next + rank;
                while (P.wbase[r + 1] <= widx) ++r;
                const int4 info = P.wrow[r];
                const uint32_t* fthr = P.m0.fthr;
                if (MULTI) {
                    const int32_t m = P.wmat[r];
                    if (m != my_m) {
                        if (my_hops) atomicAdd(P.hops + my_m, my_hops);
                        my_hops = 0;
                        my_m = m;
                    }
                    const MatWalk& mw = P.mats[m];
                    thr = mw.thr;
                    nxt = mw.nxt;
                    fthr = mw.fthr;
                    key0 = mw.key0;
                    key1 = mw.key1;
                    tag = mw.tag;
                }
                k = (uint32_t)info.x;
                w = (uint32_t)(widx - P.wbase[r]) + (P.wofs ? P.wofs[r] : 0u);
                rnd = philox4x32_10(0u, w, k, tag, key0, key1);
                const uint32_t u = rnd.v0;
                // first step: least m with u < ft_m among the upper neighbours, else the last
                const uint32_t* fb = fthr + (size_t)info.y * 8u;
                const uint4 a = ld_nc4(fb), b = ld_nc4(fb + 4);
                const uint32_t up = a.x;
                uint32_t m = (uint32_t)(a.z <= u) + (uint32_t)(a.w <= u) + (uint32_t)(b.x <= u) +
                             (uint32_t)(b.y <= u) + (uint32_t)(b.z <= u) + (uint32_t)(b.w <= u);
                if (m == 6u && up > 6u) {
                    for (uint32_t blk = 1;; ++blk) {
                        const uint4 c = ld_nc4(fb + 8u * blk), d = ld_nc4(fb + 8u * blk + 4u);
                        const uint32_t cnt = count_le8(c, d, u);
                        m += cnt;
                        if (cnt < 8u || m >= up) break;
                    }
                }
                if (m > up - 1u) m = up - 1u;
                const uint2 e = __ldg(nxt + (size_t)info.z * 8u + 1u + (uint32_t)info.w + m);
                coff = e.y;
                h = 1;
                ret = 0;
                active = true;
            }
            const int ntake = min(__popc(idle), avail);
            const unsigned tm = __ballot_sync(kFull, take);
            pool_row = __shfl_sync(kFull, r, 31 - __clz(tm));
            pool_next += ntake;
            idle = __ballot_sync(kFull, !active);
        }
        if (__ballot_sync(kFull, active) == 0u) break;

        // ---- one hop of every active lane ----
        if (active) {
            int32_t end = 0;
            bool done = false;
            if (h >= P.max_steps || ((h & 4095u) == 0u && ld_relaxed_u32(&P.st->walk_cap) != 0u)) {
                // the step cap, or another walk hit it: stop (the build reports the error)
                end = -2;
                done = true;
                if (h >= P.max_steps) atomicAdd(&P.st->walk_cap, 1u);
            } else {
                const uint32_t sidx = (uint32_t)h;
                if ((sidx & 3u) == 0u) rnd = philox4x32_10(sidx >> 2, w, k, tag, key0, key1);
                const uint32_t q = sidx & 3u;
                const uint32_t u = q == 0u ? rnd.v0 : q == 1u ? rnd.v1 : q == 2u ? rnd.v2 : rnd.v3;
                ++h;
                const uint32_t* blk = thr + (size_t)coff * 8u;
                const uint4 a = ld_nc4(blk), b = ld_nc4(blk + 4);
                const uint32_t deg = a.x;
                uint32_t m = (uint32_t)(a.y <= u) + (uint32_t)(a.z <= u) + (uint32_t)(a.w <= u) +
                             (uint32_t)(b.x <= u) + (uint32_t)(b.y <= u) + (uint32_t)(b.z <= u) +
                             (uint32_t)(b.w <= u);
                if (m == 7u && deg > 7u) {
                    for (uint32_t bi = 1;; ++bi) {
                        const uint4 c = ld_nc4(blk + 8u * bi), d = ld_nc4(blk + 8u * bi + 4u);
                        const uint32_t cnt = count_le8(c, d, u);
                        m += cnt;
                        if (cnt < 8u || m >= deg) break;
                    }
                }
                if (m >= deg) {
                    end = -1;  // ground
                    done = true;
                } else {
                    const uint2 e = __ldg(nxt + (size_t)coff * 8u + 1u + m);
                    if (e.x < k) {
                        end = (int32_t)e.x;  // home
                        done = true;
                    } else {
                        ret += (e.x == k) ? 1u : 0u;
                        coff = e.y;
                    }
                }
            }
            if (done) {
                P.rec[widx] = make_int2(end, (int32_t)(P.record_lengths ? (uint32_t)h : ret));
                my_hops += h;
                active = false;
            }
        }
    }
    if (MULTI) {
        if (my_hops) atomicAdd(P.hops + my_m, my_hops);
    } else {
        my_hops = warp_sum(my_hops);
        if (lane == 0 && my_hops) atomicAdd(P.hops, my_hops);
    }
}

rw_status run_walks(rw_context* ctx, const WalkBatch& wb, const WalkLaunch& wl, int2* rec,
                    unsigned long long* d_hops, Pool& pool, float* ms) {
    cudaStream_t s = ctx->stream;
    unsigned long long* cursor = alloc_n<unsigned long long>(pool, 1);
    if (!cursor) return RW_ERR_ALLOC;
    rw_status rc;
    if ((rc = check_cuda(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s), "memset")))
        return rc;
    if ((rc = check_cuda(cudaMemsetAsync(d_hops, 0, sizeof(unsigned long long) * wb.nmat, s),
                         "memset")))
        return rc;
    if (wb.total == 0) {
        if (ms) *ms = 0.f;
        return RW_OK;
    }
    const bool multi = wb.nmat > 1;
    WalkParams P{};
    P.mats = wb.mats;
    P.wmat = wb.wmat;
    P.wrow = wb.wrow;
    P.wbase = wb.wbase;
    P.wofs = wb.wofs;
    P.chunk_row = wb.chunk_row;
    P.total = wb.total;
    P.cursor = cursor;
    P.rec = rec;
    P.hops = d_hops;
    P.st = ctx->d_status;
    P.max_steps = wl.max_steps;
    P.record_lengths = wl.record_lengths;
    P.m0 = wb.m0;
    int per_sm = ctx->opt.walk_blocks_per_sm;
    if (per_sm <= 0) {
        if ((rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                 &per_sm, multi ? k_walk<true> : k_walk<false>, 256, 0),
                             "occupancy")))
            return rc;
        if (per_sm < 1) per_sm = 1;
    }
    int64_t blocks = (int64_t)per_sm * ctx->num_sms;
    const int64_t need = (wb.total + 255) / 256;  // never more lanes than walks
    if (blocks > need) blocks = need;
    if (ms) cudaEventRecord(ctx->ev[0], s);
    RW_COUNT_LAUNCH();
    if (multi) k_walk<true><<<(unsigned)blocks, 256, 0, s>>>(P);
    else k_walk<false><<<(unsigned)blocks, 256, 0, s>>>(P);
    if ((rc = check_launch("walk kernel"))) return rc;
    if (ms) {
        cudaEventRecord(ctx->ev[1], s);
        cudaEventSynchronize(ctx->ev[1]);
        cudaEventElapsedTime(ms, ctx->ev[0], ctx->ev[1]);
    }
    return RW_OK;
}

}  // namespace rw
