// rw_walk.cu -- the random-walk kernel (journey record of Sec. 3.1 with the
// one-step-exact first step of Sec. 5.2).
//
// Persistent kernel, one warp lane per walk.  A warp claims kWalkChunk walk
// indices at a time from a global cursor; a lane whose walk ends takes the next
// index of the warp's pool, so the warp stays full although walk lengths vary
// by orders of magnitude.  The tables hold each node's transitions in 32-byte
// group sectors of four thresholds with the four successors' words beside
// them, so the next node is known when the group arrives.  A hop to a node of
// degree <= 7 reads its group 0 (and group 1 only when the draw passes group
// 0); a hop to a node of higher degree reads the node's summary (the last
// threshold of each group; a dense node-indexed region that stays in L2), then
// the one group that holds the drawn successor, at an address the successor
// word gives without a load (nodes of more than 31 neighbours: a group base
// read beside the summary).  Random reads from HBM are limited per sector,
// not per byte, so the kernel is bound by the DRAM sectors per hop: one for
// 27-point nodes.
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
    int cache_hint;                     // tables larger than the L2: evict_last / evict_first policies
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

// Successor word: node index in bits 27..0, the node's group class in bits
// 31..28 (0: at most two groups, no summary; 3..8: its ng, groups at the
// fixed slot 3n + 8 * node; 15: more than eight groups, at gbase[node]).
constexpr uint32_t kNodeMask = 0x0FFFFFFFu;
constexpr uint32_t kHugeClass = 15u;
// Late in a launch (every walk started, at most kSpecLanes walks left in the
// warp) and on very long walks, a hop prefetches the node's groups to L2
// together with the summary read: it then waits for one DRAM round trip
// instead of an L2 read followed by a DRAM read.  The long walks set the
// launch's length; while the memory system is busy the extra sectors would
// cost more than they save.
constexpr uint64_t kSpecHops = 16384u;
constexpr int kSpecLanes = 8;

// 32 bytes (eight words) in one load; p must be 32-byte aligned (sectors are).
__device__ __forceinline__ void ld_nc8(const uint32_t* p, uint4& lo, uint4& hi) {
    asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
        : "l"(p));
}

// The same with an L2 cache-policy operand (createpolicy): evict_last keeps
// the summaries and group bases in L2 while the group sectors stream through
// with evict_first, when the tables are larger than the L2.
__device__ __forceinline__ void ld_nc8_hint(const uint32_t* p, uint4& lo, uint4& hi, uint64_t pol) {
    asm("ld.global.nc.L2::cache_hint.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
        : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
        : "l"(p), "l"(pol));
}
__device__ __forceinline__ uint32_t ld_nc_hint(const uint32_t* p, uint64_t pol) {
    uint32_t v;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_rec_hint(int2* p, int2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.s32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y), "l"(pol)
                 : "memory");
}
// Cache policies: keep (evict_last) and stream (evict_first) when `hint`,
// evict_normal for both otherwise.
__device__ __forceinline__ void walk_policies(int hint, uint64_t& keep, uint64_t& stream) {
    if (hint) {
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream));
    } else {
        asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(keep));
        stream = keep;
    }
}

// Word j (0..3) of the four words c.
__device__ __forceinline__ uint32_t pick4(const uint4 c, uint32_t j) {
    return (j & 2u) ? ((j & 1u) ? c.w : c.z) : ((j & 1u) ? c.y : c.x);
}

// Thresholds t <= u among the four words of a group.
__device__ __forceinline__ uint32_t count_le4(const uint4 t, uint32_t u) {
    return (uint32_t)(t.x <= u) + (uint32_t)(t.y <= u) + (uint32_t)(t.z <= u) + (uint32_t)(t.w <= u);
}

// Bulk prefetch of `bytes` (a multiple of 16) at p (16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const uint32_t* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes));
}

// One transition from the node of successor word cw with draw u: the least
// slot j whose threshold exceeds u (thresholds do not decrease along the
// slots, the header slot counts as passed), i.e. successor j - 1, ground if
// j > deg.  Returns that successor's word; *ground is set when the walk is
// absorbed.  n: the matrix's node count (the summaries start at sector 2n,
// the fixed group slots at 3n).  spec: prefetch the node's groups to L2
// before the summary read returns.
__device__ __forceinline__ uint32_t hop_node(const uint32_t* __restrict__ tab, const uint32_t* __restrict__ gbase,
                                             uint32_t n, uint32_t cw, uint32_t u, bool* ground, uint64_t keep,
                                             uint64_t stream, bool spec) {
    const uint32_t node = cw & kNodeMask;
    const uint32_t cls = cw >> 28;
    uint4 t, w;
    uint32_t deg, j = 0xFFFFFFFFu, nw = 0u;
    if (cls != 0u) {
        const uint32_t* sum = tab + ((size_t)2u * n + node) * 8u;
        const uint32_t* gp;
        if (cls != kHugeClass) {
            gp = tab + ((size_t)3u * n + (size_t)8u * node) * 8u;
            if (spec) prefetch_l2(gp, cls * 32u);
            ld_nc8_hint(sum, t, w, keep);  // kept in L2
        } else {
            // summary and group base together (both kept in L2)
            ld_nc8_hint(sum, t, w, keep);
            gp = tab + (size_t)ld_nc_hint(gbase + node, keep) * 8u;
        }
        deg = t.x;
        const uint32_t ng = (deg + 4u) >> 2;
        uint32_t g = (uint32_t)(t.y <= u) + (uint32_t)(t.z <= u) + (uint32_t)(t.w <= u) + count_le4(w, u);
        for (; g < ng; ++g) {  // one iteration unless the node has more than seven groups
            ld_nc8_hint(gp + (size_t)g * 8u, t, w, stream);
            if (g == 0u) t.x = 0u;
            const uint32_t c = count_le4(t, u);
            if (c < 4u) {
                j = 4u * g + c;
                nw = pick4(w, c);
                break;
            }
        }
    } else {
        // group 0 (slot 0's successor word holds deg); group 1 only when u passes group 0
        const uint32_t* g = tab + (size_t)node * 16u;
        ld_nc8(g, t, w);
        deg = w.x;
        const uint32_t c0 = count_le4(t, u);
        if (c0 < 4u) {
            j = c0;
            nw = pick4(w, c0);
        } else if (deg >= 4u) {
            ld_nc8(g + 8u, t, w);
            const uint32_t c1 = count_le4(t, u);
            j = 4u + c1;
            nw = c1 < 4u ? pick4(w, c1) : 0u;
        }
    }
    *ground = j > deg;
    return *ground ? 0u : nw;
}

// First step of a walk from the row whose group 0 is sector g0, lower degree
// lo: the successor word of successor lo + m.
__device__ __forceinline__ uint32_t first_successor(const uint32_t* __restrict__ tab, uint32_t g0, uint32_t lo,
                                                    uint32_t m) {
    const uint32_t slot = lo + m + 1u;
    return __ldg(tab + ((size_t)g0 + (slot >> 2)) * 8u + 4u + (slot & 3u));
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
    const uint32_t* tab = P.m0.tab;
    const uint32_t* gbase = P.m0.gbase;
    uint32_t key0 = P.m0.key0, key1 = P.m0.key1, tag = P.m0.tag, nn = P.m0.n;
    uint64_t h = 0;
    Philox4 rnd{0u, 0u, 0u, 0u};
    unsigned long long my_hops = 0;
    int32_t my_m = 0;  // matrix whose hops my_hops holds
    uint64_t keep, stream;
    walk_policies(P.cache_hint, keep, stream);

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
                    tab = mw.tab;
                    gbase = mw.gbase;
                    fthr = mw.fthr;
                    key0 = mw.key0;
                    key1 = mw.key1;
                    tag = mw.tag;
                    nn = mw.n;
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
                coff = first_successor(tab, (uint32_t)info.z, (uint32_t)info.w, m);
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
        const unsigned live = __ballot_sync(kFull, active);
        if (live == 0u) break;
        const bool sparse = exhausted && __popc(live) <= kSpecLanes;

        // ---- one hop of every active lane ----
        bool stepping = false;
        uint32_t u = 0u;
        if (active) {
            if (h >= P.max_steps || ((h & 4095u) == 0u && ld_relaxed_u32(&P.st->walk_cap) != 0u)) {
                // the step cap, or another walk hit it: stop (the build reports the error)
                if (h >= P.max_steps) atomicAdd(&P.st->walk_cap, 1u);
                P.rec[widx] = make_int2(-2, (int32_t)(P.record_lengths ? (uint32_t)h : ret));
                my_hops += h;
                active = false;
            } else {
                const uint32_t sidx = (uint32_t)h;
                if ((sidx & 3u) == 0u) rnd = philox4x32_10(sidx >> 2, w, k, tag, key0, key1);
                const uint32_t q = sidx & 3u;
                u = q == 0u ? rnd.v0 : q == 1u ? rnd.v1 : q == 2u ? rnd.v2 : rnd.v3;
                stepping = true;
            }
        }
        if (stepping) {
            int32_t end = 0;
            bool done = false;
            ++h;
            bool ground;
            const bool spec = sparse || h >= kSpecHops;
            const uint32_t nw = hop_node(tab, gbase, nn, coff, u, &ground, keep, stream, spec);
            const uint32_t nb = nw & kNodeMask;
            if (ground) {
                end = -1;
                done = true;
            } else if (nb < k) {
                end = (int32_t)nb;  // home
                done = true;
            } else {
                ret += (nb == k) ? 1u : 0u;
                coff = nw;
            }
            if (done) {
                st_rec_hint(P.rec + widx, make_int2(end, (int32_t)(P.record_lengths ? (uint32_t)h : ret)), stream);
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
    NvtxRange nvtx_range("rw_walk");
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
    P.cache_hint = wb.table_bytes * 4u > (uint64_t)ctx->l2_bytes * 3u ? 1 : 0;
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

// ---------------------------------------------------------------------------
// Walk reuse (Algorithm 2 of Sec. 5.3).  The simulated walk is the one k_walk
// runs; besides its own record it yields the legal sub-walks that start at a
// later node k' > k: k' is the least node of the sub-walk until it ends at a
// node below k' (a home of k') or at ground.  The lane keeps the increasing
// stack of such candidate starts above k (the top in registers, the rest in
// local memory, each with its returns so far); a hop to node e first pops
// every candidate above e -- each popped candidate is a finished sub-walk
// ending at e, counted unless it started at the previous hop (a one-step walk,
// whose contribution the first-step rule of Sec. 5.2 makes exact) -- then
// pushes e if it is above the new top, or counts a return if it equals it.
// Sub-walks of one start row never overlap (a start is popped before the same
// node can be pushed again), as the paper requires.  Finished sub-walks go to
// the warp's shared-memory stage and from there, in bulk, to the global
// extra-record arrays {start node, end node or -1, returns}.
struct ReuseParams {
    int32_t* xnode;  // start node
    int32_t* xend;   // end node, -1 ground
    uint32_t* xret;
    unsigned long long* xcount;  // records produced (may exceed xcap: then none past xcap is written)
    int64_t xcap;
    unsigned* overflow;          // walks whose stack outgrew CAP
};

constexpr int kReuseStage = 128;

template <int CAP>
__global__ void __launch_bounds__(256) k_walk_reuse(const WalkParams P, const ReuseParams R) {
    __shared__ int32_t s_node[8][kReuseStage];
    __shared__ int32_t s_end[8][kReuseStage];
    __shared__ uint32_t s_ret[8][kReuseStage];
    const unsigned lane = lane_id();
    const unsigned lt = lanemask_lt();
    const unsigned warp = threadIdx.x >> 5;

    int64_t pool_next = 0, pool_end = 0;
    int32_t pool_row = 0;
    bool exhausted = false;

    bool active = false;
    int64_t widx = 0;
    uint32_t k = 0, w = 0, coff = 0, ret = 0;
    const uint32_t* tab = P.m0.tab;
    const uint32_t* gbase = P.m0.gbase;
    const uint32_t key0 = P.m0.key0, key1 = P.m0.key1, tag = P.m0.tag, nn = P.m0.n;
    uint64_t h = 0;
    Philox4 rnd{0u, 0u, 0u, 0u};
    unsigned long long my_hops = 0;
    uint64_t keep, stream;
    walk_policies(P.cache_hint, keep, stream);

    uint2 stk[CAP];      // candidates below the top: {node, returns}
    int32_t depth = 0;   // candidates above k (the top one in registers)
    uint32_t top = 0, top_ret = 0;
    bool fresh = false;  // the top was pushed by the previous hop
    int stage_n = 0;     // warp-uniform

    auto flush = [&]() {
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(R.xcount, (unsigned long long)stage_n);
        base = __shfl_sync(kFull, base, 0);
        for (int i = (int)lane; i < stage_n; i += 32) {
            const unsigned long long p = base + (unsigned long long)i;
            if (p < (unsigned long long)R.xcap) {
                R.xnode[p] = s_node[warp][i];
                R.xend[p] = s_end[warp][i];
                R.xret[p] = s_ret[warp][i];
            }
        }
        __syncwarp();
        stage_n = 0;
    };

    for (;;) {
        unsigned idle = __ballot_sync(kFull, !active);
        while (idle != 0u && !exhausted) {
            if (pool_next >= pool_end) {
                unsigned long long base = 0;
                if (lane == 0)
                    base = (ld_relaxed_u32(&P.st->walk_cap) | ld_relaxed_u32(R.overflow)) != 0u
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
                k = (uint32_t)info.x;
                w = (uint32_t)(widx - P.wbase[r]) + (P.wofs ? P.wofs[r] : 0u);
                rnd = philox4x32_10(0u, w, k, tag, key0, key1);
                const uint32_t u = rnd.v0;
                const uint32_t* fb = P.m0.fthr + (size_t)info.y * 8u;
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
                coff = first_successor(tab, (uint32_t)info.z, (uint32_t)info.w, m);
                h = 1;
                ret = 0;
                depth = 1;  // the first step's upper neighbour starts the stack
                top = coff & kNodeMask;
                top_ret = 0;
                fresh = true;
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
        // outcome: 0 idle, 1 moved to node `to`, 2 ended at `to` (home, or -1 ground),
        // 3 stopped (step cap or stack overflow)
        int outcome = 0;
        int32_t to = 0;        // the next node (-1: ground)
        uint32_t to_word = 0;  // its successor word
        if (active) {
            if (h >= P.max_steps ||
                ((h & 4095u) == 0u && (ld_relaxed_u32(&P.st->walk_cap) | ld_relaxed_u32(R.overflow)) != 0u)) {
                outcome = 3;
                if (h >= P.max_steps) atomicAdd(&P.st->walk_cap, 1u);
            } else {
                const uint32_t sidx = (uint32_t)h;
                if ((sidx & 3u) == 0u) rnd = philox4x32_10(sidx >> 2, w, k, tag, key0, key1);
                const uint32_t q = sidx & 3u;
                const uint32_t u = q == 0u ? rnd.v0 : q == 1u ? rnd.v1 : q == 2u ? rnd.v2 : rnd.v3;
                ++h;
                bool ground;
                to_word = hop_node(tab, gbase, nn, coff, u, &ground, keep, stream, false);
                const uint32_t nb = to_word & kNodeMask;
                if (ground) {
                    outcome = 2;
                    to = -1;
                } else {
                    to = (int32_t)nb;
                    outcome = nb < k ? 2 : 1;
                }
            }
        }
        // ---- pop the candidates above `to` (warp-wide, one per round) ----
        bool pop = (outcome == 1 || outcome == 2) && depth > 0 && to < (int32_t)top;
        while (__any_sync(kFull, pop)) {
            const bool emit = pop && !fresh;
            const unsigned em = __ballot_sync(kFull, emit);
            const int cnt = __popc(em);
            if (stage_n + cnt > kReuseStage) flush();
            if (emit) {
                const int pos = stage_n + __popc(em & lt);
                s_node[warp][pos] = (int32_t)top;
                s_end[warp][pos] = to;
                s_ret[warp][pos] = top_ret;
            }
            stage_n += cnt;
            if (pop) {
                fresh = false;
                --depth;
                if (depth > 0) {
                    const uint2 t = stk[depth - 1];
                    top = t.x;
                    top_ret = t.y;
                }
                pop = depth > 0 && to < (int32_t)top;
            }
        }
        if (outcome == 1) {
            if ((uint32_t)to == k) {
                ++ret;  // every candidate is above k, so the stack is empty here
                fresh = false;
            } else if (depth > 0 && (uint32_t)to == top) {
                ++top_ret;
                fresh = false;
            } else if (depth > CAP) {
                atomicAdd(R.overflow, 1u);
                outcome = 3;
            } else {
                if (depth > 0) stk[depth - 1] = make_uint2(top, top_ret);
                ++depth;
                top = (uint32_t)to;
                top_ret = 0;
                fresh = true;
            }
            coff = to_word;
        }
        if (outcome >= 2) {
            P.rec[widx] = make_int2(outcome == 3 ? -2 : to, (int32_t)ret);
            my_hops += h;
            active = false;
            depth = 0;
        }
    }
    if (stage_n > 0) flush();
    my_hops = warp_sum(my_hops);
    if (lane == 0 && my_hops) atomicAdd(P.hops, my_hops);
}

// Extra records -> per walk row: counts, then a scatter into row order (the
// order inside a row is immaterial: the merge only sums them).
__global__ void k_extra_count(int64_t cnt, const int32_t* __restrict__ xnode, const uint32_t* __restrict__ wflag,
                              unsigned long long* rows) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(rows + wflag[xnode[i]], 1ull);
}

__global__ void k_extra_scatter(int64_t cnt, const int32_t* __restrict__ xnode, const int32_t* __restrict__ xend,
                                const uint32_t* __restrict__ xret, const uint32_t* __restrict__ wflag,
                                const int64_t* __restrict__ xbase, unsigned long long* fill, int2* xrec) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = wflag[xnode[i]];
        const int64_t p = xbase[r] + (int64_t)atomicAdd(fill + r, 1ull);
        const int32_t e = xend[i];
        xrec[p] = make_int2(e >= 0 ? e : -1, (int32_t)xret[i]);
    }
}

template <int CAP>
static rw_status launch_reuse(rw_context* ctx, const WalkParams& P, const ReuseParams& R) {
    int per_sm = ctx->opt.walk_blocks_per_sm;
    rw_status rc;
    if (per_sm <= 0) {
        if ((rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_reuse<CAP>, 256, 0),
                             "occupancy")))
            return rc;
        if (per_sm < 1) per_sm = 1;
    }
    int64_t blocks = (int64_t)per_sm * ctx->num_sms;
    const int64_t need = (P.total + 255) / 256;
    if (blocks > need) blocks = need;
    RW_COUNT_LAUNCH();
    k_walk_reuse<CAP><<<(unsigned)blocks, 256, 0, ctx->stream>>>(P, R);
    return check_launch("walk kernel (reuse)");
}

rw_status run_walks_reuse(rw_context* ctx, const WalkBatch& wb, const WalkLaunch& wl, const Tables& T, int2* rec,
                          unsigned long long* d_hops, Pool& pool, Pool& xpool, float* ms, Extras& X) {
    NvtxRange nvtx_range("rw_walk_reuse");
    cudaStream_t s = ctx->stream;
    const int32_t nw = T.n_walk_rows;
    rw_status rc;
    X = Extras{};
    X.xbase = alloc_n<int64_t>(xpool, nw + 1);
    unsigned long long* cursor = alloc_n<unsigned long long>(pool, 1);
    unsigned long long* xcount = alloc_n<unsigned long long>(pool, 1);
    unsigned* overflow = alloc_n<unsigned>(pool, 1);
    if (!X.xbase || !cursor || !xcount || !overflow) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(X.xbase, 0, sizeof(int64_t) * (size_t)(nw + 1), s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(d_hops, 0, sizeof(unsigned long long), s), "memset")))
        return rc;
    if (wb.total == 0) {
        if (ms) *ms = 0.f;
        return RW_OK;
    }
    WalkParams P{};
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
    P.record_lengths = 0;
    P.cache_hint = wb.table_bytes * 4u > (uint64_t)ctx->l2_bytes * 3u ? 1 : 0;
    P.m0 = wb.m0;
    int64_t cap = (int64_t)(ctx->reuse_ratio * (double)wb.total) + (1 << 16);
    int stack = 64;
    unsigned long long* h64 = static_cast<unsigned long long*>(ctx->h_small);
    for (int attempt = 0;; ++attempt) {
        ReuseParams R;
        R.xnode = alloc_n<int32_t>(xpool, cap);
        R.xend = alloc_n<int32_t>(xpool, cap);
        R.xret = alloc_n<uint32_t>(xpool, cap);
        if (!R.xnode || !R.xend || !R.xret) return RW_ERR_ALLOC;
        R.xcount = xcount;
        R.xcap = cap;
        R.overflow = overflow;
        if ((rc = check_cuda(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s), "memset")) ||
            (rc = check_cuda(cudaMemsetAsync(d_hops, 0, sizeof(unsigned long long), s), "memset")) ||
            (rc = check_cuda(cudaMemsetAsync(xcount, 0, sizeof(unsigned long long), s), "memset")) ||
            (rc = check_cuda(cudaMemsetAsync(overflow, 0, sizeof(unsigned), s), "memset")))
            return rc;
        if (ms) cudaEventRecord(ctx->ev[0], s);
        rc = stack == 64 ? launch_reuse<64>(ctx, P, R) : launch_reuse<1024>(ctx, P, R);
        if (rc) return rc;
        if (ms) cudaEventRecord(ctx->ev[1], s);
        if ((rc = check_cuda(cudaMemcpyAsync(h64, xcount, 8, cudaMemcpyDeviceToHost, s), "copy")) ||
            (rc = check_cuda(cudaMemcpyAsync(h64 + 1, overflow, 4, cudaMemcpyDeviceToHost, s), "copy")) ||
            (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
            return rc;
        if (ms) cudaEventElapsedTime(ms, ctx->ev[0], ctx->ev[1]);
        const uint64_t produced = h64[0];
        const unsigned over = static_cast<unsigned>(h64[1] & 0xFFFFFFFFull);
        bool again = false;
        if (over) {
            if (stack == 1024) {
                set_error("walk reuse: %u walks have more than 1024 pending sub-walk starts", over);
                return RW_ERR_CAPACITY;
            }
            stack = 1024;
            again = true;
        } else if ((int64_t)produced > cap) {
            cap = (int64_t)produced;
            again = true;
        }
        if (!again) {
            X.count = (int64_t)produced;
            X.xnode = R.xnode;
            X.xend = R.xend;
            X.xret = R.xret;
            const double ratio = 1.125 * (double)produced / (double)wb.total;
            if (ratio > ctx->reuse_ratio) ctx->reuse_ratio = ratio;
            break;
        }
        xpool.release(R.xnode);
        xpool.release(R.xend);
        xpool.release(R.xret);
        if (attempt >= 2) {
            set_error("walk reuse: extra-record capacity did not settle");
            return RW_ERR_CAPACITY;
        }
    }
    // bucket the extra records by walk row
    unsigned long long* rows = alloc_n<unsigned long long>(pool, nw);
    X.xrec = alloc_n<int2>(xpool, X.count);
    if (!rows || !X.xrec) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(rows, 0, sizeof(unsigned long long) * (size_t)nw, s), "memset")))
        return rc;
    const int g = grid_for(X.count, 256, ctx->num_sms * 16);
    if (X.count > 0) {
        RW_COUNT_LAUNCH();
        k_extra_count<<<g, 256, 0, s>>>(X.count, X.xnode, T.walk_flag, rows);
        if ((rc = check_launch("extra counts"))) return rc;
    }
    if ((rc = check_cuda(scan_i64(reinterpret_cast<const int64_t*>(rows), X.xbase, nw, s, pool), "scan")) ||
        (rc = check_cuda(cudaMemsetAsync(rows, 0, sizeof(unsigned long long) * (size_t)nw, s), "memset")))
        return rc;
    if (X.count > 0) {
        RW_COUNT_LAUNCH();
        k_extra_scatter<<<g, 256, 0, s>>>(X.count, X.xnode, X.xend, X.xret, T.walk_flag, X.xbase, rows, X.xrec);
        if ((rc = check_launch("extra scatter"))) return rc;
    }
    return RW_OK;
}

}  // namespace rw
