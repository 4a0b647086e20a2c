// rw_tables.cu -- prefix sums, matrix validation and the walk tables.
//
// The walk tables encode the transition probabilities of the walk game
// (Sec. 2.1, Eq. map) as integer thresholds of cumulative probabilities, and
// the first step of each walk over the upper neighbours only (Sec. 5.2).
#include <climits>
#include <cstdarg>
#include <cstdio>

#include "rw_internal.h"

namespace rw {

// ---------------------------------------------------------------------------
// Exclusive prefix sum: tiles of 2048 values (256 threads x 8 consecutive
// values per thread), tile totals scanned recursively.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T* total) {
    __shared__ T warp_tot[kScanThreads / 32];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T t = (lane < kScanThreads / 32) ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, ti, o);
            if ((int)lane >= o) ti += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;
        if (lane == kScanThreads / 32 - 1) *total = ti;
    }
    __syncthreads();
    T r = warp_tot[warp] + incl - v;
    __syncthreads();
    return r;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const Tin* in, int64_t n, Tout* sums) {
    __shared__ Tout tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    Tout acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) acc += (Tout)in[base + i];
    block_exclusive_scan<Tout>(acc, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads)
    k_tile_scan(const Tin* in, int64_t n, const Tout* tile_off, Tout* out) {
    __shared__ Tout tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    Tout v[kScanItems];
    Tout acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? (Tout)in[base + i] : Tout(0);
        acc += v[i];
    }
    Tout pre = block_exclusive_scan<Tout>(acc, &tot);
    if (tile_off) pre += tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) {
            out[base + i] = pre;
            if (base + i == n - 1) out[n] = pre + v[i];
        }
        pre += v[i];
    }
}

template <typename Tout>
__global__ void k_set_zero(Tout* p) { *p = 0; }

template <typename Tin, typename Tout>
static cudaError_t scan_impl(const Tin* in, Tout* out, int64_t n, cudaStream_t s, Pool& pool) {
    if (n <= 0) {
        RW_COUNT_LAUNCH();
        k_set_zero<Tout><<<1, 1, 0, s>>>(out);
        return cudaGetLastError();
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        RW_COUNT_LAUNCH();
        k_tile_scan<Tin, Tout><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        return cudaGetLastError();
    }
    Tout* sums = alloc_n<Tout>(pool, tiles + 1);
    if (!sums) return cudaErrorMemoryAllocation;
    RW_COUNT_LAUNCH();
    k_tile_sums<Tin, Tout><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_impl<Tout, Tout>(sums, sums, tiles, s, pool);
    if (e != cudaSuccess) return e;
    RW_COUNT_LAUNCH();
    k_tile_scan<Tin, Tout><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums, out);
    return cudaGetLastError();
}

cudaError_t scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s, Pool& pool) {
    return scan_impl<uint32_t, uint32_t>(in, out, n, s, pool);
}
cudaError_t scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n, cudaStream_t s,
                            Pool& pool) {
    return scan_impl<uint32_t, int64_t>(in, out, n, s, pool);
}
cudaError_t scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, Pool& pool) {
    return scan_impl<int64_t, int64_t>(in, out, n, s, pool);
}

// ---------------------------------------------------------------------------
// Validation and per-row sizes.  One thread per row.
// ---------------------------------------------------------------------------
__global__ void k_row_info(int32_t n, int64_t nnz, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const double* __restrict__ val,
                           int32_t* deg, int32_t* lowdeg, int32_t* dpos, uint32_t* blk_full,
                           uint32_t* blk_first, uint32_t* walk_flag, DevStatus* st) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || (int64_t)rp[n] != nnz))
        atomicMin(&st->bad_row, 1u);
    for (int32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        int32_t s = rp[l], e = rp[l + 1];
        bool ok = e > s && s >= 0 && (int64_t)e <= nnz;
        if (!ok) e = s;  // do not read outside the arrays
        int32_t lo = 0, up = 0, prev = -1, dp = -1;
        double dg = 0.0, sum = 0.0;
        for (int32_t p = s; p < e; ++p) {
            const int32_t c = col[p];
            const double v = val[p];
            if (c < 0 || c >= n || c <= prev) ok = false;
            prev = c;
            if (c == l) {
                dp = p;
                dg = v;
                if (!(v > 0.0) || !isfinite(v)) ok = false;
            } else {
                if (!(v < 0.0) || !isfinite(v)) ok = false;
                sum = __dadd_rn(sum, -v);
                if (c < l) ++lo; else ++up;
            }
        }
        if (dp < 0) ok = false;
        if (ok && __dadd_rn(dg, -sum) < __dmul_rn(-1e-12, dg)) ok = false;
        if (!ok) atomicMin(&st->bad_row, (unsigned)l + 1u);
        const int32_t d = lo + up;
        deg[l] = d;
        lowdeg[l] = lo;
        dpos[l] = dp;
        // groups of four slots, ceil((1 + deg) / 4); a node of more than two
        // has a summary, a node of more than eight its groups in the fourth
        // region of the tables (counted here for their prefix)
        const uint32_t ng = (uint32_t)(1 + d + 3) / 4u;
        blk_full[l] = ng > 8u ? ng : 0u;
        blk_first[l] = up > 0 ? (uint32_t)(2 + up + 7) / 8u : 0u;
        walk_flag[l] = up > 0 ? 1u : 0u;
    }
}

// Thresholds and successor words.  One thread per row; the sums run
// sequentially over the row in ascending column order, each addition and
// division rounded once (the same order the sampling rule is defined in).
__global__ void k_fill_tables(int32_t n, const int32_t* __restrict__ rp,
                              const int32_t* __restrict__ col, const double* __restrict__ val,
                              const int32_t* __restrict__ deg, const int32_t* __restrict__ lowdeg,
                              const int32_t* __restrict__ dpos, const uint32_t* __restrict__ toff,
                              const uint32_t* __restrict__ foff8, uint32_t* tab, uint32_t* gbase,
                              uint32_t* fthr, double* S, double* diag) {
    for (int32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const int32_t s = rp[l], e = rp[l + 1], dp = dpos[l], d = deg[l], lo = lowdeg[l];
        const double dg = val[dp];
        diag[l] = dg;
        const uint64_t ng = ((uint64_t)d + 4u) / 4u;
        const bool big = ng > 2u;
        const uint64_t g0 = !big      ? 2u * (uint64_t)l
                            : ng <= 8u ? 3u * (uint64_t)n + 8u * (uint64_t)l
                                       : 11u * (uint64_t)n + toff[l];
        gbase[l] = (uint32_t)g0;
        // slot j: threshold at word 8 * (g0 + j / 4) + j % 4, successor word at + 4
        auto word = [&](uint64_t j) -> uint32_t* { return tab + (g0 + j / 4u) * 8u + (j % 4u); };
        *word(0) = 0u;                 // the header slot: always passed
        word(0)[4] = (uint32_t)d;      // slot 0 has no successor: its word holds deg
        double c = 0.0;
        uint64_t j = 1;
        for (int32_t p = s; p < e; ++p) {
            if (p == dp) continue;
            c = __dadd_rn(c, -val[p]);
            uint32_t* w = word(j);
            w[0] = cumulative_threshold(c, dg);
            const int32_t jc = col[p];
            const uint32_t ngc = (uint32_t)(deg[jc] + 4) / 4u;
            // bits 31..28: the successor's group class (0: no summary, 3..8:
            // its ng, 15: more than eight groups)
            const uint32_t cls = ngc <= 2u ? 0u : ngc <= 8u ? ngc : 15u;
            w[4] = (uint32_t)jc | (cls << 28);
            ++j;
        }
        for (; j < ng * 4u; ++j) {
            uint32_t* w = word(j);
            w[0] = 0xFFFFFFFFu;
            w[4] = 0u;
        }
        if (big) {
            // summary: deg, then the threshold of the last slot of groups 0..6
            uint32_t* sw = tab + (2u * (uint64_t)n + (uint64_t)l) * 8u;
            sw[0] = (uint32_t)d;
            for (uint64_t g = 0; g < 7u; ++g) sw[1 + g] = g < ng ? *word(4u * g + 3u) : 0xFFFFFFFFu;
        }
        const int32_t up = d - lo;
        double cu = 0.0;
        if (up > 0) {
            for (int32_t p = dp + 1; p < e; ++p) cu = __dadd_rn(cu, -val[p]);
            const uint64_t fb = (uint64_t)foff8[l] * 8u;
            const uint64_t fend = (uint64_t)foff8[l + 1] * 8u;
            fthr[fb] = (uint32_t)up;
            fthr[fb + 1] = (uint32_t)lo;
            double cc = 0.0;
            uint64_t q = fb + 2;
            for (int32_t p = dp + 1; p < e; ++p) {
                cc = __dadd_rn(cc, -val[p]);
                fthr[q++] = cumulative_threshold(cc, cu);
            }
            for (; q < fend; ++q) fthr[q] = 0xFFFFFFFFu;
        }
        S[l] = -cu;
    }
}

__global__ void k_walk_rows(int32_t n, const uint32_t* __restrict__ widx,
                            const uint32_t* __restrict__ gbase, const uint32_t* __restrict__ foff8,
                            const int32_t* __restrict__ lowdeg, int4* wrow, int32_t* walk_rows) {
    for (int32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const uint32_t r = widx[l];
        if (widx[l + 1] != r) {
            wrow[r] = make_int4(l, (int)foff8[l], (int)gbase[l], lowdeg[l]);
            walk_rows[r] = l;
        }
    }
}

rw_status build_tables(rw_context* ctx, const rw_csr* A, Tables& T, Pool& pool) {
    NvtxRange nvtx_range("rw_tables");
    const int32_t n = A->n;
    cudaStream_t s = ctx->stream;
    T.n = n;
    T.deg = alloc_n<int32_t>(pool, n);
    T.lowdeg = alloc_n<int32_t>(pool, n);
    T.diag_pos = alloc_n<int32_t>(pool, n);
    T.toff = alloc_n<uint32_t>(pool, n + 1);
    T.foff8 = alloc_n<uint32_t>(pool, n + 1);
    T.walk_flag = alloc_n<uint32_t>(pool, n + 1);
    T.S = alloc_n<double>(pool, n);
    T.diag = alloc_n<double>(pool, n);
    if (!T.deg || !T.lowdeg || !T.diag_pos || !T.toff || !T.foff8 || !T.walk_flag || !T.S ||
        !T.diag)
        return RW_ERR_ALLOC;
    const int blocks = grid_for(n, 256, ctx->num_sms * 8);
    RW_COUNT_LAUNCH();
    k_row_info<<<blocks, 256, 0, s>>>(n, A->nnz, A->row_ptr, A->col, A->val, T.deg, T.lowdeg, T.diag_pos,
                                      T.toff, T.foff8, T.walk_flag, ctx->d_status);
    rw_status rc = check_launch("row info");
    if (rc) return rc;
    if ((rc = check_cuda(scan_u32(T.toff, T.toff, n, s, pool), "scan"))) return rc;
    if ((rc = check_cuda(scan_u32(T.foff8, T.foff8, n, s, pool), "scan"))) return rc;
    if ((rc = check_cuda(scan_u32(T.walk_flag, T.walk_flag, n, s, pool), "scan"))) return rc;
    uint32_t* hs = static_cast<uint32_t*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(hs, T.toff + n, 4, cudaMemcpyDeviceToHost, s), "copy")))
        return rc;
    if ((rc = check_cuda(cudaMemcpyAsync(hs + 1, T.foff8 + n, 4, cudaMemcpyDeviceToHost, s),
                         "copy")))
        return rc;
    if ((rc = check_cuda(cudaMemcpyAsync(hs + 2, T.walk_flag + n, 4, cudaMemcpyDeviceToHost, s),
                         "copy")))
        return rc;
    if ((rc = read_status(ctx, "matrix validation"))) return rc;
    T.sectors = 11u * (uint64_t)n + hs[0];
    if (n >= (1 << 28)) {
        set_error("walk tables: n = %d exceeds the 2^28 node-index range of the successor words", n);
        return RW_ERR_CAPACITY;
    }
    if (T.sectors >= 0x80000000ull) {
        set_error("walk tables: %llu sectors exceed the 2^31 sector-index range", (unsigned long long)T.sectors);
        return RW_ERR_CAPACITY;
    }
    T.first_words = (uint64_t)hs[1] * 8u;
    T.n_walk_rows = (int32_t)hs[2];
    T.tab = alloc_n<uint32_t>(pool, (int64_t)T.sectors * 8);
    T.gbase = alloc_n<uint32_t>(pool, n);
    T.fthr = alloc_n<uint32_t>(pool, (int64_t)T.first_words);
    T.wrow = alloc_n<int4>(pool, T.n_walk_rows);
    T.walk_rows = alloc_n<int32_t>(pool, T.n_walk_rows);
    if (!T.tab || !T.gbase || !T.fthr || !T.wrow || !T.walk_rows) return RW_ERR_ALLOC;
    RW_COUNT_LAUNCH();
    k_fill_tables<<<blocks, 256, 0, s>>>(n, A->row_ptr, A->col, A->val, T.deg, T.lowdeg,
                                         T.diag_pos, T.toff, T.foff8, T.tab, T.gbase, T.fthr, T.S,
                                         T.diag);
    if ((rc = check_launch("fill tables"))) return rc;
    RW_COUNT_LAUNCH();
    k_walk_rows<<<blocks, 256, 0, s>>>(n, T.walk_flag, T.gbase, T.foff8, T.lowdeg, T.wrow,
                                       T.walk_rows);
    return check_launch("walk rows");
}

// ---------------------------------------------------------------------------
// Walk index space: record index = wbase[r] + w for walk w of walk row r.
// chunk_row[c] = the walk row that holds walk c * kWalkChunk.
// ---------------------------------------------------------------------------
__global__ void k_budgets(int32_t nw, const int4* __restrict__ wrow, uint32_t uniform,
                          const uint32_t* __restrict__ budget, int64_t* out, DevStatus* st, int allow_zero) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x) {
        const uint32_t b = budget ? budget[wrow[r].x] : uniform;
        if (b == 0u && !allow_zero) atomicAdd(&st->bad_budget, 1u);
        out[r] = (int64_t)b;
    }
}

__global__ void k_chunk_rows(int32_t nw, const int64_t* __restrict__ wbase, int32_t* chunk_row) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x) {
        const int64_t c0 = (wbase[r] + kWalkChunk - 1) / kWalkChunk;
        const int64_t c1 = (wbase[r + 1] + kWalkChunk - 1) / kWalkChunk;
        for (int64_t c = c0; c < c1; ++c) chunk_row[c] = r;
    }
}

rw_status build_chunk_rows(rw_context* ctx, int32_t nw, const int64_t* wbase, int32_t* chunk_row) {
    if (nw <= 0) return RW_OK;
    RW_COUNT_LAUNCH();
    k_chunk_rows<<<grid_for(nw, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(nw, wbase, chunk_row);
    return check_launch("chunk rows");
}

rw_status build_walk_space(rw_context* ctx, const Tables& T, uint32_t uniform,
                           const uint32_t* d_budget, WalkSpace& ws, Pool& pool, bool allow_zero) {
    cudaStream_t s = ctx->stream;
    const int32_t nw = T.n_walk_rows;
    ws.wbase = alloc_n<int64_t>(pool, nw + 1);
    if (!ws.wbase) return RW_ERR_ALLOC;
    const int blocks = grid_for(nw, 256, ctx->num_sms * 8);
    rw_status rc;
    if (nw > 0) {
        RW_COUNT_LAUNCH();
        k_budgets<<<blocks, 256, 0, s>>>(nw, T.wrow, uniform, d_budget, ws.wbase, ctx->d_status, allow_zero ? 1 : 0);
        if ((rc = check_launch("budgets"))) return rc;
    }
    if ((rc = check_cuda(scan_i64(ws.wbase, ws.wbase, nw, s, pool), "scan"))) return rc;
    int64_t* hs = static_cast<int64_t*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(hs, ws.wbase + nw, 8, cudaMemcpyDeviceToHost, s), "copy")))
        return rc;
    if ((rc = read_status(ctx, "walk budgets"))) return rc;
    ws.total = hs[0];
    ws.nchunks = (ws.total + kWalkChunk - 1) / kWalkChunk;
    ws.chunk_row = alloc_n<int32_t>(pool, ws.nchunks);
    if (!ws.chunk_row) return RW_ERR_ALLOC;
    if (nw > 0) {
        RW_COUNT_LAUNCH();
        k_chunk_rows<<<blocks, 256, 0, s>>>(nw, ws.wbase, ws.chunk_row);
        if ((rc = check_launch("chunk rows"))) return rc;
    }
    return RW_OK;
}

}  // namespace rw
