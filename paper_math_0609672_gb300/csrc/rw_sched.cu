// rw_sched.cu -- schedule and kernels of the triangular solves.
//
// The paper applies the factor by forward/backward substitution (Sec. 4);
// row r of a strict triangular system (CSR rp/col/val) gives
//   x_r = rhs_r / scale_r - sum_p val_p * x_{col_p}
// (scale = D for the forward solve with Y, none for the backward solve with
// Y^T).  Rows are visited in level order (level = 1 + the largest level of a
// dependency).  The DAGs of the walk factor are tall and thin: hundreds of
// levels hold a handful of rows each, where the time is the chain of
// dependent memory round trips, not arithmetic.  The level sequence is cut
// into runs:
//   thin run: consecutive levels of at most kThinWidth rows, solved by ONE
//     block.  Phase 1 sums, in parallel, each row's dependencies that lie
//     outside the run (already final); phase 2 walks the levels with a
//     block barrier between them, keeping the run's x values in shared memory
//     and the next level's entries prefetched in registers.
//   wide run: level-synchronous over the whole co-resident grid, a group of
//     lanes per row (one lane per right-hand side and entry slice), a
//     software grid barrier between levels.
// Every row sums its terms in a fixed order, so results do not depend on
// timing.
#include <algorithm>

#include <cooperative_groups.h>

#include "rw_internal.h"

namespace rw {

constexpr int kThinWidth = 32;       // rows per level in a thin run (one warp each)
constexpr int kThinThreads = 1024;   // the block of a thin run: 32 warps
constexpr int kThinMaxRows = 4096;   // rows per thin run (shared memory)
constexpr size_t kThinSmemBudget = 200 * 1024;
constexpr int kHybridThinLevels = 64;  // hybrid schedule: shorter thin runs join the sync-free launches
static_assert(256 + (int64_t)kThinMaxRows * 16 * 8 <= kSolveWorkspaceBytes, "solve workspace");

// ---------------------------------------------------------------------------
// Schedule construction
// ---------------------------------------------------------------------------
__global__ void k_pos_of(int32_t n, const int32_t* __restrict__ order, int32_t* pos_of) {
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        pos_of[order[p]] = p;
}

__device__ __forceinline__ int run_of_pos(int64_t pos, const int64_t* run_pb, int nruns) {
    int lo = 0, hi = nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (run_pb[mid] <= pos) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Count the packed entries of each thin-run position (all its entries) and
// how many of them lie inside the run.
__global__ void k_sched_count(int32_t n, const int32_t* __restrict__ order,
                              const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const int32_t* __restrict__ pos_of, const int64_t* __restrict__ run_pb,
                              const int32_t* __restrict__ run_thin, int nruns, uint32_t* cnt,
                              int32_t* nin) {
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int r = run_of_pos(p, run_pb, nruns);
        if (!run_thin[r]) {
            cnt[p] = 0u;
            nin[p] = 0;
            continue;
        }
        const int32_t row = order[p];
        const int64_t s = rp[row], e = rp[row + 1];
        int in = 0;
        for (int64_t q = s; q < e; ++q) in += pos_of[col[q]] >= run_pb[r];
        cnt[p] = (uint32_t)(e - s);
        nin[p] = in;
    }
}

// In-run entries of each thin run (summed over the warp's lanes of the same
// run, then one atomic per run and warp).
__global__ void k_run_in(int32_t n, const int32_t* __restrict__ nin, const int64_t* __restrict__ run_pb,
                         const int32_t* __restrict__ run_thin, int nruns, unsigned long long* run_in) {
    for (int32_t b = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; b < n; b += gridDim.x * blockDim.x) {
        const int32_t p = b + (int32_t)lane_id();
        const int r = p < n ? run_of_pos(p, run_pb, nruns) : -1;
        const unsigned v = (p < n && run_thin[r]) ? (unsigned)nin[p] : 0u;
        const unsigned same = __match_any_sync(kFull, r);  // lanes of the same run
        const unsigned t = __reduce_add_sync(same, v);
        if (r >= 0 && (int)lane_id() == __ffs(same) - 1 && t) atomicAdd(run_in + r, (unsigned long long)t);
    }
}

// In-run entries first (slot = position - run start), then the external ones
// (column), each group in the row's original order.
template <typename TV>
__global__ void k_sched_fill(int32_t n, const int32_t* __restrict__ order,
                             const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const TV* __restrict__ val, const float* __restrict__ val32,
                             const int32_t* __restrict__ pos_of, const int64_t* __restrict__ run_pb,
                             const int32_t* __restrict__ run_thin, int nruns,
                             const int64_t* __restrict__ tptr, const int32_t* __restrict__ nin,
                             int32_t* tidx, double* tval, float* tval32) {
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int r = run_of_pos(p, run_pb, nruns);
        if (!run_thin[r]) continue;
        const int32_t row = order[p];
        const int64_t s = rp[row], e = rp[row + 1];
        int64_t oi = tptr[p], oe = tptr[p] + nin[p];
        for (int64_t q = s; q < e; ++q) {
            const int32_t c = col[q];
            const int32_t pc = pos_of[c];
            const int64_t o = pc >= run_pb[r] ? oi++ : oe++;
            tidx[o] = pc >= run_pb[r] ? (int32_t)(pc - run_pb[r]) : c;
            tval[o] = val[q];
            if (tval32) tval32[o] = val32[q];
        }
    }
}

rw_status build_schedule(rw_context* ctx, int32_t n, const int64_t* rp, const int32_t* col,
                         const double* val, const float* val32, const int32_t* order,
                         const int64_t* lptr_dev, int32_t depth, SolveSchedule& S, Pool& pool,
                         Pool& scratch) {
    NvtxRange nvtx_range("rw_schedule");
    cudaStream_t s = ctx->stream;
    rw_status rc;
    const int thin_levels = ctx->opt.thin_levels;
    S.n = n;
    S.depth = depth;
    S.order = order;
    S.lptr = lptr_dev;
    S.runs.clear();
    if (n == 0) return RW_OK;
    S.lptr_h.resize((size_t)depth + 1);
    if ((rc = check_cuda(cudaMemcpyAsync(S.lptr_h.data(), lptr_dev, sizeof(int64_t) * (depth + 1),
                                         cudaMemcpyDeviceToHost, s),
                         "copy")))
        return rc;
    if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
    // cut the levels into runs
    for (int32_t l = 0; l < depth;) {
        const bool thin = S.lptr_h[l + 1] - S.lptr_h[l] <= kThinWidth;
        SolveRun run{thin ? 1 : 0, l, l, S.lptr_h[l], S.lptr_h[l]};
        while (l < depth) {
            const int64_t w = S.lptr_h[l + 1] - S.lptr_h[l];
            const bool t = w <= kThinWidth;
            if (t != thin) break;
            if (thin && S.lptr_h[l + 1] - run.pos_begin > kThinMaxRows) break;
            // a cap on a thin run's levels turns the dependencies on earlier
            // levels into external ones, summed by the whole grid beforehand
            // (the one block of the run then does less FP64 arithmetic per level)
            if (thin && thin_levels > 0 && l - run.lev_begin >= thin_levels) break;
            ++l;
        }
        run.lev_end = l;
        run.pos_end = S.lptr_h[l];
        S.runs.push_back(run);
    }
    const int nruns = (int)S.runs.size();
    std::vector<int64_t> pb(nruns);
    std::vector<int32_t> th(nruns);
    for (int i = 0; i < nruns; ++i) {
        pb[i] = S.runs[i].pos_begin;
        th[i] = S.runs[i].thin;
    }
    int64_t* d_pb = alloc_n<int64_t>(scratch, nruns);
    int32_t* d_th = alloc_n<int32_t>(scratch, nruns);
    int32_t* pos_of = alloc_n<int32_t>(scratch, n);
    uint32_t* cnt = alloc_n<uint32_t>(scratch, n + 1);
    S.tptr = alloc_n<int64_t>(pool, n + 1);
    S.tnin = alloc_n<int32_t>(pool, n);
    if (!d_pb || !d_th || !pos_of || !cnt || !S.tptr || !S.tnin) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemcpyAsync(d_pb, pb.data(), sizeof(int64_t) * nruns,
                                         cudaMemcpyHostToDevice, s),
                         "copy")))
        return rc;
    if ((rc = check_cuda(cudaMemcpyAsync(d_th, th.data(), sizeof(int32_t) * nruns,
                                         cudaMemcpyHostToDevice, s),
                         "copy")))
        return rc;
    const int blocks = grid_for(n, 256, ctx->num_sms * 8);
    RW_COUNT_LAUNCH();
    k_pos_of<<<blocks, 256, 0, s>>>(n, order, pos_of);
    RW_COUNT_LAUNCH();
    k_sched_count<<<blocks, 256, 0, s>>>(n, order, rp, col, pos_of, d_pb, d_th, nruns, cnt, S.tnin);
    if ((rc = check_launch("schedule count"))) return rc;
    if ((rc = check_cuda(scan_u32_to_i64(cnt, S.tptr, n, s, scratch), "scan"))) return rc;
    int64_t* h64 = static_cast<int64_t*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(h64, S.tptr + n, 8, cudaMemcpyDeviceToHost, s), "copy")))
        return rc;
    if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
    S.thin_entries = h64[0];
    S.tidx = alloc_n<int32_t>(pool, S.thin_entries);
    S.tval = alloc_n<double>(pool, S.thin_entries);
    S.tval32 = val32 ? alloc_n<float>(pool, S.thin_entries) : nullptr;
    if (!S.tidx || !S.tval || (val32 && !S.tval32)) return RW_ERR_ALLOC;
    RW_COUNT_LAUNCH();
    k_sched_fill<double><<<blocks, 256, 0, s>>>(n, order, rp, col, val, val32, pos_of, d_pb, d_th,
                                                nruns, S.tptr, S.tnin, S.tidx, S.tval, S.tval32);
    if ((rc = check_launch("schedule fill"))) return rc;
    // in-run entries per thin run (sizes the run's shared-memory copy of them)
    unsigned long long* run_in = alloc_n<unsigned long long>(scratch, nruns);
    if (!run_in) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(run_in, 0, sizeof(unsigned long long) * nruns, s), "memset")))
        return rc;
    RW_COUNT_LAUNCH();
    k_run_in<<<blocks, 256, 0, s>>>(n, S.tnin, d_pb, d_th, nruns, run_in);
    if ((rc = check_launch("run entries"))) return rc;
    std::vector<unsigned long long> hin(nruns);
    if ((rc = check_cuda(cudaMemcpyAsync(hin.data(), run_in, sizeof(unsigned long long) * nruns,
                                         cudaMemcpyDeviceToHost, s),
                         "copy")) ||
        (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
        return rc;
    for (int i = 0; i < nruns; ++i) S.runs[i].in_entries = (int64_t)hin[i];
    return RW_OK;
}

// ---------------------------------------------------------------------------
// External sums of a thin run, by the whole grid (warp per row):
//   ext[slot][j] = sum over the row's dependencies outside the run
// ---------------------------------------------------------------------------
template <typename T, int NR>
__global__ void __launch_bounds__(256) k_thin_ext(int64_t pos_begin, int64_t pos_end,
                                                  const int64_t* __restrict__ tptr,
                                                  const int32_t* __restrict__ tnin,
                                                  const int32_t* __restrict__ tidx,
                                                  const T* __restrict__ tval, const T* x, int nrhs,
                                                  T* ext) {
    const int lane = (int)lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t pos = pos_begin + gw; pos < pos_end; pos += nw) {
        const int64_t e0 = tptr[pos] + tnin[pos], e1 = tptr[pos + 1];
        T acc[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) acc[j] = T(0);
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t c = tidx[e];
            const T y = tval[e];
#pragma unroll
            for (int j = 0; j < NR; ++j)
                if (j < nrhs) acc[j] += y * __ldcg(x + (size_t)c * nrhs + j);
        }
        const T mine = warp_sums<T, NR>(acc);
        if (lane < NR) ext[(pos - pos_begin) * NR + lane] = mine;
    }
}

// ---------------------------------------------------------------------------
// Thin run: one block.
// ---------------------------------------------------------------------------
template <typename T>
struct ThinParams {
    int64_t pos_begin, pos_end;
    int32_t lev_begin, lev_end;
    const int64_t* __restrict__ lptr;
    const int32_t* __restrict__ order;
    const int64_t* __restrict__ tptr;
    const int32_t* __restrict__ tnin;
    const int32_t* __restrict__ tidx;
    const T* __restrict__ tval;
    const T* __restrict__ ext;
    const T* __restrict__ rhs;
    const T* __restrict__ scale;
    T* x;
    int nrhs;
    int stage;  // 1: copy the run's in-run entries to shared memory first
    int stage_entries;
    int flags;  // 1: per-row ready flags in shared memory instead of a barrier per level
    DevStatus* st;
};

// Shared memory of a thin run: x values [rows][NR], row ids, entry offsets and
// counts, level starts, staged-entry offsets, ready flags; then (staged) the
// in-run values and their slot indices.
template <typename T, int NR>
__host__ __device__ __forceinline__ size_t thin_stage_offset(int rows, int nlev) {
    const size_t base = (size_t)rows * NR * sizeof(T) + (size_t)rows * 12 + (size_t)(nlev + 1) * 4 +
                        (size_t)(rows + 1) * 4 + (size_t)rows * 4;
    return (base + 15) & ~(size_t)15;
}

// in-run entries of one row held in registers: up to 32*U, prefetched ahead
template <typename T, int U>
struct RowRegs {
    int slot;
    int n;
    int32_t e0;   // first packed entry, relative to the run
    int32_t s[U];
    T y[U];
};

// NR values of one slot of the shared-memory x array, read as vectors
template <typename T, int NR>
__device__ __forceinline__ void load_slot(const T* p, T (&v)[NR]) {
    if constexpr (sizeof(T) == 8 && NR % 2 == 0) {
#pragma unroll
        for (int j = 0; j < NR; j += 2) {
            const double2 d = *reinterpret_cast<const double2*>(p + j);
            v[j] = d.x;
            v[j + 1] = d.y;
        }
    } else if constexpr (sizeof(T) == 4 && NR % 4 == 0) {
#pragma unroll
        for (int j = 0; j < NR; j += 4) {
            const float4 d = *reinterpret_cast<const float4*>(p + j);
            v[j] = d.x;
            v[j + 1] = d.y;
            v[j + 2] = d.z;
            v[j + 3] = d.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < NR; ++j) v[j] = p[j];
    }
}

// warp_sums over each group of G lanes (G a power of two, NR <= G): value j
// of a group ends in the group's lane j.  G = 32 is warp_sums.
template <typename T, int NR, int G>
__device__ __forceinline__ T group_sums(T (&v)[NR]) {
    const unsigned lane = lane_id();
    int cnt = NR;
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) {
        if (cnt > 1) {
            const int half = cnt / 2;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < NR / 2; ++i) {
                if (i < half) {
                    const T send = upper ? v[i] : v[i + half];
                    const T keep = upper ? v[i + half] : v[i];
                    v[i] = keep + __shfl_xor_sync(kFull, send, o);
                }
            }
            cnt = half;
        } else {
            v[0] += __shfl_xor_sync(kFull, v[0], o);
        }
    }
    constexpr unsigned span = G / NR;  // value j sits in the group's lanes j * span ...
    const unsigned src = (lane & ~(unsigned)(G - 1)) + (((lane & (G - 1)) * span) & (G - 1));
    return __shfl_sync(kFull, v[0], src);
}

// CL: the run is solved by a thread-block cluster instead of one block.  Every
// CTA keeps the whole run's x values in its shared memory; row q of a level
// belongs to CTA q mod csize (warp q / csize), which writes the new value into
// every CTA's copy through distributed shared memory; a cluster barrier ends
// each level.  The level's FP64 work is thereby spread over csize SMs.
//
// G: lanes per row (32 / G rows per warp, without clusters).  The run's one SM
// is bound by its FP64 rate (one warp-wide FP64 instruction per 19 cycles per
// SM on GB300, whatever the lanes active), and a row of a thin run has few
// in-run entries, so G = 8 lets each FP64 instruction serve four rows: the
// entry terms and a three-step reduction per group instead of a five-step one
// per row.
template <typename T, int NR, bool CL, int G = 32>
__global__ void __launch_bounds__(kThinThreads) k_thin(const ThinParams<T> P) {
    static_assert(G == 32 || !CL, "cluster thin runs take one row per warp");
    static_assert(NR <= G && (G & (G - 1)) == 0, "lane groups");
    constexpr int U = 6;
    constexpr int RPW = 32 / G;  // rows per warp
    extern __shared__ __align__(16) unsigned char smem[];
    namespace cg = cooperative_groups;
    const unsigned crank = CL ? cg::this_cluster().block_rank() : 0u;
    const unsigned csz = CL ? cg::this_cluster().num_blocks() : 1u;
    const int rows = (int)(P.pos_end - P.pos_begin);
    const int nlev = P.lev_end - P.lev_begin;
    T* xs = reinterpret_cast<T*>(smem);                                    // [rows][NR]
    int32_t* rowid = reinterpret_cast<int32_t*>(xs + (size_t)rows * NR);   // [rows]
    int32_t* eoff = rowid + rows;                                          // [rows] first in-run entry
    int32_t* ecnt = eoff + rows;                                           // [rows] in-run entries
    int32_t* lstart = ecnt + rows;                                         // [nlev + 1] slots
    const int lane = (int)lane_id();
    const int warp = threadIdx.x >> 5;
    const int gl = lane % G, grp = lane / G;  // lane in its group, group in the warp
    const int64_t run_e0 = P.tptr[P.pos_begin];
    const int32_t* tidx = P.tidx + run_e0;
    const T* tval = P.tval + run_e0;
    int32_t* soff = lstart + nlev + 1;  // [rows + 1] staged: first entry of each slot
    volatile int32_t* ready = soff + rows + 1;  // [rows] flags mode: slot finished

    for (int i = threadIdx.x; i <= nlev; i += blockDim.x)
        lstart[i] = (int32_t)(P.lptr[P.lev_begin + i] - P.pos_begin);
    // phase 1: right-hand side minus the external sums; per-row entry ranges
    for (int slot = threadIdx.x; slot < rows; slot += blockDim.x) {
        const int64_t pos = P.pos_begin + slot;
        const int32_t row = P.order[pos];
        rowid[slot] = row;
        ready[slot] = 0;
        eoff[slot] = (int32_t)(P.tptr[pos] - run_e0);
        ecnt[slot] = P.tnin[pos];
        for (int j = 0; j < P.nrhs && j < NR; ++j) {
            T b = P.rhs[(size_t)row * P.nrhs + j];
            if (P.scale) b = b / P.scale[row];
            xs[(size_t)slot * NR + j] = b - P.ext[(size_t)slot * NR + j];
        }
    }
    __syncthreads();
    if (P.stage) {
        // the run's in-run entries to shared memory: offsets by a block scan of
        // the per-slot counts, then every entry copied by one thread (its slot
        // found by binary search), so the copy is one round of loads
        T* sval = reinterpret_cast<T*>(smem + thin_stage_offset<T, NR>(rows, nlev));
        int32_t* sidx = reinterpret_cast<int32_t*>(sval + P.stage_entries);
        constexpr int kPer = (kThinMaxRows + kThinThreads - 1) / kThinThreads;
        int loc[kPer];
        int sum = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int sl = threadIdx.x * kPer + i;
            loc[i] = sl < rows ? ecnt[sl] : 0;
            sum += loc[i];
        }
        __shared__ int wtot[kThinThreads / 32];
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wtot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int t = wtot[lane];
            int ti = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, ti, o);
                if (lane >= o) ti += y;
            }
            wtot[lane] = ti - t;
        }
        __syncthreads();
        int pre = wtot[warp] + incl - sum;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int sl = threadIdx.x * kPer + i;
            if (sl < rows) soff[sl] = pre;
            if (sl == rows - 1) soff[rows] = pre + loc[i];
            pre += loc[i];
        }
        __syncthreads();
        const int total = soff[rows];
        for (int g = threadIdx.x; g < total; g += blockDim.x) {
            int lo = 0, hi = rows - 1;  // the last slot whose offset is <= g
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (soff[mid] <= g) lo = mid;
                else hi = mid - 1;
            }
            const int src = eoff[lo] + (g - soff[lo]);
            sidx[g] = tidx[src];
            sval[g] = tval[src];
        }
        __syncthreads();
        for (int sl = threadIdx.x; sl < rows; sl += blockDim.x) eoff[sl] = soff[sl];
        tidx = sidx;
        tval = sval;
        __syncthreads();
    }

    // every CTA's copy is initialised before any row value is written into it
    if constexpr (CL) cg::this_cluster().sync();
    // phase 2: the levels in order; in each level warp w takes rows w, w+32, ...
    // (with a cluster: slot q = warp * csize + rank of the level)
    auto fetch = [&](int li, RowRegs<T, U>& R) {
        R.slot = -1;
        R.n = 0;
        if (li < nlev) {
            const int sl = lstart[li] + (warp * RPW + grp) * (int)csz + (int)crank;
            if (sl < lstart[li + 1]) {
                R.slot = sl;
                R.e0 = eoff[sl];
                R.n = ecnt[sl];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = gl + G * u;
            const bool ok = R.slot >= 0 && k < R.n;
            R.s[u] = ok ? tidx[R.e0 + k] : -1;
            R.y[u] = ok ? tval[R.e0 + k] : T(0);
        }
    };
    auto finish = [&](int slot, T mine) {
        if (slot >= 0 && gl < P.nrhs && gl < NR) {
            const T v = xs[(size_t)slot * NR + gl] - mine;
            if constexpr (CL) {
                for (unsigned r = 0; r < csz; ++r)
                    cg::this_cluster().map_shared_rank(xs, r)[(size_t)slot * NR + gl] = v;
            } else {
                xs[(size_t)slot * NR + gl] = v;
            }
            __stcg(P.x + (size_t)rowid[slot] * P.nrhs + gl, v);
        }
    };
    // flags mode: a lane reads an in-run value only once its slot is flagged
    // (bounded wait; the warp holding the lowest unfinished slot always has its
    // dependencies, so the run progresses without a barrier per level)
    // (after one wait gives up, the others of the block give up at once)
    const bool flags = !CL && P.flags != 0;
    __shared__ int gave_up;
    if (threadIdx.x == 0) gave_up = 0;
    __syncthreads();
    const unsigned spin_limit = P.st->spin_limit;
    auto wait_slot = [&](int32_t sl) {
        if (!flags) return;
        unsigned spins = 0;
        while (ready[sl] == 0) {
            if (*(volatile int*)&gave_up) break;
            if (++spins > spin_limit) {
                *(volatile int*)&gave_up = 1;
                atomicAdd(&P.st->timeout, 1u);
                break;
            }
        }
        __threadfence_block();
    };
    RowRegs<T, U> r0, r1;
    fetch(0, r0);
    for (int li = 0; li < nlev; ++li) {
        fetch(li + 1, r1);  // the next level's entries: in flight while this level computes
        if (__any_sync(kFull, r0.slot >= 0)) {  // G = 32: r0.slot is warp-uniform
            T acc[NR];
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[j] = T(0);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (r0.s[u] >= 0) {
                    wait_slot(r0.s[u]);
                    T v[NR];
                    load_slot<T, NR>(xs + (size_t)r0.s[u] * NR, v);
#pragma unroll
                    for (int j = 0; j < NR; ++j) acc[j] += r0.y[u] * v[j];
                }
            if (r0.slot >= 0) {
                for (int k = gl + G * U; k < r0.n; k += G) {  // rows longer than G*U
                    const int32_t sl = tidx[r0.e0 + k];
                    const T y = tval[r0.e0 + k];
                    wait_slot(sl);
                    T v[NR];
                    load_slot<T, NR>(xs + (size_t)sl * NR, v);
#pragma unroll
                    for (int j = 0; j < NR; ++j) acc[j] += y * v[j];
                }
            }
            finish(r0.slot, group_sums<T, NR, G>(acc));
            if (flags) {
                __syncwarp();
                __threadfence_block();
                if (gl == 0 && r0.slot >= 0) ready[r0.slot] = 1;
            }
        }
        // the cluster barrier also keeps every CTA alive until the last remote write
        if constexpr (CL) cg::this_cluster().sync();
        else if (!flags) __syncthreads();
        r0 = r1;
    }
}

// ---------------------------------------------------------------------------
// Wide run: level-synchronous over the co-resident grid.
// ---------------------------------------------------------------------------
template <typename T>
struct WideParams {
    int32_t lev_begin, lev_end;
    const int64_t* __restrict__ lptr;
    const int32_t* __restrict__ order;
    const int64_t* __restrict__ rp;
    const int32_t* __restrict__ col;
    const T* __restrict__ val;
    const T* __restrict__ rhs;
    const T* __restrict__ scale;
    T* x;
    int nrhs;
    unsigned* bar;
    DevStatus* st;
};

// Wide and cluster runs: a group of G = NR * ES lanes per row, 32 / G rows
// per warp.  Lane (es, j) of a group owns right-hand side j and entries
// s + es, s + es + ES, ...: the NR values of x a row entry needs arrive in one
// contiguous load, and only the ES entry slices are summed across lanes.
//
// A level's own chain after the barrier is one round of x loads; the row
// structure it reads (position -> row -> row pointers -> first entries) does
// not depend on x and is loaded two levels ahead, so its dependent loads
// overlap the levels in between.
constexpr int kPreEntries = 4;  // entries per lane held ahead

template <typename T>
struct RowPre {
    int32_t row;  // -1: no row for this group in that level
    int64_t s, e;
    int32_t c[kPreEntries];
    T y[kPreEntries];
};

template <typename T, int NR, int ES>
struct RowGroup {
    static constexpr int G = NR * ES;
    static constexpr int R = 32 / G;
    int j, es;
    unsigned gmask;
    bool jok;
    __device__ RowGroup(int lane, int nrhs) {
        const int gl = lane % G;
        j = gl % NR;
        es = gl / NR;
        gmask = G == 32 ? kFull : (((1u << G) - 1u) << (lane - gl));
        jok = j < nrhs;
    }
    __device__ __forceinline__ void load(const WideParams<T>& P, int32_t row, RowPre<T>& R0) const {
        R0.row = row;
        R0.s = P.rp[row];
        R0.e = P.rp[row + 1];
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u) {
            const int64_t q = R0.s + es + (int64_t)u * ES;
            R0.c[u] = q < R0.e ? P.col[q] : 0;
            R0.y[u] = q < R0.e ? P.val[q] : T(0);
        }
    }
    // x_row = rhs_row / scale_row - sum_q val_q x_{col_q}
    __device__ __forceinline__ void row(const WideParams<T>& P, const RowPre<T>& R0) const {
        const T* __restrict__ x = P.x;
        const int nr = P.nrhs;
        T acc = T(0);
        T v[kPreEntries];
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u)
            v[u] = (jok && R0.s + es + (int64_t)u * ES < R0.e) ? __ldcg(x + (size_t)R0.c[u] * nr + j) : T(0);
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u) acc += R0.y[u] * v[u];
        int64_t q = R0.s + es + (int64_t)kPreEntries * ES;
        for (; q + 3 * ES < R0.e; q += 4 * ES) {
            int32_t c[4];
            T y[4], w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c[u] = P.col[q + u * ES];
                y[u] = P.val[q + u * ES];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = jok ? __ldcg(x + (size_t)c[u] * nr + j) : T(0);
#pragma unroll
            for (int u = 0; u < 4; ++u) acc += y[u] * w[u];
        }
        for (; q < R0.e; q += ES) {
            const int32_t c = P.col[q];
            const T y = P.val[q];
            if (jok) acc += y * __ldcg(x + (size_t)c * nr + j);
        }
#pragma unroll
        for (int o = NR; o < G; o <<= 1) acc += __shfl_xor_sync(gmask, acc, o);
        if (es == 0 && jok) {
            T b = P.rhs[(size_t)R0.row * nr + j];
            if (P.scale) b = b / P.scale[R0.row];
            __stcg(P.x + (size_t)R0.row * nr + j, b - acc);
        }
    }
};

// Vector rows (rw_options.wide_slices = -1): one warp per row; lane l owns
// entries s + l, s + l + 32, ... and reads all right-hand sides of each entry
// in one vector load, so each entry's column and value are loaded once (not
// once per right-hand side) and 4 entries per lane prefetched cover rows of
// up to 128 entries: a long row costs one round of x loads like a short one.
// The NR partial sums are reduced by the halving butterfly of warp_sums;
// lane j * 32 / NR ends with the sum of right-hand side j.
template <typename T, int NR>
struct RowVec {
    static constexpr int G = 32;
    static constexpr int R = 1;
    int lane;
    __device__ RowVec(int lane_, int) : lane(lane_) {}
    __device__ __forceinline__ void load(const WideParams<T>& P, int32_t row, RowPre<T>& R0) const {
        R0.row = row;
        R0.s = P.rp[row];
        R0.e = P.rp[row + 1];
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u) {
            const int64_t q = R0.s + lane + (int64_t)u * 32;
            R0.c[u] = q < R0.e ? P.col[q] : 0;
            R0.y[u] = q < R0.e ? P.val[q] : T(0);
        }
    }
    // the nrhs values of x at node c (vector loads when nrhs == NR)
    __device__ __forceinline__ void xload(const WideParams<T>& P, int32_t c, T (&v)[NR]) const {
        const T* p = P.x + (size_t)c * P.nrhs;
        if constexpr (NR >= 2 && sizeof(T) == 8) {
            if (P.nrhs == NR) {
#pragma unroll
                for (int j = 0; j < NR; j += 2) {
                    const double2 d = __ldcg(reinterpret_cast<const double2*>(p + j));
                    v[j] = d.x;
                    v[j + 1] = d.y;
                }
                return;
            }
        } else if constexpr (NR >= 4 && sizeof(T) == 4) {
            if (P.nrhs == NR) {
#pragma unroll
                for (int j = 0; j < NR; j += 4) {
                    const float4 d = __ldcg(reinterpret_cast<const float4*>(p + j));
                    v[j] = d.x;
                    v[j + 1] = d.y;
                    v[j + 2] = d.z;
                    v[j + 3] = d.w;
                }
                return;
            }
        }
#pragma unroll
        for (int j = 0; j < NR; ++j) v[j] = j < P.nrhs ? __ldcg(p + j) : T(0);
    }
    __device__ __forceinline__ void row(const WideParams<T>& P, const RowPre<T>& R0) const {
        T acc[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) acc[j] = T(0);
        T v[kPreEntries][NR];
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u) {
            if (R0.s + lane + (int64_t)u * 32 < R0.e) {
                xload(P, R0.c[u], v[u]);
            } else {
#pragma unroll
                for (int j = 0; j < NR; ++j) v[u][j] = T(0);
            }
        }
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[j] += R0.y[u] * v[u][j];
        for (int64_t q = R0.s + lane + (int64_t)kPreEntries * 32; q < R0.e; q += 4 * 32) {
            int32_t c[4];
            T y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = q + u * 32 < R0.e;
                c[u] = ok ? P.col[q + u * 32] : 0;
                y[u] = ok ? P.val[q + u * 32] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                // padding slots past the row's end read nothing: x of column 0
                // may still be unset (0 * NaN would poison the sum)
                if (q + u * 32 < R0.e) {
                    T w[NR];
                    xload(P, c[u], w);
#pragma unroll
                    for (int j = 0; j < NR; ++j) acc[j] += y[u] * w[j];
                }
            }
        }
        const T sum = warp_sums_spread<T, NR>(acc);
        constexpr int span = 32 / NR;
        const int j = lane / span;
        if (lane % span == 0 && j < P.nrhs) {
            T b = P.rhs[(size_t)R0.row * P.nrhs + j];
            if (P.scale) b = b / P.scale[R0.row];
            __stcg(P.x + (size_t)R0.row * P.nrhs + j, b - sum);
        }
    }
};

// The row type of a wide or cluster run: lane groups of NR * ES lanes, or
// vector rows when ES == 0.
template <typename T, int NR, int ES>
struct RowSel {
    using type = RowGroup<T, NR, ES>;
};
template <typename T, int NR>
struct RowSel<T, NR, 0> {
    using type = RowVec<T, NR>;
};
template <int NR, int ES>
constexpr int group_lanes() {
    return ES == 0 ? 32 : NR * ES;
}

// The levels of a run over `ngroups` row groups numbered from gid, with a
// barrier between levels.  Returns false if a barrier gave up.
template <typename T, typename Group, typename Barrier>
__device__ __forceinline__ bool run_levels(const WideParams<T>& P, int64_t gid, int64_t ngroups, const Group& g,
                                           Barrier barrier) {
    RowPre<T> pre[2];
    auto prefetch = [&](int32_t l, RowPre<T>& R0) {
        R0.row = -1;
        if (l < P.lev_end) {
            const int64_t pos = P.lptr[l] + gid;
            if (pos < P.lptr[l + 1]) g.load(P, P.order[pos], R0);
        }
    };
    prefetch(P.lev_begin, pre[0]);
    prefetch(P.lev_begin + 1, pre[1]);
    for (int32_t l = P.lev_begin; l < P.lev_end; ++l) {
        const RowPre<T> cur = pre[0];
        pre[0] = pre[1];
        prefetch(l + 2, pre[1]);  // in flight during this level and the next
        if (cur.row >= 0) {
            g.row(P, cur);
            const int64_t le = P.lptr[l + 1];
            for (int64_t pos = P.lptr[l] + gid + ngroups; pos < le; pos += ngroups) {
                RowPre<T> more;
                g.load(P, P.order[pos], more);
                g.row(P, more);
            }
        }
        if (l + 1 < P.lev_end && !barrier()) return false;
    }
    return true;
}

// Wide run: the whole co-resident grid, a software grid barrier between levels.
constexpr int kWideThreads = 512;  // one block per SM: fewer arrivals per grid barrier

template <typename T, int NR, int ES>
__global__ void __launch_bounds__(kWideThreads, 1) k_wide(const WideParams<T> P) {
    using Group = typename RowSel<T, NR, ES>::type;
    const Group g((int)lane_id(), P.nrhs);
    constexpr int R = Group::R;
    const int64_t gid = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * R + lane_id() / (32 / R);
    const int64_t ngroups = (((int64_t)gridDim.x * blockDim.x) >> 5) * R;
    unsigned epoch = 0;
    run_levels<T>(P, gid, ngroups, g, [&]() { return grid_barrier(P.bar, ++epoch, P.st); });
}

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Cluster run: one thread-block cluster (launched as the whole grid); the
// hardware cluster barrier with release / acquire semantics orders each
// level's x stores before the next level's loads (both through L2).  It waits
// only for the CTAs of the cluster, which the hardware schedules together.
template <typename T, int NR, int ES>
__global__ void __launch_bounds__(1024, 1) k_cluster(const WideParams<T> P) {
    using Group = typename RowSel<T, NR, ES>::type;
    const Group g((int)lane_id(), P.nrhs);
    constexpr int R = Group::R;
    const int64_t warps = blockDim.x >> 5;
    const int64_t gid = ((int64_t)cluster_rank() * warps + (threadIdx.x >> 5)) * R + lane_id() / (32 / R);
    const int64_t ngroups = (int64_t)cluster_size() * warps * R;
    run_levels<T>(P, gid, ngroups, g, []() {
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
        return true;
    });
}

// ---------------------------------------------------------------------------
// Sync-free solve (rw_options.solve_mode = 1): one cooperative launch for the
// whole solve.  x starts as the "pending" marker; warp w takes the rows at
// positions w, w + W, ... of the level order; a row loads all its
// dependencies at once, re-polls (bounded) only those still pending, and
// publishes its value with one relaxed store.  Rows are taken in level order
// and all warps are co-resident, so the lowest unfinished position can always
// proceed.  Each warp loads the structure of its next two rows while it waits,
// so a level on the critical path costs one hand-off through L2.
// ---------------------------------------------------------------------------
template <typename T>
struct FreeParams {
    int64_t n;
    const int32_t* __restrict__ order;
    const int64_t* __restrict__ rp;
    const int32_t* __restrict__ col;
    const T* __restrict__ val;
    const T* __restrict__ rhs;
    const T* __restrict__ scale;
    T* x;
    int nrhs;
    DevStatus* st;
};

template <typename T, int NR>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_syncfree(const FreeParams<T> P) {
    constexpr int ES = 32 / NR;
    const int lane = (int)lane_id();
    const int j = lane % NR, es = lane / NR;
    const bool jok = j < P.nrhs;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned spin_limit = P.st->spin_limit;
    struct Pre {
        int32_t row;
        int64_t s, e;
        int32_t c[kPreEntries];
        T y[kPreEntries];
        T b;
    };
    auto load = [&](int64_t pos, Pre& R0) {
        R0.row = -1;
        if (pos >= P.n) return;
        const int32_t row = P.order[pos];
        R0.row = row;
        R0.s = P.rp[row];
        R0.e = P.rp[row + 1];
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u) {
            const int64_t q = R0.s + es + (int64_t)u * ES;
            R0.c[u] = q < R0.e ? P.col[q] : 0;
            R0.y[u] = q < R0.e ? P.val[q] : T(0);
        }
        R0.b = T(0);
        if (es == 0 && jok) {
            R0.b = P.rhs[(size_t)row * P.nrhs + j];
            if (P.scale) R0.b = R0.b / P.scale[row];
        }
    };
    // polls back off after the first few so that waiting warps leave L2
    // bandwidth to the rows being computed
    auto wait_value = [&](const T* src, T v) -> T {
        unsigned spins = 0;
        while (is_pending(v)) {
            if (wait_gives_up(spins, spin_limit, &P.st->timeout)) return T(0);
            if (spins > 4) __nanosleep(64);
            v = ld_relaxed(src);
        }
        return v;
    };
    Pre pre[2];
    load(gw, pre[0]);
    load(gw + nw, pre[1]);
    for (int64_t pos = gw; pos < P.n; pos += nw) {
        const Pre cur = pre[0];
        pre[0] = pre[1];
        load(pos + 2 * nw, pre[1]);
        const int nr = P.nrhs;
        T v[kPreEntries];
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u)
            v[u] = (jok && cur.s + es + (int64_t)u * ES < cur.e) ? ld_relaxed(P.x + (size_t)cur.c[u] * nr + j) : T(0);
        T acc = T(0);
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u) {
            if (jok && cur.s + es + (int64_t)u * ES < cur.e)
                v[u] = wait_value(P.x + (size_t)cur.c[u] * nr + j, v[u]);
            acc += cur.y[u] * v[u];
        }
        for (int64_t q = cur.s + es + (int64_t)kPreEntries * ES; q < cur.e; q += ES) {
            const int32_t c = P.col[q];
            const T y = P.val[q];
            if (jok) {
                const T* src = P.x + (size_t)c * nr + j;
                acc += y * wait_value(src, ld_relaxed(src));
            }
        }
#pragma unroll
        for (int o = NR; o < 32; o <<= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (es == 0 && jok) st_relaxed(P.x + (size_t)cur.row * nr + j, cur.b - acc);
    }
}

// Vector-row variant (rw_options.wide_slices = -1): one warp per row, lane l
// owns entries s + l, s + l + 32, ... and reads all right-hand sides of an
// entry in one relaxed vector load, so 4 entries per lane held ahead cover
// rows of up to 128 entries and a long row on the critical path costs one
// round of loads, not one per few entries.
template <typename T, int NR>
__device__ __forceinline__ void xload_relaxed(const T* x, int nrhs, int32_t c, T (&v)[NR]) {
    const T* p = x + (size_t)c * nrhs;
    if constexpr (NR >= 2 && sizeof(T) == 8) {
        if (nrhs == NR) {
#pragma unroll
            for (int j = 0; j < NR; j += 2) ld_relaxed_v2(reinterpret_cast<const double*>(p + j), v[j], v[j + 1]);
            return;
        }
    } else if constexpr (NR >= 4 && sizeof(T) == 4) {
        if (nrhs == NR) {
#pragma unroll
            for (int j = 0; j < NR; j += 4)
                ld_relaxed_v4(reinterpret_cast<const float*>(p + j), v[j], v[j + 1], v[j + 2], v[j + 3]);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) v[j] = j < nrhs ? ld_relaxed(p + j) : T(0);
}

template <typename T, int NR>
__device__ __forceinline__ bool any_pending(const T (&v)[NR], int nrhs) {
    bool pend = false;
#pragma unroll
    for (int j = 0; j < NR; ++j) pend |= (j < nrhs) && is_pending(v[j]);
    return pend;
}

// MINB = 2 caps the registers so that two 512-thread blocks share an SM:
// twice the rows in flight, at the cost of some spilled prefetch state.
template <typename T, int NR, int MINB>
__global__ void __launch_bounds__(512, MINB) k_syncfree_vec(const FreeParams<T> P) {
    const int lane = (int)lane_id();
    constexpr int span = 32 / NR;
    const int jo = lane / span;  // the right-hand side this lane stores
    const bool owner = (lane % span) == 0 && jo < P.nrhs;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned spin_limit = P.st->spin_limit;
    struct Pre {
        int32_t row;
        int64_t s, e;
        int32_t c[kPreEntries];
        T y[kPreEntries];
        T b;
    };
    auto load = [&](int64_t pos, Pre& R0) {
        R0.row = -1;
        if (pos >= P.n) return;
        const int32_t row = P.order[pos];
        R0.row = row;
        R0.s = P.rp[row];
        R0.e = P.rp[row + 1];
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u) {
            const int64_t q = R0.s + lane + (int64_t)u * 32;
            R0.c[u] = q < R0.e ? P.col[q] : 0;
            R0.y[u] = q < R0.e ? P.val[q] : T(0);
        }
        R0.b = T(0);
        if (owner) {
            R0.b = P.rhs[(size_t)row * P.nrhs + jo];
            if (P.scale) R0.b = R0.b / P.scale[row];
        }
    };
    // re-polls (bounded, backing off) while any of the vector is pending
    auto wait_vec = [&](int32_t c, T (&v)[NR]) {
        unsigned spins = 0;
        while (any_pending<T, NR>(v, P.nrhs)) {
            if (wait_gives_up(spins, spin_limit, &P.st->timeout)) {
#pragma unroll
                for (int j = 0; j < NR; ++j) v[j] = T(0);
                return;
            }
            if (spins > 4) __nanosleep(32);
            xload_relaxed<T, NR>(P.x, P.nrhs, c, v);
        }
    };
    Pre pre[2];
    load(gw, pre[0]);
    load(gw + nw, pre[1]);
    for (int64_t pos = gw; pos < P.n; pos += nw) {
        const Pre cur = pre[0];
        pre[0] = pre[1];
        load(pos + 2 * nw, pre[1]);
        T acc[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) acc[j] = T(0);
        T v[kPreEntries][NR];
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u) {
            if (cur.s + lane + (int64_t)u * 32 < cur.e) {
                xload_relaxed<T, NR>(P.x, P.nrhs, cur.c[u], v[u]);
            } else {
#pragma unroll
                for (int j = 0; j < NR; ++j) v[u][j] = T(0);
            }
        }
#pragma unroll
        for (int u = 0; u < kPreEntries; ++u) {
            if (cur.s + lane + (int64_t)u * 32 < cur.e) wait_vec(cur.c[u], v[u]);
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[j] += cur.y[u] * v[u][j];
        }
        for (int64_t q = cur.s + lane + (int64_t)kPreEntries * 32; q < cur.e; q += 4 * 32) {
            int32_t c[4];
            T y[4], w[4][NR];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = q + u * 32 < cur.e;
                c[u] = ok ? P.col[q + u * 32] : 0;
                y[u] = ok ? P.val[q + u * 32] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (q + u * 32 < cur.e) {
                    xload_relaxed<T, NR>(P.x, P.nrhs, c[u], w[u]);
                } else {
#pragma unroll
                    for (int j = 0; j < NR; ++j) w[u][j] = T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (q + u * 32 < cur.e) wait_vec(c[u], w[u]);
#pragma unroll
                for (int j = 0; j < NR; ++j) acc[j] += y[u] * w[u][j];
            }
        }
        const T sum = warp_sums_spread<T, NR>(acc);
        if (owner) st_relaxed(P.x + (size_t)cur.row * P.nrhs + jo, cur.b - sum);
    }
}

template <typename T>
__global__ void k_inverse_diag(T* w, const T* __restrict__ d, int64_t n, int nrhs) {
    const int64_t cnt = n * nrhs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = w[i] / d[i / nrhs];
}

template <typename T>
rw_status apply_inverse_diag(rw_context* ctx, T* w, const T* d, int64_t n, int nrhs) {
    const int64_t cnt = n * nrhs;
    if (cnt == 0) return RW_OK;
    RW_COUNT_LAUNCH();
    k_inverse_diag<T><<<grid_for(cnt, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(w, d, n, nrhs);
    return check_launch("inverse diagonal");
}
template rw_status apply_inverse_diag<double>(rw_context*, double*, const double*, int64_t, int);
template rw_status apply_inverse_diag<float>(rw_context*, float*, const float*, int64_t, int);

template <typename T>
__global__ void k_fill_pending_sched(T* x, int64_t cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = pending_value(T(0));
}

// Positions [pos_begin, pos_end) of the level order, sync-free; the rows of
// the range must hold the pending marker (fill = true marks the whole vector
// first) and every dependency outside the range must be final.
template <typename T, int NR, bool VEC>
static rw_status solve_syncfree(rw_context* ctx, const SolveSchedule& S, const int64_t* rp, const int32_t* col,
                                const T* val, const T* rhs, const T* scale, T* x, int nrhs,
                                int64_t pos_begin, int64_t pos_end, bool fill) {
    cudaStream_t s = ctx->stream;
    const int two = VEC && ctx->opt.solve_blocks_per_sm >= 2 ? 1 : 0;
    const void* kern;
    if constexpr (VEC) kern = two ? (const void*)k_syncfree_vec<T, NR, 2> : (const void*)k_syncfree_vec<T, NR, 1>;
    else kern = (const void*)k_syncfree<T, NR>;
    static int per_sm_of[2] = {-1, -1};
    int& per_sm = per_sm_of[two];
    if (per_sm < 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, 0);
        if (per_sm < 1) per_sm = 1;
    }
    if (fill) {
        const int64_t cnt = (int64_t)S.n * nrhs;
        RW_COUNT_LAUNCH();
        k_fill_pending_sched<T><<<grid_for(cnt, 256, ctx->num_sms * 8), 256, 0, s>>>(x, cnt);
        rw_status rc = check_launch("pending fill");
        if (rc) return rc;
    }
    const int64_t rows = pos_end - pos_begin;
    int64_t blocks = (int64_t)std::min(per_sm, 2) * ctx->num_sms;
    const int64_t need = (rows + 15) / 16;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    FreeParams<T> P{rows, S.order + pos_begin, rp, col, val, rhs, scale, x, nrhs, ctx->d_status};
    void* args[] = {(void*)&P};
    RW_COUNT_LAUNCH();
    return check_cuda(cudaLaunchCooperativeKernel(kern, dim3((unsigned)blocks), dim3(512), args, 0, s),
                      "sync-free solve");
}

// ---------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------
// Entry slices of the lane groups: an explicit option, else 32 / NR (one
// row per warp), as a power of two with NR * ES <= 32.
static int lane_slices(int opt, int NR) {
    if (opt < 0) return 0;  // vector rows
    const int es = opt > 0 ? opt : 32 / NR;
    int p = 1;
    while (p * 2 <= es && p * 2 * NR <= 32) p *= 2;
    return p;
}

template <typename T, int NR, int ES>
static rw_status launch_wide(rw_context* ctx, const SolveSchedule& S, int32_t lev_begin, int32_t lev_end,
                             const int64_t* rp, const int32_t* col, const T* val, const T* rhs, const T* scale,
                             T* x, int nrhs, unsigned* bar) {
    if constexpr (NR * ES > 32) {
        return RW_ERR_ARG;
    } else {
        cudaStream_t s = ctx->stream;
        static int per_sm = -1;
        if (per_sm < 0) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wide<T, NR, ES>, kWideThreads, 0);
            if (per_sm < 1) per_sm = 1;
        }
        rw_status rc;
        if ((rc = check_cuda(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s), "memset"))) return rc;
        const int bps = ctx->opt.solve_blocks_per_sm > 0 ? ctx->opt.solve_blocks_per_sm : 1;
        int64_t blocks = (int64_t)std::min(per_sm, bps) * ctx->num_sms;
        int64_t maxw = 0;
        for (int32_t l = lev_begin; l < lev_end; ++l) maxw = std::max(maxw, S.lptr_h[l + 1] - S.lptr_h[l]);
        constexpr int64_t rows_per_block = (kWideThreads / 32) * (32 / group_lanes<NR, ES>());
        const int64_t need = (maxw + rows_per_block - 1) / rows_per_block;
        if (blocks > need) blocks = need;
        if (blocks < 1) blocks = 1;
        WideParams<T> P{lev_begin, lev_end, S.lptr, S.order, rp, col, val, rhs, scale, x, nrhs, bar, ctx->d_status};
        void* args[] = {(void*)&P};
        RW_COUNT_LAUNCH();
        return check_cuda(cudaLaunchCooperativeKernel((const void*)k_wide<T, NR, ES>, dim3((unsigned)blocks),
                                                      dim3(kWideThreads), args, 0, s),
                          "wide-run solve");
    }
}

template <typename T, int NR, int ES>
static rw_status launch_cluster(rw_context* ctx, const SolveSchedule& S, int32_t lev_begin, int32_t lev_end,
                                const int64_t* rp, const int32_t* col, const T* val, const T* rhs,
                                const T* scale, T* x, int nrhs, unsigned* bar, int csize) {
    if constexpr (NR * ES > 32) {
        return RW_ERR_ARG;
    } else {
        rw_status arc = set_kernel_attr_once(ctx->device, (const void*)k_cluster<T, NR, ES>,
                                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (arc) return arc;
        WideParams<T> P{lev_begin, lev_end, S.lptr, S.order, rp, col, val, rhs, scale, x, nrhs, bar, ctx->d_status};
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(NR >= 8 ? 512u : 1024u);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = ctx->stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        // the largest size up to csize that the device can place (once per size)
        static int placeable[17] = {};
        if (csize < 1 || csize > 16) csize = 16;
        while (csize > 1) {
            if (placeable[csize] == 0) {
                cfg.gridDim = dim3((unsigned)csize);
                at[0].val.clusterDim.x = (unsigned)csize;
                int nc = 0;
                placeable[csize] =
                    (cudaOccupancyMaxActiveClusters(&nc, k_cluster<T, NR, ES>, &cfg) == cudaSuccess && nc >= 1) ? 1 : -1;
                cudaGetLastError();
            }
            if (placeable[csize] > 0) break;
            csize >>= 1;
        }
        cfg.gridDim = dim3((unsigned)csize);
        at[0].val.clusterDim.x = (unsigned)csize;
        RW_COUNT_LAUNCH();
        return check_cuda(cudaLaunchKernelEx(&cfg, k_cluster<T, NR, ES>, P), "cluster-run solve");
    }
}

template <typename T, int NR, int ES>
static rw_status launch_nonthin(rw_context* ctx, const SolveSchedule& S, const SolveRun& run, const int64_t* rp,
                                const int32_t* col, const T* val, const T* rhs, const T* scale, T* x, int nrhs,
                                unsigned* bar) {
    // consecutive levels up to the cluster width go to one cluster, the rest
    // to the whole grid
    const int64_t cw = ctx->opt.cluster_width > 0 ? ctx->opt.cluster_width : 0;
    const int csize = ctx->opt.cluster_size > 0 ? ctx->opt.cluster_size : 16;
    int32_t l = run.lev_begin;
    while (l < run.lev_end) {
        const bool narrow = cw > 0 && S.lptr_h[l + 1] - S.lptr_h[l] <= cw;
        int32_t e = l + 1;
        while (e < run.lev_end && (cw > 0 && S.lptr_h[e + 1] - S.lptr_h[e] <= cw) == narrow) ++e;
        // cluster runs (1024-thread blocks, 64 registers) keep lane groups
        constexpr int CES = ES == 0 ? 32 / NR : ES;
        rw_status rc = narrow ? launch_cluster<T, NR, CES>(ctx, S, l, e, rp, col, val, rhs, scale, x, nrhs, bar, csize)
                              : launch_wide<T, NR, ES>(ctx, S, l, e, rp, col, val, rhs, scale, x, nrhs, bar);
        if (rc) return rc;
        l = e;
    }
    return RW_OK;
}

// CTAs of a thin run's cluster (rw_options.thin_cluster, a power of two
// <= 16), reduced to the largest size the device can place with this shared
// memory; 1 = one block.
template <typename T, int NR>
static int thin_cluster_size(rw_context* ctx, size_t smem) {
    int want = ctx->opt.thin_cluster;
    if (want < 2) return 1;
    if (want > 16) want = 16;
    int c = 1;
    while (c * 2 <= want) c *= 2;
    static int placeable[17][2] = {};  // per size: 0 unknown, 1 yes, -1 no (by smem above or below 128 KB)
    const int big = smem > 128 * 1024 ? 1 : 0;
    while (c > 1) {
        if (placeable[c][big] == 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)c);
            cfg.blockDim = dim3(kThinThreads);
            cfg.dynamicSmemBytes = big ? kThinSmemBudget + 16 * 1024 : 128 * 1024;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = (unsigned)c;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            placeable[c][big] =
                (cudaOccupancyMaxActiveClusters(&nc, k_thin<T, NR, true>, &cfg) == cudaSuccess && nc >= 1) ? 1 : -1;
            cudaGetLastError();
        }
        if (placeable[c][big] > 0) return c;
        c >>= 1;
    }
    return 1;
}

template <typename T, int NR>
static rw_status solve_runs_nr(rw_context* ctx, const SolveSchedule& S, const int64_t* rp,
                               const int32_t* col, const T* val, const T* tval, const T* rhs,
                               const T* scale, T* x, int nrhs, unsigned* bar, int mode) {
    cudaStream_t s = ctx->stream;
    T* ext = reinterpret_cast<T*>(bar + 64);  // the factor's solve workspace (see build_factor)
    rw_status rc;
    if (mode == 1) {
        if (S.n == 0) return RW_OK;
        // vector rows while one entry's right-hand sides fit in 32 bytes of registers
        if constexpr (NR * sizeof(T) <= 32) {
            if (ctx->opt.wide_slices < 0)
                return solve_syncfree<T, NR, true>(ctx, S, rp, col, val, rhs, scale, x, nrhs, 0, S.n, true);
        }
        return solve_syncfree<T, NR, false>(ctx, S, rp, col, val, rhs, scale, x, nrhs, 0, S.n, true);
    }
    // mode 2 (hybrid): thin runs of at least kHybridThinLevels levels as in the
    // level schedule; everything between them (wide runs and short thin runs,
    // contiguous positions) as one sync-free launch each, so short runs cost no
    // launch of their own.  The whole vector is marked pending once, before
    // the first run (a launch reads only rows of earlier launches, final by
    // then, and its own rows).
    if (mode == 2 && S.n > 0) {
        const int64_t cnt = (int64_t)S.n * nrhs;
        RW_COUNT_LAUNCH();
        k_fill_pending_sched<T><<<grid_for(cnt, 256, ctx->num_sms * 8), 256, 0, s>>>(x, cnt);
        if ((rc = check_launch("pending fill"))) return rc;
    }
    // one-block thin runs: lanes per row (rw_options.thin_lanes), at least NR
    int tl = ctx->opt.thin_lanes == 8 || ctx->opt.thin_lanes == 16 ? ctx->opt.thin_lanes : 32;
    if (tl < NR) tl = 32;
    const void* thin_kern = (const void*)k_thin<T, NR, false>;
    if constexpr (NR <= 8) {
        if (tl == 8) thin_kern = (const void*)k_thin<T, NR, false, 8>;
    }
    if constexpr (NR <= 16) {
        if (tl == 16) thin_kern = (const void*)k_thin<T, NR, false, 16>;
    }
    if ((rc = set_kernel_attr_once(ctx->device, thin_kern,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kThinSmemBudget + 16 * 1024)) ||
        (rc = set_kernel_attr_once(ctx->device, (const void*)k_thin<T, NR, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kThinSmemBudget + 16 * 1024)) ||
        (rc = set_kernel_attr_once(ctx->device, (const void*)k_thin<T, NR, true>,
                                   cudaFuncAttributeNonPortableClusterSizeAllowed, 1)))
        return rc;
    const int es = lane_slices(ctx->opt.wide_slices, NR);
    int64_t free_b = 0, free_e = 0;  // hybrid: positions waiting for one sync-free launch
    auto flush_free = [&]() -> rw_status {
        if (free_e <= free_b) return RW_OK;
        rw_status r2;
        if constexpr (NR * sizeof(T) <= 32) {
            r2 = ctx->opt.wide_slices < 0
                     ? solve_syncfree<T, NR, true>(ctx, S, rp, col, val, rhs, scale, x, nrhs, free_b, free_e, false)
                     : solve_syncfree<T, NR, false>(ctx, S, rp, col, val, rhs, scale, x, nrhs, free_b, free_e, false);
        } else {
            r2 = solve_syncfree<T, NR, false>(ctx, S, rp, col, val, rhs, scale, x, nrhs, free_b, free_e, false);
        }
        free_b = free_e = 0;
        return r2;
    };
    for (const SolveRun& run : S.runs) {
        const int64_t rows = run.pos_end - run.pos_begin;
        if (rows == 0) continue;
        const int nlev = run.lev_end - run.lev_begin;
        size_t smem = thin_stage_offset<T, NR>((int)rows, nlev);
        const size_t staged = smem + (size_t)run.in_entries * (sizeof(T) + 4);
        const int tc = thin_cluster_size<T, NR>(ctx, smem);  // 1: one block
        const bool stage = run.thin && tc == 1 && staged <= kThinSmemBudget + 16 * 1024;
        if (stage) smem = staged;
        const bool thin_ok = run.thin && smem <= kThinSmemBudget + 16 * 1024 && rows <= kThinMaxRows;
        if (mode == 2 && !(thin_ok && nlev >= kHybridThinLevels)) {
            if (free_e <= free_b) free_b = run.pos_begin;
            free_e = run.pos_end;
            continue;
        }
        if (mode == 2 && (rc = flush_free())) return rc;
        if (thin_ok) {
            const int eb = grid_for(rows * 32, 256, ctx->num_sms * 4);
            RW_COUNT_LAUNCH();
            k_thin_ext<T, NR><<<eb, 256, 0, s>>>(run.pos_begin, run.pos_end, S.tptr, S.tnin, S.tidx,
                                                  tval, x, nrhs, ext);
            ThinParams<T> P{run.pos_begin, run.pos_end, run.lev_begin, run.lev_end, S.lptr, S.order,
                            S.tptr, S.tnin, S.tidx, tval, ext, rhs, scale, x, nrhs, stage ? 1 : 0,
                            (int)run.in_entries, ctx->opt.thin_flags ? 1 : 0, ctx->d_status};
            RW_COUNT_LAUNCH();
            if (tc > 1) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)tc);
                cfg.blockDim = dim3(kThinThreads);
                cfg.dynamicSmemBytes = smem;
                cfg.stream = s;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = (unsigned)tc;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                if ((rc = check_cuda(cudaLaunchKernelEx(&cfg, k_thin<T, NR, true>, P), "thin-run cluster solve")))
                    return rc;
            } else {
                void* args[] = {(void*)&P};
                if ((rc = check_cuda(cudaLaunchKernel(thin_kern, dim3(1), dim3(kThinThreads), args, smem, s),
                                     "thin-run solve")))
                    return rc;
            }
            if ((rc = check_launch("thin-run solve"))) return rc;
        } else {
            switch (es) {
                case 0:
                    // vector rows while one entry's right-hand sides fit in 64 bytes of registers
                    if constexpr (NR * sizeof(T) <= 64)
                        rc = launch_nonthin<T, NR, 0>(ctx, S, run, rp, col, val, rhs, scale, x, nrhs, bar);
                    else
                        rc = launch_nonthin<T, NR, 32 / NR>(ctx, S, run, rp, col, val, rhs, scale, x, nrhs, bar);
                    break;
                case 1: rc = launch_nonthin<T, NR, 1>(ctx, S, run, rp, col, val, rhs, scale, x, nrhs, bar); break;
                case 2: rc = launch_nonthin<T, NR, 2>(ctx, S, run, rp, col, val, rhs, scale, x, nrhs, bar); break;
                case 4: rc = launch_nonthin<T, NR, 4>(ctx, S, run, rp, col, val, rhs, scale, x, nrhs, bar); break;
                case 8: rc = launch_nonthin<T, NR, 8>(ctx, S, run, rp, col, val, rhs, scale, x, nrhs, bar); break;
                case 16: rc = launch_nonthin<T, NR, 16>(ctx, S, run, rp, col, val, rhs, scale, x, nrhs, bar); break;
                default: rc = launch_nonthin<T, NR, 32>(ctx, S, run, rp, col, val, rhs, scale, x, nrhs, bar); break;
            }
            if (rc) return rc;
        }
    }
    if (mode == 2 && (rc = flush_free())) return rc;
    return RW_OK;
}

template <typename T>
rw_status solve_runs(rw_context* ctx, const SolveSchedule& S, const int64_t* rp, const int32_t* col,
                     const T* val, const T* tval, const T* rhs, const T* scale, T* x, int nrhs,
                     unsigned* bar, bool backward) {
    NvtxRange nvtx_range(backward ? "rw_solve_bwd" : "rw_solve_fwd");
    const int mode = backward && ctx->opt.solve_mode_bwd >= 0 ? ctx->opt.solve_mode_bwd : ctx->opt.solve_mode;
    int nr = 1;
    while (nr < nrhs) nr <<= 1;
    switch (nr) {
        case 1: return solve_runs_nr<T, 1>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar, mode);
        case 2: return solve_runs_nr<T, 2>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar, mode);
        case 4: return solve_runs_nr<T, 4>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar, mode);
        case 8: return solve_runs_nr<T, 8>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar, mode);
        default: return solve_runs_nr<T, 16>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar, mode);
    }
}

template rw_status solve_runs<double>(rw_context*, const SolveSchedule&, const int64_t*,
                                      const int32_t*, const double*, const double*, const double*,
                                      const double*, double*, int, unsigned*, bool);
template rw_status solve_runs<float>(rw_context*, const SolveSchedule&, const int64_t*,
                                     const int32_t*, const float*, const float*, const float*,
                                     const float*, float*, int, unsigned*, bool);

}  // namespace rw
