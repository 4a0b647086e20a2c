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
//   wide run: level-synchronous over the whole co-resident grid, one warp
//     per row, a software grid barrier between levels.
// Every row sums its terms in a fixed order, so results do not depend on
// timing.
#include <algorithm>

#include "rw_internal.h"

namespace rw {

constexpr int kThinWidth = 32;       // rows per level in a thin run (one warp each)
constexpr int kThinThreads = 1024;   // the block of a thin run: 32 warps
constexpr int kThinMaxRows = 4096;   // rows per thin run (shared memory)
constexpr size_t kThinSmemBudget = 200 * 1024;
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
    cudaStream_t s = ctx->stream;
    rw_status rc;
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
    return check_launch("schedule fill");
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
};

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

template <typename T, int NR>
__global__ void __launch_bounds__(kThinThreads) k_thin(const ThinParams<T> P) {
    constexpr int U = 6;
    extern __shared__ __align__(16) unsigned char smem[];
    const int rows = (int)(P.pos_end - P.pos_begin);
    const int nlev = P.lev_end - P.lev_begin;
    T* xs = reinterpret_cast<T*>(smem);                                    // [rows][NR]
    int32_t* rowid = reinterpret_cast<int32_t*>(xs + (size_t)rows * NR);   // [rows]
    int32_t* eoff = rowid + rows;                                          // [rows] first in-run entry
    int32_t* ecnt = eoff + rows;                                           // [rows] in-run entries
    int32_t* lstart = ecnt + rows;                                         // [nlev + 1] slots
    const int lane = (int)lane_id();
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int64_t run_e0 = P.tptr[P.pos_begin];
    const int32_t* tidx = P.tidx + run_e0;
    const T* tval = P.tval + run_e0;

    for (int i = threadIdx.x; i <= nlev; i += blockDim.x)
        lstart[i] = (int32_t)(P.lptr[P.lev_begin + i] - P.pos_begin);
    // phase 1: right-hand side minus the external sums; per-row entry ranges
    for (int slot = threadIdx.x; slot < rows; slot += blockDim.x) {
        const int64_t pos = P.pos_begin + slot;
        const int32_t row = P.order[pos];
        rowid[slot] = row;
        eoff[slot] = (int32_t)(P.tptr[pos] - run_e0);
        ecnt[slot] = P.tnin[pos];
        for (int j = 0; j < P.nrhs && j < NR; ++j) {
            T b = P.rhs[(size_t)row * P.nrhs + j];
            if (P.scale) b = b / P.scale[row];
            xs[(size_t)slot * NR + j] = b - P.ext[(size_t)slot * NR + j];
        }
    }
    __syncthreads();

    // phase 2: the levels in order; in each level warp w takes rows w, w+32, ...
    auto fetch = [&](int li, RowRegs<T, U>& R) {
        R.slot = -1;
        R.n = 0;
        if (li < nlev) {
            const int sl = lstart[li] + warp;
            if (sl < lstart[li + 1]) {
                R.slot = sl;
                R.e0 = eoff[sl];
                R.n = ecnt[sl];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = lane + 32 * u;
            const bool ok = R.slot >= 0 && k < R.n;
            R.s[u] = ok ? tidx[R.e0 + k] : -1;
            R.y[u] = ok ? tval[R.e0 + k] : T(0);
        }
    };
    auto finish = [&](int slot, T mine) {
        if (lane < P.nrhs && lane < NR) {
            const T v = xs[(size_t)slot * NR + lane] - mine;
            xs[(size_t)slot * NR + lane] = v;
            __stcg(P.x + (size_t)rowid[slot] * P.nrhs + lane, v);
        }
    };
    RowRegs<T, U> r0, r1;
    fetch(0, r0);
    for (int li = 0; li < nlev; ++li) {
        fetch(li + 1, r1);  // the next level's entries: in flight while this level computes
        if (r0.slot >= 0) {
            T acc[NR];
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[j] = T(0);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (r0.s[u] >= 0) {
                    T v[NR];
                    load_slot<T, NR>(xs + (size_t)r0.s[u] * NR, v);
#pragma unroll
                    for (int j = 0; j < NR; ++j) acc[j] += r0.y[u] * v[j];
                }
            for (int k = lane + 32 * U; k < r0.n; k += 32) {  // rows longer than 32*U
                const int32_t sl = tidx[r0.e0 + k];
                const T y = tval[r0.e0 + k];
                T v[NR];
                load_slot<T, NR>(xs + (size_t)sl * NR, v);
#pragma unroll
                for (int j = 0; j < NR; ++j) acc[j] += y * v[j];
            }
            finish(r0.slot, warp_sums<T, NR>(acc));
        }
        __syncthreads();
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

template <typename T, int NR>
__global__ void __launch_bounds__(256) k_wide(const WideParams<T> P) {
    const int lane = (int)lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the first row of this warp in the next level and its first 32 entries are
    // loaded before the barrier that precedes that level
    int32_t nrow = -1;
    int64_t ns = 0, ne = 0;
    int32_t nc = 0;
    T ny = T(0);
    auto prefetch = [&](int32_t l) {
        nrow = -1;
        if (l < P.lev_end) {
            const int64_t pos = P.lptr[l] + gw;
            if (pos < P.lptr[l + 1]) {
                nrow = P.order[pos];
                ns = P.rp[nrow];
                ne = P.rp[nrow + 1];
                const int64_t q = ns + lane;
                nc = q < ne ? P.col[q] : 0;
                ny = q < ne ? P.val[q] : T(0);
            }
        }
    };
    prefetch(P.lev_begin);
    for (int32_t l = P.lev_begin; l < P.lev_end; ++l) {
        const int64_t lb = P.lptr[l], le = P.lptr[l + 1];
        const int32_t row0 = nrow;
        const int64_t s0 = ns, e0 = ne;
        const int32_t c0 = nc;
        const T y0 = ny;
        for (int64_t pos = lb + gw; pos < le; pos += nw) {
            int32_t row;
            int64_t s, e;
            if (pos == lb + gw) {
                row = row0;
                s = s0;
                e = e0;
            } else {
                row = P.order[pos];
                s = P.rp[row];
                e = P.rp[row + 1];
            }
            T acc[NR];
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[j] = T(0);
            for (int64_t q = s + lane; q < e; q += 32) {
                const bool first = pos == lb + gw && q == s + lane;
                const int32_t c = first ? c0 : P.col[q];
                const T y = first ? y0 : P.val[q];
#pragma unroll
                for (int j = 0; j < NR; ++j)
                    if (j < P.nrhs) acc[j] += y * __ldcg(P.x + (size_t)c * P.nrhs + j);
            }
            const T mine = warp_sums<T, NR>(acc);
            if (lane < P.nrhs && lane < NR) {
                T b = P.rhs[(size_t)row * P.nrhs + lane];
                if (P.scale) b = b / P.scale[row];
                __stcg(P.x + (size_t)row * P.nrhs + lane, b - mine);
            }
        }
        prefetch(l + 1);
        if (l + 1 < P.lev_end && !grid_barrier(P.bar, P.st)) return;
    }
}

// ---------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------
template <typename T, int NR>
static rw_status solve_runs_nr(rw_context* ctx, const SolveSchedule& S, const int64_t* rp,
                               const int32_t* col, const T* val, const T* tval, const T* rhs,
                               const T* scale, T* x, int nrhs, unsigned* bar) {
    cudaStream_t s = ctx->stream;
    T* ext = reinterpret_cast<T*>(bar + 64);  // the factor's solve workspace (see build_factor)
    rw_status rc;
    static int wide_per_sm = -1;
    if (wide_per_sm < 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wide_per_sm, k_wide<T, NR>, 256, 0);
        if (wide_per_sm < 1) wide_per_sm = 1;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_thin<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kThinSmemBudget + 16 * 1024);
        attr = true;
    }
    for (const SolveRun& run : S.runs) {
        const int64_t rows = run.pos_end - run.pos_begin;
        if (rows == 0) continue;
        const int nlev = run.lev_end - run.lev_begin;
        const size_t smem =
            (size_t)rows * NR * sizeof(T) + (size_t)rows * 12 + (size_t)(nlev + 1) * 4;
        if (run.thin && smem <= kThinSmemBudget + 16 * 1024 && rows <= kThinMaxRows) {
            const int eb = grid_for(rows * 32, 256, ctx->num_sms * 4);
            RW_COUNT_LAUNCH();
            k_thin_ext<T, NR><<<eb, 256, 0, s>>>(run.pos_begin, run.pos_end, S.tptr, S.tnin, S.tidx,
                                                  tval, x, nrhs, ext);
            ThinParams<T> P{run.pos_begin, run.pos_end, run.lev_begin, run.lev_end, S.lptr, S.order,
                            S.tptr, S.tnin, S.tidx, tval, ext, rhs, scale, x, nrhs};
            RW_COUNT_LAUNCH();
            k_thin<T, NR><<<1, kThinThreads, smem, s>>>(P);
            if ((rc = check_launch("thin-run solve"))) return rc;
        } else {
            if ((rc = check_cuda(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s), "memset")))
                return rc;
            int64_t blocks = (int64_t)std::min(wide_per_sm, 2) * ctx->num_sms;
            int64_t maxw = 0;
            for (int32_t l = run.lev_begin; l < run.lev_end; ++l)
                maxw = std::max(maxw, S.lptr_h[l + 1] - S.lptr_h[l]);
            const int64_t need = (maxw + 7) / 8;
            if (blocks > need) blocks = need;
            if (blocks < 1) blocks = 1;
            WideParams<T> P{run.lev_begin, run.lev_end, S.lptr, S.order, rp, col, val, rhs, scale,
                            x, nrhs, bar, ctx->d_status};
            void* args[] = {(void*)&P};
            RW_COUNT_LAUNCH();
            if ((rc = check_cuda(cudaLaunchCooperativeKernel((const void*)k_wide<T, NR>,
                                                             dim3((unsigned)blocks), dim3(256),
                                                             args, 0, s),
                                 "wide-run solve")))
                return rc;
        }
    }
    return RW_OK;
}

template <typename T>
rw_status solve_runs(rw_context* ctx, const SolveSchedule& S, const int64_t* rp, const int32_t* col,
                     const T* val, const T* tval, const T* rhs, const T* scale, T* x, int nrhs,
                     unsigned* bar) {
    int nr = 1;
    while (nr < nrhs) nr <<= 1;
    switch (nr) {
        case 1: return solve_runs_nr<T, 1>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar);
        case 2: return solve_runs_nr<T, 2>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar);
        case 4: return solve_runs_nr<T, 4>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar);
        case 8: return solve_runs_nr<T, 8>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar);
        default: return solve_runs_nr<T, 16>(ctx, S, rp, col, val, tval, rhs, scale, x, nrhs, bar);
    }
}

template rw_status solve_runs<double>(rw_context*, const SolveSchedule&, const int64_t*,
                                      const int32_t*, const double*, const double*, const double*,
                                      const double*, double*, int, unsigned*);
template rw_status solve_runs<float>(rw_context*, const SolveSchedule&, const int64_t*,
                                     const int32_t*, const float*, const float*, const float*,
                                     const float*, float*, int, unsigned*);

}  // namespace rw
