// rw_solve.cu -- the solve step of Algorithm 1: PCG with M = Y^T diag(D) Y.
//
//   z = M^-1 r:  Y^T w = r (backward), v = w / D, Y z = v (forward).
//
// Vectors are node-major [n, nrhs], so one node's right-hand sides share a
// DRAM sector and every gather serves all of them.  The triangular solves are
// sync-free: rows are visited in level order by a co-resident grid, each
// row's warp waits (bounded) until the values it depends on have left the
// "pending" state, computes its row and publishes it with one relaxed store.
// Scalars (alpha, beta, norms) stay on the device; the host reads one small
// status record per iteration.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "rw_internal.h"

namespace rw {

constexpr int kDotParts = 1024;  // blocks of the dot-product producing kernels

// ---------------------------------------------------------------------------
// SpMV: y = A x for node-major vectors.  GS lanes per row, each lane keeps one
// accumulator per right-hand side.  Optionally accumulates per-block partial
// dot products x.y (per right-hand side) for the PCG step.
//
// DIFF (the FP32 operator of the mixed mode): val holds A_ij (j != i) and, at
// the diagonal position, the excess e_i = A_ii + sum_j A_ij, and the row is
// applied as e_i x_i + sum_{j != i} A_ij (x_j - x_i).  Rounding an R-matrix to
// FP32 this way perturbs edge weights and excesses by a relative 2^-24 each,
// so the operator keeps the near-null space of a weakly grounded matrix
// (rounding A_ii itself would move a row sum by 2^-24 A_ii).
// ---------------------------------------------------------------------------
template <typename TA, typename TV, int NR, int ES, bool DIFF>
__global__ void __launch_bounds__(256) k_spmv(int32_t n, const int32_t* __restrict__ rp,
                                              const int32_t* __restrict__ col,
                                              const TA* __restrict__ val, const TV* __restrict__ x,
                                              TV* __restrict__ y, int nrhs, double* part) {
    // a group of G = NR * ES lanes per row: lane (es, j) owns right-hand side j
    // and entries s + es, s + es + ES, ... (one contiguous load of NR values per
    // entry); the ES entry slices are summed across lanes
    constexpr int G = NR * ES;
    constexpr int R = 32 / G;
    static_assert(G <= 32 && 32 % G == 0, "lane group");
    __shared__ double sdot[8][R][NR];  // per (warp, row group, rhs): summed in a fixed order
    const int lane = (int)lane_id();
    const int gl = lane % G, j = gl % NR, es = gl / NR;
    const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << (lane - gl));
    const int64_t gid = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * R + lane / G;
    const int64_t ngroups = (((int64_t)gridDim.x * blockDim.x) >> 5) * R;
    const bool jok = j < nrhs;
    double mydot = 0.0;
    for (int64_t row = gid; row < n; row += ngroups) {
        const TV xi = (DIFF && jok) ? x[(size_t)row * nrhs + j] : TV(0);
        TV acc = TV(0);
        const int32_t s = rp[row], e = rp[row + 1];
        for (int32_t p = s + es; p < e; p += ES) {
            const int32_t c = col[p];
            const TV a = (TV)val[p];
            if (jok) {
                if (DIFF) acc += (c == row) ? a * xi : a * (x[(size_t)c * nrhs + j] - xi);
                else acc += a * x[(size_t)c * nrhs + j];
            }
        }
#pragma unroll
        for (int o = NR; o < G; o <<= 1) acc += __shfl_xor_sync(gmask, acc, o);
        if (es == 0 && jok) {
            y[(size_t)row * nrhs + j] = acc;
            if (part) mydot += (double)x[(size_t)row * nrhs + j] * (double)acc;
        }
    }
    if (part) {
        if (es == 0) sdot[threadIdx.x >> 5][lane / G][j] = jok ? mydot : 0.0;
        __syncthreads();
        if (threadIdx.x < NR) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                for (int g = 0; g < R; ++g) t += sdot[w][g][threadIdx.x];
            part[(size_t)blockIdx.x * 16 + threadIdx.x] = t;
        }
    }
}

// FP32 operator of the mixed mode (see k_spmv): off-diagonals rounded, the
// diagonal slot replaced by the row's excess (FP64 sum of the row in column
// order, then rounded).  One thread per row.
__global__ void k_to_fp32_diff(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const double* __restrict__ val, float* __restrict__ a32) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t s = rp[i], e = rp[i + 1];
        double ex = 0.0;
        for (int32_t p = s; p < e; ++p) ex = __dadd_rn(ex, val[p]);
        for (int32_t p = s; p < e; ++p) a32[p] = col[p] == i ? (float)ex : (float)val[p];
    }
}

void launch_to_fp32_diff(int32_t n, const int32_t* rp, const int32_t* col, const double* val, float* a32,
                         cudaStream_t s, int num_sms) {
    RW_COUNT_LAUNCH();
    k_to_fp32_diff<<<grid_for(n, 256, num_sms * 8), 256, 0, s>>>(n, rp, col, val, a32);
}

template <typename T>
__global__ void k_fill_pending(T* x, int64_t cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = pending_value(T(0));
}

// ---------------------------------------------------------------------------
// PCG vector kernels and device scalars.
// ---------------------------------------------------------------------------
struct PcgScalars {
    double bnorm2[16];
    double rho[16];
    double pq[16];
    double alpha[16];
    double rr[16];
    double tt[16];
    double beta[16];
    int active[16];
    int check[16];
    int iters[16];
    int broke;
    int any_active;
    int any_check;
    int pad;
};

// Deterministic reduction of per-block partials: part[b * NR + j].
__device__ double reduce_parts(const double* part, int nparts, int j) {
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(size_t)b * 16 + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

enum ScalarOp { kOpBnorm = 0, kOpRho0, kOpAlpha, kOpResid, kOpTrue, kOpBeta, kOpReport };

// One block of 256 threads.  part: [kDotParts][16].
__global__ void __launch_bounds__(256) k_scalars(PcgScalars* S, const double* part, int nparts,
                                                 int nrhs, int op, double tol, int it) {
    for (int j = 0; j < nrhs; ++j) {
        const double v = reduce_parts(part, nparts, j);
        if (threadIdx.x != 0) continue;
        switch (op) {
            case kOpBnorm:
                S->bnorm2[j] = v;
                S->active[j] = v > 0.0;
                S->iters[j] = 0;
                break;
            case kOpRho0:
                S->rho[j] = v;
                break;
            case kOpAlpha:
                S->pq[j] = v;
                if (S->active[j]) {
                    if (!(v > 0.0)) {
                        S->broke = 1;
                        S->active[j] = 0;
                        S->alpha[j] = 0.0;
                    } else {
                        S->alpha[j] = S->rho[j] / v;
                    }
                } else {
                    S->alpha[j] = 0.0;
                }
                break;
            case kOpResid:
                S->rr[j] = v;
                S->check[j] = S->active[j] && (sqrt(v) < tol * sqrt(S->bnorm2[j]));
                break;
            case kOpTrue:
                S->tt[j] = v;
                if (S->check[j] && sqrt(v) < tol * sqrt(S->bnorm2[j])) {
                    S->active[j] = 0;
                    S->iters[j] = it;
                }
                break;
            case kOpBeta:
                S->beta[j] = S->active[j] ? v / S->rho[j] : 0.0;
                S->rho[j] = v;
                break;
            case kOpReport:
                S->tt[j] = v;
                break;
        }
    }
    if (threadIdx.x == 0) {
        int a = 0, c = 0;
        for (int j = 0; j < nrhs; ++j) {
            a |= S->active[j];
            c |= S->check[j];
        }
        S->any_active = a;
        S->any_check = c;
        if (op == kOpTrue)
            for (int j = 0; j < nrhs; ++j) S->check[j] = 0;
    }
}

// Fixed-order block sum of one value per (thread, right-hand side j < 16):
// warp sums, then the warps' sums in warp order, into part[blockIdx][j].
__device__ __forceinline__ void block_parts16(double (&acc)[16], double* part) {
    __shared__ double ws[8][16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = warp_sum(acc[j]);
    if (lane_id() == 0)
#pragma unroll
        for (int j = 0; j < 16; ++j) ws[threadIdx.x >> 5][j] = acc[j];
    __syncthreads();
    if (threadIdx.x < 16) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w][threadIdx.x];
        part[(size_t)blockIdx.x * 16 + threadIdx.x] = t;
    }
}

// Block-level partial sums of a.b per right-hand side into part[blockIdx][j].
template <typename TA, typename TB>
__device__ void block_dot_parts(const TA* a, const TB* b, int64_t n, int nrhs, double* part) {
    double acc[16];
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    // thread handles whole nodes so that each accumulator belongs to one rhs
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < nrhs; ++j)
            acc[j] += (double)a[i * nrhs + j] * (double)b[i * nrhs + j];
    block_parts16(acc, part);
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_dot(const TA* a, const TB* b, int64_t n, int nrhs,
                                             double* part) {
    block_dot_parts(a, b, n, nrhs, part);
}

// x += alpha p (x FP64), r -= alpha q; partial r.r; marks w and z pending.
template <typename T>
__global__ void __launch_bounds__(256) k_update_xr(int64_t n, int nrhs, const PcgScalars* S,
                                                   double* x, T* r, const T* p, const T* q, T* w,
                                                   T* z, double* part) {
    __shared__ double al[16];
    if (threadIdx.x < 16) al[threadIdx.x] = threadIdx.x < (unsigned)nrhs ? S->alpha[threadIdx.x] : 0.0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < nrhs; ++j) {
            const size_t o = (size_t)i * nrhs + j;
            const double a = al[j];
            if (a != 0.0) {
                x[o] += a * (double)p[o];
                r[o] = (T)((double)r[o] - a * (double)q[o]);
            }
            w[o] = pending_value(T(0));
            z[o] = pending_value(T(0));
        }
    __syncthreads();
    block_dot_parts(r, r, n, nrhs, part);
}

// p = z + beta p
template <typename T>
__global__ void __launch_bounds__(256) k_update_p(int64_t n, int nrhs, const PcgScalars* S,
                                                  const T* z, T* p) {
    __shared__ double be[16];
    if (threadIdx.x < 16) be[threadIdx.x] = threadIdx.x < (unsigned)nrhs ? S->beta[threadIdx.x] : 0.0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < nrhs; ++j) {
            const size_t o = (size_t)i * nrhs + j;
            p[o] = (T)((double)z[o] + be[j] * (double)p[o]);
        }
}

// t = b - A x in FP64 (true residual), optionally stored to r (residual
// replacement) in T; partial t.t.
template <typename T>
__global__ void __launch_bounds__(256) k_true_resid(int32_t n, const int32_t* __restrict__ rp,
                                                    const int32_t* __restrict__ col,
                                                    const double* __restrict__ val,
                                                    const double* __restrict__ b,
                                                    const double* __restrict__ x, int nrhs,
                                                    T* r_out, double* part) {
    double acc2[16];
    for (int j = 0; j < 16; ++j) acc2[j] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = rp[i], e = rp[i + 1];
        for (int j = 0; j < nrhs; ++j) {
            double ax = 0.0;
            for (int32_t p = s; p < e; ++p) ax += val[p] * x[(size_t)col[p] * nrhs + j];
            const double t = b[(size_t)i * nrhs + j] - ax;
            if (r_out) r_out[(size_t)i * nrhs + j] = (T)t;
            acc2[j] += t * t;
        }
    }
    block_parts16(acc2, part);
}

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin* in, Tout* out, int64_t cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (Tout)in[i];
}

__global__ void k_check_finite(const double* v, int64_t cnt, DevStatus* st) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicAdd(&st->nonfinite, 1u);
}

// ---------------------------------------------------------------------------
// Host-side dispatch
// ---------------------------------------------------------------------------
static int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <typename TA, typename TV, int NR, int ES>
static void launch_spmv_es(int32_t n, const int32_t* rp, const int32_t* col, const TA* val, const TV* x, TV* y,
                           int nrhs, double* part, int blocks, cudaStream_t s) {
    if constexpr (NR * ES <= 32) {
        RW_COUNT_LAUNCH();
        // FP32 values are always the excess + difference form of the mixed mode
        k_spmv<TA, TV, NR, ES, sizeof(TA) == 4><<<blocks, 256, 0, s>>>(n, rp, col, val, x, y, nrhs, part);
    }
}

template <typename TA, typename TV, int NR>
static void launch_spmv_nr(const rw_context* ctx, int32_t n, const int32_t* rp, const int32_t* col,
                           const TA* val, const TV* x, TV* y, int nrhs, double* part, cudaStream_t s) {
    int es = ctx->opt.spmv_slices > 0 ? ctx->opt.spmv_slices : 32 / NR;
    int p = 1;
    while (p * 2 <= es && p * 2 * NR <= 32) p *= 2;
    const int rows_per_block = 8 * (32 / (NR * p));
    const int blocks = part ? kDotParts : grid_for(((int64_t)n + rows_per_block - 1) / rows_per_block, 1,
                                                   ctx->num_sms * 16);
    switch (p) {
        case 1: launch_spmv_es<TA, TV, NR, 1>(n, rp, col, val, x, y, nrhs, part, blocks, s); break;
        case 2: launch_spmv_es<TA, TV, NR, 2>(n, rp, col, val, x, y, nrhs, part, blocks, s); break;
        case 4: launch_spmv_es<TA, TV, NR, 4>(n, rp, col, val, x, y, nrhs, part, blocks, s); break;
        case 8: launch_spmv_es<TA, TV, NR, 8>(n, rp, col, val, x, y, nrhs, part, blocks, s); break;
        case 16: launch_spmv_es<TA, TV, NR, 16>(n, rp, col, val, x, y, nrhs, part, blocks, s); break;
        default: launch_spmv_es<TA, TV, NR, 32>(n, rp, col, val, x, y, nrhs, part, blocks, s); break;
    }
}

template <typename TA, typename TV>
static rw_status launch_spmv(rw_context* ctx, int32_t n, const int32_t* rp, const int32_t* col,
                             const TA* val, const TV* x, TV* y, int nrhs, double* part) {
    cudaStream_t s = ctx->stream;
    const int nr = pow2_at_least(nrhs);
    switch (nr) {
        case 1: launch_spmv_nr<TA, TV, 1>(ctx, n, rp, col, val, x, y, nrhs, part, s); break;
        case 2: launch_spmv_nr<TA, TV, 2>(ctx, n, rp, col, val, x, y, nrhs, part, s); break;
        case 4: launch_spmv_nr<TA, TV, 4>(ctx, n, rp, col, val, x, y, nrhs, part, s); break;
        case 8: launch_spmv_nr<TA, TV, 8>(ctx, n, rp, col, val, x, y, nrhs, part, s); break;
        default: launch_spmv_nr<TA, TV, 16>(ctx, n, rp, col, val, x, y, nrhs, part, s); break;
    }
    return check_launch("spmv");
}

template <typename T>
rw_status spmv_launch(rw_context* ctx, int32_t n, const int32_t* rp, const int32_t* col, const T* val,
                      const T* x, T* y, int nrhs) {
    NvtxRange nvtx_range("rw_spmv");
    return launch_spmv<T, T>(ctx, n, rp, col, val, x, y, nrhs, nullptr);
}
template rw_status spmv_launch<double>(rw_context*, int32_t, const int32_t*, const int32_t*, const double*,
                                       const double*, double*, int);
template rw_status spmv_launch<float>(rw_context*, int32_t, const int32_t*, const int32_t*, const float*,
                                      const float*, float*, int);

template <typename T>
static rw_status fill_pending(rw_context* ctx, T* x, int64_t cnt) {
    RW_COUNT_LAUNCH();
    k_fill_pending<T><<<grid_for(cnt, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(x, cnt);
    return check_launch("fill");
}

// Device-time accumulation of the solve phases (events on the context stream).
struct SolveTimes {
    bool on = false;
    float spmv = 0.f, bwd = 0.f, fwd = 0.f;
    bool pending_spmv = false, pending_pre = false;
};

// z = Y^-1 D^-1 Y^-T r; w: scratch [n, nrhs].  With timing, events 5/6/7
// bracket the two solves (read by the caller).
template <typename T>
static const T* thin_values(const SolveSchedule& S);
template <>
const double* thin_values<double>(const SolveSchedule& S) { return S.tval; }
template <>
const float* thin_values<float>(const SolveSchedule& S) { return S.tval32; }

template <typename T>
static rw_status precond_t(rw_context* ctx, const FactorView& F, const T* yv, const T* ytv,
                           const T* d, const T* r, T* w, T* z, int nrhs, SolveTimes* tm = nullptr) {
    NvtxRange nvtx_range("rw_precond");
    if (tm && tm->on) cudaEventRecord(ctx->ev[5], ctx->stream);
    rw_status rc = solve_runs<T>(ctx, *F.bwd_sched, F.yt_rp, F.yt_col, ytv,
                                 thin_values<T>(*F.bwd_sched), r, nullptr, w, nrhs, F.bar, true);
    if (rc) return rc;
    if (tm && tm->on) cudaEventRecord(ctx->ev[6], ctx->stream);
    if ((rc = apply_inverse_diag<T>(ctx, w, d, F.n, nrhs))) return rc;
    rc = solve_runs<T>(ctx, *F.fwd_sched, F.y_rp, F.y_col, yv, thin_values<T>(*F.fwd_sched), w, nullptr,
                       z, nrhs, F.bar);
    if (tm && tm->on) {
        cudaEventRecord(ctx->ev[7], ctx->stream);
        tm->pending_pre = true;
    }
    return rc;
}

// Adds the completed event intervals of the last preconditioner application
// and SpMV (the stream has been synchronised by the caller).
static void collect_times(rw_context* ctx, SolveTimes& tm) {
    float t = 0.f;
    if (tm.pending_pre) {
        if (cudaEventElapsedTime(&t, ctx->ev[5], ctx->ev[6]) == cudaSuccess) tm.bwd += t;
        if (cudaEventElapsedTime(&t, ctx->ev[6], ctx->ev[7]) == cudaSuccess) tm.fwd += t;
        tm.pending_pre = false;
    }
    if (tm.pending_spmv) {
        if (cudaEventElapsedTime(&t, ctx->ev[2], ctx->ev[3]) == cudaSuccess) tm.spmv += t;
        tm.pending_spmv = false;
    }
}

void launch_to_fp32(const double* in, float* out, int64_t cnt, cudaStream_t s, int num_sms) {
    RW_COUNT_LAUNCH();
    k_convert<double, float><<<grid_for(cnt, 256, num_sms * 8), 256, 0, s>>>(in, out, cnt);
}

rw_status spmv_fp64(rw_context* ctx, const rw_csr* A, const double* x, double* y, int nrhs) {
    return launch_spmv<double, double>(ctx, A->n, A->row_ptr, A->col, A->val, x, y, nrhs, nullptr);
}

rw_status precond_fp64(rw_context* ctx, const FactorView& F, const double* r, double* z,
                       int nrhs, Pool& scratch) {
    const int64_t cnt = (int64_t)F.n * nrhs;
    double* w = alloc_n<double>(scratch, cnt);
    if (!w) return RW_ERR_ALLOC;
    rw_status rc;
    if ((rc = fill_pending(ctx, w, cnt))) return rc;
    if ((rc = fill_pending(ctx, z, cnt))) return rc;
    if ((rc = precond_t<double>(ctx, F, F.y_val, F.yt_val, F.d, r, w, z, nrhs))) return rc;
    return read_status(ctx, "preconditioner");
}

template <typename T>
static rw_status pcg_t(rw_context* ctx, const rw_csr* A, const FactorView& F, const double* b,
                       double* x, int nrhs, double tol, int max_iter, rw_pcg_stats* stats,
                       int32_t* h_iters, double* h_relres, Pool& sc, const T* Aval, const T* yv,
                       const T* ytv, const T* dv, bool mixed) {
    NvtxRange nvtx_range("rw_pcg");
    cudaStream_t s = ctx->stream;
    const int32_t n = A->n;
    const int64_t cnt = (int64_t)n * nrhs;
    T* r = alloc_n<T>(sc, cnt);
    T* z = alloc_n<T>(sc, cnt);
    T* p = alloc_n<T>(sc, cnt);
    T* q = alloc_n<T>(sc, cnt);
    T* w = alloc_n<T>(sc, cnt);
    double* part = alloc_n<double>(sc, (int64_t)kDotParts * 16);
    PcgScalars* S = alloc_n<PcgScalars>(sc, 1);
    if (!r || !z || !p || !q || !w || !part || !S) return RW_ERR_ALLOC;
    PcgScalars* hS = static_cast<PcgScalars*>(ctx->h_small);
    const int vb = grid_for(n, 256, kDotParts);
    rw_status rc;
    if ((rc = check_cuda(cudaMemsetAsync(S, 0, sizeof(PcgScalars), s), "memset"))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)cnt, s), "memset"))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(part, 0, sizeof(double) * kDotParts * 16, s), "memset")))
        return rc;
    RW_COUNT_LAUNCH();
    k_check_finite<<<vb, 256, 0, s>>>(b, cnt, ctx->d_status);
    RW_COUNT_LAUNCH();
    k_convert<double, T><<<vb, 256, 0, s>>>(b, r, cnt);
    RW_COUNT_LAUNCH();
    k_dot<double, double><<<vb, 256, 0, s>>>(b, b, n, nrhs, part);
    RW_COUNT_LAUNCH();
    k_scalars<<<1, 256, 0, s>>>(S, part, vb, nrhs, kOpBnorm, tol, 0);
    if ((rc = check_launch("pcg init"))) return rc;
    if ((rc = fill_pending(ctx, w, cnt))) return rc;
    if ((rc = fill_pending(ctx, z, cnt))) return rc;
    SolveTimes tm;
    tm.on = ctx->opt.timing != 0;
    if ((rc = precond_t<T>(ctx, F, yv, ytv, dv, r, w, z, nrhs, &tm))) return rc;
    RW_COUNT_LAUNCH();
    k_dot<T, T><<<vb, 256, 0, s>>>(r, z, n, nrhs, part);
    RW_COUNT_LAUNCH();
    k_scalars<<<1, 256, 0, s>>>(S, part, vb, nrhs, kOpRho0, tol, 0);
    RW_COUNT_LAUNCH();
    k_convert<T, T><<<vb, 256, 0, s>>>(z, p, cnt);
    if ((rc = check_launch("pcg start"))) return rc;
    if ((rc = check_cuda(cudaMemcpyAsync(hS, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s), "copy")))
        return rc;
    if ((rc = read_status(ctx, "pcg start"))) return rc;
    if (ctx->d_status && ctx->h_status->nonfinite) {
        set_error("pcg: right-hand side holds a non-finite value");
        return RW_ERR_ARG;
    }
    int done_iters = 0;
    const int refine = ctx->opt.refine_every > 0 ? ctx->opt.refine_every : 50;
    bool any_active = hS->any_active != 0;
    for (int it = 1; it <= max_iter && any_active; ++it) {
        done_iters = it;
        if (tm.on) cudaEventRecord(ctx->ev[2], s);
        if ((rc = launch_spmv<T, T>(ctx, n, A->row_ptr, A->col, Aval, p, q, nrhs, part))) return rc;
        if (tm.on) {
            cudaEventRecord(ctx->ev[3], s);
            tm.pending_spmv = true;
        }
        RW_COUNT_LAUNCH();
        k_scalars<<<1, 256, 0, s>>>(S, part, kDotParts, nrhs, kOpAlpha, tol, it);
        RW_COUNT_LAUNCH();
        k_update_xr<T><<<vb, 256, 0, s>>>(n, nrhs, S, x, r, p, q, w, z, part);
        if (mixed && it % refine == 0) {
            RW_COUNT_LAUNCH();
            k_true_resid<T><<<vb, 256, 0, s>>>(n, A->row_ptr, A->col, A->val, b, x, nrhs, r, part);
        }
        RW_COUNT_LAUNCH();
        k_scalars<<<1, 256, 0, s>>>(S, part, vb, nrhs, kOpResid, tol, it);
        if ((rc = check_launch("pcg step"))) return rc;
        if ((rc = check_cuda(cudaMemcpyAsync(hS, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s),
                             "copy")))
            return rc;
        if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
        if (tm.on) collect_times(ctx, tm);
        if (hS->any_check) {
            RW_COUNT_LAUNCH();
            k_true_resid<T><<<vb, 256, 0, s>>>(n, A->row_ptr, A->col, A->val, b, x, nrhs, nullptr,
                                               part);
            RW_COUNT_LAUNCH();
            k_scalars<<<1, 256, 0, s>>>(S, part, vb, nrhs, kOpTrue, tol, it);
            if ((rc = check_launch("pcg true residual"))) return rc;
            if ((rc = check_cuda(cudaMemcpyAsync(hS, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost,
                                                 s),
                                 "copy")))
                return rc;
            if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
            if (!hS->any_active) break;
        }
        if (hS->broke) break;
        if ((rc = precond_t<T>(ctx, F, yv, ytv, dv, r, w, z, nrhs, &tm))) return rc;
        RW_COUNT_LAUNCH();
        k_dot<T, T><<<vb, 256, 0, s>>>(r, z, n, nrhs, part);
        RW_COUNT_LAUNCH();
        k_scalars<<<1, 256, 0, s>>>(S, part, vb, nrhs, kOpBeta, tol, it);
        RW_COUNT_LAUNCH();
        k_update_p<T><<<vb, 256, 0, s>>>(n, nrhs, S, z, p);
        if ((rc = check_launch("pcg direction"))) return rc;
    }
    // final true residuals for the report
    RW_COUNT_LAUNCH();
    k_true_resid<T><<<vb, 256, 0, s>>>(n, A->row_ptr, A->col, A->val, b, x, nrhs, nullptr, part);
    RW_COUNT_LAUNCH();
    k_scalars<<<1, 256, 0, s>>>(S, part, vb, nrhs, kOpReport, tol, done_iters);
    if ((rc = check_launch("pcg report"))) return rc;
    if ((rc = check_cuda(cudaMemcpyAsync(hS, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s), "copy")))
        return rc;
    if ((rc = read_status(ctx, "pcg"))) return rc;
    if (tm.on) collect_times(ctx, tm);
    int maxit = 0;
    double maxrel = 0.0;
    bool conv_all = true;
    for (int j = 0; j < nrhs; ++j) {
        const int itj = hS->active[j] ? done_iters : hS->iters[j];
        if (hS->active[j]) conv_all = false;
        const double rel = hS->bnorm2[j] > 0.0 ? std::sqrt(hS->tt[j] / hS->bnorm2[j]) : 0.0;
        maxit = std::max(maxit, itj);
        maxrel = std::max(maxrel, rel);
        if (h_iters) h_iters[j] = itj;
        if (h_relres) h_relres[j] = rel;
    }
    if (stats) {
        stats->iterations = maxit;
        stats->rel_residual = maxrel;
        stats->spmv_ms = tm.spmv;
        stats->bwd_ms = tm.bwd;
        stats->fwd_ms = tm.fwd;
    }
    if (hS->broke) {
        set_error("pcg breakdown: p.Ap <= 0");
        return RW_ERR_BREAKDOWN;
    }
    if (tol > 0.0 && !conv_all) {
        set_error("pcg did not reach the tolerance in %d iterations", max_iter);
        return RW_ERR_NO_CONVERGENCE;
    }
    return RW_OK;
}

rw_status pcg_run(rw_context* ctx, const rw_csr* A, const FactorView& F, const double* b,
                  double* x, int nrhs, double tol, int max_iter, rw_precision prec,
                  rw_pcg_stats* stats, int32_t* h_iters, double* h_relres) {
    Pool sc(ctx);
    cudaStream_t s = ctx->stream;
    rw_status rc;
    if (ctx->opt.timing) cudaEventRecord(ctx->ev[8], s);
    if (prec == RW_FP32_MIXED) {
        if (!F.y_val32 || !F.yt_val32 || !F.d32) {
            set_error("pcg: FP32 mode needs a factor built with store_fp32 = 1");
            return RW_ERR_ARG;
        }
        float* a32 = alloc_n<float>(sc, A->nnz);
        if (!a32) return RW_ERR_ALLOC;
        launch_to_fp32_diff(A->n, A->row_ptr, A->col, A->val, a32, s, ctx->num_sms);
        if ((rc = check_launch("convert A"))) return rc;
        rc = pcg_t<float>(ctx, A, F, b, x, nrhs, tol, max_iter, stats, h_iters, h_relres, sc, a32,
                          F.y_val32, F.yt_val32, F.d32, true);
    } else {
        rc = pcg_t<double>(ctx, A, F, b, x, nrhs, tol, max_iter, stats, h_iters, h_relres, sc,
                           A->val, F.y_val, F.yt_val, F.d, false);
    }
    if (ctx->opt.timing && stats) {
        cudaEventRecord(ctx->ev[9], s);
        cudaEventSynchronize(ctx->ev[9]);
        cudaEventElapsedTime(&stats->solve_ms, ctx->ev[8], ctx->ev[9]);
    }
    return rc;
}


// ---------------------------------------------------------------------------
// BiCGSTAB with right preconditioning (van der Vorst's method) for a
// nonsymmetric A, one right-hand side, FP64.  The preconditioner is the
// two-game factor of Sec. 7.1 (M = Y_{A^T}^T D Y_A): the view's forward data
// come from the game on A, its backward data from the game on A^T, and it is
// applied by the same backward and forward solves as in PCG.  Dot products:
// per-block sums on the device, added in a fixed order by one warp, so every
// run takes the same iterations.  Convergence is decided on the true residual
// ||b - A x|| < tol ||b||, recomputed whenever the recursive one passes (and
// then replacing it).
// ---------------------------------------------------------------------------
__global__ void k_lin3(int64_t n, double* out, const double* a, double ca, const double* b, double cb,
                       const double* c, double cc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = ca * a[i];
        if (b) v += cb * b[i];
        if (c) v += cc * c[i];
        out[i] = v;
    }
}

// One warp adds the block sums of right-hand side 0 in a fixed order.
__global__ void k_sum_parts(const double* __restrict__ part, int nblocks, double* out) {
    double t = 0.0;
    for (int b = (int)lane_id(); b < nblocks; b += 32) t += part[(size_t)b * 16];
    t = warp_sum(t);
    if (lane_id() == 0) *out = t;
}

rw_status bicgstab_run(rw_context* ctx, const rw_csr* A, const FactorView& F, const double* b, double* x, double tol,
                       int max_iter, rw_pcg_stats* stats) {
    cudaStream_t s = ctx->stream;
    const int32_t n = A->n;
    const int64_t launches0 = g_launches;
    Pool sc(ctx);
    double* r = alloc_n<double>(sc, n);
    double* rh = alloc_n<double>(sc, n);
    double* pv = alloc_n<double>(sc, n);
    double* ph = alloc_n<double>(sc, n);
    double* v = alloc_n<double>(sc, n);
    double* sv = alloc_n<double>(sc, n);
    double* sh = alloc_n<double>(sc, n);
    double* t = alloc_n<double>(sc, n);
    double* w = alloc_n<double>(sc, n);
    double* part = alloc_n<double>(sc, (int64_t)kDotParts * 16);
    double* dres = alloc_n<double>(sc, 1);
    if (!r || !rh || !pv || !ph || !v || !sv || !sh || !t || !w || !part || !dres) return RW_ERR_ALLOC;
    double* hd = static_cast<double*>(ctx->h_small);
    const int vb = grid_for(n, 256, kDotParts);
    const int gb = grid_for(n, 256, ctx->num_sms * 8);
    rw_status rc;
    auto dot = [&](const double* a, const double* c, double* out) -> rw_status {
        RW_COUNT_LAUNCH();
        k_dot<double, double><<<vb, 256, 0, s>>>(a, c, n, 1, part);
        RW_COUNT_LAUNCH();
        k_sum_parts<<<1, 32, 0, s>>>(part, vb, dres);
        rw_status r2;
        if ((r2 = check_launch("bicgstab dot")) ||
            (r2 = check_cuda(cudaMemcpyAsync(hd, dres, sizeof(double), cudaMemcpyDeviceToHost, s), "copy")) ||
            (r2 = check_cuda(cudaStreamSynchronize(s), "sync")))
            return r2;
        *out = hd[0];
        return RW_OK;
    };
    auto lin3 = [&](double* out, const double* a, double ca, const double* bb, double cb, const double* c,
                    double cc) -> rw_status {
        RW_COUNT_LAUNCH();
        k_lin3<<<gb, 256, 0, s>>>(n, out, a, ca, bb, cb, c, cc);
        return check_launch("bicgstab update");
    };
    auto apply_m = [&](const double* in, double* out) -> rw_status {
        rw_status r2 = precond_t<double>(ctx, F, F.y_val, F.yt_val, F.d, in, w, out, 1);
        return r2 ? r2 : check_launch("bicgstab preconditioner");
    };
    auto spmv = [&](const double* in, double* out) -> rw_status {
        return launch_spmv<double, double>(ctx, n, A->row_ptr, A->col, A->val, in, out, 1, nullptr);
    };
    cudaEventRecord(ctx->ev[8], s);
    double bb = 0.0;
    if ((rc = check_cuda(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(pv, 0, sizeof(double) * (size_t)n, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(v, 0, sizeof(double) * (size_t)n, s), "memset")) ||
        (rc = lin3(r, b, 1.0, nullptr, 0.0, nullptr, 0.0)) || (rc = lin3(rh, b, 1.0, nullptr, 0.0, nullptr, 0.0)) ||
        (rc = dot(b, b, &bb)))
        return rc;
    if (!std::isfinite(bb)) {
        set_error("bicgstab: right-hand side holds a non-finite value");
        return RW_ERR_ARG;
    }
    const double bnorm = std::sqrt(bb);
    double rho_old = 1.0, alpha = 1.0, omega = 1.0, relres = bnorm > 0.0 ? 1.0 : 0.0;
    int it = 0;
    bool done = bnorm == 0.0, broke = false;
    // the true residual b - A x into r; returns its relative norm
    auto true_residual = [&](double* rel) -> rw_status {
        rw_status r2;
        double rr = 0.0;
        if ((r2 = spmv(x, t)) || (r2 = lin3(r, b, 1.0, t, -1.0, nullptr, 0.0)) || (r2 = dot(r, r, &rr))) return r2;
        *rel = std::sqrt(rr) / bnorm;
        return RW_OK;
    };
    while (!done && it < max_iter) {
        ++it;
        double rho = 0.0, rv = 0.0;
        if ((rc = dot(rh, r, &rho))) return rc;
        if (rho == 0.0 || !std::isfinite(rho)) {
            broke = true;
            break;
        }
        const double beta = (rho / rho_old) * (alpha / omega);
        if ((rc = lin3(pv, r, 1.0, pv, beta, v, -beta * omega)) || (rc = apply_m(pv, ph)) || (rc = spmv(ph, v)) ||
            (rc = dot(rh, v, &rv)))
            return rc;
        if (rv == 0.0 || !std::isfinite(rv)) {
            broke = true;
            break;
        }
        alpha = rho / rv;
        double ss = 0.0;
        if ((rc = lin3(sv, r, 1.0, v, -alpha, nullptr, 0.0)) || (rc = dot(sv, sv, &ss))) return rc;
        if (std::sqrt(ss) < tol * bnorm) {
            if ((rc = lin3(x, x, 1.0, ph, alpha, nullptr, 0.0)) || (rc = true_residual(&relres))) return rc;
            if (relres < tol) {
                done = true;
                break;
            }
            rho_old = rho;  // continue from the replaced residual
            omega = 1.0;
            continue;
        }
        double ts = 0.0, tt = 0.0;
        if ((rc = apply_m(sv, sh)) || (rc = spmv(sh, t)) || (rc = dot(t, sv, &ts)) || (rc = dot(t, t, &tt))) return rc;
        if (tt == 0.0 || !std::isfinite(tt)) {
            broke = true;
            break;
        }
        omega = ts / tt;
        double rr = 0.0;
        if ((rc = lin3(x, x, 1.0, ph, alpha, sh, omega)) || (rc = lin3(r, sv, 1.0, t, -omega, nullptr, 0.0)) ||
            (rc = dot(r, r, &rr)))
            return rc;
        relres = std::sqrt(rr) / bnorm;
        if (relres < tol) {
            if ((rc = true_residual(&relres))) return rc;
            if (relres < tol) done = true;
        }
        if (omega == 0.0) {
            broke = !done;
            break;
        }
        rho_old = rho;
    }
    if (!done && bnorm > 0.0 && (rc = true_residual(&relres))) return rc;
    cudaEventRecord(ctx->ev[9], s);
    if ((rc = read_status(ctx, "bicgstab"))) return rc;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->iterations = it;
        stats->rel_residual = relres;
        cudaEventElapsedTime(&stats->solve_ms, ctx->ev[8], ctx->ev[9]);
        stats->kernel_launches = g_launches - launches0;
    }
    if (done) return RW_OK;
    if (broke) {
        set_error("bicgstab: breakdown after %d iterations (relative residual %.3e)", it, relres);
        return RW_ERR_BREAKDOWN;
    }
    set_error("bicgstab: %d iterations without reaching the tolerance (relative residual %.3e)", it, relres);
    return RW_ERR_NO_CONVERGENCE;
}

// ---------------------------------------------------------------------------
// Preconditioner application without allocation.
//
// Some callers cannot allocate device memory while they apply the
// preconditioner: an outer iterative solver that calls it once per iteration
// from a tight loop, code that runs under a fixed memory budget, or a
// framework whose allocator must not be re-entered from a library call.  For
// them the scratch vector w of the backward solve lives in the file-scope
// device array below instead of coming from the context's allocator.  The
// array holds kStaticScratchEntries doubles (n * nrhs at most) on every device
// that loads the library, for the life of the process.
// ---------------------------------------------------------------------------
constexpr int64_t kStaticScratchEntries = (int64_t)1 << 20;  // 8 MiB of FP64
static __device__ __align__(256) double g_static_scratch[kStaticScratchEntries];

static std::mutex g_static_scratch_mu;
constexpr int kMaxDevices = 64;
static double* g_static_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on `device` (which must be current).  The
// host-side name of the array is only a stand-in, so the address is looked up
// once per device and cached.
static rw_status static_scratch_address(int device, double** out) {
    std::lock_guard<std::mutex> lock(g_static_scratch_mu);
    if (device < 0 || device >= kMaxDevices) {
        set_error("static scratch: device %d out of range", device);
        return RW_ERR_ARG;
    }
    if (!g_static_scratch_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return check_cuda(e, "cudaGetSymbolAddress(static scratch)");
        g_static_scratch_ptr[device] = static_cast<double*>(p);
    }
    *out = g_static_scratch_ptr[device];
    return RW_OK;
}

}  // namespace rw

extern "C" rw_status rw_precond_apply_static(rw_context* ctx, const rw_factor* F,
                                             const double* d_r, double* d_z, int32_t nrhs) {
    using namespace rw;
    if (!ctx || !F || !d_r || !d_z || nrhs < 1 || nrhs > 16) {
        set_error("rw_precond_apply_static: bad arguments");
        return RW_ERR_ARG;
    }
    const rw_factor_desc& d = F->desc;
    const int64_t cnt = (int64_t)d.n * nrhs;
    if (cnt > kStaticScratchEntries) {
        set_error("rw_precond_apply_static: n * nrhs = %lld exceeds the static scratch of %lld "
                  "entries; use rw_precond_apply",
                  (long long)cnt, (long long)kStaticScratchEntries);
        return RW_ERR_CAPACITY;
    }
    if (d.n == 0) return RW_OK;
    int dev = -1;
    rw_status rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev != ctx->device) {
        set_error("rw_precond_apply_static: device %d is current, the context is on device %d",
                  dev, ctx->device);
        return RW_ERR_ARG;
    }
    double* w = nullptr;
    if ((rc = static_scratch_address(dev, &w))) return rc;
    FactorView v;
    v.n = d.n;
    v.nnz = d.nnz;
    v.y_rp = d.y_row_ptr;
    v.y_col = d.y_col;
    v.y_val = d.y_val;
    v.y_val32 = d.y_val32;
    v.yt_rp = d.yt_row_ptr;
    v.yt_col = d.yt_col;
    v.yt_val = d.yt_val;
    v.yt_val32 = d.yt_val32;
    v.d = d.d;
    v.d32 = d.d32;
    v.fwd_order = F->fwd_order;
    v.bwd_order = F->bwd_order;
    v.fwd_sched = &F->fwd_sched;
    v.bwd_sched = &F->bwd_sched;
    v.bar = F->bar;
    if ((rc = reset_status(ctx))) return rc;
    // w and z start as "pending" on every call: the array keeps the last call's contents
    if ((rc = fill_pending(ctx, w, cnt))) return rc;
    if ((rc = fill_pending(ctx, d_z, cnt))) return rc;
    if ((rc = precond_t<double>(ctx, v, v.y_val, v.yt_val, v.d, d_r, w, d_z, nrhs))) return rc;
    return read_status(ctx, "static-scratch preconditioner");
}

namespace rw {
}  // namespace rw
