// rw_batch.cu -- PCG (Algorithm 1) over many matrices and right-hand sides at once.
//
// The matrices of a batch form one block-diagonal system: their CSR arrays,
// factors (Y, Y^T, D) and vectors are concatenated, and one level schedule
// covers all factors (level l of the union is the union of the levels l, so
// its depth is the largest single depth).  Every PCG step is then one SpMV,
// one backward and one forward solve and a few vector kernels over all
// matrices, whatever their number.  Scalars (rho, alpha, beta, norms,
// convergence) are per system = (matrix, right-hand side), reduced per matrix
// from fixed row chunks in a fixed order (deterministic).  Every kernel of an
// iteration reads the iteration state from the device, so the iteration is
// captured once in a CUDA graph and replayed; the host reads one flag word
// per iteration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rw_internal.h"

namespace rw {

constexpr int kChunkRows = 2048;  // rows per reduction chunk (never across matrices)
constexpr int kMaxRhs = 16;

// Per-matrix input of the concatenation kernels.
struct CatDesc {
    const void* rp;     // int32 (A) or int64 (factor) row pointers of the matrix
    const int32_t* col;
    const double* val;
    const double* d;    // factor diagonal (factor only)
    int64_t nz0;        // first entry in the combined arrays
    int32_t row0;       // first row in the combined system
    int32_t n;
};

__device__ __forceinline__ int find_seg(const int32_t* __restrict__ row0, int nmat, int32_t row) {
    int lo = 0, hi = nmat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row0[mid] <= row) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One warp per combined row: row pointer, shifted columns, values; the
// segment of every row; with a factor, its diagonal.
template <typename RP_IN, typename RP_OUT>
__global__ void k_cat(int nmat, const CatDesc* __restrict__ md, const int32_t* __restrict__ row0,
                      int32_t N, RP_OUT* rp_out, int32_t* col_out, double* val_out, double* d_out,
                      int32_t* rowseg) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    for (int64_t row = gw; row < N; row += nw) {
        const int m = find_seg(row0, nmat, (int32_t)row);
        const CatDesc D = md[m];
        const int32_t i = (int32_t)row - D.row0;
        const RP_IN* rp = static_cast<const RP_IN*>(D.rp);
        const int64_t s = (int64_t)rp[i], e = (int64_t)rp[i + 1];
        const int64_t o = D.nz0 + s;
        for (int64_t p = s + lane; p < e; p += 32) {
            col_out[o + (p - s)] = D.col[p] + D.row0;
            val_out[o + (p - s)] = D.val[p];
        }
        if (lane == 0) {
            rp_out[row] = (RP_OUT)o;
            if (row == N - 1) rp_out[N] = (RP_OUT)(D.nz0 + (int64_t)rp[D.n]);
            rowseg[row] = m;
            if (d_out) d_out[row] = D.d[i];
        }
    }
}

// ---------------------------------------------------------------------------
// Iteration state on the device.
// ---------------------------------------------------------------------------
struct BatchState {
    double* bnorm2;
    double* rho;
    double* alpha;
    double* beta;
    double* rr;
    double* tt;
    int* active;
    int* check;
    int* iters;
    int* flags;  // [0] any active, [1] any check, [2] breakdown, [3] iteration, [4] max_iter
};
enum { kFlagActive = 0, kFlagCheck, kFlagBroke, kFlagIter, kFlagMaxIter, kFlagWords = 8 };

// Per-chunk partial dot products a.b per right-hand side: part[c * 16 + j].
// One block per chunk; thread t takes rows t, t + 256, ...; fixed-order sums
// (FP64 products and sums).  NR: the right-hand sides rounded up to a power
// of two, so that only those accumulators are reduced.
template <typename TA, typename TB, int NR>
__global__ void __launch_bounds__(256) k_seg_dot(const TA* __restrict__ a, const TB* __restrict__ b,
                                                 int nrhs, const int32_t* __restrict__ chunk_row0,
                                                 double* __restrict__ part) {
    __shared__ double sm[8][NR];
    const int32_t r0 = chunk_row0[blockIdx.x], r1 = chunk_row0[blockIdx.x + 1];
    double acc[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] = 0.0;
    for (int32_t i = r0 + (int32_t)threadIdx.x; i < r1; i += blockDim.x)
#pragma unroll
        for (int j = 0; j < NR; ++j)
            if (j < nrhs) acc[j] += (double)a[(size_t)i * nrhs + j] * (double)b[(size_t)i * nrhs + j];
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] = warp_sum(acc[j]);
    if (lane_id() == 0)
#pragma unroll
        for (int j = 0; j < NR; ++j) sm[threadIdx.x >> 5][j] = acc[j];
    __syncthreads();
    if (threadIdx.x < kMaxRhs) {
        double s = 0.0;
        if ((int)threadIdx.x < NR)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w][threadIdx.x];
        part[(size_t)blockIdx.x * kMaxRhs + threadIdx.x] = s;
    }
}

template <typename TA, typename TB>
static void seg_dot(int nch, cudaStream_t s, const TA* a, const TB* b, int nrhs, const int32_t* chunk_row0,
                    double* part) {
    RW_COUNT_LAUNCH();
    if (nrhs == 1) k_seg_dot<TA, TB, 1><<<nch, 256, 0, s>>>(a, b, nrhs, chunk_row0, part);
    else if (nrhs == 2) k_seg_dot<TA, TB, 2><<<nch, 256, 0, s>>>(a, b, nrhs, chunk_row0, part);
    else if (nrhs <= 4) k_seg_dot<TA, TB, 4><<<nch, 256, 0, s>>>(a, b, nrhs, chunk_row0, part);
    else if (nrhs <= 8) k_seg_dot<TA, TB, 8><<<nch, 256, 0, s>>>(a, b, nrhs, chunk_row0, part);
    else k_seg_dot<TA, TB, 16><<<nch, 256, 0, s>>>(a, b, nrhs, chunk_row0, part);
}

enum BatchOp { kBOpBnorm = 0, kBOpRho0, kBOpAlpha, kBOpResid, kBOpTrue, kBOpBeta, kBOpReport };

// The step of Algorithm 1 for system sys given the sum v of its chunks.
__device__ __forceinline__ void seg_step(const BatchState& S, int sys, double v, int op, int it, double tol,
                                         int& broke) {
    switch (op) {
        case kBOpBnorm:
            S.bnorm2[sys] = v;
            S.active[sys] = v > 0.0;
            S.iters[sys] = 0;
            S.check[sys] = 0;
            break;
        case kBOpRho0:
            S.rho[sys] = v;
            break;
        case kBOpAlpha:
            if (S.active[sys]) {
                if (!(v > 0.0)) {
                    broke = 1;
                    S.active[sys] = 0;
                    S.alpha[sys] = 0.0;
                } else {
                    S.alpha[sys] = S.rho[sys] / v;
                }
            } else {
                S.alpha[sys] = 0.0;
            }
            break;
        case kBOpResid:
            S.rr[sys] = v;
            S.check[sys] = S.active[sys] && (sqrt(v) < tol * sqrt(S.bnorm2[sys]));
            break;
        case kBOpTrue:
            S.tt[sys] = v;
            if (S.check[sys] && sqrt(v) < tol * sqrt(S.bnorm2[sys])) {
                S.active[sys] = 0;
                S.iters[sys] = it;
            }
            S.check[sys] = 0;
            break;
        case kBOpBeta:
            S.beta[sys] = S.active[sys] ? v / S.rho[sys] : 0.0;
            S.rho[sys] = v;
            break;
        case kBOpReport:
            S.tt[sys] = v;
            break;
    }
}

// One block of 1024 threads over all systems s = m * nrhs + j: sums the
// chunks of matrix m in a fixed order and applies the step of Algorithm 1.
// WIDE (matrices of more than 64 chunks): a warp per system, lane l summing
// chunks l, l + 32, ... before a fixed-order warp reduction; otherwise a
// thread per system summing its chunks in order.
template <bool WIDE>
__global__ void __launch_bounds__(1024) k_seg_scalars(BatchState S, const double* __restrict__ part,
                                                      const int32_t* __restrict__ seg_chunk0, int nmat,
                                                      int nrhs, int op, double tol) {
    __shared__ int s_skip, s_it;
    if (threadIdx.x == 0) {
        int it = S.flags[kFlagIter];
        if (op == kBOpAlpha) ++it;
        s_it = it;
        // the true-residual step runs only when some residual passed its test;
        // steps beyond max_iter change nothing
        s_skip = (op == kBOpTrue && !S.flags[kFlagCheck]) ||
                 ((op == kBOpAlpha || op == kBOpResid || op == kBOpTrue || op == kBOpBeta) &&
                  it > S.flags[kFlagMaxIter]);
    }
    __syncthreads();
    const int it = s_it;
    const int nsys = nmat * nrhs;
    int any_act = 0, any_chk = 0, broke = 0;
    if (!s_skip) {
        if (WIDE) {
            const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
            for (int sys = warp; sys < nsys; sys += (int)(blockDim.x >> 5)) {
                const int m = sys / nrhs, j = sys - m * nrhs;
                double v = 0.0;
                for (int32_t c = seg_chunk0[m] + lane; c < seg_chunk0[m + 1]; c += 32)
                    v += part[(size_t)c * kMaxRhs + j];
                v = warp_sum(v);
                if (lane == 0) {
                    seg_step(S, sys, v, op, it, tol, broke);
                    any_act |= S.active[sys];
                    any_chk |= S.check[sys];
                }
            }
        } else {
            for (int sys = threadIdx.x; sys < nsys; sys += blockDim.x) {
                const int m = sys / nrhs, j = sys - m * nrhs;
                double v = 0.0;
                for (int32_t c = seg_chunk0[m]; c < seg_chunk0[m + 1]; ++c) v += part[(size_t)c * kMaxRhs + j];
                seg_step(S, sys, v, op, it, tol, broke);
                any_act |= S.active[sys];
                any_chk |= S.check[sys];
            }
        }
    } else if (op == kBOpAlpha) {
        // past max_iter: every step is a no-op
        for (int sys = threadIdx.x; sys < nsys; sys += blockDim.x) S.alpha[sys] = 0.0;
    }
    any_act = __syncthreads_or(any_act);
    any_chk = __syncthreads_or(any_chk);
    broke = __syncthreads_or(broke);
    if (threadIdx.x == 0) {
        if (op == kBOpAlpha) S.flags[kFlagIter] = it;
        if (broke) S.flags[kFlagBroke] = 1;
        if (!s_skip) {
            S.flags[kFlagActive] = any_act;
            S.flags[kFlagCheck] = any_chk;
        }
    }
}

static void seg_scalars(bool wide, cudaStream_t s, const BatchState& S, const double* part,
                        const int32_t* seg_chunk0, int nmat, int nrhs, int op, double tol) {
    RW_COUNT_LAUNCH();
    if (wide) k_seg_scalars<true><<<1, 1024, 0, s>>>(S, part, seg_chunk0, nmat, nrhs, op, tol);
    else k_seg_scalars<false><<<1, 1024, 0, s>>>(S, part, seg_chunk0, nmat, nrhs, op, tol);
}

// x += alpha p (x FP64), r -= alpha q, per system.
template <typename T>
__global__ void __launch_bounds__(256) k_seg_update_xr(int32_t N, int nrhs, const int32_t* __restrict__ rowseg,
                                                       const double* __restrict__ alpha, double* x, T* r,
                                                       const T* __restrict__ p, const T* __restrict__ q) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double* al = alpha + (rowseg ? (size_t)rowseg[i] * nrhs : 0);
        for (int j = 0; j < nrhs; ++j) {
            const double a = al[j];
            if (a != 0.0) {
                const size_t o = (size_t)i * nrhs + j;
                x[o] += a * (double)p[o];
                r[o] = (T)((double)r[o] - a * (double)q[o]);
            }
        }
    }
}

// p = z + beta p, per system.
template <typename T>
__global__ void __launch_bounds__(256) k_seg_update_p(int32_t N, int nrhs, const int32_t* __restrict__ rowseg,
                                                      const double* __restrict__ beta, const T* __restrict__ z,
                                                      T* p) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double* be = beta + (rowseg ? (size_t)rowseg[i] * nrhs : 0);
        for (int j = 0; j < nrhs; ++j) {
            const size_t o = (size_t)i * nrhs + j;
            p[o] = (T)((double)z[o] + be[j] * (double)p[o]);
        }
    }
}

enum TrueMode { kTrueCheck = 0, kTrueRefine = 1, kTrueAlways = 2 };

// t = b - A x in FP64 per chunk (one block per chunk, thread per row), the
// partials t.t, and in refine mode r = (T) t.  Check mode runs only when a
// residual passed its test; refine mode only on iterations that are a
// multiple of `refine` (and not beyond max_iter).
template <typename T>
__global__ void __launch_bounds__(256) k_seg_true_resid(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                        const double* __restrict__ val, const double* __restrict__ b,
                                                        const double* __restrict__ x, int nrhs,
                                                        const int32_t* __restrict__ chunk_row0, T* r_out,
                                                        double* __restrict__ part, const int* __restrict__ flags,
                                                        int mode, int refine) {
    if (mode == kTrueCheck && !flags[kFlagCheck]) return;
    if (mode == kTrueRefine) {
        const int it = flags[kFlagIter];
        if (it % refine != 0 || it > flags[kFlagMaxIter]) return;
    }
    __shared__ double sm[8][kMaxRhs];
    const int32_t r0 = chunk_row0[blockIdx.x], r1 = chunk_row0[blockIdx.x + 1];
    double acc[kMaxRhs];
#pragma unroll
    for (int j = 0; j < kMaxRhs; ++j) acc[j] = 0.0;
    for (int32_t i = r0 + (int32_t)threadIdx.x; i < r1; i += blockDim.x) {
        const int32_t s = rp[i], e = rp[i + 1];
#pragma unroll
        for (int j = 0; j < kMaxRhs; ++j) {
            if (j >= nrhs) break;
            double ax = 0.0;
            for (int32_t p = s; p < e; ++p) ax += val[p] * x[(size_t)col[p] * nrhs + j];
            const double t = b[(size_t)i * nrhs + j] - ax;
            if (mode == kTrueRefine) r_out[(size_t)i * nrhs + j] = (T)t;
            acc[j] += t * t;
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxRhs; ++j) acc[j] = warp_sum(acc[j]);
    if (lane_id() == 0)
#pragma unroll
        for (int j = 0; j < kMaxRhs; ++j) sm[threadIdx.x >> 5][j] = acc[j];
    __syncthreads();
    if (threadIdx.x < kMaxRhs) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w][threadIdx.x];
        part[(size_t)blockIdx.x * kMaxRhs + threadIdx.x] = s;
    }
}

// Gather the matrices' right-hand sides into the combined FP64 b and r = (T) b;
// zero x.  Counts non-finite values of b.
template <typename T>
__global__ void k_seg_gather_b(int32_t N, int nrhs, const int32_t* __restrict__ rowseg,
                               const int32_t* __restrict__ row0, const double* const* __restrict__ bs,
                               double* b, T* r, double* x, DevStatus* st) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int m = rowseg ? rowseg[i] : 0;
        const double* src = bs[m] + (size_t)(i - row0[m]) * nrhs;
        for (int j = 0; j < nrhs; ++j) {
            const double v = src[j];
            if (!isfinite(v)) atomicAdd(&st->nonfinite, 1u);
            b[(size_t)i * nrhs + j] = v;
            r[(size_t)i * nrhs + j] = (T)v;
            x[(size_t)i * nrhs + j] = 0.0;
        }
    }
}

__global__ void k_seg_scatter_x(int32_t N, int nrhs, const int32_t* __restrict__ rowseg,
                                const int32_t* __restrict__ row0, const double* __restrict__ x,
                                double* const* __restrict__ xs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int m = rowseg ? rowseg[i] : 0;
        double* dst = xs[m] + (size_t)(i - row0[m]) * nrhs;
        for (int j = 0; j < nrhs; ++j) dst[j] = x[(size_t)i * nrhs + j];
    }
}

template <typename T>
__global__ void k_copy_vec(const T* __restrict__ a, T* __restrict__ b, int64_t cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

}  // namespace rw

// ---------------------------------------------------------------------------
// The combined system.
// ---------------------------------------------------------------------------
struct rw_batch {
    rw_context* ctx = nullptr;
    rw::Pool pool;
    int32_t nmat = 0;
    int32_t N = 0;
    int64_t nnzA = 0, nnzY = 0;
    std::vector<int32_t> row0_h;
    int32_t* row0 = nullptr;    // [nmat + 1]
    int32_t* rowseg = nullptr;  // [N] (NULL for a batch of one matrix)
    int32_t nchunks = 0;
    int32_t* chunk_row0 = nullptr;  // [nchunks + 1]
    int32_t* seg_chunk0 = nullptr;  // [nmat + 1]
    int32_t max_seg_chunks = 0;     // chunks of the largest matrix
    // combined A (FP64 and FP32 values)
    int32_t* a_rp = nullptr;
    int32_t* a_col = nullptr;
    double* a_val = nullptr;
    float* a_val32 = nullptr;
    // combined factor
    int64_t* y_rp = nullptr;
    int32_t* y_col = nullptr;
    double* y_val = nullptr;
    float* y_val32 = nullptr;
    int64_t* yt_rp = nullptr;
    int32_t* yt_col = nullptr;
    double* yt_val = nullptr;
    float* yt_val32 = nullptr;
    double* d = nullptr;
    float* d32 = nullptr;
    int32_t* fwd_order = nullptr;
    int32_t* bwd_order = nullptr;
    int32_t fwd_depth = 0, bwd_depth = 0;
    rw::SolveSchedule fwd_sched, bwd_sched;
    unsigned* bar = nullptr;
    bool refs = false;  // one matrix: the arrays and schedules are the caller's matrix and factor
    explicit rw_batch(rw_context* c) : ctx(c), pool(c) {}
};

using namespace rw;

namespace rw {
rw_status batch_tune_target(const rw_batch* B, TuneTarget* X) {
    if (!B) {
        set_error("autotune: NULL batch");
        return RW_ERR_ARG;
    }
    *X = TuneTarget{B->N, B->a_rp, B->a_col, B->a_val, B->a_val32, B->y_rp, B->y_col, B->y_val, B->y_val32,
                    B->yt_rp, B->yt_col, B->yt_val, B->yt_val32, B->d, B->d32, &B->fwd_sched, &B->bwd_sched,
                    B->bar, B->nnzY, std::max(B->fwd_depth, B->bwd_depth)};
    return RW_OK;
}
}  // namespace rw

namespace {

template <typename T>
rw_status pcg_batch_t(rw_context* ctx, rw_batch* B, const double* const* d_b, double* const* d_x,
                      int nrhs, double tol, int max_iter, rw_pcg_stats* stats, int32_t* h_iters,
                      double* h_relres, const T* Aval, const T* yv, const T* ytv, const T* dv,
                      const T* tv_fwd, const T* tv_bwd, bool mixed, Pool& sc) {
    NvtxRange nvtx_range("rw_pcg_batch");
    cudaStream_t s = ctx->stream;
    const int32_t N = B->N;
    const int nmat = B->nmat;
    const int64_t cnt = (int64_t)N * nrhs;
    const int nsys = nmat * nrhs;
    double* b = alloc_n<double>(sc, cnt);
    double* x = alloc_n<double>(sc, cnt);
    T* r = alloc_n<T>(sc, cnt);
    T* z = alloc_n<T>(sc, cnt);
    T* p = alloc_n<T>(sc, cnt);
    T* q = alloc_n<T>(sc, cnt);
    T* w = alloc_n<T>(sc, cnt);
    double* part = alloc_n<double>(sc, (int64_t)B->nchunks * kMaxRhs);
    double* dbl = alloc_n<double>(sc, (int64_t)nsys * 6);
    int* ints = alloc_n<int>(sc, (int64_t)nsys * 3 + kFlagWords);
    const double** bptr = alloc_n<const double*>(sc, nmat);
    double** xptr = alloc_n<double*>(sc, nmat);
    if (!b || !x || !r || !z || !p || !q || !w || !part || !dbl || !ints || !bptr || !xptr)
        return RW_ERR_ALLOC;
    BatchState S{dbl, dbl + nsys, dbl + 2 * nsys, dbl + 3 * nsys, dbl + 4 * nsys, dbl + 5 * nsys,
                 ints, ints + nsys, ints + 2 * nsys, ints + 3 * nsys};
    rw_status rc;
    std::vector<int> hflags_init(kFlagWords, 0);
    hflags_init[kFlagMaxIter] = max_iter;
    if ((rc = check_cuda(cudaMemsetAsync(dbl, 0, sizeof(double) * (size_t)nsys * 6, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(ints, 0, sizeof(int) * (size_t)nsys * 3, s), "memset")) ||
        (rc = check_cuda(cudaMemcpyAsync(S.flags, hflags_init.data(), sizeof(int) * kFlagWords,
                                         cudaMemcpyHostToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(bptr, d_b, sizeof(double*) * nmat, cudaMemcpyHostToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(xptr, d_x, sizeof(double*) * nmat, cudaMemcpyHostToDevice, s),
                         "copy")))
        return rc;
    const int vb = grid_for(N, 256, ctx->num_sms * 8);
    const int nch = B->nchunks;
    const bool wide = B->max_seg_chunks > 64;
    const int refine = ctx->opt.refine_every > 0 ? ctx->opt.refine_every : 50;
    const bool timing = ctx->opt.timing != 0;
    const int64_t l0 = g_launches;

    // start: r = b, x = 0, ||b||, z = M^-1 r, rho = r.z, p = z
    RW_COUNT_LAUNCH();
    k_seg_gather_b<T><<<vb, 256, 0, s>>>(N, nrhs, B->rowseg, B->row0, bptr, b, r, x, ctx->d_status);
    seg_dot<double, double>(nch, s, b, b, nrhs, B->chunk_row0, part);
    seg_scalars(wide, s, S, part, B->seg_chunk0, nmat, nrhs, kBOpBnorm, tol);
    if ((rc = check_launch("batch pcg init"))) return rc;
    auto precond = [&]() -> rw_status {
        rw_status r2 = solve_runs<T>(ctx, B->bwd_sched, B->yt_rp, B->yt_col, ytv, tv_bwd, r, nullptr, w,
                                     nrhs, B->bar, true);
        if (r2) return r2;
        if ((r2 = apply_inverse_diag<T>(ctx, w, dv, B->fwd_sched.n, nrhs))) return r2;
        return solve_runs<T>(ctx, B->fwd_sched, B->y_rp, B->y_col, yv, tv_fwd, w, nullptr, z, nrhs, B->bar);
    };
    if ((rc = precond())) return rc;
    seg_dot<T, T>(nch, s, r, z, nrhs, B->chunk_row0, part);
    seg_scalars(wide, s, S, part, B->seg_chunk0, nmat, nrhs, kBOpRho0, tol);
    RW_COUNT_LAUNCH();
    k_copy_vec<T><<<vb, 256, 0, s>>>(z, p, cnt);
    if ((rc = check_launch("batch pcg start"))) return rc;
    if ((rc = read_status(ctx, "batch pcg start"))) return rc;
    if (ctx->h_status->nonfinite) {
        set_error("pcg: right-hand side holds a non-finite value");
        return RW_ERR_ARG;
    }

    // one iteration of Algorithm 1 for every system; every decision on the device
    auto iteration = [&]() -> rw_status {
        rw_status r2;
        if ((r2 = spmv_launch<T>(ctx, N, B->a_rp, B->a_col, Aval, p, q, nrhs))) return r2;
        seg_dot<T, T>(nch, s, p, q, nrhs, B->chunk_row0, part);
        seg_scalars(wide, s, S, part, B->seg_chunk0, nmat, nrhs, kBOpAlpha, tol);
        RW_COUNT_LAUNCH();
        k_seg_update_xr<T><<<vb, 256, 0, s>>>(N, nrhs, B->rowseg, S.alpha, x, r, p, q);
        seg_dot<T, T>(nch, s, r, r, nrhs, B->chunk_row0, part);
        if (mixed) {
            RW_COUNT_LAUNCH();
            k_seg_true_resid<T><<<nch, 256, 0, s>>>(B->a_rp, B->a_col, B->a_val, b, x, nrhs, B->chunk_row0,
                                                    r, part, S.flags, kTrueRefine, refine);
        }
        seg_scalars(wide, s, S, part, B->seg_chunk0, nmat, nrhs, kBOpResid, tol);
        RW_COUNT_LAUNCH();
        k_seg_true_resid<T><<<nch, 256, 0, s>>>(B->a_rp, B->a_col, B->a_val, b, x, nrhs, B->chunk_row0,
                                                r, part, S.flags, kTrueCheck, refine);
        seg_scalars(wide, s, S, part, B->seg_chunk0, nmat, nrhs, kBOpTrue, tol);
        if ((r2 = precond())) return r2;
        seg_dot<T, T>(nch, s, r, z, nrhs, B->chunk_row0, part);
        seg_scalars(wide, s, S, part, B->seg_chunk0, nmat, nrhs, kBOpBeta, tol);
        RW_COUNT_LAUNCH();
        k_seg_update_p<T><<<vb, 256, 0, s>>>(N, nrhs, B->rowseg, S.beta, z, p);
        return check_launch("batch pcg step");
    };

    // capture one iteration in a graph (fall back to direct launches if the
    // capture is refused)
    cudaGraphExec_t gexec = nullptr;
    int64_t per_iter = 0;
    if (ctx->opt.graphs) {
        cudaGraph_t graph = nullptr;
        const int64_t c0 = g_launches;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            rw_status r2 = iteration();
            const cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (r2 == RW_OK && e == cudaSuccess && graph &&
                cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess) {
                per_iter = g_launches - c0;
            } else {
                gexec = nullptr;
            }
            if (graph) cudaGraphDestroy(graph);
        }
        g_launches = c0;
        cudaGetLastError();  // a refused capture leaves no sticky error
    }
    int* hflags = static_cast<int*>(ctx->h_small);
    int done = 0;
    bool any_active = true;
    float ms_loop = 0.f;
    if (timing) cudaEventRecord(ctx->ev[2], s);
    for (int it = 1; it <= max_iter && any_active; ++it) {
        if (gexec) {
            if ((rc = check_cuda(cudaGraphLaunch(gexec, s), "graph launch"))) break;
            g_launches += per_iter;
        } else if ((rc = iteration())) {
            break;
        }
        done = it;
        if ((rc = check_cuda(cudaMemcpyAsync(hflags, S.flags, sizeof(int) * kFlagWords, cudaMemcpyDeviceToHost, s),
                             "copy")) ||
            (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
            break;
        any_active = hflags[kFlagActive] != 0;
    }
    if (timing) {
        cudaEventRecord(ctx->ev[3], s);
        cudaEventSynchronize(ctx->ev[3]);
        cudaEventElapsedTime(&ms_loop, ctx->ev[2], ctx->ev[3]);
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (rc) return rc;

    // final true residuals, x back to the callers
    RW_COUNT_LAUNCH();
    k_seg_true_resid<T><<<nch, 256, 0, s>>>(B->a_rp, B->a_col, B->a_val, b, x, nrhs, B->chunk_row0, r, part,
                                            S.flags, kTrueAlways, refine);
    seg_scalars(wide, s, S, part, B->seg_chunk0, nmat, nrhs, kBOpReport, tol);
    RW_COUNT_LAUNCH();
    k_seg_scatter_x<<<vb, 256, 0, s>>>(N, nrhs, B->rowseg, B->row0, x, xptr);
    if ((rc = check_launch("batch pcg report"))) return rc;
    std::vector<double> hb2(nsys), htt(nsys);
    std::vector<int> hact(nsys), hit(nsys), hfl(kFlagWords);
    if ((rc = check_cuda(cudaMemcpyAsync(hb2.data(), S.bnorm2, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(htt.data(), S.tt, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(hact.data(), S.active, sizeof(int) * nsys, cudaMemcpyDeviceToHost, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(hit.data(), S.iters, sizeof(int) * nsys, cudaMemcpyDeviceToHost, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(hfl.data(), S.flags, sizeof(int) * kFlagWords, cudaMemcpyDeviceToHost, s),
                         "copy")))
        return rc;
    if ((rc = read_status(ctx, "batch pcg"))) return rc;
    bool conv_all = true;
    for (int m = 0; m < nmat; ++m) {
        int maxit = 0;
        double maxrel = 0.0;
        for (int j = 0; j < nrhs; ++j) {
            const int sys = m * nrhs + j;
            const int itj = hact[sys] ? done : hit[sys];
            if (hact[sys]) conv_all = false;
            const double rel = hb2[sys] > 0.0 ? std::sqrt(htt[sys] / hb2[sys]) : 0.0;
            maxit = std::max(maxit, itj);
            maxrel = std::max(maxrel, rel);
            if (h_iters) h_iters[sys] = itj;
            if (h_relres) h_relres[sys] = rel;
        }
        if (stats) {
            stats[m].iterations = maxit;
            stats[m].rel_residual = maxrel;
            stats[m].solve_ms = ms_loop;
            stats[m].kernel_launches = g_launches - l0;
        }
    }
    if (hfl[kFlagBroke]) {
        set_error("pcg breakdown: p.Ap <= 0");
        return RW_ERR_BREAKDOWN;
    }
    if (tol > 0.0 && !conv_all) {
        set_error("pcg did not reach the tolerance in %d iterations", max_iter);
        return RW_ERR_NO_CONVERGENCE;
    }
    return RW_OK;
}

}  // namespace

extern "C" {

rw_status rw_batch_create(rw_context* ctx, int32_t nmat, const rw_csr* As, const rw_factor* const* Fs,
                          rw_batch** out) {
    NvtxRange nvtx_range("rw_batch_create");
    if (!ctx || nmat < 1 || !As || !Fs || !out) {
        set_error("rw_batch_create: bad arguments");
        return RW_ERR_ARG;
    }
    *out = nullptr;
    int64_t N = 0, nnzA = 0, nnzY = 0;
    bool fp32 = true;
    for (int32_t m = 0; m < nmat; ++m) {
        rw_status rc = check_csr(&As[m]);
        if (rc) return rc;
        if (!Fs[m] || Fs[m]->desc.n != As[m].n) {
            set_error("rw_batch_create: factor %d does not match its matrix", m);
            return RW_ERR_ARG;
        }
        N += As[m].n;
        nnzA += As[m].nnz;
        nnzY += Fs[m]->desc.nnz;
        fp32 = fp32 && Fs[m]->desc.y_val32;
    }
    if (N > 0x7FFFFFFF - 1 || nnzA > 0x7FFFFFFF) {
        set_error("rw_batch_create: combined system too large for 32-bit row pointers");
        return RW_ERR_ARG;
    }
    rw_batch* B = new (std::nothrow) rw_batch(ctx);
    if (!B) return RW_ERR_ALLOC;
    auto fail = [&](rw_status rc) {
        delete B;
        return rc;
    };
    cudaStream_t s = ctx->stream;
    Pool sc(ctx);
    rw_status rc0 = reset_status(ctx);
    if (rc0) return fail(rc0);
    if (nmat == 1) {
        // a batch of one matrix uses the matrix and its factor in place (both
        // must outlive it): no concatenation, the factor's own schedules
        const rw_factor* F = Fs[0];
        const rw_factor_desc& d = F->desc;
        const int32_t n = As[0].n;
        B->refs = true;
        B->nmat = 1;
        B->N = n;
        B->nnzA = As[0].nnz;
        B->nnzY = d.nnz;
        B->row0_h = {0, n};
        std::vector<int32_t> chunk_row0, seg_chunk0 = {0, 0};
        for (int64_t c = 0; c < n; c += kChunkRows) chunk_row0.push_back((int32_t)c);
        seg_chunk0[1] = (int32_t)chunk_row0.size();
        B->nchunks = (int32_t)chunk_row0.size();
        B->max_seg_chunks = B->nchunks;
        chunk_row0.push_back(n);
        Pool& P = B->pool;
        B->row0 = alloc_n<int32_t>(P, 2);
        B->chunk_row0 = alloc_n<int32_t>(P, B->nchunks + 1);
        B->seg_chunk0 = alloc_n<int32_t>(P, 2);
        if (!B->row0 || !B->chunk_row0 || !B->seg_chunk0) return fail(RW_ERR_ALLOC);
        rw_status rc;
        if ((rc = check_cuda(cudaMemcpyAsync(B->row0, B->row0_h.data(), sizeof(int32_t) * 2, cudaMemcpyHostToDevice, s),
                             "copy")) ||
            (rc = check_cuda(cudaMemcpyAsync(B->chunk_row0, chunk_row0.data(), sizeof(int32_t) * chunk_row0.size(),
                                             cudaMemcpyHostToDevice, s),
                             "copy")) ||
            (rc = check_cuda(cudaMemcpyAsync(B->seg_chunk0, seg_chunk0.data(), sizeof(int32_t) * 2,
                                             cudaMemcpyHostToDevice, s),
                             "copy")))
            return fail(rc);
        B->a_rp = const_cast<int32_t*>(As[0].row_ptr);
        B->a_col = const_cast<int32_t*>(As[0].col);
        B->a_val = const_cast<double*>(As[0].val);
        B->y_rp = const_cast<int64_t*>(d.y_row_ptr);
        B->y_col = const_cast<int32_t*>(d.y_col);
        B->y_val = const_cast<double*>(d.y_val);
        B->yt_rp = const_cast<int64_t*>(d.yt_row_ptr);
        B->yt_col = const_cast<int32_t*>(d.yt_col);
        B->yt_val = const_cast<double*>(d.yt_val);
        B->d = const_cast<double*>(d.d);
        B->y_val32 = const_cast<float*>(d.y_val32);
        B->yt_val32 = const_cast<float*>(d.yt_val32);
        B->d32 = const_cast<float*>(d.d32);
        B->fwd_sched = F->fwd_sched;
        B->bwd_sched = F->bwd_sched;
        B->fwd_depth = d.fwd_levels;
        B->bwd_depth = d.bwd_levels;
        B->bar = F->bar;
        if (d.y_val32 && n > 0) {
            B->a_val32 = alloc_n<float>(P, B->nnzA);
            if (!B->a_val32) return fail(RW_ERR_ALLOC);
            launch_to_fp32_diff(n, As[0].row_ptr, As[0].col, As[0].val, B->a_val32, s, ctx->num_sms);
            if ((rc = check_launch("batch fp32 operator"))) return fail(rc);
        }
        if ((rc = read_status(ctx, "batch create"))) return fail(rc);
        *out = B;
        return RW_OK;
    }
    B->nmat = nmat;
    B->N = (int32_t)N;
    B->nnzA = nnzA;
    B->nnzY = nnzY;
    B->row0_h.resize(nmat + 1);
    std::vector<CatDesc> ha(nmat), hy(nmat), hyt(nmat);
    std::vector<int32_t> chunk_row0, seg_chunk0(nmat + 1);
    int64_t r0 = 0, za = 0, zy = 0;
    for (int32_t m = 0; m < nmat; ++m) {
        const rw_factor_desc& d = Fs[m]->desc;
        B->row0_h[m] = (int32_t)r0;
        ha[m] = CatDesc{As[m].row_ptr, As[m].col, As[m].val, nullptr, za, (int32_t)r0, As[m].n};
        hy[m] = CatDesc{d.y_row_ptr, d.y_col, d.y_val, d.d, zy, (int32_t)r0, d.n};
        hyt[m] = CatDesc{d.yt_row_ptr, d.yt_col, d.yt_val, nullptr, zy, (int32_t)r0, d.n};
        seg_chunk0[m] = (int32_t)chunk_row0.size();
        for (int64_t c = 0; c < As[m].n; c += kChunkRows) chunk_row0.push_back((int32_t)(r0 + c));
        r0 += As[m].n;
        za += As[m].nnz;
        zy += d.nnz;
    }
    B->row0_h[nmat] = (int32_t)r0;
    seg_chunk0[nmat] = (int32_t)chunk_row0.size();
    B->nchunks = (int32_t)chunk_row0.size();
    for (int32_t m = 0; m < nmat; ++m)
        B->max_seg_chunks = std::max(B->max_seg_chunks, seg_chunk0[m + 1] - seg_chunk0[m]);
    chunk_row0.push_back((int32_t)r0);
    Pool& P = B->pool;
    B->row0 = alloc_n<int32_t>(P, nmat + 1);
    B->rowseg = alloc_n<int32_t>(P, N);
    B->chunk_row0 = alloc_n<int32_t>(P, B->nchunks + 1);
    B->seg_chunk0 = alloc_n<int32_t>(P, nmat + 1);
    B->a_rp = alloc_n<int32_t>(P, N + 1);
    B->a_col = alloc_n<int32_t>(P, nnzA);
    B->a_val = alloc_n<double>(P, nnzA);
    B->y_rp = alloc_n<int64_t>(P, N + 1);
    B->y_col = alloc_n<int32_t>(P, nnzY);
    B->y_val = alloc_n<double>(P, nnzY);
    B->yt_rp = alloc_n<int64_t>(P, N + 1);
    B->yt_col = alloc_n<int32_t>(P, nnzY);
    B->yt_val = alloc_n<double>(P, nnzY);
    B->d = alloc_n<double>(P, N);
    B->fwd_order = alloc_n<int32_t>(P, N);
    B->bwd_order = alloc_n<int32_t>(P, N);
    B->bar = static_cast<unsigned*>(P.get((size_t)kSolveWorkspaceBytes));
    CatDesc* d_desc = alloc_n<CatDesc>(sc, 3 * (int64_t)nmat);
    int32_t* seg_tmp = alloc_n<int32_t>(sc, N);
    if (!B->row0 || !B->rowseg || !B->chunk_row0 || !B->seg_chunk0 || !B->a_rp || !B->a_col || !B->a_val ||
        !B->y_rp || !B->y_col || !B->y_val || !B->yt_rp || !B->yt_col || !B->yt_val || !B->d ||
        !B->fwd_order || !B->bwd_order || !B->bar || !d_desc || !seg_tmp)
        return fail(RW_ERR_ALLOC);
    rw_status rc;
    if ((rc = check_cuda(cudaMemcpyAsync(B->row0, B->row0_h.data(), sizeof(int32_t) * (nmat + 1),
                                         cudaMemcpyHostToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(B->chunk_row0, chunk_row0.data(), sizeof(int32_t) * chunk_row0.size(),
                                         cudaMemcpyHostToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(B->seg_chunk0, seg_chunk0.data(), sizeof(int32_t) * (nmat + 1),
                                         cudaMemcpyHostToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(d_desc, ha.data(), sizeof(CatDesc) * nmat, cudaMemcpyHostToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(d_desc + nmat, hy.data(), sizeof(CatDesc) * nmat, cudaMemcpyHostToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemcpyAsync(d_desc + 2 * nmat, hyt.data(), sizeof(CatDesc) * nmat,
                                         cudaMemcpyHostToDevice, s),
                         "copy")))
        return fail(rc);
    if (N > 0) {
        const int g = grid_for(N * 32, 256, ctx->num_sms * 16);
        RW_COUNT_LAUNCH();
        k_cat<int32_t, int32_t><<<g, 256, 0, s>>>(nmat, d_desc, B->row0, (int32_t)N, B->a_rp, B->a_col, B->a_val,
                                                  nullptr, B->rowseg);
        RW_COUNT_LAUNCH();
        k_cat<int64_t, int64_t><<<g, 256, 0, s>>>(nmat, d_desc + nmat, B->row0, (int32_t)N, B->y_rp, B->y_col,
                                                  B->y_val, B->d, seg_tmp);
        RW_COUNT_LAUNCH();
        k_cat<int64_t, int64_t><<<g, 256, 0, s>>>(nmat, d_desc + 2 * nmat, B->row0, (int32_t)N, B->yt_rp,
                                                  B->yt_col, B->yt_val, nullptr, seg_tmp);
        if ((rc = check_launch("batch concatenation"))) return fail(rc);
    }
    if (fp32) {
        B->a_val32 = alloc_n<float>(P, nnzA);
        B->y_val32 = alloc_n<float>(P, nnzY);
        B->yt_val32 = alloc_n<float>(P, nnzY);
        B->d32 = alloc_n<float>(P, N);
        if (!B->a_val32 || !B->y_val32 || !B->yt_val32 || !B->d32) return fail(RW_ERR_ALLOC);
        launch_to_fp32_diff((int32_t)N, B->a_rp, B->a_col, B->a_val, B->a_val32, s, ctx->num_sms);
        launch_to_fp32(B->y_val, B->y_val32, nnzY, s, ctx->num_sms);
        launch_to_fp32(B->yt_val, B->yt_val32, nnzY, s, ctx->num_sms);
        launch_to_fp32(B->d, B->d32, N, s, ctx->num_sms);
        if ((rc = check_launch("batch fp32 copies"))) return fail(rc);
    }
    int64_t* fwd_lptr = nullptr;
    int64_t* bwd_lptr = nullptr;
    if ((rc = compute_levels_pair(ctx, (int32_t)N,
                                  LevelDag{B->y_rp, B->y_col, false, B->fwd_order, &B->fwd_depth, &fwd_lptr},
                                  LevelDag{B->yt_rp, B->yt_col, true, B->bwd_order, &B->bwd_depth, &bwd_lptr}, P,
                                  sc)) ||
        (rc = build_schedule(ctx, (int32_t)N, B->y_rp, B->y_col, B->y_val, B->y_val32, B->fwd_order, fwd_lptr,
                             B->fwd_depth, B->fwd_sched, P, sc)) ||
        (rc = build_schedule(ctx, (int32_t)N, B->yt_rp, B->yt_col, B->yt_val, B->yt_val32, B->bwd_order, bwd_lptr,
                             B->bwd_depth, B->bwd_sched, P, sc)))
        return fail(rc);
    if ((rc = read_status(ctx, "batch create"))) return fail(rc);
    *out = B;
    return RW_OK;
}

void rw_batch_destroy(rw_batch* B) {
    if (!B) return;
    cudaStreamSynchronize(B->ctx->stream);
    delete B;
}

rw_status rw_batch_info(const rw_batch* B, int32_t* n_total, int64_t* nnz_y, int32_t* fwd_levels,
                        int32_t* bwd_levels) {
    if (!B) {
        set_error("rw_batch_info: NULL batch");
        return RW_ERR_ARG;
    }
    if (n_total) *n_total = B->N;
    if (nnz_y) *nnz_y = B->nnzY;
    if (fwd_levels) *fwd_levels = B->fwd_depth;
    if (bwd_levels) *bwd_levels = B->bwd_depth;
    return RW_OK;
}

rw_status pcg_solve_batch(rw_context* ctx, rw_batch* B, const double* const* d_b, double* const* d_x,
                          int32_t nrhs, double tol, int32_t max_iter, rw_precision prec, rw_pcg_stats* stats,
                          int32_t* h_iters, double* h_relres) {
    if (!ctx || !B || B->ctx != ctx || !d_b || !d_x || nrhs < 1 || nrhs > kMaxRhs || max_iter < 0 ||
        !(tol >= 0.0) || (prec != RW_FP64 && prec != RW_FP32_MIXED)) {
        set_error("pcg_solve_batch: bad arguments");
        return RW_ERR_ARG;
    }
    for (int32_t m = 0; m < B->nmat; ++m)
        if (!d_b[m] || !d_x[m]) {
            set_error("pcg_solve_batch: NULL vector of matrix %d", m);
            return RW_ERR_ARG;
        }
    if (stats) memset(stats, 0, sizeof(rw_pcg_stats) * (size_t)B->nmat);
    if (B->N == 0) return RW_OK;
    rw_status rc = reset_status(ctx);
    if (rc) return rc;
    Pool sc(ctx);
    if (prec == RW_FP32_MIXED) {
        if (!B->y_val32) {
            set_error("pcg_solve_batch: FP32 mode needs factors built with store_fp32 = 1");
            return RW_ERR_ARG;
        }
        return pcg_batch_t<float>(ctx, B, d_b, d_x, nrhs, tol, max_iter, stats, h_iters, h_relres, B->a_val32,
                                  B->y_val32, B->yt_val32, B->d32, B->fwd_sched.tval32, B->bwd_sched.tval32,
                                  true, sc);
    }
    return pcg_batch_t<double>(ctx, B, d_b, d_x, nrhs, tol, max_iter, stats, h_iters, h_relres, B->a_val,
                               B->y_val, B->yt_val, B->d, B->fwd_sched.tval, B->bwd_sched.tval, false, sc);
}

}  // extern "C"
