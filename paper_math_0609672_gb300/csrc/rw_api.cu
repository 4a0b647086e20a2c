// rw_api.cu -- C ABI of librwpc: contexts, factor construction (Algorithm 1,
// "Precondition") and the PCG solve (Algorithm 1, "solve").
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <mutex>
#include <set>
#include <tuple>
#include <vector>

#include "rw_internal.h"

namespace rw {

static thread_local char g_err[512] = "";
thread_local int64_t g_launches = 0;

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

rw_status check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return RW_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return RW_ERR_ALLOC;
    return RW_ERR_CUDA;
}

rw_status check_launch(const char* what) { return check_cuda(cudaGetLastError(), what); }

rw_status set_kernel_attr_once(int device, const void* func, cudaFuncAttribute attr, int value) {
    static std::mutex mu;
    static std::set<std::tuple<int, const void*, int, int>> done;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(device, func, (int)attr, value);
    if (done.count(key)) return RW_OK;
    rw_status rc = check_cuda(cudaFuncSetAttribute(func, attr, value), "kernel attribute");
    if (rc == RW_OK) done.insert(key);
    return rc;
}

rw_status reset_status(rw_context* ctx) {
    DevStatus init{};
    init.bad_row = UINT_MAX;
    init.spin_limit = ctx->opt.spin_limit > 0 ? (unsigned)ctx->opt.spin_limit : kSpinLimit;
    *ctx->h_status = init;
    return check_cuda(cudaMemcpyAsync(ctx->d_status, ctx->h_status, sizeof(DevStatus),
                                      cudaMemcpyHostToDevice, ctx->stream),
                      "status reset");
}

rw_status read_status(rw_context* ctx, const char* what) {
    rw_status rc = check_cuda(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(DevStatus),
                                              cudaMemcpyDeviceToHost, ctx->stream),
                              what);
    if (rc) return rc;
    if ((rc = check_cuda(cudaStreamSynchronize(ctx->stream), what))) return rc;
    const DevStatus& st = *ctx->h_status;
    if (st.bad_row != UINT_MAX) {
        set_error("%s: row %u is not in R-matrix form (sorted columns, positive diagonal, "
                  "negative off-diagonals, diagonal dominance)",
                  what, st.bad_row - 1u);
        return RW_ERR_NOT_RMATRIX;
    }
    if (st.bad_budget) {
        set_error("%s: %u rows with an upper neighbour have a zero walk budget", what,
                  st.bad_budget);
        return RW_ERR_ARG;
    }
    if (st.walk_cap) {
        set_error("%s: %u walks reached the step cap (is every component grounded?)", what,
                  st.walk_cap);
        return RW_ERR_WALK_CAP;
    }
    if (st.capacity) {
        set_error("%s: %u rows exceed the merge capacity",
                  what, st.capacity);
        return RW_ERR_CAPACITY;
    }
    if (st.timeout) {
        set_error("%s: %u device-side waits gave up", what, st.timeout);
        return RW_ERR_TIMEOUT;
    }
    return RW_OK;
}

void* Pool::get(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (ctx->alloc) {
        p = ctx->alloc(ctx->user, bytes, (void*)ctx->stream);
        if (!p) set_error("allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
        if (e != cudaSuccess) {
            set_error("cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
            p = nullptr;
        }
    }
    if (p) bufs.push_back({p, bytes});
    return p;
}

void Pool::release(void* p) {
    for (size_t i = 0; i < bufs.size(); ++i)
        if (bufs[i].p == p) {
            if (ctx->free_fn) ctx->free_fn(ctx->user, p, bufs[i].bytes, (void*)ctx->stream);
            else cudaFreeAsync(p, ctx->stream);
            bufs.erase(bufs.begin() + (long)i);
            return;
        }
}

void Pool::release_all() {
    if (!ctx) return;
    for (size_t i = bufs.size(); i-- > 0;) {
        if (ctx->free_fn) ctx->free_fn(ctx->user, bufs[i].p, bufs[i].bytes, (void*)ctx->stream);
        else cudaFreeAsync(bufs[i].p, ctx->stream);
    }
    bufs.clear();
}

rw_status check_csr(const rw_csr* A) {
    if (!A) {
        set_error("matrix is NULL");
        return RW_ERR_ARG;
    }
    if (A->n < 0 || A->nnz < A->n || A->nnz >= ((int64_t)1 << 31)) {
        set_error("matrix sizes out of range (n=%d, nnz=%lld)", A->n, (long long)A->nnz);
        return A->nnz < A->n ? RW_ERR_NOT_RMATRIX : RW_ERR_ARG;
    }
    if (A->n > 0 && (!A->row_ptr || !A->col || !A->val)) {
        set_error("matrix arrays are NULL");
        return RW_ERR_ARG;
    }
    return RW_OK;
}

}  // namespace rw

using namespace rw;

extern "C" {

void rw_options_default(rw_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->max_steps = 1ull << 24;
    opt->keep_records = 0;
    opt->record_lengths = 0;
    opt->store_fp32 = 1;
    opt->refine_every = 50;
    opt->walk_blocks_per_sm = 0;
    opt->timing = 1;
    opt->graphs = 1;
    opt->solve_mode = 2;
    opt->wide_slices = -1;
    opt->solve_mode_bwd = -1;
    opt->thin_levels = 128;
    opt->adapt_ahead = 100;
}

const char* rw_status_string(rw_status s) {
    switch (s) {
        case RW_OK: return "ok";
        case RW_ERR_ARG: return "invalid argument";
        case RW_ERR_NOT_RMATRIX: return "matrix is not an R-matrix in the required form";
        case RW_ERR_WALK_CAP: return "a walk reached the step cap";
        case RW_ERR_ALLOC: return "allocation failed";
        case RW_ERR_NO_CONVERGENCE: return "PCG did not converge";
        case RW_ERR_BREAKDOWN: return "PCG breakdown";
        case RW_ERR_CUDA: return "CUDA error";
        case RW_ERR_TIMEOUT: return "device-side wait timed out";
        case RW_ERR_CAPACITY: return "a row exceeds the merge capacity";
    }
    return "unknown status";
}

const char* rw_last_error(void) { return g_err; }

rw_status rw_context_create(rw_context** out, void* stream, rw_alloc_fn alloc, rw_free_fn free_fn,
                            void* user, const rw_options* opt) {
    if (!out || ((alloc == nullptr) != (free_fn == nullptr))) {
        set_error("rw_context_create: bad arguments");
        return RW_ERR_ARG;
    }
    *out = nullptr;
    rw_context* c = new (std::nothrow) rw_context();
    if (!c) return RW_ERR_ALLOC;
    c->stream = static_cast<cudaStream_t>(stream);
    c->alloc = alloc;
    c->free_fn = free_fn;
    c->user = user;
    if (opt) c->opt = *opt;
    else rw_options_default(&c->opt);
    if (c->opt.max_steps < 1) c->opt.max_steps = 1ull << 24;
    rw_status rc;
    int l2 = 0;
    if ((rc = check_cuda(cudaGetDevice(&c->device), "cudaGetDevice")) ||
        (rc = check_cuda(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount,
                                                c->device),
                         "device attribute")) ||
        (rc = check_cuda(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device), "device attribute")) ||
        (rc = check_cuda(cudaMalloc(&c->d_status, sizeof(DevStatus)), "cudaMalloc status")) ||
        (rc = check_cuda(cudaMallocHost(&c->h_status, sizeof(DevStatus)), "cudaMallocHost")) ||
        (rc = check_cuda(cudaMallocHost(&c->h_small, 4096), "cudaMallocHost"))) {
        rw_context_destroy(c);
        return rc;
    }
    for (auto& e : c->ev) {
        if ((rc = check_cuda(cudaEventCreate(&e), "cudaEventCreate"))) {
            rw_context_destroy(c);
            return rc;
        }
    }
    c->l2_bytes = (size_t)(l2 > 0 ? l2 : 0);
    // a fresh context reports no error until a call sets one
    if ((rc = reset_status(c)) || (rc = check_cuda(cudaStreamSynchronize(c->stream), "sync"))) {
        rw_context_destroy(c);
        return rc;
    }
    if (!alloc) {
        // keep freed stream-ordered allocations cached in the device pool
        cudaMemPool_t mp;
        if (cudaDeviceGetDefaultMemPool(&mp, c->device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    *out = c;
    return RW_OK;
}

void rw_context_destroy(rw_context* ctx) {
    if (!ctx) return;
    if (ctx->stream || true) cudaStreamSynchronize(ctx->stream);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_small) cudaFreeHost(ctx->h_small);
    delete ctx;
}

// One matrix of a (possibly batched) factor build.
struct MatBuild {
    const rw_csr* A = nullptr;
    const uint32_t* budget = nullptr;  // device [n] or NULL (uniform)
    uint64_t seed = 0;
    uint32_t matrix_index = 0;
    rw_factor* F = nullptr;
    Tables T;
    WalkSpace ws;
    int64_t rec_base = 0;   // first record of this matrix in the batch
    int64_t row_base = 0;   // first walk row of this matrix in the batch
    int64_t launches = 0;
};

}  // extern "C"

// Transpose, levels, FP32 copies and solve schedules of a factor whose rows
// (Y, D and the counters in fo) are in place; fills the description's arrays.
// Events 12-14 mark the transpose, levels and FP32/schedule phases when
// timing is on.
rw_status rw::complete_factor(rw_context* ctx, rw_factor* F, const FactorOut& fo, Pool& scratch) {
    cudaStream_t s = ctx->stream;
    const bool timing = ctx->opt.timing != 0;
    rw_factor_desc& d = F->desc;
    const int32_t n = d.n;
    int64_t* fwd_lptr = nullptr;
    int64_t* bwd_lptr = nullptr;
    float* y32 = nullptr;
    float* yt32 = nullptr;
    rw_status rc;
    int64_t* yt_rp = alloc_n<int64_t>(F->pool, n + 1);
    int32_t* yt_col = alloc_n<int32_t>(F->pool, fo.nnz);
    double* yt_val = alloc_n<double>(F->pool, fo.nnz);
    if (!yt_rp || !yt_col || !yt_val) return RW_ERR_ALLOC;
    if ((rc = transpose_factor(ctx, n, fo, yt_rp, yt_col, yt_val, scratch))) return rc;
    if (timing) cudaEventRecord(ctx->ev[12], s);
    F->fwd_order = alloc_n<int32_t>(F->pool, n);
    F->bwd_order = alloc_n<int32_t>(F->pool, n);
    if (!F->fwd_order || !F->bwd_order) return RW_ERR_ALLOC;
    if ((rc = compute_levels_pair(ctx, n, LevelDag{fo.y_rp, fo.y_col, false, F->fwd_order, &d.fwd_levels, &fwd_lptr},
                                  LevelDag{yt_rp, yt_col, true, F->bwd_order, &d.bwd_levels, &bwd_lptr}, F->pool,
                                  scratch)))
        return rc;
    if (timing) cudaEventRecord(ctx->ev[13], s);
    d.fwd_order = F->fwd_order;
    d.fwd_level_ptr = fwd_lptr;
    d.bwd_order = F->bwd_order;
    d.bwd_level_ptr = bwd_lptr;
    if (ctx->opt.store_fp32) {
        y32 = alloc_n<float>(F->pool, fo.nnz);
        yt32 = alloc_n<float>(F->pool, fo.nnz);
        float* d32 = alloc_n<float>(F->pool, n);
        if (!y32 || !yt32 || !d32) return RW_ERR_ALLOC;
        launch_to_fp32(fo.y_val, y32, fo.nnz, s, ctx->num_sms);
        launch_to_fp32(yt_val, yt32, fo.nnz, s, ctx->num_sms);
        launch_to_fp32(fo.d, d32, n, s, ctx->num_sms);
        if ((rc = check_launch("fp32 copies"))) return rc;
        d.y_val32 = y32;
        d.yt_val32 = yt32;
        d.d32 = d32;
    }
    F->bar = static_cast<unsigned*>(F->pool.get((size_t)kSolveWorkspaceBytes));
    if (!F->bar) return RW_ERR_ALLOC;
    if ((rc = build_schedule(ctx, n, fo.y_rp, fo.y_col, fo.y_val, y32, F->fwd_order, fwd_lptr,
                             d.fwd_levels, F->fwd_sched, F->pool, scratch)))
        return rc;
    if ((rc = build_schedule(ctx, n, yt_rp, yt_col, yt_val, yt32, F->bwd_order, bwd_lptr,
                             d.bwd_levels, F->bwd_sched, F->pool, scratch)))
        return rc;
    if (timing) cudaEventRecord(ctx->ev[14], s);
    d.nnz = fo.nnz;
    d.y_row_ptr = fo.y_rp;
    d.y_col = fo.y_col;
    d.y_val = fo.y_val;
    d.d = fo.d;
    d.yt_row_ptr = yt_rp;
    d.yt_col = yt_col;
    d.yt_val = yt_val;
    d.walks = fo.M;
    d.visits = fo.J;
    d.ground = fo.G;
    return RW_OK;
}

extern "C" {

// The rest of the build of one matrix after the walks: merge and emission,
// then complete_factor, and the description.
static rw_status finish_factor(rw_context* ctx, MatBuild& mb, const int2* rec, const Extras* X, bool rec_owned,
                               double drop_tol, uint64_t hops, float ms_walk, Pool& scratch) {
    cudaStream_t s = ctx->stream;
    const bool timing = ctx->opt.timing != 0;
    rw_factor* F = mb.F;
    rw_factor_desc& d = F->desc;
    const rw_csr* A = mb.A;
    FactorOut fo;
    float ms_merge = 0.f, ms_emit = 0.f;
    rw_status rc;
    const int64_t launches0 = g_launches;
    if (timing) cudaEventRecord(ctx->ev[11], s);
    if ((rc = emit_factor(ctx, A, mb.T, mb.ws, rec, X, drop_tol, fo, F->pool, scratch,
                          timing ? &ms_merge : nullptr, timing ? &ms_emit : nullptr)))
        return rc;
    if ((rc = complete_factor(ctx, F, fo, scratch))) return rc;
    if ((rc = read_status(ctx, "factor build"))) return rc;
    d.total_hops = hops;
    d.n_walk_rows = mb.T.n_walk_rows;
    d.total_walks = mb.ws.total;
    d.extra_walks = X ? X->count : 0;
    if (ctx->opt.keep_records && rec_owned) {
        d.records = reinterpret_cast<const int32_t*>(rec);
        d.walk_base = mb.ws.wbase;
        int32_t* wr = alloc_n<int32_t>(F->pool, mb.T.n_walk_rows);
        if (!wr) return RW_ERR_ALLOC;
        if (mb.T.n_walk_rows > 0 &&
            (rc = check_cuda(cudaMemcpyAsync(wr, mb.T.walk_rows,
                                             sizeof(int32_t) * (size_t)mb.T.n_walk_rows,
                                             cudaMemcpyDeviceToDevice, s),
                             "copy")))
            return rc;
        d.walk_rows = wr;
    }
    if (timing) {
        float t_tr = 0.f, t_lev = 0.f, t_fp = 0.f, t_fin = 0.f;
        cudaEventSynchronize(ctx->ev[14]);
        cudaEventElapsedTime(&t_tr, ctx->ev[11], ctx->ev[12]);
        cudaEventElapsedTime(&t_lev, ctx->ev[12], ctx->ev[13]);
        cudaEventElapsedTime(&t_fp, ctx->ev[13], ctx->ev[14]);
        cudaEventElapsedTime(&t_fin, ctx->ev[11], ctx->ev[14]);
        d.phase_ms[1] = ms_walk;
        d.phase_ms[2] = ms_merge;
        d.phase_ms[3] = ms_emit;
        d.phase_ms[4] = t_tr - ms_merge - ms_emit;
        d.phase_ms[5] = t_lev;
        d.phase_ms[6] = t_fp;
        d.phase_ms[7] = d.phase_ms[0] + ms_walk + t_fin;
    }
    mb.launches += g_launches - launches0;
    return RW_OK;
}

__global__ void k_concat_walk_rows(int32_t nw, const int4* __restrict__ wrow,
                                   const int64_t* __restrict__ wbase, int64_t rec_base, int32_t m,
                                   int4* wrow_all, int64_t* wbase_all, int32_t* wmat_all) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x) {
        wrow_all[r] = wrow[r];
        wbase_all[r] = wbase[r] + rec_base;
        wmat_all[r] = m;
    }
}

__global__ void k_set_i64(int64_t* p, int64_t v) { *p = v; }

// Build factors of one or more matrices; the walks of all of them run in one
// persistent launch (work stealing across matrices).
static rw_status build_factors(rw_context* ctx, std::vector<MatBuild>& mbs, uint32_t uniform,
                               double drop_tol) {
    cudaStream_t s = ctx->stream;
    const bool timing = ctx->opt.timing != 0;
    const int nmat = (int)mbs.size();
    rw_status rc = RW_OK;
    Pool scratch(ctx);
    Pool xpool(ctx);  // walk reuse: extra records (until the merge is done)
    Extras X;
    const bool reuse = ctx->opt.reuse != 0;
    int2* rec = nullptr;
    unsigned long long* d_hops = nullptr;
    float ms_walk = 0.f;
    WalkBatch wb;
    if (reuse && nmat != 1) {
        set_error("walk reuse applies to single-matrix builds");
        return RW_ERR_ARG;
    }
    std::vector<MatWalk> hmats(nmat);
    if ((rc = reset_status(ctx))) return rc;
    for (auto& mb : mbs) {
        mb.F = new (std::nothrow) rw_factor(ctx);
        if (!mb.F) {
            rc = RW_ERR_ALLOC;
            goto fail;
        }
        memset(&mb.F->desc, 0, sizeof(mb.F->desc));
        mb.F->desc.n = mb.A->n;
    }
    // tables and walk spaces
    {
        int64_t total = 0, rows = 0;
        for (int m = 0; m < nmat; ++m) {
            MatBuild& mb = mbs[m];
            const int64_t launches0 = g_launches;
            if (timing) cudaEventRecord(ctx->ev[10], s);
            Pool& keep = ctx->opt.keep_records ? mb.F->pool : scratch;
            if ((rc = build_tables(ctx, mb.A, mb.T, scratch))) goto fail;
            if ((rc = build_walk_space(ctx, mb.T, uniform, mb.budget, mb.ws, keep))) goto fail;
            if (timing) {
                cudaEventRecord(ctx->ev[11], s);
                cudaEventSynchronize(ctx->ev[11]);
                cudaEventElapsedTime(&mb.F->desc.phase_ms[0], ctx->ev[10], ctx->ev[11]);
            }
            mb.rec_base = total;
            mb.row_base = rows;
            total += mb.ws.total;
            rows += mb.T.n_walk_rows;
            hmats[m] = mat_walk(mb.T, mb.seed, mb.matrix_index, 0);
            mb.launches += g_launches - launches0;
        }
        wb.nmat = nmat;
        wb.total = total;
        for (const auto& mb : mbs) wb.table_bytes += table_bytes(mb.T);
        wb.nrows = (int32_t)rows;
        if (nmat == 1) {
            wb.m0 = hmats[0];
            wb.wrow = mbs[0].T.wrow;
            wb.wbase = mbs[0].ws.wbase;
            wb.chunk_row = mbs[0].ws.chunk_row;
        } else {
            int4* wrow_all = alloc_n<int4>(scratch, rows);
            int64_t* wbase_all = alloc_n<int64_t>(scratch, rows + 1);
            int32_t* wmat_all = alloc_n<int32_t>(scratch, rows);
            MatWalk* dmats = alloc_n<MatWalk>(scratch, nmat);
            const int64_t nchunks = (total + kWalkChunk - 1) / kWalkChunk;
            int32_t* chunk_row = alloc_n<int32_t>(scratch, nchunks);
            if (!wrow_all || !wbase_all || !wmat_all || !dmats || !chunk_row) {
                rc = RW_ERR_ALLOC;
                goto fail;
            }
            for (int m = 0; m < nmat; ++m) {
                const MatBuild& mb = mbs[m];
                if (mb.T.n_walk_rows == 0) continue;
                RW_COUNT_LAUNCH();
                k_concat_walk_rows<<<grid_for(mb.T.n_walk_rows, 256, ctx->num_sms * 4), 256, 0, s>>>(
                    mb.T.n_walk_rows, mb.T.wrow, mb.ws.wbase, mb.rec_base, m,
                    wrow_all + mb.row_base, wbase_all + mb.row_base, wmat_all + mb.row_base);
            }
            RW_COUNT_LAUNCH();
            k_set_i64<<<1, 1, 0, s>>>(wbase_all + rows, total);
            if ((rc = check_launch("batch walk rows"))) goto fail;
            if ((rc = check_cuda(cudaMemcpyAsync(dmats, hmats.data(), sizeof(MatWalk) * nmat,
                                                 cudaMemcpyHostToDevice, s),
                                 "copy")))
                goto fail;
            if ((rc = build_chunk_rows(ctx, (int32_t)rows, wbase_all, chunk_row))) goto fail;
            wb.mats = dmats;
            wb.wmat = wmat_all;
            wb.wrow = wrow_all;
            wb.wbase = wbase_all;
            wb.chunk_row = chunk_row;
        }
    }
    // walks of all matrices
    {
        const bool keep_rec = ctx->opt.keep_records && nmat == 1;
        rec = alloc_n<int2>(keep_rec ? mbs[0].F->pool : scratch, wb.total);
        d_hops = alloc_n<unsigned long long>(scratch, nmat);
        if (!rec || !d_hops) {
            rc = RW_ERR_ALLOC;
            goto fail;
        }
        WalkLaunch wl;
        wl.max_steps = ctx->opt.max_steps;
        wl.record_lengths = ctx->opt.record_lengths;
        const int64_t launches0 = g_launches;
        if (reuse) {
            wl.record_lengths = 0;
            if ((rc = run_walks_reuse(ctx, wb, wl, mbs[0].T, rec, d_hops, scratch, xpool,
                                      timing ? &ms_walk : nullptr, X)))
                goto fail;
        } else if ((rc = run_walks(ctx, wb, wl, rec, d_hops, scratch, timing ? &ms_walk : nullptr))) {
            goto fail;
        }
        if ((rc = read_status(ctx, "walks"))) goto fail;  // no merge of stopped walks
        mbs[0].launches += g_launches - launches0;
    }
    {
        std::vector<unsigned long long> hops(nmat);
        if ((rc = check_cuda(cudaMemcpy(hops.data(), d_hops, sizeof(unsigned long long) * nmat,
                                        cudaMemcpyDeviceToHost),
                             "copy")))
            goto fail;
        for (int m = 0; m < nmat; ++m) {
            MatBuild& mb = mbs[m];
            if ((rc = finish_factor(ctx, mb, rec + mb.rec_base, reuse ? &X : nullptr, nmat == 1, drop_tol, hops[m],
                                    ms_walk, scratch)))
                goto fail;
            mb.F->desc.kernel_launches = mb.launches;
        }
    }
    scratch.release_all();
    if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) goto fail;
    return RW_OK;
fail:
    scratch.release_all();
    cudaStreamSynchronize(s);
    for (auto& mb : mbs) {
        delete mb.F;
        mb.F = nullptr;
    }
    return rc;
}

static rw_status check_build_args(rw_context* ctx, const rw_csr* A, double drop_tol) {
    if (!ctx) {
        set_error("factor build: NULL context");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr(A);
    if (rc) return rc;
    if (!(drop_tol >= 0.0) || !(drop_tol < 1e300)) {
        set_error("drop_tol must be finite and >= 0");
        return RW_ERR_ARG;
    }
    return RW_OK;
}

static rw_status build_factor_impl(rw_context* ctx, const rw_csr* A, uint32_t uniform,
                                   const uint32_t* d_budget, uint64_t seed, double drop_tol,
                                   rw_factor** out) {
    if (!out) {
        set_error("rw_build_factor: NULL output");
        return RW_ERR_ARG;
    }
    *out = nullptr;
    rw_status rc = check_build_args(ctx, A, drop_tol);
    if (rc) return rc;
    if (!d_budget && uniform < 1) {
        set_error("walks_per_row must be >= 1");
        return RW_ERR_ARG;
    }
    std::vector<MatBuild> mbs(1);
    mbs[0].A = A;
    mbs[0].budget = d_budget;
    mbs[0].seed = seed;
    mbs[0].matrix_index = 0;
    if ((rc = build_factors(ctx, mbs, uniform, drop_tol))) return rc;
    *out = mbs[0].F;
    return RW_OK;
}

rw_status rw_build_factor(rw_context* ctx, const rw_csr* A, uint32_t walks_per_row, uint64_t seed,
                          double drop_tol, rw_factor** out) {
    return build_factor_impl(ctx, A, walks_per_row, nullptr, seed, drop_tol, out);
}

rw_status rw_build_factor_budget(rw_context* ctx, const rw_csr* A, const uint32_t* d_budget,
                                 uint64_t seed, double drop_tol, rw_factor** out) {
    if (!d_budget && A && A->n > 0) {
        set_error("rw_build_factor_budget: budget is NULL");
        return RW_ERR_ARG;
    }
    return build_factor_impl(ctx, A, 0u, d_budget, seed, drop_tol, out);
}

rw_status rw_build_factor_batched(rw_context* ctx, int32_t nmat, const rw_csr* As,
                                  const uint32_t* const* d_budgets, uint32_t walks_per_row,
                                  const uint64_t* seeds, double drop_tol, rw_factor** outs) {
    if (!ctx || nmat < 1 || !As || !seeds || !outs) {
        set_error("rw_build_factor_batched: bad arguments");
        return RW_ERR_ARG;
    }
    for (int32_t m = 0; m < nmat; ++m) outs[m] = nullptr;
    std::vector<MatBuild> mbs(nmat);
    for (int32_t m = 0; m < nmat; ++m) {
        rw_status rc = check_build_args(ctx, &As[m], drop_tol);
        if (rc) return rc;
        const uint32_t* bud = d_budgets ? d_budgets[m] : nullptr;
        if (!bud && walks_per_row < 1) {
            set_error("walks_per_row must be >= 1 for matrices without a budget");
            return RW_ERR_ARG;
        }
        mbs[m].A = &As[m];
        mbs[m].budget = bud;
        mbs[m].seed = seeds[m];
        mbs[m].matrix_index = (uint32_t)m;
    }
    rw_status rc = build_factors(ctx, mbs, walks_per_row, drop_tol);
    if (rc) return rc;
    for (int32_t m = 0; m < nmat; ++m) outs[m] = mbs[m].F;
    return RW_OK;
}

rw_status rw_factor_view(const rw_factor* F, rw_factor_desc* desc) {
    if (!F || !desc) {
        set_error("rw_factor_view: NULL argument");
        return RW_ERR_ARG;
    }
    *desc = F->desc;
    return RW_OK;
}

void rw_factor_destroy(rw_factor* F) {
    if (!F) return;
    cudaStreamSynchronize(F->ctx->stream);
    delete F;
}

static FactorView view_of(const rw_factor* F) {
    const rw_factor_desc& d = F->desc;
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
    return v;
}

// The two-game factor of Sec. 7.1: forward data (Y, its schedule, D) from the
// game on A, backward data (Y^T and its schedule) from the game on A^T.
static rw_status ldu_view(const rw_factor* FA, const rw_factor* FAT, FactorView* v) {
    if (!FA || !FAT || FA->desc.n != FAT->desc.n) {
        set_error("two-game factor: factors missing or of different sizes");
        return RW_ERR_ARG;
    }
    *v = view_of(FA);
    const FactorView t = view_of(FAT);
    v->yt_rp = t.yt_rp;
    v->yt_col = t.yt_col;
    v->yt_val = t.yt_val;
    v->yt_val32 = t.yt_val32;
    v->bwd_order = t.bwd_order;
    v->bwd_sched = t.bwd_sched;
    return RW_OK;
}

rw_status rw_csr_transpose(rw_context* ctx, const rw_csr* A, int32_t* d_row_ptr, int32_t* d_col, double* d_val) {
    if (!ctx || !d_row_ptr || !d_col || !d_val) {
        set_error("rw_csr_transpose: bad arguments");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr(A);
    if (rc) return rc;
    Pool sc(ctx);
    rc = csr_transpose(ctx, A, d_row_ptr, d_col, d_val, sc);
    sc.release_all();
    if (rc) return rc;
    return check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
}

rw_status rw_precond_apply_ldu(rw_context* ctx, const rw_factor* F_A, const rw_factor* F_AT, const double* d_r,
                               double* d_z, int32_t nrhs) {
    if (!ctx || !d_r || !d_z || nrhs < 1 || nrhs > 16) {
        set_error("rw_precond_apply_ldu: bad arguments");
        return RW_ERR_ARG;
    }
    FactorView v;
    rw_status rc = ldu_view(F_A, F_AT, &v);
    if (rc) return rc;
    if (v.n == 0) return RW_OK;
    if ((rc = reset_status(ctx))) return rc;
    Pool sc(ctx);
    rc = precond_fp64(ctx, v, d_r, d_z, nrhs, sc);
    sc.release_all();
    cudaStreamSynchronize(ctx->stream);
    return rc;
}

rw_status bicgstab_solve(rw_context* ctx, const rw_csr* A, const rw_factor* F_A, const rw_factor* F_AT,
                         const double* d_b, double* d_x, double tol, int32_t max_iter, rw_pcg_stats* stats) {
    if (!ctx || !d_b || !d_x || !(tol >= 0.0) || max_iter < 0) {
        set_error("bicgstab_solve: bad arguments");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr(A);
    if (rc) return rc;
    FactorView v;
    if ((rc = ldu_view(F_A, F_AT, &v))) return rc;
    if (v.n != A->n) {
        set_error("bicgstab_solve: matrix and factors do not match");
        return RW_ERR_ARG;
    }
    if ((rc = reset_status(ctx))) return rc;
    if (A->n == 0) {
        if (stats) memset(stats, 0, sizeof(*stats));
        return RW_OK;
    }
    return bicgstab_run(ctx, A, v, d_b, d_x, tol, max_iter, stats);
}

}  // extern "C"

namespace rw {
rw_status factor_tune_target(const rw_factor* F, const rw_csr* A, TuneTarget* X) {
    if (!F || !A || A->n != F->desc.n) {
        set_error("autotune: matrix and factor do not match");
        return RW_ERR_ARG;
    }
    const rw_factor_desc& d = F->desc;
    *X = TuneTarget{A->n, A->row_ptr, A->col, A->val, nullptr, d.y_row_ptr, d.y_col, d.y_val, d.y_val32,
                    d.yt_row_ptr, d.yt_col, d.yt_val, d.yt_val32, d.d, d.d32, &F->fwd_sched, &F->bwd_sched,
                    F->bar, d.nnz, std::max(d.fwd_levels, d.bwd_levels)};
    return RW_OK;
}
}  // namespace rw

extern "C" {

rw_status pcg_solve(rw_context* ctx, const rw_csr* A, const rw_factor* F, const double* d_b,
                    double* d_x, int32_t nrhs, double tol, int32_t max_iter, rw_precision prec,
                    rw_pcg_stats* stats, int32_t* h_iters, double* h_relres) {
    if (!ctx || !F || !d_b || !d_x) {
        set_error("pcg_solve: NULL argument");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr(A);
    if (rc) return rc;
    if (A->n != F->desc.n || nrhs < 1 || nrhs > 16 || max_iter < 0 || !(tol >= 0.0) ||
        (prec != RW_FP64 && prec != RW_FP32_MIXED)) {
        set_error("pcg_solve: bad arguments (n=%d vs factor %d, nrhs=%d, max_iter=%d)", A->n,
                  F->desc.n, nrhs, max_iter);
        return RW_ERR_ARG;
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    if (A->n == 0) return RW_OK;
    if ((rc = reset_status(ctx))) return rc;
    const int64_t launches0 = g_launches;
    rc = pcg_run(ctx, A, view_of(F), d_b, d_x, nrhs, tol, max_iter, prec, stats, h_iters, h_relres);
    if (stats) stats->kernel_launches = g_launches - launches0;
    return rc;
}

rw_status pcg_solve_batched(rw_context* ctx, int32_t nmat, const rw_csr* As,
                            const rw_factor* const* Fs, const double* const* d_b,
                            double* const* d_x, int32_t nrhs, double tol, int32_t max_iter,
                            rw_precision prec, rw_pcg_stats* stats, int32_t* h_iters,
                            double* h_relres) {
    if (!ctx || nmat < 1 || !As || !Fs || !d_b || !d_x) {
        set_error("pcg_solve_batched: bad arguments");
        return RW_ERR_ARG;
    }
    // one block-diagonal system for the whole batch
    rw_batch* B = nullptr;
    rw_status rc = rw_batch_create(ctx, nmat, As, Fs, &B);
    if (rc) return rc;
    rc = pcg_solve_batch(ctx, B, d_b, d_x, nrhs, tol, max_iter, prec, stats, h_iters, h_relres);
    rw_batch_destroy(B);
    return rc;
}

rw_status rw_precond_apply(rw_context* ctx, const rw_factor* F, const double* d_r, double* d_z,
                           int32_t nrhs) {
    if (!ctx || !F || !d_r || !d_z || nrhs < 1 || nrhs > 16) {
        set_error("rw_precond_apply: bad arguments");
        return RW_ERR_ARG;
    }
    if (F->desc.n == 0) return RW_OK;
    rw_status rc = reset_status(ctx);
    if (rc) return rc;
    Pool sc(ctx);
    rc = precond_fp64(ctx, view_of(F), d_r, d_z, nrhs, sc);
    sc.release_all();
    cudaStreamSynchronize(ctx->stream);
    return rc;
}

rw_status rw_spmv(rw_context* ctx, const rw_csr* A, const double* d_x, double* d_y, int32_t nrhs) {
    if (!ctx || !d_x || !d_y || nrhs < 1 || nrhs > 16) {
        set_error("rw_spmv: bad arguments");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr(A);
    if (rc) return rc;
    if (A->n == 0) return RW_OK;
    if ((rc = reset_status(ctx))) return rc;
    if ((rc = spmv_fp64(ctx, A, d_x, d_y, nrhs))) return rc;
    return read_status(ctx, "spmv");
}

}  // extern "C"
