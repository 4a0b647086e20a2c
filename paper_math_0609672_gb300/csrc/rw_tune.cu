// rw_tune.cu -- autotuner for the solve-step schedules.
//
// The preconditioner application (two level-scheduled triangular solves) and
// the SpMV have launch-shape parameters whose best values depend on the
// factor's level structure and the number of right-hand sides: entry slices
// per row group (lanes per row = slices x right-hand sides), blocks per SM of
// the wide-level kernel, and whether narrow levels run on one thread-block
// cluster.  The tuner times a fixed candidate list on the caller's own
// factor (or batch) with CUDA events, keeps the fastest, installs it in the
// context options, and records it in a JSON-lines cache keyed by the device
// and the problem's shape, so that later runs on similar problems skip the
// timing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rw_internal.h"

namespace rw {

namespace {

struct Candidate {
    int wide_slices, solve_blocks_per_sm, cluster_width, spmv_slices, solve_mode;
    int solve_mode_bwd = -1;  // -1: as solve_mode
    int thin_cluster = 0;
    int thin_flags = 0;
    int thin_lanes = 0;
};

std::string shape_key(const rw_context* ctx, const TuneTarget& T, int nrhs) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, ctx->device);
    int nr = 1;
    while (nr < nrhs) nr <<= 1;
    const int lg_n = (int)std::lround(std::log2(std::max(1, T.n)));
    const double per_row = T.n > 0 ? (double)T.nnz_y / T.n : 0.0;
    const int lg_per_row = (int)std::lround(std::log2(std::max(1.0, per_row)) * 2.0);
    const int lg_depth = (int)std::lround(std::log2(std::max(1, T.depth)) * 2.0);
    char buf[512];
    snprintf(buf, sizeof buf, "%s|sm%d|n2^%d|ypr%d|depth%d|nrhs%d", prop.name, prop.multiProcessorCount, lg_n,
             lg_per_row, lg_depth, nr);
    for (char* p = buf; *p; ++p)
        if (*p == '"' || *p == '\\') *p = '_';
    return buf;
}

// Reads "key": integer from a one-line JSON object (the cache format written below).
bool json_int(const std::string& line, const char* key, int* out) {
    const std::string k = std::string("\"") + key + "\":";
    const size_t p = line.find(k);
    if (p == std::string::npos) return false;
    *out = atoi(line.c_str() + p + k.size());
    return true;
}

bool cache_lookup(const char* path, const std::string& key, Candidate* c) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char buf[1024];
    bool found = false;
    const std::string kk = "\"key\":\"" + key + "\"";
    while (fgets(buf, sizeof buf, f)) {
        const std::string line(buf);
        if (line.find(kk) == std::string::npos) continue;
        Candidate t{};
        if (json_int(line, "wide_slices", &t.wide_slices) && json_int(line, "solve_blocks_per_sm", &t.solve_blocks_per_sm) &&
            json_int(line, "cluster_width", &t.cluster_width) && json_int(line, "spmv_slices", &t.spmv_slices) &&
            json_int(line, "solve_mode", &t.solve_mode) && json_int(line, "solve_mode_bwd", &t.solve_mode_bwd) &&
            json_int(line, "thin_cluster", &t.thin_cluster) && json_int(line, "thin_flags", &t.thin_flags)) {
            json_int(line, "thin_lanes", &t.thin_lanes);  // absent in older cache lines: 0
            *c = t;  // the last matching line wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& key, const Candidate& c, float ms_pre, float ms_spmv) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"key\":\"%s\",\"solve_mode\":%d,\"solve_mode_bwd\":%d,\"thin_cluster\":%d,\"thin_flags\":%d,\"thin_lanes\":%d,\"wide_slices\":%d,\"solve_blocks_per_sm\":%d,\"cluster_width\":%d,"
            "\"spmv_slices\":%d,\"precond_ms\":%.4f,\"spmv_ms\":%.4f}\n",
            key.c_str(), c.solve_mode, c.solve_mode_bwd, c.thin_cluster, c.thin_flags, c.thin_lanes, c.wide_slices, c.solve_blocks_per_sm, c.cluster_width, c.spmv_slices, ms_pre,
            ms_spmv);
    fclose(f);
}

template <typename T>
rw_status time_precond(rw_context* ctx, const TuneTarget& X, const T* yv, const T* ytv, const T* dv,
                       const T* tvf, const T* tvb, const T* r, T* w, T* z, int nrhs, int reps, float* ms) {
    cudaStream_t s = ctx->stream;
    rw_status rc;
    auto once = [&]() -> rw_status {
        rw_status r2 = solve_runs<T>(ctx, *X.bwd, X.yt_rp, X.yt_col, ytv, tvb, r, nullptr, w, nrhs, X.bar, true);
        if (r2) return r2;
        if ((r2 = apply_inverse_diag<T>(ctx, w, dv, X.fwd->n, nrhs))) return r2;
        return solve_runs<T>(ctx, *X.fwd, X.y_rp, X.y_col, yv, tvf, w, nullptr, z, nrhs, X.bar);
    };
    if ((rc = once())) return rc;
    cudaEventRecord(ctx->ev[10], s);
    for (int i = 0; i < reps; ++i)
        if ((rc = once())) return rc;
    cudaEventRecord(ctx->ev[11], s);
    if ((rc = check_cuda(cudaEventSynchronize(ctx->ev[11]), "sync"))) return rc;
    cudaEventElapsedTime(ms, ctx->ev[10], ctx->ev[11]);
    *ms /= (float)reps;
    return read_status(ctx, "autotune");
}

template <typename T>
rw_status time_spmv(rw_context* ctx, const TuneTarget& X, const T* av, const T* x, T* y, int nrhs, int reps,
                    float* ms) {
    cudaStream_t s = ctx->stream;
    rw_status rc;
    if ((rc = spmv_launch<T>(ctx, X.n, X.a_rp, X.a_col, av, x, y, nrhs))) return rc;
    cudaEventRecord(ctx->ev[10], s);
    for (int i = 0; i < reps; ++i)
        if ((rc = spmv_launch<T>(ctx, X.n, X.a_rp, X.a_col, av, x, y, nrhs))) return rc;
    cudaEventRecord(ctx->ev[11], s);
    if ((rc = check_cuda(cudaEventSynchronize(ctx->ev[11]), "sync"))) return rc;
    cudaEventElapsedTime(ms, ctx->ev[10], ctx->ev[11]);
    *ms /= (float)reps;
    return RW_OK;
}

template <typename T>
__global__ void k_tune_fill(T* v, int64_t cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (T)(1.0 + 0.001 * (double)(i % 977));
}

template <typename T>
rw_status tune_t(rw_context* ctx, const TuneTarget& X, int nrhs, const T* av, const T* yv, const T* ytv,
                 const T* dv, const T* tvf, const T* tvb, Candidate* best, float* best_pre, float* best_spmv) {
    Pool sc(ctx);
    const int64_t cnt = (int64_t)X.n * nrhs;
    T* r = alloc_n<T>(sc, cnt);
    T* w = alloc_n<T>(sc, cnt);
    T* z = alloc_n<T>(sc, cnt);
    if (!r || !w || !z) return RW_ERR_ALLOC;
    RW_COUNT_LAUNCH();
    k_tune_fill<T><<<grid_for(cnt, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(r, cnt);
    rw_status rc = check_launch("autotune fill");
    if (rc) return rc;
    int nr = 1;
    while (nr < nrhs) nr <<= 1;
    const rw_options saved = ctx->opt;
    // candidate list: the sync-free solve; the level schedule with entry
    // slices 32/NR, 16/NR, 8/NR (>= 1), 1 or 2 blocks per SM, cluster runs off
    // or for levels of up to 256 rows; vector rows with 1 or 2 blocks per SM
    std::vector<int> slices;
    for (int es = 32 / nr; es >= 1 && (int)slices.size() < 3; es /= 2) slices.push_back(es);
    float bp = 1e30f, bs = 1e30f;
    Candidate b{slices[0], 1, 0, slices[0], 0};
    const int reps = 3;
    std::vector<Candidate> cands;
    cands.push_back(Candidate{slices[0], 1, 0, 0, 1});
    for (int es : slices)
        for (int bps : {1, 2})
            for (int cw : {0, 256}) cands.push_back(Candidate{es, bps, cw, 0, 0});
    for (int bps : {1, 2}) cands.push_back(Candidate{-1, bps, 0, 0, 0});  // vector rows
    cands.push_back(Candidate{-1, 1, 0, 0, 1});                            // sync-free, vector rows
    cands.push_back(Candidate{-1, 1, 0, 0, 1, 0});  // sync-free forward, level-scheduled backward
    cands.push_back(Candidate{-1, 1, 0, 0, 0, 1});  // level-scheduled forward, sync-free backward
    cands.push_back(Candidate{-1, 1, 0, 0, 2});     // hybrid runs (thin: one block; wide: sync-free)
    cands.push_back(Candidate{-1, 2, 0, 0, 2});     // hybrid, sync-free parts with two blocks per SM
    cands.push_back(Candidate{-1, 1, 0, 0, 1, 2});  // sync-free forward, hybrid backward
    for (int tc : {4, 8}) {                          // hybrid with thin runs on clusters
        Candidate c{-1, 1, 0, 0, 2};
        c.thin_cluster = tc;
        cands.push_back(c);
    }
    for (int bps : {1, 2}) {                         // hybrid, thin runs with ready flags
        Candidate c{-1, bps, 0, 0, 2};
        c.thin_flags = 1;
        cands.push_back(c);
    }
    for (int tl : {8, 16}) {                         // hybrid, thin runs with lane groups
        if (tl < nr) continue;
        for (int bps : {1, 2})
            for (int fl : {0, 1}) {
                Candidate c{-1, bps, 0, 0, 2};
                c.thin_lanes = tl;
                c.thin_flags = fl;
                cands.push_back(c);
            }
    }
    for (const Candidate& c : cands) {
        ctx->opt.solve_mode = c.solve_mode;
        ctx->opt.solve_mode_bwd = c.solve_mode_bwd;
        ctx->opt.thin_cluster = c.thin_cluster;
        ctx->opt.thin_flags = c.thin_flags;
        ctx->opt.thin_lanes = c.thin_lanes;
        ctx->opt.wide_slices = c.wide_slices;
        ctx->opt.solve_blocks_per_sm = c.solve_blocks_per_sm;
        ctx->opt.cluster_width = c.cluster_width;
        float ms = 0.f;
        if ((rc = time_precond<T>(ctx, X, yv, ytv, dv, tvf, tvb, r, w, z, nrhs, reps, &ms))) {
            ctx->opt = saved;
            return rc;
        }
        if (ms < bp) {
            bp = ms;
            b.solve_mode = c.solve_mode;
            b.solve_mode_bwd = c.solve_mode_bwd;
            b.thin_cluster = c.thin_cluster;
            b.thin_flags = c.thin_flags;
            b.thin_lanes = c.thin_lanes;
            b.wide_slices = c.wide_slices;
            b.solve_blocks_per_sm = c.solve_blocks_per_sm;
            b.cluster_width = c.cluster_width;
        }
    }
    if (X.a_rp) {
        for (int es : slices) {
            ctx->opt.spmv_slices = es;
            float ms = 0.f;
            if ((rc = time_spmv<T>(ctx, X, av, r, z, nrhs, 5, &ms))) {
                ctx->opt = saved;
                return rc;
            }
            if (ms < bs) {
                bs = ms;
                b.spmv_slices = es;
            }
        }
    }
    ctx->opt = saved;
    *best = b;
    *best_pre = bp;
    *best_spmv = X.a_rp ? bs : 0.f;
    return RW_OK;
}

rw_status autotune(rw_context* ctx, const TuneTarget& X, int nrhs, rw_precision prec, const char* cache,
                   rw_options* out, float* ms_out) {
    const std::string key = shape_key(ctx, X, nrhs) + (prec == RW_FP32_MIXED ? "|fp32" : "|fp64");
    Candidate c{};
    float ms_pre = 0.f, ms_spmv = 0.f;
    if (!cache_lookup(cache, key, &c)) {
        rw_status rc;
        if (prec == RW_FP32_MIXED) {
            rc = tune_t<float>(ctx, X, nrhs, X.a_val32, X.y_val32, X.yt_val32, X.d32, X.fwd->tval32, X.bwd->tval32, &c,
                               &ms_pre, &ms_spmv);
        } else {
            rc = tune_t<double>(ctx, X, nrhs, X.a_val, X.y_val, X.yt_val, X.d, X.fwd->tval, X.bwd->tval, &c,
                                &ms_pre, &ms_spmv);
        }
        if (rc) return rc;
        cache_store(cache, key, c, ms_pre, ms_spmv);
    }
    ctx->opt.solve_mode = c.solve_mode;
    ctx->opt.solve_mode_bwd = c.solve_mode_bwd;
    ctx->opt.thin_cluster = c.thin_cluster;
    ctx->opt.thin_flags = c.thin_flags;
    ctx->opt.thin_lanes = c.thin_lanes;
    ctx->opt.wide_slices = c.wide_slices;
    ctx->opt.solve_blocks_per_sm = c.solve_blocks_per_sm;
    ctx->opt.cluster_width = c.cluster_width;
    ctx->opt.spmv_slices = c.spmv_slices;
    if (out) *out = ctx->opt;
    if (ms_out) ms_out[0] = ms_pre, ms_out[1] = ms_spmv;
    return RW_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Latency probes.  A triangular solve is a chain through L2: a row's value is
// stored by one SM and picked up by the polling load of another, so the two
// latencies that bound it are a dependent L2-hit load and an SM-to-SM hand-off
// through L2 (a relaxed store seen by a relaxed poll).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One thread follows `steps` dependent relaxed loads through a cyclic
// permutation that stays in L2.
__global__ void k_probe_chase(const unsigned* next, int steps, unsigned* sink, unsigned long long* ns) {
    unsigned idx = 0;
    for (int i = 0; i < 256; ++i) idx = ld_relaxed_u32(next + idx);
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < steps; ++i) idx = ld_relaxed_u32(next + idx);
    ns[0] = global_ns() - t0;
    sink[0] = idx;
}

// Blocks 0 and `partner` (distinct SMs: the dynamic shared memory admits one
// block per SM) pass a counter back and forth `iters` times; every wait is
// bounded and sets the timeout flag when it gives up.
__global__ void k_probe_pingpong(unsigned* flags, int partner, int iters, unsigned long long* ns, DevStatus* st) {
    extern __shared__ unsigned probe_pad[];
    const int b = (int)blockIdx.x;
    if (threadIdx.x != 0 || (b != 0 && b != partner)) return;
    probe_pad[0] = (unsigned)b;
    const bool first = b == 0;
    unsigned* mine = flags + (first ? 0 : 32);
    const unsigned* theirs = flags + (first ? 32 : 0);
    const unsigned limit = st->spin_limit;
    const unsigned long long t0 = global_ns();
    for (int i = 1; i <= iters; ++i) {
        if (first) st_relaxed_u32(mine, (unsigned)i);
        unsigned spins = 0;
        while (ld_relaxed_u32(theirs) != (unsigned)i)
            if (wait_gives_up(spins, limit, &st->timeout)) return;
        if (!first) st_relaxed_u32(mine, (unsigned)i);
    }
    if (first) ns[0] = global_ns() - t0;
}

// Random-gather throughput: every thread runs kGatherStreams independent
// address streams (a 64-bit LCG each) and per step loads one aligned unit of
// W * 32 bytes from a random unit of the buffer per stream, folding the words
// into a checksum so that no load is dead.  The loads of a step are
// independent, so kGatherStreams of them are in flight per thread.
constexpr int kGatherStreams = 4;

__device__ __forceinline__ void ld_gather8(const uint32_t* p, uint4& lo, uint4& hi) {
    asm volatile("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
                 : "l"(p));
}

template <int W>
__global__ void __launch_bounds__(256) k_probe_gather(const uint32_t* __restrict__ buf, uint64_t nunits, int steps,
                                                      unsigned* sink) {
    uint64_t st[kGatherStreams];
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int c = 0; c < kGatherStreams; ++c) st[c] = (tid * kGatherStreams + c) * 0x9E3779B97F4A7C15ull + 1u;
    uint32_t acc = 0;
    for (int i = 0; i < steps; ++i) {
#pragma unroll
        for (int c = 0; c < kGatherStreams; ++c) {
            st[c] = st[c] * 6364136223846793005ull + 1442695040888963407ull;
            const uint64_t unit = ((st[c] >> 32) * nunits) >> 32;  // < nunits
            const uint32_t* p = buf + unit * (uint64_t)(W * 8);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint4 a, b;
                ld_gather8(p + 8 * w, a, b);
                acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
            }
        }
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);
}

}  // namespace rw

using namespace rw;

extern "C" {

rw_status rw_probe_gather(rw_context* ctx, uint64_t buffer_bytes, int32_t access_bytes, double* h_gbs) {
    if (!ctx || !h_gbs || buffer_bytes < ((uint64_t)1 << 20) || buffer_bytes > ((uint64_t)1 << 37) ||
        (access_bytes != 32 && access_bytes != 64 && access_bytes != 128)) {
        set_error("rw_probe_gather: bad arguments (buffer 1 MiB .. 128 GiB, access 32, 64 or 128 bytes)");
        return RW_ERR_ARG;
    }
    cudaStream_t s = ctx->stream;
    rw_status rc;
    if ((rc = reset_status(ctx))) return rc;
    Pool sc(ctx);
    const uint64_t nunits = buffer_bytes / (uint64_t)access_bytes;
    uint32_t* buf = static_cast<uint32_t*>(sc.get((size_t)(nunits * (uint64_t)access_bytes)));
    unsigned* sink = alloc_n<unsigned>(sc, 1);
    if (!buf || !sink) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(buf, 0x5A, (size_t)(nunits * (uint64_t)access_bytes), s), "memset")))
        return rc;
    const void* fn = access_bytes == 32 ? (const void*)k_probe_gather<1>
                     : access_bytes == 64 ? (const void*)k_probe_gather<2> : (const void*)k_probe_gather<4>;
    int per_sm = 0;
    if ((rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0), "occupancy")))
        return rc;
    if (per_sm < 1) per_sm = 1;
    const unsigned blocks = (unsigned)(per_sm * ctx->num_sms);
    const uint64_t threads = (uint64_t)blocks * 256u;
    // about 2^28 accessed units per launch
    int steps = (int)(((uint64_t)1 << 28) / (threads * kGatherStreams));
    if (steps < 16) steps = 16;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms the caches and the TLB
        cudaEventRecord(ctx->ev[0], s);
        RW_COUNT_LAUNCH();
        if (access_bytes == 32) k_probe_gather<1><<<blocks, 256, 0, s>>>(buf, nunits, steps, sink);
        else if (access_bytes == 64) k_probe_gather<2><<<blocks, 256, 0, s>>>(buf, nunits, steps, sink);
        else k_probe_gather<4><<<blocks, 256, 0, s>>>(buf, nunits, steps, sink);
        if ((rc = check_launch("gather probe"))) return rc;
        cudaEventRecord(ctx->ev[1], s);
        if ((rc = check_cuda(cudaEventSynchronize(ctx->ev[1]), "gather probe"))) return rc;
        cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    }
    const double bytes = (double)threads * (double)steps * kGatherStreams * (double)access_bytes;
    *h_gbs = ms > 0.f ? bytes / ((double)ms * 1e-3) / 1e9 : 0.0;
    return read_status(ctx, "gather probe");
}

rw_status rw_probe_latency(rw_context* ctx, int32_t iters, double* h_handoff_ns, double* h_l2_ns) {
    if (!ctx || iters < 1 || iters > (1 << 20) || !h_handoff_ns || !h_l2_ns) {
        set_error("rw_probe_latency: bad arguments (1 <= iters <= 2^20, both outputs)");
        return RW_ERR_ARG;
    }
    cudaStream_t s = ctx->stream;
    rw_status rc;
    if ((rc = reset_status(ctx))) return rc;
    Pool sc(ctx);
    constexpr unsigned kChase = 1u << 16;  // 256 KB: L2-resident
    unsigned* next = alloc_n<unsigned>(sc, kChase);
    unsigned* flags = alloc_n<unsigned>(sc, 64);
    unsigned long long* ns = alloc_n<unsigned long long>(sc, 8);
    if (!next || !flags || !ns) return RW_ERR_ALLOC;
    // one cycle through all entries (Sattolo's shuffle, fixed LCG)
    std::vector<unsigned> perm(kChase);
    for (unsigned i = 0; i < kChase; ++i) perm[i] = i;
    uint64_t lcg = 0x9E3779B97F4A7C15ull;
    for (unsigned i = kChase - 1; i > 0; --i) {
        lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
        const unsigned j = (unsigned)((lcg >> 33) % i);
        std::swap(perm[i], perm[j]);
    }
    if ((rc = check_cuda(cudaMemcpyAsync(next, perm.data(), sizeof(unsigned) * kChase, cudaMemcpyHostToDevice, s),
                         "copy")))
        return rc;
    RW_COUNT_LAUNCH();
    k_probe_chase<<<1, 1, 0, s>>>(next, iters, flags + 48, ns);
    if ((rc = check_launch("latency probe"))) return rc;
    const int smem = 120 * 1024;
    if ((rc = check_cuda(cudaFuncSetAttribute(k_probe_pingpong, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                         "attribute")))
        return rc;
    const int nsm = ctx->num_sms;
    int partners[4] = {1, nsm / 4, nsm / 2, nsm - 1};
    int np = 0;
    for (int i = 0; i < 4; ++i) {
        bool dup = partners[i] < 1 || partners[i] >= nsm;
        for (int j = 0; j < np; ++j) dup = dup || partners[j] == partners[i];
        if (!dup) partners[np++] = partners[i];
    }
    for (int i = 0; i < np; ++i) {
        if ((rc = check_cuda(cudaMemsetAsync(flags, 0, sizeof(unsigned) * 48, s), "memset"))) return rc;
        unsigned long long* out = ns + 1 + i;
        int partner = partners[i], it = iters;
        DevStatus* st = ctx->d_status;
        void* args[] = {(void*)&flags, (void*)&partner, (void*)&it, (void*)&out, (void*)&st};
        RW_COUNT_LAUNCH();
        if ((rc = check_cuda(cudaLaunchCooperativeKernel((const void*)k_probe_pingpong, dim3((unsigned)nsm), dim3(32),
                                                         args, (size_t)smem, s),
                             "latency probe")))
            return rc;
    }
    unsigned long long h[8] = {0};
    if ((rc = check_cuda(cudaMemcpyAsync(h, ns, sizeof(h), cudaMemcpyDeviceToHost, s), "copy")) ||
        (rc = read_status(ctx, "latency probe")))
        return rc;
    *h_l2_ns = (double)h[0] / iters;
    double sum = 0.0;
    for (int i = 0; i < np; ++i) sum += (double)h[1 + i] / (2.0 * iters);
    *h_handoff_ns = np ? sum / np : 0.0;
    return RW_OK;
}

rw_status rw_autotune(rw_context* ctx, const rw_csr* A, const rw_factor* F, int32_t nrhs, rw_precision prec,
                      const char* cache_path, rw_options* out, float* h_ms) {
    NvtxRange nvtx_range("rw_autotune");
    if (!ctx || !A || !F || nrhs < 1 || nrhs > 16 || (prec != RW_FP64 && prec != RW_FP32_MIXED)) {
        set_error("rw_autotune: bad arguments");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr(A);
    if (rc) return rc;
    TuneTarget X{};
    if ((rc = factor_tune_target(F, A, &X))) return rc;
    if (X.n == 0) return RW_OK;
    if (prec == RW_FP32_MIXED && !X.y_val32) {
        set_error("rw_autotune: FP32 tuning needs a factor built with store_fp32 = 1");
        return RW_ERR_ARG;
    }
    if ((rc = reset_status(ctx))) return rc;
    Pool sc(ctx);
    if (prec == RW_FP32_MIXED) {
        float* a32 = alloc_n<float>(sc, A->nnz);
        if (!a32) return RW_ERR_ALLOC;
        launch_to_fp32_diff(A->n, A->row_ptr, A->col, A->val, a32, ctx->stream, ctx->num_sms);
        X.a_val32 = a32;
    }
    return autotune(ctx, X, nrhs, prec, cache_path, out, h_ms);
}

rw_status rw_batch_autotune(rw_context* ctx, const rw_batch* B, int32_t nrhs, rw_precision prec,
                            const char* cache_path, rw_options* out, float* h_ms) {
    NvtxRange nvtx_range("rw_autotune");
    if (!ctx || !B || nrhs < 1 || nrhs > 16 || (prec != RW_FP64 && prec != RW_FP32_MIXED)) {
        set_error("rw_batch_autotune: bad arguments");
        return RW_ERR_ARG;
    }
    TuneTarget X{};
    rw_status rc = batch_tune_target(B, &X);
    if (rc) return rc;
    if (X.n == 0) return RW_OK;
    if (prec == RW_FP32_MIXED && (!X.y_val32 || !X.a_val32)) {
        set_error("rw_batch_autotune: FP32 tuning needs factors built with store_fp32 = 1");
        return RW_ERR_ARG;
    }
    if ((rc = reset_status(ctx))) return rc;
    return autotune(ctx, X, nrhs, prec, cache_path, out, h_ms);
}

}  // extern "C"
