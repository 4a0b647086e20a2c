// rw_adapt.cu -- the adaptive walk count of Sec. 5.1.
//
// The paper runs walks from row k until the mean walk length Xi'_k of its M_k
// walks is within a relative margin Delta of its expectation at confidence
// alpha (Eq. lengthdelta), checked as Delta Xi'_k sqrt(M_k) / sigma_k > z with
// z = Q^-1((1 - alpha)/2), with a lower bound on M_k.  Each walk row makes a
// sequence of decisions: the first after min_walks walks; a row whose walks do
// not yet meet the criterion asks for the number its current estimates give,
// z^2 sigma^2 / (Delta^2 Xi'^2) (at least one more, at most max_walks in
// total), and is decided again when it has that many; at most max_rounds
// decisions.  A walk is a function of (seed, row, walk index) only, so the
// factor built afterwards with these counts consists of the very walks that
// fixed them.  The sums of lengths and squared lengths are exact integers and
// the test is evaluated in FP64 with every operation rounded once, so the
// counts are reproducible bit for bit.
//
// The GPU runs the rows in launch rounds, each running ahead of the row's next
// decision point T: walks A, A+1, ... up to T + (adapt_ahead % of T), capped,
// A being the walks run so far.  One warp per row then replays the decisions
// in walk order over the new lengths, as many as the walks run allow, so a row
// whose estimate moves by a few walks is decided again in the same round.
// Walks beyond the final count are discarded; the counts and the decision
// count are those of the one-decision-per-round schedule.
#include <cmath>

#include "rw_internal.h"

namespace rw {

// Per walk row: A = walks run, T = next decision point (0 once decided for
// good, the count then in M), S1/S2 = exact sums of the lengths and squared
// lengths of walks 0 .. A-1, D = decisions made.
struct AdaptRows {
    uint32_t* A;
    uint32_t* T;
    uint32_t* M;
    uint32_t* D;
    unsigned long long* S1;
    unsigned long long* S2;
};

// The Sec. 5.1 test after m walks with sums s1, s2: 0 if the row is decided,
// else the walk count its estimates ask for.
__device__ __forceinline__ uint32_t adapt_target(uint32_t m, unsigned long long s1, unsigned long long s2, double d2,
                                                 double z2, uint32_t max_walks) {
    if (m <= 1u || m >= max_walks) return 0u;
    const double Md = (double)m;
    const double mean = __ddiv_rn((double)s1, Md);
    const double var = __ddiv_rn(__dadd_rn((double)s2, -__dmul_rn((double)s1, mean)), __dadd_rn(Md, -1.0));
    const double lhs = __dmul_rn(__dmul_rn(d2, __dmul_rn(mean, mean)), Md);
    const double rhs = __dmul_rn(z2, var);
    if (lhs > rhs) return 0u;
    const double need = __ddiv_rn(rhs, __dmul_rn(d2, __dmul_rn(mean, mean)));
    uint32_t target = need >= (double)max_walks ? max_walks : (uint32_t)ceil(need);
    return target < m + 1u ? m + 1u : target;
}

// Walks a row runs up to: its decision point t and `pct` percent of t beyond.
__device__ __forceinline__ uint32_t adapt_ahead(uint32_t t, uint32_t pct, uint32_t max_walks) {
    const uint64_t a = (uint64_t)t + (uint64_t)t * pct / 100u;
    return a > max_walks ? max_walks : (uint32_t)a;
}

// One warp per walk row: consumes this launch round's lengths (walks A .. A+cnt-1 in
// rec[wbase[r] ..]) in walk order, deciding at every decision point reached;
// sets the row's next request in inc[node] and counts the rows still pending.
__global__ void k_adapt_chain(int32_t nw, const int4* __restrict__ wrow, const int64_t* __restrict__ wbase,
                              const int2* __restrict__ rec, AdaptRows R, double d2, double z2, uint32_t max_walks,
                              uint32_t pct, int32_t max_rounds, uint32_t* inc, unsigned* pending, unsigned* dmax) {
    const int32_t gw = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nwarps = (int32_t)((gridDim.x * blockDim.x) >> 5);
    for (int32_t r = gw; r < nw; r += nwarps) {
        uint32_t t = R.T[r];
        if (t == 0u) {
            if (lane_id() == 0) inc[wrow[r].x] = 0u;
            continue;
        }
        const int64_t b0 = wbase[r], b1 = wbase[r + 1];
        const uint32_t a0 = R.A[r], a1 = a0 + (uint32_t)(b1 - b0);
        uint32_t a = a0, d = R.D[r];
        unsigned long long s1 = R.S1[r], s2 = R.S2[r];
        bool done = false;
        for (;;) {
            if (a == t) {  // a decision point: walks 0 .. t-1 are summed
                ++d;
                const uint32_t nt = adapt_target(t, s1, s2, d2, z2, max_walks);
                if (nt == 0u || d >= (uint32_t)max_rounds) {
                    done = true;
                    break;
                }
                t = nt;
                continue;
            }
            if (a == a1) break;
            const uint32_t e = t < a1 ? t : a1;
            unsigned long long p1 = 0, p2 = 0;
            for (int64_t i = b0 + (a - a0) + lane_id(); i < b0 + (e - a0); i += 32) {
                const unsigned long long l = (uint32_t)rec[i].y;
                p1 += l;
                p2 += l * l;
            }
            s1 += warp_sum(p1);
            s2 += warp_sum(p2);
            a = e;
        }
        if (lane_id() == 0) {
            R.D[r] = d;
            atomicMax(dmax, d);
            if (done) {
                R.T[r] = 0u;
                R.M[r] = t;
                inc[wrow[r].x] = 0u;
            } else {
                R.T[r] = t;
                R.A[r] = a1;
                R.S1[r] = s1;
                R.S2[r] = s2;
                inc[wrow[r].x] = adapt_ahead(t, pct, max_walks) - a1;
                atomicAdd(pending, 1u);
            }
        }
    }
}

__global__ void k_adapt_budget(int32_t n, uint32_t* budget) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) budget[k] = 0u;
}
// Every walk row: first decision after `first` walks, run ahead of it.
__global__ void k_adapt_first(int32_t nw, const int4* __restrict__ wrow, uint32_t first, uint32_t pct,
                              uint32_t max_walks, uint32_t* T, uint32_t* inc) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x) {
        T[r] = first;
        inc[wrow[r].x] = adapt_ahead(first, pct, max_walks);
    }
}
__global__ void k_adapt_budget_rows(int32_t nw, const int4* __restrict__ wrow, const uint32_t* __restrict__ M,
                                    uint32_t* budget) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x)
        budget[wrow[r].x] = M[r];
}

}  // namespace rw

using namespace rw;

extern "C" {

rw_status rw_adaptive_budget(rw_context* ctx, const rw_csr* A, uint64_t seed, double delta, double z,
                             uint32_t min_walks, uint32_t max_walks, int32_t max_rounds, uint32_t* d_budget,
                             int32_t* h_rounds) {
    NvtxRange nvtx_range("rw_adaptive_budget");
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
    k_adapt_budget<<<g, 256, 0, s>>>(n, d_budget);
    if ((rc = check_launch("adaptive budget"))) return rc;
    if (nw == 0) return check_cuda(cudaStreamSynchronize(s), "sync");
    AdaptRows R;
    R.A = alloc_n<uint32_t>(sc, nw);
    R.T = alloc_n<uint32_t>(sc, nw);
    R.M = alloc_n<uint32_t>(sc, nw);
    R.D = alloc_n<uint32_t>(sc, nw);
    R.S1 = alloc_n<unsigned long long>(sc, nw);
    R.S2 = alloc_n<unsigned long long>(sc, nw);
    uint32_t* inc = alloc_n<uint32_t>(sc, n);
    unsigned* flags = alloc_n<unsigned>(sc, 2);  // pending rows, most decisions of a row
    unsigned long long* hops = alloc_n<unsigned long long>(sc, 1);
    if (!R.A || !R.T || !R.M || !R.D || !R.S1 || !R.S2 || !inc || !flags || !hops) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(R.A, 0, sizeof(uint32_t) * (size_t)nw, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(R.M, 0, sizeof(uint32_t) * (size_t)nw, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(R.D, 0, sizeof(uint32_t) * (size_t)nw, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(R.S1, 0, sizeof(unsigned long long) * (size_t)nw, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(R.S2, 0, sizeof(unsigned long long) * (size_t)nw, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(inc, 0, sizeof(uint32_t) * (size_t)n, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(flags, 0, sizeof(unsigned) * 2, s), "memset")))
        return rc;
    const int gw = grid_for(nw, 256, ctx->num_sms * 8);
    const uint32_t pct = ctx->opt.adapt_ahead > 0 ? (uint32_t)ctx->opt.adapt_ahead : 0u;
    RW_COUNT_LAUNCH();
    k_adapt_first<<<gw, 256, 0, s>>>(nw, T.wrow, min_walks, pct, max_walks, R.T, inc);
    if ((rc = check_launch("adaptive start"))) return rc;
    const double d2 = delta * delta, z2 = z * z;
    unsigned* hp = static_cast<unsigned*>(ctx->h_small);
    hp[0] = hp[1] = 0u;
    // Every launch round reaches each pending row's decision point at least
    // once, so max_rounds launch rounds decide every row.
    for (int32_t round = 0; round < max_rounds; ++round) {
        Pool rp(ctx);  // this launch round's walk space and records
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
        wb.wofs = R.A;  // walks A, A+1, ... of each row
        wb.chunk_row = ws.chunk_row;
        wb.total = ws.total;
        WalkLaunch wl;
        wl.max_steps = ctx->opt.max_steps;
        wl.record_lengths = 1;
        if ((rc = run_walks(ctx, wb, wl, rec, hops, rp, nullptr)) || (rc = read_status(ctx, "adaptive walks")))
            return rc;
        if ((rc = check_cuda(cudaMemsetAsync(flags, 0, sizeof(unsigned), s), "memset"))) return rc;
        RW_COUNT_LAUNCH();
        k_adapt_chain<<<grid_for((int64_t)nw * 32, 256, ctx->num_sms * 8), 256, 0, s>>>(
            nw, T.wrow, ws.wbase, rec, R, d2, z2, max_walks, pct, max_rounds, inc, flags, flags + 1);
        if ((rc = check_launch("adaptive decisions"))) return rc;
        if ((rc = check_cuda(cudaMemcpyAsync(hp, flags, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s), "copy")) ||
            (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
            return rc;
        if (hp[0] == 0u) break;
    }
    RW_COUNT_LAUNCH();
    k_adapt_budget_rows<<<gw, 256, 0, s>>>(nw, T.wrow, R.M, d_budget);
    if ((rc = check_launch("adaptive budget"))) return rc;
    if (h_rounds) *h_rounds = (int32_t)hp[1];
    return read_status(ctx, "adaptive budget");
}

}  // extern "C"
