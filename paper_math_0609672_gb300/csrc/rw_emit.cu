// rw_emit.cu -- journey record -> incomplete factor.
//
// For every walk row k the per-walk records are merged into end-point counts
// H'_ki (warp-level __match_any_sync, then a shared-memory hash table), the
// union of the end points and the lower neighbours of k is sorted, and the
// factor row follows the one-step-exact estimator (Sec. 5.2):
//   a    = S_k / A_kk,  S_k = sum_{j>k} A_kj
//   Y_ki = A_ki / A_kk + a * (H'_ki / M'_k)          (Eq. newy)
//   D_kk = A_kk / (1 + a * (1 - J'_k / M'_k))        (Eq. newz with Eq. d: D = 1/Z)
// each operation rounded once, in this order.  Entries with |Y_ki| < drop_tol
// are dropped (post-processing drop, footnote of Sec. 4).  Rows without an
// upper neighbour are exact: Y_ki = A_ki / A_kk, D_kk = A_kk.
#include <algorithm>
#include <climits>
#include <utility>
#include <vector>

#include "rw_internal.h"

namespace rw {

constexpr uint32_t kNbrFlag = 0x80000000u;
constexpr uint32_t kCountMask = 0x7FFFFFFFu;
constexpr int kLog2SmallHash = 10;              // 1024 slots per warp
constexpr int kSmallCap = 768;                  // distinct keys a warp table accepts
constexpr int kLog2BigHash = 14;                // 16384 slots per block
constexpr int kBigCap = 12288;
// Rows with more possible keys go to a block with a global-memory table of at
// least twice their bound (the huge path); those tables take at most this much.
constexpr size_t kHugeTableBytes = size_t(1) << 30;

struct MergeParams {
    const int32_t* __restrict__ rp;
    const int32_t* __restrict__ col;
    const double* __restrict__ val;
    const int32_t* __restrict__ dpos;
    const int4* __restrict__ wrow;
    const int64_t* __restrict__ wbase;
    const int64_t* __restrict__ tbase;
    const int2* __restrict__ rec;
    const int64_t* __restrict__ xbase;  // walk reuse: extra records per walk row (NULL: none)
    const int2* __restrict__ xrec;
    const double* __restrict__ S;
    const double* __restrict__ diag;
    double drop_tol;
    int32_t nw;
    int32_t* tcol;
    double* tval;
    int64_t* ycnt;
    double* D;
    uint32_t* M;
    uint64_t* J;
    uint32_t* G;
    int32_t* big_rows;
    int32_t* n_big;
    int32_t* huge_rows;
    int32_t* n_huge;
    unsigned long long* huge_bound;  // largest key bound of the huge rows
    DevStatus* st;
};

// Upper bound on the distinct keys of walk row r: its walks' end points and
// its lower neighbours are all columns below k.
__device__ __forceinline__ int64_t row_walks(const MergeParams& P, int32_t r) {
    return P.wbase[r + 1] - P.wbase[r] + (P.xbase ? P.xbase[r + 1] - P.xbase[r] : 0);
}

__device__ __forceinline__ int64_t key_bound(const MergeParams& P, int32_t r) {
    const int4 info = P.wrow[r];
    const int64_t m = row_walks(P, r);
    return min(m + (int64_t)info.w, (int64_t)info.x);
}

// Slots of the global table of a huge row with key bound b: a power of two >= 2b + 2.
__host__ __device__ __forceinline__ int huge_log2_slots(int64_t b) {
    int lg = 1;
    while ((int64_t(1) << lg) < 2 * b + 2) ++lg;
    return lg;
}

template <int TEAM>
__device__ __forceinline__ void team_sync() {
    if (TEAM == 32) __syncwarp();
    else __syncthreads();
}

template <int TEAM>
__device__ __forceinline__ int team_rank() {
    return TEAM == 32 ? (int)lane_id() : (int)threadIdx.x;
}

// Exclusive count of `f` over the team in thread order; total in *total.
template <int TEAM>
__device__ __forceinline__ int team_prefix(bool f, int* total, int* wsm) {
    const unsigned b = __ballot_sync(kFull, f);
    const int in_warp = __popc(b & lanemask_lt());
    if (TEAM == 32) {
        *total = __popc(b);
        return in_warp;
    }
    const int warp = threadIdx.x >> 5;
    if (lane_id() == 0) wsm[warp] = __popc(b);
    __syncthreads();
    int pre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < TEAM / 32; ++i) {
        const int c = wsm[i];
        pre += (i < warp) ? c : 0;
        tot += c;
    }
    __syncthreads();
    *total = tot;
    return pre + in_warp;
}

template <int TEAM, typename T>
__device__ __forceinline__ T team_sum(T v, T* sm) {
    v = warp_sum(v);
    if (TEAM == 32) return v;
    if (threadIdx.x == 0) *sm = T(0);
    __syncthreads();
    if (lane_id() == 0) atomicAdd(sm, v);
    __syncthreads();
    const T r = *sm;
    __syncthreads();
    return r;
}

// Table of 2^lg slots; at most half of them ever hold a key (the callers'
// key bounds), so the probe always finds the key or an empty slot.
__device__ __forceinline__ void hash_insert(int* keys, uint32_t* vals, int key, uint32_t add,
                                            bool flag, int lg) {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = ((uint32_t)key * 2654435761u) >> (32 - lg);
    for (;;) {
        const int prev = atomicCAS(&keys[h], -1, key);
        if (prev == -1 || prev == key) {
            if (flag) atomicOr(&vals[h], kNbrFlag);
            else atomicAdd(&vals[h], add);
            return;
        }
        h = (h + 1u) & mask;
    }
}

// Bitonic sort of keys[0..P) (with vals) ascending, P a power of two.
template <int TEAM>
__device__ void team_bitonic(int* keys, uint32_t* vals, int P) {
    const int t = team_rank<TEAM>();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = t; i < (P >> 1); i += TEAM) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const int a = keys[lo], b = keys[hi];
                if ((a > b) == asc) {
                    keys[lo] = b;
                    keys[hi] = a;
                    const uint32_t va = vals[lo];
                    vals[lo] = vals[hi];
                    vals[hi] = va;
                }
            }
            team_sync<TEAM>();
        }
    }
}

// Merge the records of walk row r and write its kept entries (ascending
// columns) to the row's slot of the temporary area.
// LOG2HC > 0: a table of 2^LOG2HC slots; LOG2HC == 0: 2^lg_rt slots.
template <int TEAM, int LOG2HC>
__device__ void merge_row(const MergeParams& P, int32_t r, int* keys, uint32_t* vals, int* wsm,
                          unsigned long long* sm64, int lg_rt = 0) {
    const int lg = LOG2HC > 0 ? LOG2HC : lg_rt;
    const int HC = 1 << lg;
    const int t = team_rank<TEAM>();
    const int4 info = P.wrow[r];
    const int32_t k = info.x;
    const int64_t b0 = P.wbase[r], b1 = P.wbase[r + 1];
    const int32_t rs = P.rp[k], dp = P.dpos[k];

    for (int i = t; i < HC; i += TEAM) {
        keys[i] = -1;
        vals[i] = 0u;
    }
    team_sync<TEAM>();
    for (int32_t p = rs + t; p < dp; p += TEAM) hash_insert(keys, vals, P.col[p], 0u, true, lg);

    unsigned long long jsum = 0;
    unsigned gsum = 0, csum = 0;
    // the row's own walks, then (walk reuse) the sub-walks that start at k
    const int2* src = P.rec;
    int64_t e0 = b0, e1 = b1;
    for (int part = 0; part < 2; ++part) {
        if (part == 1) {
            if (!P.xbase) break;
            src = P.xrec;
            e0 = P.xbase[r];
            e1 = P.xbase[r + 1];
        }
        for (int64_t base = e0; base < e1; base += TEAM) {
            const int64_t idx = base + t;
            const bool valid = idx < e1;
            int2 rc = make_int2(-3, 0);
            if (valid) rc = src[idx];
            if (valid) {
                jsum += (unsigned)rc.y;
                gsum += rc.x == -1;
                csum += (rc.x < -1 || rc.x >= k);  // step cap (or a record that is not an end node)
            }
            const bool ep = valid && rc.x >= 0 && rc.x < k;
            const unsigned em = __ballot_sync(kFull, ep);
            if (ep) {
                const unsigned g = __match_any_sync(em, rc.x);
                if ((int)lane_id() == __ffs(g) - 1) hash_insert(keys, vals, rc.x, __popc(g), false, lg);
            }
        }
    }
    team_sync<TEAM>();

    // move the occupied slots to the front, in slot order
    int u = 0;
    for (int base = 0; base < HC; base += TEAM) {
        const int key = keys[base + t];
        const uint32_t v = vals[base + t];
        const bool occ = key != -1;
        int tot;
        const int pos = team_prefix<TEAM>(occ, &tot, wsm);
        team_sync<TEAM>();
        if (occ) {
            keys[u + pos] = key;
            vals[u + pos] = v;
        }
        u += tot;
        team_sync<TEAM>();
    }
    int Pw = 1;
    while (Pw < u) Pw <<= 1;
    for (int i = u + t; i < Pw; i += TEAM) {
        keys[i] = 0x7FFFFFFF;
        vals[i] = 0u;
    }
    team_sync<TEAM>();
    team_bitonic<TEAM>(keys, vals, Pw);

    const double akk = P.diag[k];
    const int64_t walks = row_walks(P, r);
    const double Mk = (double)walks;
    const int64_t tb = P.tbase[r];
    // The row's quotients in one warp-wide FP64 division (each lane one IEEE
    // quotient; the FP64 pipe is narrow, so the per-row divisions are packed):
    // lane 0: a = S_k / A_kk; lanes 1..8: h / M' for the small counts h almost
    // every end point has; lanes 9..31: A_ki / A_kk for the first 23 lower
    // neighbours (in column order).  Rarer quotients are divided where needed.
    constexpr int kQuotSmall = 8, kQuotNbr = 9;
    const int nlow = dp - rs;
    const int ql = (int)lane_id();
    double qnum = 1.0, qden = 1.0;
    if (ql == 0) {
        qnum = P.S[k];
        qden = akk;
    } else if (ql <= kQuotSmall) {
        qnum = (double)ql;
        qden = Mk;
    } else if (ql - kQuotNbr < nlow) {
        qnum = P.val[rs + ql - kQuotNbr];
        qden = akk;
    }
    const double quot = __ddiv_rn(qnum, qden);
    const double a = __shfl_sync(kFull, quot, 0);
    int kept = 0;
    int nbr_before = 0;  // lower neighbours among the keys of earlier chunks
    for (int base = 0; base < u; base += TEAM) {
        const int s = base + t;
        bool keep = false;
        int key = 0;
        double y = 0.0;
        const uint32_t v = s < u ? vals[s] : 1u;
        const uint32_t hcount = v & kCountMask;
        // the keys are sorted, and so are the row's lower entries (CSR positions
        // rs .. dp - 1): the i-th key flagged as a neighbour is entry rs + i
        const bool nb = s < u && (v & kNbrFlag) != 0u;
        int nb_tot;
        const int nb_rank = nbr_before + team_prefix<TEAM>(nb, &nb_tot, wsm);
        nbr_before += nb_tot;
        double ratio = __shfl_sync(kFull, quot, (int)(1u + ((hcount - 1u) & 7u)));
        double d = __shfl_sync(kFull, quot, kQuotNbr + (nb_rank < 32 - kQuotNbr ? nb_rank : 0));
        const bool div_ratio = s < u && hcount > (uint32_t)kQuotSmall;
        const bool div_d = nb && nb_rank >= 32 - kQuotNbr;
        if (__any_sync(kFull, div_ratio || div_d)) {
            if (div_ratio) ratio = __ddiv_rn((double)hcount, Mk);
            if (div_d) d = __ddiv_rn(P.val[rs + nb_rank], akk);
        }
        if (hcount == 0u) ratio = 0.0;  // a neighbour no walk ended at
        if (s < u) {
            key = keys[s];
            // y = A_ki/A_kk + a * H'/M' (a non-neighbour's first term is +0 and
            // the product is non-zero, so the sum is the product itself)
            const double prod = __dmul_rn(a, ratio);
            y = nb ? __dadd_rn(d, prod) : prod;
            keep = fabs(y) >= P.drop_tol;
        }
        int tot;
        const int pos = team_prefix<TEAM>(keep, &tot, wsm);
        if (keep) {
            P.tcol[tb + kept + pos] = key;
            P.tval[tb + kept + pos] = y;
        }
        kept += tot;
    }
    jsum = team_sum<TEAM, unsigned long long>(jsum, sm64);
    const unsigned long long g_all = team_sum<TEAM, unsigned long long>(gsum, sm64);
    const unsigned long long c_all = team_sum<TEAM, unsigned long long>(csum, sm64);
    if (t == 0) {  // D_kk follows in k_walk_row_d, 32 rows per FP64 instruction
        const uint64_t Jk = (uint64_t)walks + jsum;
        P.M[k] = (uint32_t)walks;
        P.J[k] = Jk;
        P.G[k] = (uint32_t)g_all;
        P.ycnt[k] = kept;
        if (c_all) atomicAdd(&P.st->walk_cap, (unsigned)c_all);
    }
    team_sync<TEAM>();
}

constexpr int kMergeWarps = 8;

__global__ void __launch_bounds__(32 * kMergeWarps) k_merge_small(const MergeParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int HC = 1 << kLog2SmallHash;
    const int warp = threadIdx.x >> 5;
    int* keys = reinterpret_cast<int*>(smem) + warp * HC;
    uint32_t* vals = reinterpret_cast<uint32_t*>(smem + kMergeWarps * HC * sizeof(int)) + warp * HC;
    const int32_t gw = blockIdx.x * kMergeWarps + warp;
    const int32_t nwarps = gridDim.x * kMergeWarps;
    for (int32_t r = gw; r < P.nw; r += nwarps) {
        if (key_bound(P, r) > kSmallCap) {
            if (lane_id() == 0) P.big_rows[atomicAdd(P.n_big, 1)] = r;
            continue;
        }
        merge_row<32, kLog2SmallHash>(P, r, keys, vals, nullptr, nullptr);
    }
}

__global__ void __launch_bounds__(256) k_merge_big(const MergeParams P, int32_t nbig) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int HC = 1 << kLog2BigHash;
    int* keys = reinterpret_cast<int*>(smem);
    uint32_t* vals = reinterpret_cast<uint32_t*>(smem + HC * sizeof(int));
    __shared__ int wsm[8];
    __shared__ unsigned long long sm64;
    for (int32_t i = blockIdx.x; i < nbig; i += gridDim.x) {
        const int32_t r = P.big_rows[i];
        const int64_t b = key_bound(P, r);
        if (b > kBigCap) {
            if (threadIdx.x == 0) {
                P.huge_rows[atomicAdd(P.n_huge, 1)] = r;
                atomicMax(P.huge_bound, (unsigned long long)b);
            }
            continue;
        }
        merge_row<256, kLog2BigHash>(P, r, keys, vals, wsm, &sm64);
    }
}

// Huge rows: one block per row, the table in this block's part of a global
// area (2 * 2^lg_max words per block), sized per row by its key bound.
__global__ void __launch_bounds__(256) k_merge_huge(const MergeParams P, int32_t nhuge, int* area,
                                                    int64_t words_per_block) {
    __shared__ int wsm[8];
    __shared__ unsigned long long sm64;
    int* base = area + (size_t)blockIdx.x * (size_t)words_per_block;
    for (int32_t i = blockIdx.x; i < nhuge; i += gridDim.x) {
        const int32_t r = P.huge_rows[i];
        const int lg = huge_log2_slots(key_bound(P, r));
        int* keys = base;
        uint32_t* vals = reinterpret_cast<uint32_t*>(base + (size_t(1) << lg));
        merge_row<256, 0>(P, r, keys, vals, wsm, &sm64, lg);
    }
}

// D_kk of the walk rows (Eq. newz with Eq. d): D = A_kk / (1 + a (1 - J'/M')),
// a = S_k / A_kk, one thread per row after the merge has counted J'_k -- the
// same operations as inside the merge, but each FP64 instruction serves 32
// rows (GB300 issues one warp-wide FP64 instruction per 19 cycles per SM,
// whatever the lanes active).
__global__ void k_walk_row_d(int32_t nw, const int4* __restrict__ wrow, const int64_t* __restrict__ wbase,
                             const int64_t* __restrict__ xbase, const double* __restrict__ S,
                             const double* __restrict__ diag, const uint64_t* __restrict__ J, double* D) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x) {
        const int32_t k = wrow[r].x;
        const int64_t walks = wbase[r + 1] - wbase[r] + (xbase ? xbase[r + 1] - xbase[r] : 0);
        const double Mk = (double)walks;
        const double akk = diag[k];
        const double a = __ddiv_rn(S[k], akk);
        const double q = __ddiv_rn((double)J[k], Mk);
        D[k] = __ddiv_rn(akk, __dadd_rn(1.0, __dmul_rn(a, __dadd_rn(1.0, -q))));
    }
}

// Temporary slot capacity per walk row: walks + lower neighbours.
__global__ void k_slot_sizes(int32_t nw, const int4* __restrict__ wrow,
                             const int64_t* __restrict__ wbase, const int64_t* __restrict__ xbase, int64_t* cap) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nw; r += gridDim.x * blockDim.x)
        cap[r] = wbase[r + 1] - wbase[r] + (xbase ? xbase[r + 1] - xbase[r] : 0) + wrow[r].w;
}

// Exact rows (no upper neighbour, Sec. 5.2): count pass and fill pass.
__global__ void k_exact_rows(int32_t n, const uint32_t* __restrict__ wflag,
                             const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const int32_t* __restrict__ dpos,
                             double drop_tol, int64_t* ycnt, double* D, uint32_t* M, uint64_t* J,
                             uint32_t* G, const int64_t* y_rp, int32_t* y_col, double* y_val) {
    for (int32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        if (wflag[l + 1] != wflag[l]) continue;
        const int32_t s = rp[l], dp = dpos[l];
        const double dg = val[dp];
        if (!y_rp) {
            int64_t c = 0;
            for (int32_t p = s; p < dp; ++p) c += fabs(__ddiv_rn(val[p], dg)) >= drop_tol;
            ycnt[l] = c;
            D[l] = dg;
            M[l] = 0u;
            J[l] = 0u;
            G[l] = 0u;
        } else {
            int64_t o = y_rp[l];
            for (int32_t p = s; p < dp; ++p) {
                const double y = __ddiv_rn(val[p], dg);
                if (fabs(y) >= drop_tol) {
                    y_col[o] = col[p];
                    y_val[o] = y;
                    ++o;
                }
            }
        }
    }
}

// Copy each walk row's kept entries from its slot to the final CSR.
__global__ void k_copy_rows(int32_t nw, const int4* __restrict__ wrow,
                            const int64_t* __restrict__ tbase, const int32_t* __restrict__ tcol,
                            const double* __restrict__ tval, const int64_t* __restrict__ y_rp,
                            int32_t* y_col, double* y_val) {
    const int32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int32_t r = gw; r < nw; r += nwarps) {
        const int32_t k = wrow[r].x;
        const int64_t o = y_rp[k], c = y_rp[k + 1] - o, tb = tbase[r];
        for (int64_t i = lane_id(); i < c; i += 32) {
            y_col[o + i] = tcol[tb + i];
            y_val[o + i] = tval[tb + i];
        }
    }
}

rw_status emit_factor(rw_context* ctx, const rw_csr* A, const Tables& T, const WalkSpace& ws,
                      const int2* rec, const Extras* X, double drop_tol, FactorOut& fo, Pool& pool,
                      Pool& scratch, float* ms_merge, float* ms_emit) {
    NvtxRange nvtx_range("rw_merge_emit");
    cudaStream_t s = ctx->stream;
    const int32_t n = A->n, nw = T.n_walk_rows;
    rw_status rc;
    fo.y_rp = alloc_n<int64_t>(pool, n + 1);
    fo.d = alloc_n<double>(pool, n);
    fo.M = alloc_n<uint32_t>(pool, n);
    fo.J = alloc_n<uint64_t>(pool, n);
    fo.G = alloc_n<uint32_t>(pool, n);
    int64_t* tbase = alloc_n<int64_t>(scratch, nw + 1);
    int32_t* big_rows = alloc_n<int32_t>(scratch, nw);
    int32_t* huge_rows = alloc_n<int32_t>(scratch, nw);
    // n_big, n_huge, huge_bound (as 64-bit words)
    unsigned long long* counters = alloc_n<unsigned long long>(scratch, 3);
    if (!fo.y_rp || !fo.d || !fo.M || !fo.J || !fo.G || !tbase || !big_rows || !huge_rows || !counters)
        return RW_ERR_ALLOC;
    int32_t* n_big = reinterpret_cast<int32_t*>(counters);
    int32_t* n_huge = reinterpret_cast<int32_t*>(counters + 1);
    const int blocks = grid_for(std::max(n, nw), 256, ctx->num_sms * 8);
    if (nw > 0) {
        RW_COUNT_LAUNCH();
        k_slot_sizes<<<blocks, 256, 0, s>>>(nw, T.wrow, ws.wbase, X ? X->xbase : nullptr, tbase);
        if ((rc = check_launch("slot sizes"))) return rc;
    }
    if ((rc = check_cuda(scan_i64(tbase, tbase, nw, s, scratch), "scan"))) return rc;
    int64_t* h64 = static_cast<int64_t*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(h64, tbase + nw, 8, cudaMemcpyDeviceToHost, s), "copy")))
        return rc;
    if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
    const int64_t tslots = h64[0];
    int32_t* tcol = alloc_n<int32_t>(scratch, tslots);
    double* tval = alloc_n<double>(scratch, tslots);
    if (!tcol || !tval) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned long long), s), "memset")))
        return rc;

    MergeParams P;
    P.rp = A->row_ptr;
    P.col = A->col;
    P.val = A->val;
    P.dpos = T.diag_pos;
    P.wrow = T.wrow;
    P.wbase = ws.wbase;
    P.tbase = tbase;
    P.rec = rec;
    P.xbase = X ? X->xbase : nullptr;
    P.xrec = X ? X->xrec : nullptr;
    P.S = T.S;
    P.diag = T.diag;
    P.drop_tol = drop_tol;
    P.nw = nw;
    P.tcol = tcol;
    P.tval = tval;
    P.ycnt = fo.y_rp;
    P.D = fo.d;
    P.M = fo.M;
    P.J = fo.J;
    P.G = fo.G;
    P.big_rows = big_rows;
    P.n_big = n_big;
    P.huge_rows = huge_rows;
    P.n_huge = n_huge;
    P.huge_bound = counters + 2;
    P.st = ctx->d_status;

    if (ms_merge) cudaEventRecord(ctx->ev[2], s);
    if (nw > 0) {
        const size_t sm_small = (size_t)kMergeWarps * (1 << kLog2SmallHash) * 8;
        if ((rc = set_kernel_attr_once(ctx->device, (const void*)k_merge_small,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_small)))
            return rc;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_merge_small, 32 * kMergeWarps,
                                                      sm_small);
        if (per_sm < 1) per_sm = 1;
        const int mblocks = grid_for(nw, kMergeWarps, ctx->num_sms * per_sm);
        RW_COUNT_LAUNCH();
        k_merge_small<<<mblocks, 32 * kMergeWarps, sm_small, s>>>(P);
        if ((rc = check_launch("merge (warp tables)"))) return rc;
        int32_t* h32 = static_cast<int32_t*>(ctx->h_small);
        if ((rc = check_cuda(cudaMemcpyAsync(h32, n_big, 4, cudaMemcpyDeviceToHost, s), "copy")))
            return rc;
        if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
        const int32_t nbig = h32[0];
        if (nbig > 0) {
            const size_t sm_big = (size_t)(1 << kLog2BigHash) * 8;
            if ((rc = set_kernel_attr_once(ctx->device, (const void*)k_merge_big,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_big)))
                return rc;
            RW_COUNT_LAUNCH();
            k_merge_big<<<grid_for(nbig, 1, ctx->num_sms), 256, sm_big, s>>>(P, nbig);
            if ((rc = check_launch("merge (block tables)"))) return rc;
            unsigned long long* hc = static_cast<unsigned long long*>(ctx->h_small);
            if ((rc = check_cuda(cudaMemcpyAsync(hc, counters, 3 * sizeof(unsigned long long),
                                                 cudaMemcpyDeviceToHost, s),
                                 "copy")))
                return rc;
            if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
            const int32_t nhuge = (int32_t)(uint32_t)hc[1];
            if (nhuge > 0) {
                const int lg = huge_log2_slots((int64_t)hc[2]);
                if (lg > 30) {
                    set_error("merge: a row has %llu possible end points, above the 2^29 limit", hc[2]);
                    return RW_ERR_CAPACITY;
                }
                const int64_t words = int64_t(2) << lg;  // keys and values
                int64_t blocks_h = (int64_t)(kHugeTableBytes / (sizeof(int) * (size_t)words));
                blocks_h = std::max<int64_t>(1, std::min<int64_t>(blocks_h, std::min(nhuge, 2 * ctx->num_sms)));
                int* area = alloc_n<int>(scratch, blocks_h * words);
                if (!area) return RW_ERR_ALLOC;
                RW_COUNT_LAUNCH();
                k_merge_huge<<<(int)blocks_h, 256, 0, s>>>(P, nhuge, area, words);
                if ((rc = check_launch("merge (global tables)"))) return rc;
            }
        }
    }
    if (nw > 0) {
        RW_COUNT_LAUNCH();
        k_walk_row_d<<<blocks, 256, 0, s>>>(nw, T.wrow, ws.wbase, X ? X->xbase : nullptr, T.S, T.diag, fo.J, fo.d);
        if ((rc = check_launch("walk-row diagonal"))) return rc;
    }
    RW_COUNT_LAUNCH();
    k_exact_rows<<<blocks, 256, 0, s>>>(n, T.walk_flag, A->row_ptr, A->col, A->val, T.diag_pos,
                                        drop_tol, fo.y_rp, fo.d, fo.M, fo.J, fo.G, nullptr, nullptr,
                                        nullptr);
    if ((rc = check_launch("exact rows"))) return rc;
    if (ms_merge) cudaEventRecord(ctx->ev[3], s);
    if ((rc = check_cuda(scan_i64(fo.y_rp, fo.y_rp, n, s, scratch), "scan"))) return rc;
    if ((rc = check_cuda(cudaMemcpyAsync(h64, fo.y_rp + n, 8, cudaMemcpyDeviceToHost, s), "copy")))
        return rc;
    if ((rc = read_status(ctx, "merge"))) return rc;
    fo.nnz = h64[0];
    fo.y_col = alloc_n<int32_t>(pool, fo.nnz);
    fo.y_val = alloc_n<double>(pool, fo.nnz);
    if (!fo.y_col || !fo.y_val) return RW_ERR_ALLOC;
    if (nw > 0) {
        RW_COUNT_LAUNCH();
        k_copy_rows<<<grid_for((int64_t)nw * 32, 256, ctx->num_sms * 8), 256, 0, s>>>(
            nw, T.wrow, tbase, tcol, tval, fo.y_rp, fo.y_col, fo.y_val);
        if ((rc = check_launch("copy rows"))) return rc;
    }
    RW_COUNT_LAUNCH();
    k_exact_rows<<<blocks, 256, 0, s>>>(n, T.walk_flag, A->row_ptr, A->col, A->val, T.diag_pos,
                                        drop_tol, nullptr, nullptr, nullptr, nullptr, nullptr,
                                        fo.y_rp, fo.y_col, fo.y_val);
    if ((rc = check_launch("exact rows fill"))) return rc;
    if (ms_merge || ms_emit) {
        cudaEventRecord(ctx->ev[4], s);
        cudaEventSynchronize(ctx->ev[4]);
        if (ms_merge) cudaEventElapsedTime(ms_merge, ctx->ev[2], ctx->ev[3]);
        if (ms_emit) cudaEventElapsedTime(ms_emit, ctx->ev[3], ctx->ev[4]);
    }
    return RW_OK;
}

// ---------------------------------------------------------------------------
// Transpose: Y^T in CSR with each row's columns ascending.  The entries of Y
// are in row order, so a stable sort of (column, position) pairs by column
// gives Y^T with rows ascending inside every column: a least-significant-digit
// radix sort, 9 bits per pass, each pass = tile histograms, a prefix sum over
// (digit, tile), and a stable scatter ranked inside each tile.
// ---------------------------------------------------------------------------
constexpr int kRadixBits = 9;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;

__global__ void __launch_bounds__(kRadixThreads)
    k_radix_hist(const uint32_t* __restrict__ keys, int64_t cnt, int shift, int64_t ntiles,
                 uint32_t* hist) {
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += kRadixThreads) h[i] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
        if (i < cnt) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kRadixThreads)
        hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter of one tile: elements are ranked in index order (round-major,
// thread-minor), warp ranks from __match_any_sync, warp offsets from shared
// per-warp digit counts.
__global__ void __launch_bounds__(kRadixThreads)
    k_radix_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                    int64_t cnt, int shift, int64_t ntiles, const uint32_t* __restrict__ offs,
                    uint32_t* okeys, uint32_t* ovals) {
    constexpr int NW = kRadixThreads / 32;
    __shared__ uint32_t wcnt[NW][kRadix];
    __shared__ uint32_t run[kRadix];
    __shared__ uint32_t goff[kRadix];
    const int warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    for (int d = threadIdx.x; d < kRadix; d += kRadixThreads) {
        run[d] = 0u;
        goff[d] = offs[(int64_t)d * ntiles + blockIdx.x];
        for (int w = 0; w < NW; ++w) wcnt[w][d] = 0u;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixItems; ++r) {
        const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
        const bool valid = i < cnt;
        const uint32_t key = valid ? keys[i] : 0u;
        const uint32_t val = valid ? vals[i] : 0u;
        const uint32_t d = valid ? ((key >> shift) & (kRadix - 1)) : (uint32_t)kRadix;
        const unsigned peers = __match_any_sync(kFull, d);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t before = 0;
            for (int w = 0; w < warp; ++w) before += wcnt[w][d];
            const uint32_t pos = goff[d] + run[d] + before + rank;
            okeys[pos] = key;
            ovals[pos] = val;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < kRadix; dd += kRadixThreads) {
            uint32_t t = 0;
            for (int w = 0; w < NW; ++w) {
                t += wcnt[w][dd];
                wcnt[w][dd] = 0u;
            }
            run[dd] += t;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Transpose of the factor: every entry (k, c) of Y goes to row c of Y^T at a
// position taken with an atomic counter of that row (one warp per row of Y,
// reads coalesced, one 16-byte record {k, Y_kc} written per entry); then each
// row of Y^T is sorted by k while it is copied into the column and value
// arrays, so the result lists the rows of Y in ascending order -- the same
// arrays a stable sort by column gives.  Rows of at most 32 entries are sorted
// in the registers of one warp, rows of at most kSortWarp entries by one warp
// in its shared memory, rows of at most kSortSmem entries by one block in
// shared memory, longer rows by one block through a global scratch copy
// (bitonic networks throughout; the keys of a row are distinct).
// ---------------------------------------------------------------------------
constexpr int kSortWarp = 1024;
constexpr int kSortSmem = 4096;
constexpr int kSortWarpsPerBlock = 4;

struct TRec {
    int32_t k;
    int32_t pad;
    double v;
};

__global__ void k_transpose_place(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, unsigned long long* fill, TRec* tr) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    for (int64_t k = gw; k < n; k += nw) {
        const int64_t s = rp[k], e = rp[k + 1];
        for (int64_t p = s + lane; p < e; p += 32) {
            const unsigned long long q = atomicAdd(&fill[col[p]], 1ull);
            TRec r;
            r.k = (int32_t)k;
            r.pad = 0;
            r.v = val[p];
            tr[q] = r;
        }
    }
}

// Rows of at most 32 entries: a bitonic network across the lanes of a warp.
// Longer rows are listed for the shared-memory sorts (by size class).
__global__ void k_sort_rows_warp(int32_t n, const int64_t* __restrict__ trp, const TRec* __restrict__ tr,
                                 int32_t* tcol, double* tval, int32_t* lists, int32_t* counts) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    for (int64_t c = gw; c < n; c += nw) {
        const int64_t s = trp[c], L = trp[c + 1] - s;
        if (L == 0) continue;
        if (L > 32) {
            if (lane == 0) {
                const int cls = L <= kSortWarp ? 0 : L <= kSortSmem ? 1 : 2;
                lists[(int64_t)cls * n + atomicAdd(&counts[cls], 1)] = (int32_t)c;
            }
            continue;
        }
        int32_t key = INT32_MAX;
        double v = 0.0;
        if (lane < L) {
            const TRec r = tr[s + lane];
            key = r.k;
            v = r.v;
        }
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int32_t ok = __shfl_xor_sync(kFull, key, j);
                const double ov = __shfl_xor_sync(kFull, v, j);
                const bool asc = (lane & k) == 0;
                const bool low = (lane & j) == 0;
                // the lower lane of a pair keeps the smaller key in an ascending block
                const bool take = low == asc ? ok < key : ok > key;
                if (take) {
                    key = ok;
                    v = ov;
                }
            }
        }
        if (lane < L) {
            tcol[s + lane] = key;
            tval[s + lane] = v;
        }
    }
}

// Rows of at most 256 entries, one warp per row, keys in registers: entry e
// of the row becomes the 32-bit key (k << ibits) | e (k < 2^(32-ibits),
// e < 2^ibits), so sorting the keys alone orders the row by k, and the value
// of each sorted entry is read back by its index.  Element t * 32 + lane lives
// in register t of the lane: partners closer than 32 are exchanged by a
// shuffle, farther ones inside the lane (bitonic network, fully unrolled).
template <int EPL>
__device__ __forceinline__ void reg_bitonic(uint32_t (&v)[EPL], int lane) {
    constexpr int P = 32 * EPL;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int t = 0; t < EPL; ++t) {
                    const int t2 = t ^ (j >> 5);
                    if (t2 > t) {
                        const bool asc = ((t * 32 + lane) & k) == 0;
                        const uint32_t a = v[t], b = v[t2];
                        v[t] = asc ? min(a, b) : max(a, b);
                        v[t2] = asc ? max(a, b) : min(a, b);
                    }
                }
            } else {
#pragma unroll
                for (int t = 0; t < EPL; ++t) {
                    const uint32_t o = __shfl_xor_sync(kFull, v[t], j);
                    const bool asc = ((t * 32 + lane) & k) == 0;
                    const bool low = (lane & j) == 0;
                    v[t] = (low == asc) ? min(v[t], o) : max(v[t], o);
                }
            }
        }
    }
}

template <int EPL>
__device__ __forceinline__ void sort_row_reg(int64_t s, int64_t L, const TRec* __restrict__ tr, int32_t* tcol,
                                             double* tval, int ibits, int lane) {
    uint32_t v[EPL];
#pragma unroll
    for (int t = 0; t < EPL; ++t) {
        const int e = t * 32 + lane;
        v[t] = e < L ? (((uint32_t)tr[s + e].k << ibits) | (uint32_t)e) : 0xFFFFFFFFu;
    }
    reg_bitonic<EPL>(v, lane);
    const uint32_t imask = (1u << ibits) - 1u;
#pragma unroll
    for (int t = 0; t < EPL; ++t) {
        const int e = t * 32 + lane;
        if (e < L) {
            tcol[s + e] = (int32_t)(v[t] >> ibits);
            tval[s + e] = tr[s + (v[t] & imask)].v;
        }
    }
}

// Size classes of the Yt rows (packed-key path): 3..6 = at most 32, 64, 128,
// 256 entries (register sorts); 0..2 = the shared-memory and global sorts of
// k_sort_rows_warp.  One thread per row, one atomic per class and warp.
__global__ void __launch_bounds__(256) k_sort_classify(int32_t n, const int64_t* __restrict__ trp, int32_t* lists,
                                                       int32_t* counts) {
    const unsigned lt = lanemask_lt();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = b + threadIdx.x;
        int cls = -1;
        if (c < n) {
            const int64_t L = trp[c + 1] - trp[c];
            if (L > 0)
                cls = L <= 32 ? 3 : L <= 64 ? 4 : L <= 128 ? 5 : L <= 256 ? 6 : L <= kSortWarp ? 0 : L <= kSortSmem ? 1 : 2;
        }
        const unsigned same = __match_any_sync(kFull, cls);
        const int leader = __ffs(same) - 1;
        int base = 0;
        if (cls >= 0 && (int)lane_id() == leader) base = atomicAdd(&counts[cls], __popc(same));
        base = __shfl_sync(kFull, base, leader);
        if (cls >= 0) lists[(int64_t)cls * n + base + __popc(same & lt)] = (int32_t)c;
    }
}

// The rows of one class, one warp per row, sorted in registers.
template <int EPL>
__global__ void __launch_bounds__(256) k_sort_rows_reg(const int32_t* __restrict__ rows,
                                                       const int32_t* __restrict__ n_rows,
                                                       const int64_t* __restrict__ trp,
                                                       const TRec* __restrict__ tr, int32_t* tcol, double* tval,
                                                       int ibits) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    const int32_t nr = *n_rows;
    for (int64_t r = gw; r < nr; r += nw) {
        const int32_t c = rows[r];
        const int64_t s = trp[c], L = trp[c + 1] - s;
        sort_row_reg<EPL>(s, L, tr, tcol, tval, ibits, lane);
    }
}

struct WarpSync {
    __device__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
    __device__ void operator()() const { __syncthreads(); }
};

// Bitonic sort of P (a power of two) keys with payloads, in place, by
// `threads` cooperating threads of index t; sync() separates the stages.
template <typename Sync>
__device__ __forceinline__ void bitonic(int32_t* key, double* val, int64_t P, int t, int threads, Sync sync) {
    for (int64_t k = 2; k <= P; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t i = t; i < P / 2; i += threads) {
                const int64_t a = 2 * i - (i & (j - 1));  // the lower index of pair i (j a power of two)
                const int64_t b = a + j;
                const bool asc = (a & k) == 0;
                const int32_t ka = key[a], kb = key[b];
                if ((ka > kb) == asc) {
                    key[a] = kb;
                    key[b] = ka;
                    const double x = val[a];
                    val[a] = val[b];
                    val[b] = x;
                }
            }
            sync();
        }
    }
}

// Rows of 33 .. kSortWarp entries: one warp per row, in its shared memory.
__global__ void __launch_bounds__(32 * kSortWarpsPerBlock) k_sort_rows_wsmem(const int64_t* __restrict__ trp,
                                                                            const int32_t* __restrict__ rows,
                                                                            const int32_t* __restrict__ n_rows,
                                                                            const TRec* __restrict__ tr,
                                                                            int32_t* tcol, double* tval) {
    __shared__ int32_t skey[kSortWarpsPerBlock][kSortWarp];
    __shared__ double sval[kSortWarpsPerBlock][kSortWarp];
    const int warp = (int)(threadIdx.x >> 5), lane = (int)lane_id();
    int32_t* key = skey[warp];
    double* val = sval[warp];
    const int32_t nr = *n_rows;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = gw; r < nr; r += nw) {
        const int32_t c = rows[r];
        const int64_t s = trp[c], L = trp[c + 1] - s;
        int64_t P = 64;
        while (P < L) P <<= 1;
        for (int64_t i = lane; i < P; i += 32) {
            if (i < L) {
                const TRec x = tr[s + i];
                key[i] = x.k;
                val[i] = x.v;
            } else {
                key[i] = INT32_MAX;
                val[i] = 0.0;
            }
        }
        __syncwarp();
        bitonic(key, val, P, lane, 32, WarpSync{});
        for (int64_t i = lane; i < L; i += 32) {
            tcol[s + i] = key[i];
            tval[s + i] = val[i];
        }
        __syncwarp();
    }
}

// Rows of kSortWarp + 1 .. kSortSmem entries: one block per row, in shared memory.
__global__ void __launch_bounds__(512) k_sort_rows_smem(const int64_t* __restrict__ trp, const int32_t* __restrict__ rows,
                                                        const int32_t* __restrict__ n_rows,
                                                        const TRec* __restrict__ tr, int32_t* tcol, double* tval) {
    __shared__ int32_t skey[kSortSmem];
    __shared__ double sval[kSortSmem];
    const int32_t nr = *n_rows;
    for (int32_t r = blockIdx.x; r < nr; r += gridDim.x) {
        const int32_t c = rows[r];
        const int64_t s = trp[c], L = trp[c + 1] - s;
        int64_t P = 64;
        while (P < L) P <<= 1;
        for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
            if (i < L) {
                const TRec x = tr[s + i];
                skey[i] = x.k;
                sval[i] = x.v;
            } else {
                skey[i] = INT32_MAX;
                sval[i] = 0.0;
            }
        }
        __syncthreads();
        bitonic(skey, sval, P, (int)threadIdx.x, (int)blockDim.x, BlockSync{});
        for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
            tcol[s + i] = skey[i];
            tval[s + i] = sval[i];
        }
        __syncthreads();
    }
}

// Rows longer than kSortSmem: one block per row over a padded global copy
// (scratch of 2^ceil(log2 L) entries per row, placed at sbase[r]).
__global__ void __launch_bounds__(1024) k_sort_rows_global(const int64_t* __restrict__ trp,
                                                           const int32_t* __restrict__ rows,
                                                           const int64_t* __restrict__ sbase, int32_t nr,
                                                           const TRec* __restrict__ tr, int32_t* skey_all,
                                                           double* sval_all, int32_t* tcol, double* tval) {
    for (int32_t r = blockIdx.x; r < nr; r += gridDim.x) {
        const int32_t c = rows[r];
        const int64_t s = trp[c], L = trp[c + 1] - s;
        const int64_t P = sbase[r + 1] - sbase[r];
        int32_t* key = skey_all + sbase[r];
        double* val = sval_all + sbase[r];
        for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
            if (i < L) {
                const TRec x = tr[s + i];
                key[i] = x.k;
                val[i] = x.v;
            } else {
                key[i] = INT32_MAX;
                val[i] = 0.0;
            }
        }
        __syncthreads();
        bitonic(key, val, P, (int)threadIdx.x, (int)blockDim.x, BlockSync{});
        for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
            tcol[s + i] = key[i];
            tval[s + i] = val[i];
        }
        __syncthreads();
    }
}

__global__ void k_col_counts(int64_t nnz, const int32_t* __restrict__ col, uint32_t* cnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[p]], 1u);
}

__global__ void k_transpose_gather(int64_t nnz, const uint32_t* __restrict__ pos,
                                   const int32_t* __restrict__ row_of,
                                   const double* __restrict__ val, int32_t* tcol, double* tval) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = pos[q];
        tcol[q] = row_of[p];
        tval[q] = val[p];
    }
}

__global__ void k_transpose_pairs32(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    uint32_t* keys, uint32_t* vals, int32_t* row_of) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        for (int32_t p = rp[k]; p < rp[k + 1]; ++p) {
            keys[p] = (uint32_t)col[p];
            vals[p] = (uint32_t)p;
            row_of[p] = k;
        }
}

rw_status radix_sort_pairs(rw_context* ctx, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t cnt,
                           int bits, Pool& scratch, uint32_t** ko, uint32_t** vo) {
    cudaStream_t s = ctx->stream;
    rw_status rc;
    const int64_t ntiles = (cnt + kRadixTile - 1) / kRadixTile;
    uint32_t* hist = alloc_n<uint32_t>(scratch, ntiles * kRadix + 1);
    if (!hist) return RW_ERR_ALLOC;
    for (int shift = 0; shift < bits && cnt > 0; shift += kRadixBits) {
        RW_COUNT_LAUNCH();
        k_radix_hist<<<(unsigned)ntiles, kRadixThreads, 0, s>>>(k0, cnt, shift, ntiles, hist);
        if ((rc = check_launch("radix histogram"))) return rc;
        if ((rc = check_cuda(scan_u32(hist, hist, ntiles * kRadix, s, scratch), "scan"))) return rc;
        RW_COUNT_LAUNCH();
        k_radix_scatter<<<(unsigned)ntiles, kRadixThreads, 0, s>>>(k0, v0, cnt, shift, ntiles, hist, k1, v1);
        if ((rc = check_launch("radix scatter"))) return rc;
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    *ko = k0;
    *vo = v0;
    return RW_OK;
}

rw_status transpose_factor(rw_context* ctx, int32_t n, const FactorOut& fo, int64_t* yt_rp,
                           int32_t* yt_col, double* yt_val, Pool& scratch) {
    NvtxRange nvtx_range("rw_transpose");
    cudaStream_t s = ctx->stream;
    const int64_t nnz = fo.nnz;
    rw_status rc;
    uint32_t* cnt = alloc_n<uint32_t>(scratch, n + 1);
    if (!cnt) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(n + 1), s), "memset")))
        return rc;
    if (nnz > 0) {
        RW_COUNT_LAUNCH();
        k_col_counts<<<grid_for(nnz, 256, ctx->num_sms * 8), 256, 0, s>>>(nnz, fo.y_col, cnt);
        if ((rc = check_launch("transpose counts"))) return rc;
    }
    if ((rc = check_cuda(scan_u32_to_i64(cnt, yt_rp, n, s, scratch), "scan"))) return rc;
    if (nnz == 0) return RW_OK;
    unsigned long long* fill = alloc_n<unsigned long long>(scratch, n);
    TRec* tr = alloc_n<TRec>(scratch, nnz);
    int32_t* lists = alloc_n<int32_t>(scratch, 7 * (int64_t)n);
    int32_t* counts = alloc_n<int32_t>(scratch, 7);
    if (!fill || !tr || !lists || !counts) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemcpyAsync(fill, yt_rp, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemsetAsync(counts, 0, 7 * sizeof(int32_t), s), "memset")))
        return rc;
    const int wblocks = grid_for((int64_t)n * 32, 256, ctx->num_sms * 16);
    RW_COUNT_LAUNCH();
    k_transpose_place<<<wblocks, 256, 0, s>>>(n, fo.y_rp, fo.y_col, fo.y_val, fill, tr);
    // packed 32-bit keys (k, entry) when k fits beside 8 or more index bits
    int kbits = 1;
    while (kbits < 32 && (1ll << kbits) < (int64_t)n) ++kbits;
    if (kbits <= 24) {
        // rows by size class, then one register sort per class (one unrolled
        // network per kernel)
        RW_COUNT_LAUNCH();
        k_sort_classify<<<grid_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(n, yt_rp, lists, counts);
        const int rb = ctx->num_sms * 16;
        RW_COUNT_LAUNCH();
        k_sort_rows_reg<1><<<rb, 256, 0, s>>>(lists + 3 * (int64_t)n, counts + 3, yt_rp, tr, yt_col, yt_val, 32 - kbits);
        RW_COUNT_LAUNCH();
        k_sort_rows_reg<2><<<rb, 256, 0, s>>>(lists + 4 * (int64_t)n, counts + 4, yt_rp, tr, yt_col, yt_val, 32 - kbits);
        RW_COUNT_LAUNCH();
        k_sort_rows_reg<4><<<rb, 256, 0, s>>>(lists + 5 * (int64_t)n, counts + 5, yt_rp, tr, yt_col, yt_val, 32 - kbits);
        RW_COUNT_LAUNCH();
        k_sort_rows_reg<8><<<rb, 256, 0, s>>>(lists + 6 * (int64_t)n, counts + 6, yt_rp, tr, yt_col, yt_val, 32 - kbits);
    } else {
        RW_COUNT_LAUNCH();
        k_sort_rows_warp<<<wblocks, 256, 0, s>>>(n, yt_rp, tr, yt_col, yt_val, lists, counts);
    }
    RW_COUNT_LAUNCH();
    k_sort_rows_wsmem<<<ctx->num_sms * 4, 32 * kSortWarpsPerBlock, 0, s>>>(yt_rp, lists, counts, tr, yt_col,
                                                                            yt_val);
    RW_COUNT_LAUNCH();
    k_sort_rows_smem<<<ctx->num_sms * 2, 512, 0, s>>>(yt_rp, lists + n, counts + 1, tr, yt_col, yt_val);
    if ((rc = check_launch("transpose"))) return rc;
    // rows longer than the shared-memory sorts (none on most factors)
    int32_t* h = static_cast<int32_t*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(h, counts + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "copy")) ||
        (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
        return rc;
    const int32_t nbig = h[0];
    if (nbig > 0) {
        std::vector<int32_t> rows(nbig);
        std::vector<int64_t> trp((size_t)n + 1);
        if ((rc = check_cuda(cudaMemcpy(rows.data(), lists + 2 * (int64_t)n, sizeof(int32_t) * nbig,
                                        cudaMemcpyDeviceToHost),
                             "copy")) ||
            (rc = check_cuda(cudaMemcpy(trp.data(), yt_rp, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost),
                             "copy")))
            return rc;
        std::sort(rows.begin(), rows.end());
        std::vector<int64_t> sbase(nbig + 1, 0);
        for (int32_t r = 0; r < nbig; ++r) {
            int64_t P = 1;
            while (P < trp[rows[r] + 1] - trp[rows[r]]) P <<= 1;
            sbase[r + 1] = sbase[r] + P;
        }
        int32_t* d_rows = alloc_n<int32_t>(scratch, nbig);
        int64_t* d_sbase = alloc_n<int64_t>(scratch, nbig + 1);
        int32_t* skey = alloc_n<int32_t>(scratch, sbase[nbig]);
        double* sval = alloc_n<double>(scratch, sbase[nbig]);
        if (!d_rows || !d_sbase || !skey || !sval) return RW_ERR_ALLOC;
        if ((rc = check_cuda(cudaMemcpyAsync(d_rows, rows.data(), sizeof(int32_t) * nbig, cudaMemcpyHostToDevice, s),
                             "copy")) ||
            (rc = check_cuda(cudaMemcpyAsync(d_sbase, sbase.data(), sizeof(int64_t) * (nbig + 1),
                                             cudaMemcpyHostToDevice, s),
                             "copy")))
            return rc;
        RW_COUNT_LAUNCH();
        k_sort_rows_global<<<std::min(nbig, ctx->num_sms * 2), 1024, 0, s>>>(yt_rp, d_rows, d_sbase, nbig, tr, skey,
                                                                            sval, yt_col, yt_val);
        if ((rc = check_launch("transpose long rows"))) return rc;
        // the host copies of rows and sbase are read by the launch: keep them until it is done
        if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
    }
    return RW_OK;
}

// A^T of a CSR matrix (int32 row pointers): entries sorted by column with a
// stable radix sort, so each row of the result lists its columns (the rows of
// A) in ascending order.
rw_status csr_transpose(rw_context* ctx, const rw_csr* A, int32_t* rp, int32_t* col, double* val, Pool& scratch) {
    cudaStream_t s = ctx->stream;
    const int32_t n = A->n;
    const int64_t nnz = A->nnz;
    rw_status rc;
    uint32_t* cnt = alloc_n<uint32_t>(scratch, n + 1);
    if (!cnt) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(n + 1), s), "memset"))) return rc;
    if (nnz > 0) {
        RW_COUNT_LAUNCH();
        k_col_counts<<<grid_for(nnz, 256, ctx->num_sms * 8), 256, 0, s>>>(nnz, A->col, cnt);
        if ((rc = check_launch("transpose counts"))) return rc;
    }
    // nnz < 2^31, so the prefix sums fit the int32 row pointers
    if ((rc = check_cuda(scan_u32(cnt, reinterpret_cast<uint32_t*>(rp), n, s, scratch), "scan"))) return rc;
    if (nnz == 0) return RW_OK;
    uint32_t* k0 = alloc_n<uint32_t>(scratch, nnz);
    uint32_t* v0 = alloc_n<uint32_t>(scratch, nnz);
    uint32_t* k1 = alloc_n<uint32_t>(scratch, nnz);
    uint32_t* v1 = alloc_n<uint32_t>(scratch, nnz);
    int32_t* row_of = alloc_n<int32_t>(scratch, nnz);
    if (!k0 || !v0 || !k1 || !v1 || !row_of) return RW_ERR_ALLOC;
    RW_COUNT_LAUNCH();
    k_transpose_pairs32<<<grid_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(n, A->row_ptr, A->col, k0, v0, row_of);
    if ((rc = check_launch("transpose pairs"))) return rc;
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;
    if ((rc = radix_sort_pairs(ctx, k0, v0, k1, v1, nnz, bits, scratch, &k0, &v0))) return rc;
    RW_COUNT_LAUNCH();
    k_transpose_gather<<<grid_for(nnz, 256, ctx->num_sms * 8), 256, 0, s>>>(nnz, v0, row_of, A->val, col, val);
    return check_launch("transpose gather");
}

}  // namespace rw
