// rw_io.cu -- factor files, SHA-256, seeded random orderings.
//
// A factor file holds the rows of a built factor (Y in CSR, D, and the
// journey-record counters M', J', G' of Sec. 3.1) with a header and the
// SHA-256 of the payload; loading rebuilds the transpose, levels and solve
// schedules with the same code as a fresh build.  The random symmetric
// ordering (the paper's choice, Sec. 5.4) is drawn from Philox-4x32-10 with
// the generator tag 2 and applied to a matrix as B = P A P^T.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "rw_internal.h"

namespace rw {

// ---------------------------------------------------------------------------
// SHA-256 (FIPS 180-4).  The initial hash words and round constants are, by
// definition, the first 32 bits of the fractional parts of the square roots
// of the first 8 primes and of the cube roots of the first 64 primes; they are
// computed here exactly with integer roots: floor(root(p) * 2^32) is the
// largest x with x^2 <= p 2^64 (or x^3 <= p 2^96), and its low 32 bits are the
// fraction's first 32 bits.
// ---------------------------------------------------------------------------
namespace {

typedef unsigned __int128 u128;

uint64_t iroot(u128 v, int deg) {
    uint64_t lo = 0, hi = (uint64_t)1 << (deg == 2 ? 40 : 36);
    while (lo < hi) {  // largest x with x^deg <= v
        const uint64_t mid = lo + (hi - lo + 1) / 2;
        u128 m = mid;
        u128 pw = deg == 2 ? m * m : m * m * m;
        if (pw <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct ShaConst {
    uint32_t H0[8], K[64];
    ShaConst() {
        int primes[64], np = 0;
        for (int c = 2; np < 64; ++c) {
            bool pr = true;
            for (int d = 2; d * d <= c; ++d)
                if (c % d == 0) {
                    pr = false;
                    break;
                }
            if (pr) primes[np++] = c;
        }
        for (int i = 0; i < 8; ++i) H0[i] = (uint32_t)iroot((u128)primes[i] << 64, 2);
        for (int i = 0; i < 64; ++i) K[i] = (uint32_t)iroot((u128)primes[i] << 96, 3);
    }
};
const ShaConst& sha_const() {
    static const ShaConst c;
    return c;
}

inline uint32_t rotr(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

struct Sha256 {
    uint32_t h[8];
    uint8_t buf[64];
    size_t nbuf = 0;
    uint64_t total = 0;
    Sha256() { memcpy(h, sha_const().H0, sizeof h); }
    void block(const uint8_t* p) {
        const uint32_t* K = sha_const().K;
        uint32_t w[64];
        for (int t = 0; t < 16; ++t)
            w[t] = ((uint32_t)p[4 * t] << 24) | ((uint32_t)p[4 * t + 1] << 16) | ((uint32_t)p[4 * t + 2] << 8) |
                   (uint32_t)p[4 * t + 3];
        for (int t = 16; t < 64; ++t) {
            const uint32_t s0 = rotr(w[t - 15], 7) ^ rotr(w[t - 15], 18) ^ (w[t - 15] >> 3);
            const uint32_t s1 = rotr(w[t - 2], 17) ^ rotr(w[t - 2], 19) ^ (w[t - 2] >> 10);
            w[t] = s1 + w[t - 7] + s0 + w[t - 16];
        }
        uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
        for (int t = 0; t < 64; ++t) {
            const uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
            const uint32_t ch = (e & f) ^ (~e & g);
            const uint32_t t1 = hh + S1 + ch + K[t] + w[t];
            const uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
            const uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
            const uint32_t t2 = S0 + mj;
            hh = g;
            g = f;
            f = e;
            e = d + t1;
            d = c;
            c = b;
            b = a;
            a = t1 + t2;
        }
        h[0] += a;
        h[1] += b;
        h[2] += c;
        h[3] += d;
        h[4] += e;
        h[5] += f;
        h[6] += g;
        h[7] += hh;
    }
    void update(const void* data, size_t len) {
        const uint8_t* p = static_cast<const uint8_t*>(data);
        total += len;
        while (len > 0) {
            if (nbuf == 0 && len >= 64) {
                block(p);
                p += 64;
                len -= 64;
                continue;
            }
            const size_t take = std::min(len, 64 - nbuf);
            memcpy(buf + nbuf, p, take);
            nbuf += take;
            p += take;
            len -= take;
            if (nbuf == 64) {
                block(buf);
                nbuf = 0;
            }
        }
    }
    void final(uint8_t out[32]) {
        const uint64_t bits = total * 8;
        const uint8_t one = 0x80, zero = 0;
        update(&one, 1);
        while (nbuf != 56) update(&zero, 1);
        uint8_t lenb[8];
        for (int i = 0; i < 8; ++i) lenb[i] = (uint8_t)(bits >> (56 - 8 * i));
        update(lenb, 8);
        for (int i = 0; i < 8; ++i) {
            out[4 * i] = (uint8_t)(h[i] >> 24);
            out[4 * i + 1] = (uint8_t)(h[i] >> 16);
            out[4 * i + 2] = (uint8_t)(h[i] >> 8);
            out[4 * i + 3] = (uint8_t)h[i];
        }
    }
};

// ---------------------------------------------------------------------------
// Factor file
// ---------------------------------------------------------------------------
constexpr char kMagic[8] = {'R', 'W', 'P', 'C', 'F', 'A', 'C', '1'};

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int32_t n;
    int32_t n_walk_rows;
    int64_t nnz;
    int64_t total_walks;
    uint64_t total_hops;
    int32_t fwd_levels, bwd_levels;
};
static_assert(sizeof(FileHeader) == 56, "header layout");

struct Section {
    const void* dev;
    size_t bytes;
};

std::vector<Section> sections(const rw_factor_desc& d) {
    const size_t n = (size_t)d.n, nnz = (size_t)d.nnz;
    return {{d.y_row_ptr, 8 * (n + 1)}, {d.y_col, 4 * nnz}, {d.y_val, 8 * nnz}, {d.d, 8 * n},
            {d.walks, 4 * n},           {d.visits, 8 * n},  {d.ground, 4 * n}};
}

// ---------------------------------------------------------------------------
// Orderings
// ---------------------------------------------------------------------------
__global__ void k_perm_keys(int64_t n, uint32_t key0, uint32_t key1, uint32_t* keys, uint32_t* vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = philox4x32_10((uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, 2u, key0, key1).v0;
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_perm_invert(int64_t n, const uint32_t* __restrict__ order, int32_t* perm) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        perm[order[j]] = (int32_t)j;
}

__global__ void k_perm_lengths(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ perm,
                               uint32_t* len, int32_t* bad) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t t = perm[i];
        if (t < 0 || t >= n) {
            atomicExch(bad, 1);
            continue;
        }
        len[t] = (uint32_t)(rp[i + 1] - rp[i]);
    }
}

// Row i of A becomes row perm[i] of B with columns perm[c], sorted (insertion
// sort inside the row).
__global__ void k_perm_rows(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ brp, int32_t* bcol, double* bval) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t s = rp[i], e = rp[i + 1], o = brp[perm[i]];
        for (int32_t p = s; p < e; ++p) {
            const int32_t c = perm[col[p]];
            const double v = val[p];
            int32_t q = o + (p - s);
            while (q > o && bcol[q - 1] > c) {
                bcol[q] = bcol[q - 1];
                bval[q] = bval[q - 1];
                --q;
            }
            bcol[q] = c;
            bval[q] = v;
        }
    }
}

__global__ void k_perm_check(int64_t n, const int32_t* __restrict__ perm, uint32_t* seen, int32_t* bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = perm[i];
        if (t < 0 || t >= n || atomicAdd(&seen[t], 1u) != 0u) atomicExch(bad, 1);
    }
}

}  // namespace
}  // namespace rw

using namespace rw;

extern "C" {

void rw_sha256(const void* data, size_t len, uint8_t out[32]) {
    Sha256 h;
    h.update(data, len);
    h.final(out);
}

rw_status rw_factor_save(const rw_factor* F, const char* path) {
    if (!F || !path) {
        set_error("rw_factor_save: bad arguments");
        return RW_ERR_ARG;
    }
    const rw_factor_desc& d = F->desc;
    FileHeader hd{};
    memcpy(hd.magic, kMagic, 8);
    hd.version = 1;
    hd.header_bytes = sizeof(FileHeader);
    hd.n = d.n;
    hd.n_walk_rows = d.n_walk_rows;
    hd.nnz = d.nnz;
    hd.total_walks = d.total_walks;
    hd.total_hops = d.total_hops;
    hd.fwd_levels = d.fwd_levels;
    hd.bwd_levels = d.bwd_levels;
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error("rw_factor_save: cannot open %s", path);
        return RW_ERR_ARG;
    }
    Sha256 sha;
    bool ok = fwrite(&hd, sizeof hd, 1, f) == 1;
    std::vector<uint8_t> host;
    for (const Section& sec : sections(d)) {
        if (!ok) break;
        host.resize(sec.bytes);
        if (sec.bytes > 0) {
            rw_status rc = check_cuda(cudaMemcpy(host.data(), sec.dev, sec.bytes, cudaMemcpyDeviceToHost), "copy");
            if (rc) {
                fclose(f);
                return rc;
            }
        }
        sha.update(host.data(), sec.bytes);
        ok = sec.bytes == 0 || fwrite(host.data(), 1, sec.bytes, f) == sec.bytes;
    }
    uint8_t dig[32];
    sha.final(dig);
    ok = ok && fwrite(dig, 1, 32, f) == 32;
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("rw_factor_save: write to %s failed", path);
        return RW_ERR_ARG;
    }
    return RW_OK;
}

rw_status rw_factor_load(rw_context* ctx, const char* path, rw_factor** out) {
    if (!ctx || !path || !out) {
        set_error("rw_factor_load: bad arguments");
        return RW_ERR_ARG;
    }
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error("rw_factor_load: cannot open %s", path);
        return RW_ERR_ARG;
    }
    FileHeader hd{};
    if (fread(&hd, sizeof hd, 1, f) != 1 || memcmp(hd.magic, kMagic, 8) != 0 || hd.version != 1 ||
        hd.header_bytes != sizeof(FileHeader) || hd.n < 0 || hd.nnz < 0 || hd.nnz >= ((int64_t)1 << 32)) {
        fclose(f);
        set_error("rw_factor_load: %s is not a factor file of this version", path);
        return RW_ERR_ARG;
    }
    rw_factor* F = new (std::nothrow) rw_factor(ctx);
    if (!F) {
        fclose(f);
        return RW_ERR_ALLOC;
    }
    auto fail = [&](rw_status rc) {
        fclose(f);
        delete F;
        return rc;
    };
    const int32_t n = hd.n;
    FactorOut fo;
    fo.nnz = hd.nnz;
    fo.y_rp = alloc_n<int64_t>(F->pool, (int64_t)n + 1);
    fo.y_col = alloc_n<int32_t>(F->pool, hd.nnz);
    fo.y_val = alloc_n<double>(F->pool, hd.nnz);
    fo.d = alloc_n<double>(F->pool, n);
    fo.M = alloc_n<uint32_t>(F->pool, n);
    fo.J = alloc_n<uint64_t>(F->pool, n);
    fo.G = alloc_n<uint32_t>(F->pool, n);
    if (!fo.y_rp || !fo.y_col || !fo.y_val || !fo.d || !fo.M || !fo.J || !fo.G) return fail(RW_ERR_ALLOC);
    const std::vector<Section> secs = {{fo.y_rp, 8 * ((size_t)n + 1)}, {fo.y_col, 4 * (size_t)hd.nnz},
                                       {fo.y_val, 8 * (size_t)hd.nnz}, {fo.d, 8 * (size_t)n},
                                       {fo.M, 4 * (size_t)n},          {fo.J, 8 * (size_t)n},
                                       {fo.G, 4 * (size_t)n}};
    Sha256 sha;
    std::vector<std::vector<uint8_t>> host(secs.size());
    for (size_t i = 0; i < secs.size(); ++i) {
        host[i].resize(secs[i].bytes);
        if (secs[i].bytes && fread(host[i].data(), 1, secs[i].bytes, f) != secs[i].bytes) {
            set_error("rw_factor_load: %s is truncated", path);
            return fail(RW_ERR_ARG);
        }
        sha.update(host[i].data(), secs[i].bytes);
    }
    uint8_t want[32], got[32];
    if (fread(want, 1, 32, f) != 32) {
        set_error("rw_factor_load: %s is truncated", path);
        return fail(RW_ERR_ARG);
    }
    sha.final(got);
    if (memcmp(want, got, 32) != 0) {
        set_error("rw_factor_load: %s fails its SHA-256 check", path);
        return fail(RW_ERR_ARG);
    }
    // the row pointers must describe the entries before any kernel reads them
    const int64_t* rp = reinterpret_cast<const int64_t*>(host[0].data());
    bool sane = rp[0] == 0 && rp[n] == hd.nnz;
    for (int32_t i = 0; sane && i < n; ++i) sane = rp[i + 1] >= rp[i];
    const int32_t* cl = reinterpret_cast<const int32_t*>(host[1].data());
    for (int32_t i = 0; sane && i < n; ++i)
        for (int64_t p = rp[i]; sane && p < rp[i + 1]; ++p) sane = cl[p] >= 0 && cl[p] < i;
    if (!sane) {
        set_error("rw_factor_load: %s holds an inconsistent factor", path);
        return fail(RW_ERR_ARG);
    }
    fclose(f);
    cudaStream_t s = ctx->stream;
    rw_status rc;
    for (size_t i = 0; i < secs.size(); ++i)
        if (secs[i].bytes &&
            (rc = check_cuda(cudaMemcpyAsync(const_cast<void*>(secs[i].dev), host[i].data(), secs[i].bytes,
                                             cudaMemcpyHostToDevice, s),
                             "copy"))) {
            delete F;
            return rc;
        }
    if ((rc = reset_status(ctx))) {
        delete F;
        return rc;
    }
    F->desc.n = n;
    Pool scratch(ctx);
    if ((rc = complete_factor(ctx, F, fo, scratch)) || (rc = read_status(ctx, "factor load"))) {
        scratch.release_all();
        delete F;
        return rc;
    }
    F->desc.n_walk_rows = hd.n_walk_rows;
    F->desc.total_walks = hd.total_walks;
    F->desc.total_hops = hd.total_hops;
    *out = F;
    return RW_OK;
}

rw_status rw_random_permutation(rw_context* ctx, int32_t n, uint64_t seed, int32_t* d_perm) {
    if (!ctx || n < 0 || (n > 0 && !d_perm)) {
        set_error("rw_random_permutation: bad arguments");
        return RW_ERR_ARG;
    }
    if (n == 0) return RW_OK;
    cudaStream_t s = ctx->stream;
    Pool sc(ctx);
    uint32_t* k0 = alloc_n<uint32_t>(sc, n);
    uint32_t* v0 = alloc_n<uint32_t>(sc, n);
    uint32_t* k1 = alloc_n<uint32_t>(sc, n);
    uint32_t* v1 = alloc_n<uint32_t>(sc, n);
    if (!k0 || !v0 || !k1 || !v1) return RW_ERR_ALLOC;
    RW_COUNT_LAUNCH();
    k_perm_keys<<<grid_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(n, (uint32_t)seed, (uint32_t)(seed >> 32), k0, v0);
    rw_status rc = check_launch("permutation keys");
    if (rc) return rc;
    uint32_t *ko = nullptr, *vo = nullptr;
    if ((rc = radix_sort_pairs(ctx, k0, v0, k1, v1, n, 32, sc, &ko, &vo))) return rc;
    RW_COUNT_LAUNCH();
    k_perm_invert<<<grid_for(n, 256, ctx->num_sms * 8), 256, 0, s>>>(n, vo, d_perm);
    if ((rc = check_launch("permutation"))) return rc;
    return check_cuda(cudaStreamSynchronize(s), "sync");
}

rw_status rw_permute_csr(rw_context* ctx, const rw_csr* A, const int32_t* d_perm, int32_t* d_row_ptr, int32_t* d_col,
                         double* d_val) {
    if (!ctx || !d_perm || !d_row_ptr || !d_col || !d_val) {
        set_error("rw_permute_csr: bad arguments");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr(A);
    if (rc) return rc;
    const int32_t n = A->n;
    cudaStream_t s = ctx->stream;
    Pool sc(ctx);
    uint32_t* len = alloc_n<uint32_t>(sc, (int64_t)n + 1);
    uint32_t* seen = alloc_n<uint32_t>(sc, n);
    int32_t* bad = alloc_n<int32_t>(sc, 1);
    if (!len || !seen || !bad) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(seen, 0, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1), s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(bad, 0, sizeof(int32_t), s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(len, 0, sizeof(uint32_t) * ((size_t)n + 1), s), "memset")))
        return rc;
    const int g = grid_for(n, 256, ctx->num_sms * 8);
    if (n > 0) {
        RW_COUNT_LAUNCH();
        k_perm_check<<<g, 256, 0, s>>>(n, d_perm, seen, bad);
        RW_COUNT_LAUNCH();
        k_perm_lengths<<<g, 256, 0, s>>>(n, A->row_ptr, d_perm, len, bad);
        if ((rc = check_launch("permutation check"))) return rc;
    }
    int32_t* hb = static_cast<int32_t*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(hb, bad, 4, cudaMemcpyDeviceToHost, s), "copy")) ||
        (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
        return rc;
    if (hb[0]) {
        set_error("rw_permute_csr: d_perm is not a permutation of 0..n-1");
        return RW_ERR_ARG;
    }
    // row pointers of B (uint32 scan; nnz < 2^31 by check_csr)
    if ((rc = check_cuda(scan_u32(len, len, n, s, sc), "scan"))) return rc;
    if ((rc = check_cuda(cudaMemcpyAsync(d_row_ptr, len, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s),
                         "copy")))
        return rc;
    if (n > 0) {
        RW_COUNT_LAUNCH();
        k_perm_rows<<<g, 256, 0, s>>>(n, A->row_ptr, A->col, A->val, d_perm, d_row_ptr, d_col, d_val);
        if ((rc = check_launch("permute rows"))) return rc;
    }
    return check_cuda(cudaStreamSynchronize(s), "sync");
}

}  // extern "C"
