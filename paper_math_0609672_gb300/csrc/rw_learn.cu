// rw_learn.cu -- learned walk budget: per-row graph features, pilot-walk
// statistics, a 12 -> 64 -> 64 -> 1 MLP (BF16 weights, FP32 accumulation on
// the tensor cores) with hand-written training, and the budget normaliser.
//
// The label follows the accuracy criterion of Sec. 5.1 (Eq. lengthdelta):
// walks from row k are enough once the relative confidence interval of the
// mean walk length is below Delta at confidence alpha, which needs
//     M*_k = (z_alpha sigma_k / (Delta Xi'_k))^2
// walks.  The network predicts log((sigma_k / Xi'_k)^2); the constant
// (z_alpha / Delta)^2 is set by normalising the budgets to a requested mean,
// and the lower bound on M_k (Sec. 5.1) is the normaliser's minimum.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "rw_internal.h"

namespace rw {

// ---------------------------------------------------------------------------
// Row features: one thread per row, FP64 arithmetic, FP32 output [n][16]
// (entries 12..15 zero).
//  0 log(1 + degree)              1 upper neighbours / degree
//  2 lower neighbours / degree    3 excess / A_kk
//  4 -S_k / A_kk                  5 entropy of the transition probabilities
//  6 largest weight / weight sum  7 k / (n - 1)
//  8 mean over neighbours c of (row sum of c) / A_cc
//  9 log(1 + mean neighbour degree)
// 10 log(1 + sum over upper neighbours c of #{entries of row c with column > k})
// 11 log A_kk
// ---------------------------------------------------------------------------
// Per node c: its off-diagonal count and (A_cc + sum_j A_cj) / A_cc, the sum
// taken in column order (what feature 8 averages over a row's neighbours).
__global__ void k_node_info(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ val, int32_t* ndeg, double* exr) {
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double cd = 0.0, csum = 0.0;
        for (int32_t q = rp[c]; q < rp[c + 1]; ++q) {
            if (col[q] == c) cd = val[q];
            else csum += val[q];
        }
        ndeg[c] = rp[c + 1] - rp[c] - 1;
        exr[c] = (cd + csum) / cd;
    }
}

// One thread per row k (FP64).  Feature 8 averages the neighbours' excess
// ratios and feature 9 their degrees (per-node arrays from k_node_info);
// feature 10 counts, over the upper neighbours c, the off-diagonal entries of
// row c with column > k: a binary search of row c's ascending columns.
__global__ void k_features(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const int32_t* __restrict__ ndeg_of,
                           const double* __restrict__ exr, float* __restrict__ feat) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int32_t s = rp[k], e = rp[k + 1];
        double diag = 0.0, wsum = 0.0, wup = 0.0, wmax = 0.0;
        int up = 0, lo = 0;
        for (int32_t p = s; p < e; ++p) {
            const int32_t c = col[p];
            if (c == k) {
                diag = val[p];
                continue;
            }
            const double w = -val[p];
            wsum += w;
            wmax = fmax(wmax, w);
            if (c > k) {
                ++up;
                wup += w;
            } else {
                ++lo;
            }
        }
        const int deg = up + lo;
        double ent = 0.0, nex = 0.0, ndeg = 0.0;
        int64_t up2 = 0;
        const double inv = 1.0 / wsum;  // one division per row (FP64 division is long on GB300)
        for (int32_t p = s; p < e; ++p) {
            const int32_t c = col[p];
            if (c == k) continue;
            const double pr = -val[p] * inv;
            if (pr > 0.0) ent -= pr * log(pr);
            nex += exr[c];
            ndeg += (double)ndeg_of[c];
            if (c > k) {
                // first position of row c with column > k (the diagonal c > k is among them)
                int32_t a = rp[c], b = rp[c + 1];
                const int32_t ce = b;
                while (a < b) {
                    const int32_t m = (a + b) >> 1;
                    if (col[m] > k) b = m;
                    else a = m + 1;
                }
                up2 += ce - a - 1;
            }
        }
        float* f = feat + (size_t)k * kFeatStride;
        f[0] = (float)log1p((double)deg);
        f[1] = deg ? (float)((double)up / deg) : 0.f;
        f[2] = deg ? (float)((double)lo / deg) : 0.f;
        f[3] = (float)((diag - wsum) / diag);
        f[4] = (float)(wup / diag);
        f[5] = (float)ent;
        f[6] = wsum > 0.0 ? (float)(wmax / wsum) : 0.f;
        f[7] = (float)((double)k / (double)(n > 1 ? n - 1 : 1));
        f[8] = deg ? (float)(nex / deg) : 0.f;
        f[9] = (float)log1p(deg ? ndeg / deg : 0.0);
        f[10] = (float)log1p((double)up2);
        f[11] = (float)log(diag);
#pragma unroll
        for (int i = kFeatures; i < kFeatStride; ++i) f[i] = 0.f;
    }
}

// Pilot-walk statistics of each walk row (one warp per row) from a per-walk
// quantity: the walk length (records hold lengths; plus = 0) or the visits to
// the start row, J = 1 + returns (records hold returns; plus = 1).  Mean,
// sample standard deviation (two passes, FP64), and the label
// log((sd / mean)^2 + 1e-6).
__global__ void k_pilot_stats(int32_t nw, const int4* __restrict__ wrow,
                              const int64_t* __restrict__ wbase, const int2* __restrict__ rec, uint32_t plus,
                              float* mean_out, float* sd_out, float* label, float* has) {
    const int32_t gw = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nwarps = (int32_t)((gridDim.x * blockDim.x) >> 5);
    for (int32_t r = gw; r < nw; r += nwarps) {
        const int32_t k = wrow[r].x;
        const int64_t b0 = wbase[r], b1 = wbase[r + 1];
        unsigned long long s1 = 0;
        for (int64_t i = b0 + lane_id(); i < b1; i += 32) s1 += (unsigned long long)(uint32_t)rec[i].y + plus;
        s1 = warp_sum(s1);
        const double m = (double)(b1 - b0);
        const double mean = (double)s1 / m;
        double s2 = 0.0;
        for (int64_t i = b0 + lane_id(); i < b1; i += 32) {
            const double d = (double)((unsigned long long)(uint32_t)rec[i].y + plus) - mean;
            s2 += d * d;
        }
        s2 = warp_sum(s2);
        if (lane_id() == 0) {
            const double var = m > 1.0 ? s2 / (m - 1.0) : 0.0;
            mean_out[k] = (float)mean;
            sd_out[k] = (float)sqrt(var);
            label[k] = (float)log(var / (mean * mean) + 1e-6);
            has[k] = 1.f;
        }
    }
}

// Cost-aware label (quantity 2): half of (the visits label minus log of the
// mean walk length), so that exp(label) is proportional to sqrt(relative
// variance of the visits / walk cost) -- the allocation of a fixed number of
// hops that minimises the summed relative variances.
__global__ void k_label_cost(int32_t n, const float* __restrict__ mean_len, const float* __restrict__ has,
                             float* label) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        if (has[k] > 0.f) label[k] = (float)(0.5 * ((double)label[k] - log((double)mean_len[k])));
}

// ---------------------------------------------------------------------------
// MLP.  Parameters (FP32 master copy, one flat vector of kMlpParams):
//   W1 [64][16] (output-major, inputs 12..15 unused), b1 [64],
//   W2 [64][64] (output-major), b2 [64], w3 [64], b3.
// Forward: x = bf16((f - mu) * inv_sd); h1 = bf16(relu(W1 x + b1));
//          h2 = relu(W2 h1 + b2); y = w3 . h2 + b3, with W1, W2 in BF16 and
//          FP32 accumulation (m16n8k16 tensor-core products).
// ---------------------------------------------------------------------------
constexpr int kH = 64;
constexpr int kIn = 16;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kH * kIn;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kH;
static_assert(kOffB3 + 1 == kMlpParams, "parameter count");
static_assert(kIn == kFeatStride, "input width");

struct MlpSmem {
    __nv_bfloat16 w1[kH][kIn];   // [out][in]
    __nv_bfloat16 w2[kH][kH];    // [out][in]
    __nv_bfloat16 w2t[kH][kH];   // [in][out]
    float b1[kH], b2[kH], w3[kH];
    float mu[kIn], inv_sd[kIn];
    float b3;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

// d += a b: m16n8k16, A row-major (4 registers), B column-major (2), FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ void mlp_load_smem(MlpSmem& S, const float* __restrict__ P, const float* __restrict__ norm) {
    for (int i = threadIdx.x; i < kH * kIn; i += blockDim.x)
        S.w1[i / kIn][i % kIn] = __float2bfloat16_rn((i % kIn) < kFeatures ? P[kOffW1 + i] : 0.f);
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
        const __nv_bfloat16 v = __float2bfloat16_rn(P[kOffW2 + i]);
        S.w2[i / kH][i % kH] = v;
        S.w2t[i % kH][i / kH] = v;
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        S.b1[i] = P[kOffB1 + i];
        S.b2[i] = P[kOffB2 + i];
        S.w3[i] = P[kOffW3 + i];
    }
    for (int i = threadIdx.x; i < kIn; i += blockDim.x) {
        S.mu[i] = i < kFeatures ? norm[i] : 0.f;
        S.inv_sd[i] = i < kFeatures ? norm[kIn + i] : 0.f;
    }
    if (threadIdx.x == 0) S.b3 = P[kOffB3];
    __syncthreads();
}

// Activations of the 16 rows one warp holds.  Fragment coordinates: g = lane/4,
// q = lane%4; the lane owns rows g (index 0) and g+8 (index 1), and in n-tile t
// the hidden units 8t+2q and 8t+2q+1.
struct MlpRows {
    float xn[2][4];   // inputs at columns 2q, 2q+1, 2q+8, 2q+9
    float h1[8][4];   // accumulator layout: {row g: 2 units, row g+8: 2 units}
    float h2[8][4];
    float out[2];
};

// fa, fb: feature rows of the warp's rows g and g+8 (nullptr: padding row)
__device__ __forceinline__ void mlp_forward(const MlpSmem& S, const float* fa, const float* fb,
                                           MlpRows& R) {
    const int lane = (int)lane_id(), g = lane >> 2, q = lane & 3;
    const int cols[4] = {2 * q, 2 * q + 1, 2 * q + 8, 2 * q + 9};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int f = cols[c];
        R.xn[0][c] = (fa && f < kFeatures) ? bf16_round((fa[f] - S.mu[f]) * S.inv_sd[f]) : 0.f;
        R.xn[1][c] = (fb && f < kFeatures) ? bf16_round((fb[f] - S.mu[f]) * S.inv_sd[f]) : 0.f;
    }
    const uint32_t a1[4] = {pack_bf16(R.xn[0][0], R.xn[0][1]), pack_bf16(R.xn[1][0], R.xn[1][1]),
                            pack_bf16(R.xn[0][2], R.xn[0][3]), pack_bf16(R.xn[1][2], R.xn[1][3])};
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int n0 = 8 * t + 2 * q;
        R.h1[t][0] = S.b1[n0];
        R.h1[t][1] = S.b1[n0 + 1];
        R.h1[t][2] = S.b1[n0];
        R.h1[t][3] = S.b1[n0 + 1];
        mma_bf16(R.h1[t], a1, ld_pair(&S.w1[8 * t + g][2 * q]), ld_pair(&S.w1[8 * t + g][2 * q + 8]));
#pragma unroll
        for (int c = 0; c < 4; ++c) R.h1[t][c] = bf16_round(fmaxf(R.h1[t][c], 0.f));
    }
    // the layer-1 accumulators are already in the A-fragment layout of layer 2
    uint32_t a2[4][4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        a2[s][0] = pack_bf16(R.h1[2 * s][0], R.h1[2 * s][1]);
        a2[s][1] = pack_bf16(R.h1[2 * s][2], R.h1[2 * s][3]);
        a2[s][2] = pack_bf16(R.h1[2 * s + 1][0], R.h1[2 * s + 1][1]);
        a2[s][3] = pack_bf16(R.h1[2 * s + 1][2], R.h1[2 * s + 1][3]);
    }
    float o0 = 0.f, o1 = 0.f;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int n0 = 8 * t + 2 * q;
        R.h2[t][0] = S.b2[n0];
        R.h2[t][1] = S.b2[n0 + 1];
        R.h2[t][2] = S.b2[n0];
        R.h2[t][3] = S.b2[n0 + 1];
#pragma unroll
        for (int s = 0; s < 4; ++s)
            mma_bf16(R.h2[t], a2[s], ld_pair(&S.w2[8 * t + g][16 * s + 2 * q]),
                     ld_pair(&S.w2[8 * t + g][16 * s + 8 + 2 * q]));
#pragma unroll
        for (int c = 0; c < 4; ++c) R.h2[t][c] = fmaxf(R.h2[t][c], 0.f);
        o0 += R.h2[t][0] * S.w3[n0] + R.h2[t][1] * S.w3[n0 + 1];
        o1 += R.h2[t][2] * S.w3[n0] + R.h2[t][3] * S.w3[n0 + 1];
    }
    o0 += __shfl_xor_sync(kFull, o0, 1);
    o0 += __shfl_xor_sync(kFull, o0, 2);
    o1 += __shfl_xor_sync(kFull, o1, 1);
    o1 += __shfl_xor_sync(kFull, o1, 2);
    R.out[0] = o0 + S.b3;
    R.out[1] = o1 + S.b3;
}

__global__ void __launch_bounds__(256) k_mlp_predict(const float* __restrict__ P,
                                                     const float* __restrict__ norm,
                                                     const float* __restrict__ feat, int64_t nrows,
                                                     float* __restrict__ out) {
    __shared__ MlpSmem S;
    mlp_load_smem(S, P, norm);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id(), g = lane >> 2, q = lane & 3;
    for (int64_t base = gw * 16; base < nrows; base += nw * 16) {
        const int64_t ra = base + g, rb = base + g + 8;
        MlpRows R;
        mlp_forward(S, ra < nrows ? feat + ra * kFeatStride : nullptr,
                    rb < nrows ? feat + rb * kFeatStride : nullptr, R);
        if (q == 0) {
            if (ra < nrows) out[ra] = R.out[0];
            if (rb < nrows) out[rb] = R.out[1];
        }
    }
}

// Training, part 1: forward and backward through the activations for the
// batch rows idx[0..B); loss = (1/B) sum (y - label)^2.  Per batch row r the
// kernel stores what the weight gradients need:
//   act[r] = {x[16], h1[64], dh1[64], h2[64], dh2[64], dy, pad[3]}
// dh1 = (bf16(dh2) W2) * [h1 > 0] is a tensor-core product, like the forward.
constexpr int kActX = 0, kActH1 = 16, kActDH1 = 80, kActH2 = 144, kActDH2 = 208, kActDY = 272;
constexpr int kActStride = 276;

__global__ void __launch_bounds__(256) k_mlp_train_act(const float* __restrict__ P,
                                                       const float* __restrict__ norm,
                                                       const float* __restrict__ feat,
                                                       const float* __restrict__ label,
                                                       const uint32_t* __restrict__ idx, int64_t B,
                                                       float* __restrict__ act,
                                                       float* __restrict__ loss_part) {
    __shared__ MlpSmem S;
    __shared__ float wloss[8];
    mlp_load_smem(S, P, norm);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id(), g = lane >> 2, q = lane & 3;
    float myloss = 0.f;
    for (int64_t base = gw * 16; base < B; base += nw * 16) {
        const int64_t ra = base + g, rb = base + g + 8;
        const uint32_t ia = ra < B ? idx[ra] : 0u, ib = rb < B ? idx[rb] : 0u;
        MlpRows R;
        mlp_forward(S, ra < B ? feat + (size_t)ia * kFeatStride : nullptr,
                    rb < B ? feat + (size_t)ib * kFeatStride : nullptr, R);
        const float ea = ra < B ? R.out[0] - label[ia] : 0.f;
        const float eb = rb < B ? R.out[1] - label[ib] : 0.f;
        if (q == 0) myloss += ea * ea + eb * eb;
        const float da = 2.f * ea / (float)B, db = 2.f * eb / (float)B;
        float dh2[8][4];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int n0 = 8 * t + 2 * q;
            dh2[t][0] = R.h2[t][0] > 0.f ? da * S.w3[n0] : 0.f;
            dh2[t][1] = R.h2[t][1] > 0.f ? da * S.w3[n0 + 1] : 0.f;
            dh2[t][2] = R.h2[t][2] > 0.f ? db * S.w3[n0] : 0.f;
            dh2[t][3] = R.h2[t][3] > 0.f ? db * S.w3[n0 + 1] : 0.f;
        }
        uint32_t ad[4][4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            ad[s][0] = pack_bf16(dh2[2 * s][0], dh2[2 * s][1]);
            ad[s][1] = pack_bf16(dh2[2 * s][2], dh2[2 * s][3]);
            ad[s][2] = pack_bf16(dh2[2 * s + 1][0], dh2[2 * s + 1][1]);
            ad[s][3] = pack_bf16(dh2[2 * s + 1][2], dh2[2 * s + 1][3]);
        }
        float dh1[8][4];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            dh1[t][0] = dh1[t][1] = dh1[t][2] = dh1[t][3] = 0.f;
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_bf16(dh1[t], ad[s], ld_pair(&S.w2t[8 * t + g][16 * s + 2 * q]),
                         ld_pair(&S.w2t[8 * t + g][16 * s + 8 + 2 * q]));
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (!(R.h1[t][c] > 0.f)) dh1[t][c] = 0.f;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t r = base + g + 8 * h;
            if (r >= B) continue;
            float* a = act + (size_t)r * kActStride;
            *reinterpret_cast<float2*>(a + kActX + 2 * q) = make_float2(R.xn[h][0], R.xn[h][1]);
            *reinterpret_cast<float2*>(a + kActX + 2 * q + 8) = make_float2(R.xn[h][2], R.xn[h][3]);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int n0 = 8 * t + 2 * q;
                *reinterpret_cast<float2*>(a + kActH1 + n0) = make_float2(R.h1[t][2 * h], R.h1[t][2 * h + 1]);
                *reinterpret_cast<float2*>(a + kActDH1 + n0) = make_float2(dh1[t][2 * h], dh1[t][2 * h + 1]);
                *reinterpret_cast<float2*>(a + kActH2 + n0) = make_float2(R.h2[t][2 * h], R.h2[t][2 * h + 1]);
                *reinterpret_cast<float2*>(a + kActDH2 + n0) = make_float2(dh2[t][2 * h], dh2[t][2 * h + 1]);
            }
            if (q == 0) a[kActDY] = h == 0 ? da : db;
        }
    }
    myloss = warp_sum(myloss);
    if (lane == 0) wloss[threadIdx.x >> 5] = myloss;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wloss[w];
        loss_part[blockIdx.x] = s;
    }
}

// Training, part 2: weight gradients, each a sum over the batch rows.  Block
// (x, y) computes entries x*256.. over the rows of slice y; the slices are
// summed in a fixed order afterwards (deterministic).
__global__ void __launch_bounds__(256) k_mlp_wgrad(const float* __restrict__ act, int64_t B,
                                                   int64_t rows_per_slice, float* __restrict__ part) {
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_slice;
    const int64_t r1 = min(B, r0 + rows_per_slice);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kMlpParams) return;
    int ia, ib;  // product of act[ia] and act[ib]; ib == -1: act[ia] alone; -2: zero
    if (e < kOffB1) {
        ia = kActDH1 + e / kIn;
        ib = (e % kIn) < kFeatures ? kActX + e % kIn : -2;
    } else if (e < kOffW2) {
        ia = kActDH1 + (e - kOffB1);
        ib = -1;
    } else if (e < kOffB2) {
        ia = kActDH2 + (e - kOffW2) / kH;
        ib = kActH1 + (e - kOffW2) % kH;
    } else if (e < kOffW3) {
        ia = kActDH2 + (e - kOffB2);
        ib = -1;
    } else if (e < kOffB3) {
        ia = kActDY;
        ib = kActH2 + (e - kOffW3);
    } else {
        ia = kActDY;
        ib = -1;
    }
    float s = 0.f;
    if (ib >= 0) {
        for (int64_t r = r0; r < r1; ++r) s += act[r * kActStride + ia] * act[r * kActStride + ib];
    } else if (ib == -1) {
        for (int64_t r = r0; r < r1; ++r) s += act[r * kActStride + ia];
    }
    part[(size_t)blockIdx.y * kMlpParams + e] = s;
}

// Sum the slices in order into grad; with do_step, an Adam step on P
// (beta1 0.9, beta2 0.999, eps 1e-8; b1t, b2t = beta^t for bias correction).
// Block 0 also sums the loss partials into *loss (when loss is not null).
__global__ void k_mlp_adam(int nslices, const float* __restrict__ part, float* __restrict__ grad,
                           float* __restrict__ P, float* __restrict__ m1, float* __restrict__ m2,
                           float lr, float b1t, float b2t, int do_step, int nloss,
                           const float* __restrict__ loss_part, float* __restrict__ loss) {
    constexpr float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    if (loss && blockIdx.x == 0 && threadIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < nloss; ++i) s += loss_part[i];
        *loss = s;
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kMlpParams; e += gridDim.x * blockDim.x) {
        float gsum = 0.f;
        for (int sl = 0; sl < nslices; ++sl) gsum += part[(size_t)sl * kMlpParams + e];
        grad[e] = gsum;
        if (!do_step) continue;
        const float a = beta1 * m1[e] + (1.f - beta1) * gsum;
        const float v = beta2 * m2[e] + (1.f - beta2) * gsum * gsum;
        m1[e] = a;
        m2[e] = v;
        P[e] -= lr * (a / (1.f - b1t)) / (sqrtf(v / (1.f - b2t)) + eps);
    }
}

// Per-feature sums of f and f^2 over the rows with mask > 0 (block partials).
__global__ void __launch_bounds__(256) k_feat_moments(int64_t n, const float* __restrict__ feat,
                                                      const float* __restrict__ mask,
                                                      double* __restrict__ part) {
    constexpr int kW = 2 * kFeatures + 1;
    __shared__ double sm[8][kW];
    double acc[kW];
#pragma unroll
    for (int i = 0; i < kW; ++i) acc[i] = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (!(mask[r] > 0.f)) continue;
        acc[2 * kFeatures] += 1.0;
#pragma unroll
        for (int f = 0; f < kFeatures; ++f) {
            const double v = feat[r * kFeatStride + f];
            acc[f] += v;
            acc[kFeatures + f] += v * v;
        }
    }
#pragma unroll
    for (int i = 0; i < kW; ++i) acc[i] = warp_sum(acc[i]);
    if (lane_id() == 0)
        for (int i = 0; i < kW; ++i) sm[threadIdx.x >> 5][i] = acc[i];
    __syncthreads();
    if (threadIdx.x < kW) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w][threadIdx.x];
        part[(size_t)blockIdx.x * kW + threadIdx.x] = s;
    }
}

__global__ void k_exp_weights(int64_t n, const float* pred, float* w) {  // may run in place
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        w[k] = expf(fminf(fmaxf(pred[k], -60.f), 60.f));
}

// ---------------------------------------------------------------------------
// Budget normaliser.  For the walk rows (rows with an upper neighbour), with
// T = floor(mean * #walk rows + 1/2) walks in total:
//   quota q_k(s) = min(cap, max(min_b, s w_k)),  cap = min(T, 2^31),
//   V_k(s) = round_half_even(q_k(s) 2^20)  (fixed point, exact integer sums),
//   s = the result of a fixed doubling-then-bisection search for the largest
//       s whose total sum_k V_k(s) is not above T 2^20,
//   floor_k = V_k >> 20, frac_k = V_k mod 2^20, R = T - sum floor_k,
//   budget_k = floor_k + R / nw + [rank_k < R mod nw], ranks by (frac desc, k asc)
// (largest-remainder apportionment).  Rows without walks get 0.  Every step
// is exact in double or integer arithmetic, so the result does not depend on
// the order of any sum.
// ---------------------------------------------------------------------------
constexpr int kFracBits = 20;
constexpr int kFracBins = 1 << kFracBits;

__device__ __forceinline__ bool row_has_upper(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                              int32_t k) {
    for (int32_t p = rp[k + 1] - 1; p >= rp[k]; --p)
        if (col[p] > k) return true;
    return false;
}

__device__ __forceinline__ int64_t quota_fixed(float w, double s, double min_b, double cap) {
    const double v = fmin(cap, fmax(min_b, __dmul_rn(s, (double)w)));
    return llrint(ldexp(v, kFracBits));
}

__device__ __forceinline__ unsigned long long sat_add(unsigned long long a, unsigned long long b,
                                                      unsigned long long sat) {
    return (a >= sat || b >= sat - a) ? sat : a + b;
}

// The walk rows' weights in a row-indexed array (-1 for the other rows), read
// by every pass of the search instead of the matrix; out[3 block + {0,1,2}] =
// {0, walk rows, invalid weights}.
__global__ void __launch_bounds__(256) k_norm_prep(int32_t n, const int32_t* __restrict__ rp,
                                                   const int32_t* __restrict__ col, const float* __restrict__ w,
                                                   float* __restrict__ wv, unsigned long long* __restrict__ out) {
    unsigned long long cnt = 0, bad = 0;
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        float v = -1.0f;
        if (row_has_upper(rp, col, k)) {
            ++cnt;
            v = w[k];
            if (!(v >= 0.f) || isinf(v)) {
                ++bad;
                v = -1.0f;
            }
        }
        wv[k] = v;
    }
    __shared__ unsigned long long sm[2][8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(kFull, cnt, o);
        bad += __shfl_xor_sync(kFull, bad, o);
    }
    const int wid = threadIdx.x >> 5;
    if (lane_id() == 0) {
        sm[0][wid] = cnt;
        sm[1][wid] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long c = 0, b = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            c += sm[0][i];
            b += sm[1][i];
        }
        out[3 * blockIdx.x] = 0;
        out[3 * blockIdx.x + 1] = c;
        out[3 * blockIdx.x + 2] = b;
    }
}

// out[3 block] = sum over the walk rows (wv >= 0) of V_k(s), saturated at sat.
__global__ void __launch_bounds__(256) k_norm_sum(int32_t n, const float* __restrict__ wv, double s, double min_b,
                                                  double cap, unsigned long long sat,
                                                  unsigned long long* __restrict__ out) {
    unsigned long long sum = 0;
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float wk = wv[k];
        if (wk >= 0.f) sum = sat_add(sum, (unsigned long long)quota_fixed(wk, s, min_b, cap), sat);
    }
    __shared__ unsigned long long sm[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum = sat_add(sum, __shfl_xor_sync(kFull, sum, o), sat);
    const int wid = threadIdx.x >> 5;
    if (lane_id() == 0) sm[wid] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a = sat_add(a, sm[i], sat);
        out[3 * blockIdx.x] = a;
        out[3 * blockIdx.x + 1] = 0;
        out[3 * blockIdx.x + 2] = 0;
    }
}

// floor parts into budget, fractional parts into frac (0xFFFFFFFF for rows
// without walks), their histogram, and the sum of the floors (exact integer
// atomics).
__global__ void k_norm_split(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const float* __restrict__ w, double s, double min_b, double cap,
                             uint32_t* __restrict__ budget, uint32_t* __restrict__ frac,
                             uint32_t* __restrict__ hist, unsigned long long* __restrict__ fsum) {
    unsigned long long acc = 0;
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (!row_has_upper(rp, col, k)) {
            budget[k] = 0u;
            frac[k] = 0xFFFFFFFFu;
            continue;
        }
        const int64_t v = quota_fixed(w[k], s, min_b, cap);
        const uint32_t fl = (uint32_t)(v >> kFracBits), fr = (uint32_t)(v & (kFracBins - 1));
        budget[k] = fl;
        frac[k] = fr;
        atomicAdd(&hist[fr], 1u);
        acc += fl;
    }
    acc = warp_sum(acc);
    if (lane_id() == 0) atomicAdd(fsum, acc);
}

// One block of 1024 threads: the bin t holding the r-th largest fractional
// part (1 <= r <= walk rows) and the number of walk rows above bin t.
// res = {t, count above t}.
__global__ void __launch_bounds__(1024) k_norm_select(const uint32_t* __restrict__ hist, uint64_t r,
                                                      uint64_t* __restrict__ res) {
    constexpr int kPer = kFracBins / 1024;
    __shared__ unsigned long long sm[1024];
    const int t = threadIdx.x;
    // thread t owns bins [(1023 - t) kPer, (1024 - t) kPer): thread 0 the top bins
    const int lo = (1023 - t) * kPer;
    unsigned long long c = 0;
    for (int b = 0; b < kPer; ++b) c += hist[lo + b];
    sm[t] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan from the top bins down
        const unsigned long long add = t >= o ? sm[t - o] : 0ull;
        __syncthreads();
        sm[t] += add;
        __syncthreads();
    }
    const unsigned long long above = t > 0 ? sm[t - 1] : 0ull;
    if (above < r && sm[t] >= r) {
        unsigned long long acc = above;
        for (int b = kPer - 1; b >= 0; --b) {
            const unsigned long long h = hist[lo + b];
            if (acc + h >= r) {
                res[0] = (uint64_t)(lo + b);
                res[1] = acc;
                break;
            }
            acc += h;
        }
    }
}

__global__ void k_norm_ties(int32_t n, const uint32_t* __restrict__ frac, uint32_t t,
                            uint32_t* __restrict__ flag) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        flag[k] = frac[k] == t ? 1u : 0u;
}

// budget_k += qa + [frac > t or (frac == t and tie rank < rt)] for walk rows
__global__ void k_norm_final(int32_t n, const uint32_t* __restrict__ frac,
                             const uint32_t* __restrict__ tie_rank, uint32_t qa, int use_sel, uint32_t t,
                             uint32_t rt, uint32_t* __restrict__ budget) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t f = frac[k];
        if (f == 0xFFFFFFFFu) continue;
        uint32_t add = qa;
        if (use_sel && (f > t || (f == t && tie_rank[k] < rt))) ++add;
        budget[k] += add;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static rw_status features_run(rw_context* ctx, const rw_csr* A, float* feat) {
    NvtxRange nvtx_range("rw_features");
    Pool sc(ctx);
    int32_t* ndeg = alloc_n<int32_t>(sc, A->n);
    double* exr = alloc_n<double>(sc, A->n);
    if (!ndeg || !exr) return RW_ERR_ALLOC;
    RW_COUNT_LAUNCH();
    k_node_info<<<grid_for(A->n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(A->n, A->row_ptr, A->col, A->val,
                                                                                 ndeg, exr);
    RW_COUNT_LAUNCH();
    k_features<<<grid_for(A->n, 128, ctx->num_sms * 16), 128, 0, ctx->stream>>>(A->n, A->row_ptr, A->col,
                                                                                 A->val, ndeg, exr, feat);
    return check_launch("row features");
}

static rw_status pilot_run(rw_context* ctx, const rw_csr* A, uint32_t walks, uint64_t seed, int quantity,
                           float* mean, float* sd, float* label, float* has);

// quantity 2: the same walks twice (lengths, then visits), combined
static rw_status pilot_cost(rw_context* ctx, const rw_csr* A, uint32_t walks, uint64_t seed, float* mean, float* sd,
                            float* label, float* has) {
    Pool sc(ctx);
    float* mlen = alloc_n<float>(sc, A->n);
    float* t1 = alloc_n<float>(sc, A->n);
    float* t2 = alloc_n<float>(sc, A->n);
    if (!mlen || !t1 || !t2) return RW_ERR_ALLOC;
    rw_status rc;
    if ((rc = pilot_run(ctx, A, walks, seed, 0, mlen, t1, t2, has))) return rc;
    if ((rc = pilot_run(ctx, A, walks, seed, 1, mean, sd, label, has))) return rc;
    RW_COUNT_LAUNCH();
    k_label_cost<<<grid_for(A->n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(A->n, mlen, has, label);
    if ((rc = check_launch("cost label"))) return rc;
    return read_status(ctx, "pilot statistics");
}

static rw_status pilot_run(rw_context* ctx, const rw_csr* A, uint32_t walks, uint64_t seed, int quantity,
                           float* mean, float* sd, float* label, float* has) {
    NvtxRange nvtx_range("rw_pilot");
    cudaStream_t s = ctx->stream;
    Pool scratch(ctx);
    Tables T;
    WalkSpace ws;
    rw_status rc;
    if ((rc = reset_status(ctx))) return rc;
    if ((rc = build_tables(ctx, A, T, scratch))) return rc;
    if ((rc = read_status(ctx, "walk tables"))) return rc;
    if ((rc = build_walk_space(ctx, T, walks, nullptr, ws, scratch))) return rc;
    const size_t nb = sizeof(float) * (size_t)A->n;
    if ((rc = check_cuda(cudaMemsetAsync(has, 0, nb, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(mean, 0, nb, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(sd, 0, nb, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(label, 0, nb, s), "memset")))
        return rc;
    if (T.n_walk_rows == 0) return check_cuda(cudaStreamSynchronize(s), "sync");
    int2* rec = alloc_n<int2>(scratch, ws.total);
    unsigned long long* hops = alloc_n<unsigned long long>(scratch, 1);
    if (!rec || !hops) return RW_ERR_ALLOC;
    WalkBatch wb;
    wb.m0 = mat_walk(T, seed, 0, 1);  // kind 1: pilot walks
    wb.table_bytes = table_bytes(T);
    wb.nrows = T.n_walk_rows;
    wb.wrow = T.wrow;
    wb.wbase = ws.wbase;
    wb.chunk_row = ws.chunk_row;
    wb.total = ws.total;
    WalkLaunch wl;
    wl.max_steps = ctx->opt.max_steps;
    wl.record_lengths = quantity == 0 ? 1 : 0;
    if ((rc = run_walks(ctx, wb, wl, rec, hops, scratch, nullptr))) return rc;
    if ((rc = read_status(ctx, "pilot walks"))) return rc;
    RW_COUNT_LAUNCH();
    k_pilot_stats<<<grid_for((int64_t)T.n_walk_rows * 32, 256, ctx->num_sms * 8), 256, 0, s>>>(
        T.n_walk_rows, T.wrow, ws.wbase, rec, quantity == 0 ? 0u : 1u, mean, sd, label, has);
    if ((rc = check_launch("pilot statistics"))) return rc;
    return read_status(ctx, "pilot statistics");
}

static rw_status normalize_run(rw_context* ctx, const rw_csr* A, const float* w, double mean_budget,
                               uint32_t min_budget, uint32_t* budget, Pool& sc) {
    NvtxRange nvtx_range("rw_budget_normalize");
    cudaStream_t s = ctx->stream;
    const int32_t n = A->n;
    const int blocks = grid_for(n, 256, ctx->num_sms * 4);
    unsigned long long* part = alloc_n<unsigned long long>(sc, 3 * (int64_t)blocks);
    if (!part) return RW_ERR_ALLOC;
    std::vector<unsigned long long> hp(3 * (size_t)blocks);
    const double min_b = (double)min_budget;
    unsigned long long sat = ~0ull;
    double cap = min_b;
    rw_status rc;
    float* wv = alloc_n<float>(sc, n);
    if (!wv) return RW_ERR_ALLOC;
    // the partial results of one launch summed on the host (saturating the first)
    auto reduce = [&](unsigned long long* sum, unsigned long long* cnt, unsigned long long* bad) -> rw_status {
        rw_status r2;
        if ((r2 = check_cuda(cudaMemcpyAsync(hp.data(), part, sizeof(unsigned long long) * hp.size(),
                                             cudaMemcpyDeviceToHost, s),
                             "copy")) ||
            (r2 = check_cuda(cudaStreamSynchronize(s), "sync")))
            return r2;
        unsigned long long a = 0, c = 0, b = 0;
        for (int i = 0; i < blocks; ++i) {
            a = (a >= sat || hp[3 * i] >= sat - a) ? sat : a + hp[3 * i];
            c += hp[3 * i + 1];
            b += hp[3 * i + 2];
        }
        if (sum) *sum = a;
        if (cnt) *cnt = c;
        if (bad) *bad = b;
        return RW_OK;
    };
    // total(s) = sum of V_k(s) over the walk rows, saturated at sat
    auto total = [&](double sv, unsigned long long* sum) -> rw_status {
        RW_COUNT_LAUNCH();
        k_norm_sum<<<blocks, 256, 0, s>>>(n, wv, sv, min_b, cap, sat, part);
        rw_status r2 = check_launch("budget total");
        if (r2) return r2;
        return reduce(sum, nullptr, nullptr);
    };
    unsigned long long sum = 0, nw = 0, bad = 0;
    RW_COUNT_LAUNCH();
    k_norm_prep<<<blocks, 256, 0, s>>>(n, A->row_ptr, A->col, w, wv, part);
    if ((rc = check_launch("budget weights"))) return rc;
    if ((rc = reduce(nullptr, &nw, &bad))) return rc;
    if (bad) {
        set_error("rw_budget_normalize: %llu walk rows with a negative, infinite or NaN weight", bad);
        return RW_ERR_ARG;
    }
    if (nw == 0) {
        if ((rc = check_cuda(cudaMemsetAsync(budget, 0, sizeof(uint32_t) * (size_t)n, s), "memset")))
            return rc;
        return check_cuda(cudaStreamSynchronize(s), "sync");
    }
    const double tot = std::floor(mean_budget * (double)nw + 0.5);
    if (tot > 1099511627776.0) {  // 2^40 walks
        set_error("rw_budget_normalize: %.0f walks in total, above 2^40", tot);
        return RW_ERR_ARG;
    }
    const uint64_t T = (uint64_t)tot;
    const unsigned long long target = (unsigned long long)T << kFracBits;
    // totals saturate far above the target (only the comparison with the
    // target is used), so that they can be interpolated
    sat = 1ull << 62;
    cap = std::min((double)T, 2147483648.0);
    if ((rc = total(0.0, &sum))) return rc;
    double lo = 0.0;
    if (sum < target) {
        double hi = 1.0;
        unsigned long long sum_lo = sum;
        for (;;) {  // doubling: the first hi with total(hi) > target
            if ((rc = total(hi, &sum))) return rc;
            if (sum > target) break;
            lo = hi;
            sum_lo = sum;
            if (sum == target || hi > 1e300) break;
            hi *= 2.0;
        }
        if (sum > target) {
            // total(lo) <= target < total(hi): the answer is the largest double
            // s in [lo, hi) with total(s) <= target (total does not decrease
            // in s), the point where plain bisection stops, so the search may
            // take any points inside the bracket.  Odd steps interpolate the
            // totals, even steps bisect (the bracket at least halves every two
            // steps); it stops when lo and hi are adjacent doubles.
            unsigned long long sum_hi = sum;
            for (int it = 0; it < 4400; ++it) {
                double mid = 0.5 * (lo + hi);
                if ((it & 1) && sum_hi > sum_lo) {
                    const double f = (double)(target - sum_lo) / (double)(sum_hi - sum_lo);
                    const double g = lo + f * (hi - lo);
                    if (g > lo && g < hi) mid = g;
                }
                if (!(mid > lo && mid < hi)) break;
                if ((rc = total(mid, &sum))) return rc;
                if (sum <= target) {
                    lo = mid;
                    sum_lo = sum;
                } else {
                    hi = mid;
                    sum_hi = sum;
                }
            }
        }
    }
    uint32_t* frac = alloc_n<uint32_t>(sc, n);
    uint32_t* hist = alloc_n<uint32_t>(sc, kFracBins);
    uint32_t* ties = alloc_n<uint32_t>(sc, (int64_t)n + 1);
    unsigned long long* fsum = alloc_n<unsigned long long>(sc, 1);
    uint64_t* sel = alloc_n<uint64_t>(sc, 2);
    if (!frac || !hist || !ties || !fsum || !sel) return RW_ERR_ALLOC;
    if ((rc = check_cuda(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kFracBins, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(fsum, 0, sizeof(unsigned long long), s), "memset")))
        return rc;
    RW_COUNT_LAUNCH();
    k_norm_split<<<blocks, 256, 0, s>>>(n, A->row_ptr, A->col, w, lo, min_b, cap, budget, frac, hist, fsum);
    if ((rc = check_launch("budget split"))) return rc;
    unsigned long long* hF = static_cast<unsigned long long*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(hF, fsum, 8, cudaMemcpyDeviceToHost, s), "copy")) ||
        (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
        return rc;
    const uint64_t F = hF[0];
    if (F > T) {
        set_error("rw_budget_normalize: internal error (floor sum above the total)");
        return RW_ERR_CUDA;
    }
    const uint64_t R = T - F;
    const uint64_t qa = R / nw, r = R % nw;
    if ((double)qa + cap + 1.0 > 4294967295.0) {
        set_error("rw_budget_normalize: a budget above 2^32 - 1");
        return RW_ERR_ARG;
    }
    uint64_t* hsel = static_cast<uint64_t*>(ctx->h_small);
    uint64_t t = 0, above = 0;
    if (r > 0) {
        RW_COUNT_LAUNCH();
        k_norm_select<<<1, 1024, 0, s>>>(hist, r, sel);
        if ((rc = check_launch("budget select"))) return rc;
        if ((rc = check_cuda(cudaMemcpyAsync(hsel, sel, 16, cudaMemcpyDeviceToHost, s), "copy")) ||
            (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
            return rc;
        t = hsel[0];
        above = hsel[1];
        RW_COUNT_LAUNCH();
        k_norm_ties<<<blocks, 256, 0, s>>>(n, frac, (uint32_t)t, ties);
        if ((rc = check_launch("budget ties"))) return rc;
        if ((rc = check_cuda(scan_u32(ties, ties, n, s, sc), "scan"))) return rc;
    }
    RW_COUNT_LAUNCH();
    k_norm_final<<<blocks, 256, 0, s>>>(n, frac, ties, (uint32_t)qa, r > 0 ? 1 : 0, (uint32_t)t,
                                        (uint32_t)(r - above), budget);
    if ((rc = check_launch("budget final"))) return rc;
    return check_cuda(cudaStreamSynchronize(s), "sync");
}

}  // namespace rw

struct rw_mlp {
    rw_context* ctx = nullptr;
    rw::Pool pool;
    float* P = nullptr;     // [kMlpParams] FP32 master weights
    float* m1 = nullptr;    // Adam moments
    float* m2 = nullptr;
    float* grad = nullptr;  // gradient of the last step
    float* norm = nullptr;  // [32]: feature means, inverse standard deviations
    int64_t steps = 0;
    explicit rw_mlp(rw_context* c) : ctx(c), pool(c) {}
};

using namespace rw;

namespace {

rw_status check_csr_args(const rw_csr* A, const char* who) {
    if (!A || A->n < 0 || (A->n > 0 && (!A->row_ptr || !A->col || !A->val))) {
        set_error("%s: bad matrix", who);
        return RW_ERR_ARG;
    }
    return RW_OK;
}

struct StepBuffers {
    float* act = nullptr;
    float* lpart = nullptr;
    float* part = nullptr;
};

constexpr int64_t kGradSlice = 256;

int act_blocks(rw_context* ctx, int64_t B) { return grid_for((B + 15) / 16 * 32, 256, ctx->num_sms * 2); }

rw_status step_buffers(rw_context* ctx, int64_t B, Pool& sc, StepBuffers& b) {
    const int64_t nslices = (B + kGradSlice - 1) / kGradSlice;
    b.act = alloc_n<float>(sc, B * kActStride);
    b.lpart = alloc_n<float>(sc, act_blocks(ctx, B));
    b.part = alloc_n<float>(sc, nslices * kMlpParams);
    return (b.act && b.lpart && b.part) ? RW_OK : RW_ERR_ALLOC;
}

// One training step over the batch rows idx[0..B): gradient into M->grad, the
// batch's loss sum into *d_loss (optional), an Adam step if step.
rw_status mlp_step(rw_context* ctx, rw_mlp* M, const float* feat, const float* label, const uint32_t* idx,
                   int64_t B, float lr, bool step, float* d_loss, const StepBuffers& b) {
    cudaStream_t s = ctx->stream;
    const int blocks = act_blocks(ctx, B);
    const int nslices = (int)((B + kGradSlice - 1) / kGradSlice);
    RW_COUNT_LAUNCH();
    k_mlp_train_act<<<blocks, 256, 0, s>>>(M->P, M->norm, feat, label, idx, B, b.act, b.lpart);
    RW_COUNT_LAUNCH();
    k_mlp_wgrad<<<dim3((kMlpParams + 255) / 256, nslices), 256, 0, s>>>(b.act, B, kGradSlice, b.part);
    if (step) ++M->steps;
    const double t = (double)(M->steps > 0 ? M->steps : 1);
    RW_COUNT_LAUNCH();
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(nslices, b.part, M->grad, M->P, M->m1, M->m2, lr,
                                                        (float)std::pow(0.9, t), (float)std::pow(0.999, t),
                                                        step ? 1 : 0, blocks, b.lpart, d_loss);
    return check_launch("mlp step");
}

uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

rw_status rw_row_features(rw_context* ctx, const rw_csr* A, float* d_feat) {
    if (!ctx || !d_feat) {
        set_error("rw_row_features: bad arguments");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr_args(A, "rw_row_features");
    if (rc || A->n == 0) return rc;
    if ((rc = reset_status(ctx))) return rc;
    if ((rc = features_run(ctx, A, d_feat))) return rc;
    return read_status(ctx, "row features");
}

rw_status rw_pilot_stats(rw_context* ctx, const rw_csr* A, uint32_t pilot_walks, uint64_t seed, int32_t quantity,
                         float* d_mean, float* d_sd, float* d_label, float* d_has) {
    if (!ctx || !d_mean || !d_sd || !d_label || !d_has || pilot_walks < 2 || quantity < 0 || quantity > 2) {
        set_error("rw_pilot_stats: bad arguments (pilot_walks >= 2, quantity 0, 1 or 2)");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr_args(A, "rw_pilot_stats");
    if (rc || A->n == 0) return rc;
    if (quantity == 2) return pilot_cost(ctx, A, pilot_walks, seed, d_mean, d_sd, d_label, d_has);
    return pilot_run(ctx, A, pilot_walks, seed, quantity, d_mean, d_sd, d_label, d_has);
}

rw_status rw_mlp_create(rw_context* ctx, uint64_t seed, rw_mlp** out) {
    if (!ctx || !out) {
        set_error("rw_mlp_create: bad arguments");
        return RW_ERR_ARG;
    }
    *out = nullptr;
    rw_mlp* M = new (std::nothrow) rw_mlp(ctx);
    if (!M) return RW_ERR_ALLOC;
    M->P = alloc_n<float>(M->pool, kMlpParams);
    M->m1 = alloc_n<float>(M->pool, kMlpParams);
    M->m2 = alloc_n<float>(M->pool, kMlpParams);
    M->grad = alloc_n<float>(M->pool, kMlpParams);
    M->norm = alloc_n<float>(M->pool, 2 * kIn);
    if (!M->P || !M->m1 || !M->m2 || !M->grad || !M->norm) {
        delete M;
        return RW_ERR_ALLOC;
    }
    // He-uniform weights from a splitmix64 stream, zero biases, identity standardisation
    std::vector<float> h(kMlpParams, 0.f), nrm(2 * kIn, 0.f);
    uint64_t st = seed;
    auto uni = [&]() { return (float)((double)(splitmix64(st) >> 11) * 0x1.0p-53 * 2.0 - 1.0); };
    for (int o = 0; o < kH; ++o)
        for (int f = 0; f < kFeatures; ++f) h[kOffW1 + o * kIn + f] = uni() * std::sqrt(6.f / kFeatures);
    for (int i = 0; i < kH * kH; ++i) h[kOffW2 + i] = uni() * std::sqrt(6.f / kH);
    for (int i = 0; i < kH; ++i) h[kOffW3 + i] = uni() * std::sqrt(3.f / kH);
    for (int i = 0; i < kFeatures; ++i) nrm[kIn + i] = 1.f;
    cudaStream_t s = ctx->stream;
    rw_status rc;
    if ((rc = check_cuda(cudaMemcpyAsync(M->P, h.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaMemsetAsync(M->m1, 0, sizeof(float) * kMlpParams, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(M->m2, 0, sizeof(float) * kMlpParams, s), "memset")) ||
        (rc = check_cuda(cudaMemsetAsync(M->grad, 0, sizeof(float) * kMlpParams, s), "memset")) ||
        (rc = check_cuda(cudaMemcpyAsync(M->norm, nrm.data(), sizeof(float) * 2 * kIn, cudaMemcpyHostToDevice, s),
                         "copy")) ||
        (rc = check_cuda(cudaStreamSynchronize(s), "sync"))) {
        delete M;
        return rc;
    }
    *out = M;
    return RW_OK;
}

void rw_mlp_destroy(rw_mlp* M) {
    if (!M) return;
    cudaStreamSynchronize(M->ctx->stream);
    delete M;
}

rw_status rw_mlp_params(rw_mlp* M, float* h_params, float* h_norm, const float* h_set_params,
                        const float* h_set_norm) {
    if (!M) {
        set_error("rw_mlp_params: NULL model");
        return RW_ERR_ARG;
    }
    cudaStream_t s = M->ctx->stream;
    rw_status rc = RW_OK;
    if (h_set_params) {
        if ((rc = check_cuda(cudaMemcpyAsync(M->P, h_set_params, sizeof(float) * kMlpParams,
                                             cudaMemcpyHostToDevice, s),
                             "copy")) ||
            (rc = check_cuda(cudaMemsetAsync(M->m1, 0, sizeof(float) * kMlpParams, s), "memset")) ||
            (rc = check_cuda(cudaMemsetAsync(M->m2, 0, sizeof(float) * kMlpParams, s), "memset")))
            return rc;
        M->steps = 0;
    }
    if (h_set_norm && (rc = check_cuda(cudaMemcpyAsync(M->norm, h_set_norm, sizeof(float) * 2 * kIn,
                                                       cudaMemcpyHostToDevice, s),
                                       "copy")))
        return rc;
    if (h_params && (rc = check_cuda(cudaMemcpyAsync(h_params, M->P, sizeof(float) * kMlpParams,
                                                     cudaMemcpyDeviceToHost, s),
                                     "copy")))
        return rc;
    if (h_norm && (rc = check_cuda(cudaMemcpyAsync(h_norm, M->norm, sizeof(float) * 2 * kIn,
                                                   cudaMemcpyDeviceToHost, s),
                                   "copy")))
        return rc;
    return check_cuda(cudaStreamSynchronize(s), "sync");
}

rw_status rw_mlp_predict(rw_context* ctx, const rw_mlp* M, const float* d_feat, int64_t nrows,
                         float* d_out) {
    NvtxRange nvtx_range("rw_mlp_predict");
    if (!ctx || !M || !d_feat || !d_out || nrows < 0) {
        set_error("rw_mlp_predict: bad arguments");
        return RW_ERR_ARG;
    }
    if (nrows == 0) return RW_OK;
    RW_COUNT_LAUNCH();
    k_mlp_predict<<<grid_for((nrows + 15) / 16 * 32, 256, ctx->num_sms * 4), 256, 0, ctx->stream>>>(
        M->P, M->norm, d_feat, nrows, d_out);
    rw_status rc = check_launch("mlp predict");
    if (rc) return rc;
    return check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
}

rw_status rw_mlp_gradient(rw_context* ctx, rw_mlp* M, const float* d_feat, const float* d_label,
                          const uint32_t* d_rows, int64_t nrows, float* h_grad, float* h_loss) {
    if (!ctx || !M || !d_feat || !d_label || !d_rows || nrows < 1 || !h_grad) {
        set_error("rw_mlp_gradient: bad arguments");
        return RW_ERR_ARG;
    }
    Pool sc(ctx);
    StepBuffers b;
    float* dl = alloc_n<float>(sc, 1);
    if (!dl || step_buffers(ctx, nrows, sc, b)) return RW_ERR_ALLOC;
    rw_status rc;
    if ((rc = mlp_step(ctx, M, d_feat, d_label, d_rows, nrows, 0.f, false, dl, b))) return rc;
    cudaStream_t s = ctx->stream;
    if ((rc = check_cuda(cudaMemcpyAsync(h_grad, M->grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s),
                         "copy")))
        return rc;
    float* hl = static_cast<float*>(ctx->h_small);
    if ((rc = check_cuda(cudaMemcpyAsync(hl, dl, 4, cudaMemcpyDeviceToHost, s), "copy")) ||
        (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
        return rc;
    if (h_loss) *h_loss = hl[0] / (float)nrows;
    return RW_OK;
}

rw_status rw_mlp_train(rw_context* ctx, rw_mlp* M, const float* d_feat, const float* d_label,
                       const float* d_mask, int64_t nrows, int32_t epochs, int32_t batch, float lr,
                       uint64_t seed, int32_t set_norm, float* h_epoch_loss) {
    NvtxRange nvtx_range("rw_mlp_train");
    if (!ctx || !M || !d_feat || !d_label || !d_mask || nrows < 1 || epochs < 0 || batch < 16 ||
        !(lr > 0.f) || nrows > 0xFFFFFFFFll) {
        set_error("rw_mlp_train: bad arguments");
        return RW_ERR_ARG;
    }
    cudaStream_t s = ctx->stream;
    Pool sc(ctx);
    rw_status rc;
    std::vector<float> hmask((size_t)nrows);
    if ((rc = check_cuda(cudaMemcpyAsync(hmask.data(), d_mask, sizeof(float) * (size_t)nrows,
                                         cudaMemcpyDeviceToHost, s),
                         "copy")) ||
        (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
        return rc;
    std::vector<uint32_t> rows;
    for (int64_t i = 0; i < nrows; ++i)
        if (hmask[(size_t)i] > 0.f) rows.push_back((uint32_t)i);
    const int64_t N = (int64_t)rows.size();
    if (N < batch) {
        set_error("rw_mlp_train: %lld training rows, fewer than one batch", (long long)N);
        return RW_ERR_ARG;
    }
    if (set_norm) {
        const int blocks = grid_for(nrows, 256, ctx->num_sms * 2);
        constexpr int kW = 2 * kFeatures + 1;
        double* part = alloc_n<double>(sc, (int64_t)blocks * kW);
        if (!part) return RW_ERR_ALLOC;
        RW_COUNT_LAUNCH();
        k_feat_moments<<<blocks, 256, 0, s>>>(nrows, d_feat, d_mask, part);
        if ((rc = check_launch("feature moments"))) return rc;
        std::vector<double> hp((size_t)blocks * kW);
        if ((rc = check_cuda(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s),
                             "copy")) ||
            (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
            return rc;
        std::vector<double> acc(kW, 0.0);
        for (int b = 0; b < blocks; ++b)
            for (int i = 0; i < kW; ++i) acc[i] += hp[(size_t)b * kW + i];
        std::vector<float> nrm(2 * kIn, 0.f);
        for (int f = 0; f < kFeatures; ++f) {
            const double mu = acc[f] / acc[2 * kFeatures];
            const double var = std::max(0.0, acc[kFeatures + f] / acc[2 * kFeatures] - mu * mu);
            nrm[f] = (float)mu;
            nrm[kIn + f] = var > 1e-12 ? (float)(1.0 / std::sqrt(var)) : 1.f;
        }
        if ((rc = check_cuda(cudaMemcpyAsync(M->norm, nrm.data(), sizeof(float) * 2 * kIn, cudaMemcpyHostToDevice, s),
                             "copy")) ||
            (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
            return rc;
    }
    const int64_t nb = N / batch;
    uint32_t* perm = alloc_n<uint32_t>(sc, N);
    float* dloss = alloc_n<float>(sc, nb);
    StepBuffers b;
    if (!perm || !dloss || step_buffers(ctx, batch, sc, b)) return RW_ERR_ALLOC;
    std::vector<uint32_t> hperm(rows);
    std::vector<float> hloss((size_t)nb);
    uint64_t st = seed;
    for (int32_t ep = 0; ep < epochs; ++ep) {
        // Fisher-Yates shuffle of the training rows (splitmix64 stream)
        for (int64_t i = N - 1; i > 0; --i) {
            const uint64_t j = splitmix64(st) % (uint64_t)(i + 1);
            std::swap(hperm[(size_t)i], hperm[(size_t)j]);
        }
        if ((rc = check_cuda(cudaMemcpyAsync(perm, hperm.data(), sizeof(uint32_t) * (size_t)N,
                                             cudaMemcpyHostToDevice, s),
                             "copy")))
            return rc;
        for (int64_t bi = 0; bi < nb; ++bi)
            if ((rc = mlp_step(ctx, M, d_feat, d_label, perm + bi * batch, batch, lr, true, dloss + bi, b)))
                return rc;
        // also orders the next epoch's shuffle after this epoch's upload
        if ((rc = check_cuda(cudaMemcpyAsync(hloss.data(), dloss, sizeof(float) * (size_t)nb, cudaMemcpyDeviceToHost, s),
                             "copy")) ||
            (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
            return rc;
        if (h_epoch_loss) {
            double l = 0.0;
            for (float v : hloss) l += v;
            h_epoch_loss[ep] = (float)(l / (double)(nb * batch));
        }
    }
    return check_cuda(cudaStreamSynchronize(s), "sync");
}

rw_status rw_budget_normalize(rw_context* ctx, const rw_csr* A, const float* d_weight, double mean_budget,
                              uint32_t min_budget, uint32_t* d_budget) {
    if (!ctx || !d_weight || !d_budget || min_budget < 1 || !(mean_budget >= (double)min_budget) ||
        !(mean_budget <= 2147483648.0)) {
        set_error("rw_budget_normalize: bad arguments (need 1 <= min_budget <= mean_budget <= 2^31)");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr_args(A, "rw_budget_normalize");
    if (rc || A->n == 0) return rc;
    Pool sc(ctx);
    return normalize_run(ctx, A, d_weight, mean_budget, min_budget, d_budget, sc);
}

rw_status rw_budget_predict(rw_context* ctx, const rw_csr* A, const rw_mlp* M, double mean_budget,
                            uint32_t min_budget, uint32_t* d_budget) {
    if (!ctx || !M || !d_budget || min_budget < 1 || !(mean_budget >= (double)min_budget) ||
        !(mean_budget <= 2147483648.0)) {
        set_error("rw_budget_predict: bad arguments (need 1 <= min_budget <= mean_budget <= 2^31)");
        return RW_ERR_ARG;
    }
    rw_status rc = check_csr_args(A, "rw_budget_predict");
    if (rc || A->n == 0) return rc;
    Pool sc(ctx);
    float* feat = alloc_n<float>(sc, (int64_t)A->n * kFeatStride);
    float* pred = alloc_n<float>(sc, A->n);
    if (!feat || !pred) return RW_ERR_ALLOC;
    if ((rc = reset_status(ctx))) return rc;
    if ((rc = features_run(ctx, A, feat))) return rc;
    RW_COUNT_LAUNCH();
    k_mlp_predict<<<grid_for(((int64_t)A->n + 15) / 16 * 32, 256, ctx->num_sms * 4), 256, 0, ctx->stream>>>(
        M->P, M->norm, feat, A->n, pred);
    if ((rc = check_launch("mlp predict"))) return rc;
    RW_COUNT_LAUNCH();
    k_exp_weights<<<grid_for(A->n, 256, ctx->num_sms * 4), 256, 0, ctx->stream>>>(A->n, pred, pred);
    if ((rc = check_launch("budget weights"))) return rc;
    if ((rc = read_status(ctx, "budget features"))) return rc;
    return normalize_run(ctx, A, pred, mean_budget, min_budget, d_budget, sc);
}

}  // extern "C"
