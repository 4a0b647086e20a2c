// rw_common.cuh -- device-side building blocks shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rw {

constexpr unsigned kFull = 0xffffffffu;

// Device-side error record, zeroed at the start of every library call and read
// back by the host before the call returns.
struct DevStatus {
    unsigned int bad_row;      // min over invalid rows of (row + 1); UINT_MAX = none
    unsigned int walk_cap;     // walks that reached the step cap
    unsigned int capacity;     // rows whose merge table would overflow
    unsigned int timeout;      // bounded waits that gave up
    unsigned int bad_budget;   // walk rows with a zero budget
    unsigned int breakdown;    // PCG p.Ap <= 0
    unsigned int nonfinite;    // non-finite right-hand-side entries
    unsigned int spin_limit;   // polls of one bounded wait before it gives up (set by the host)
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).  A round
// takes the 64-bit products of words 0 and 2 with the two Philox multipliers;
// the new words are (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1,
// lo(M0*x0)); the key advances by the two Weyl increments between rounds.
struct Philox4 {
    uint32_t v0, v1, v2, v3;
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a_lo = 0xD2511F53u * c0;
        const uint32_t a_hi = __umulhi(0xD2511F53u, c0);
        const uint32_t b_lo = 0xCD9E8D57u * c2;
        const uint32_t b_hi = __umulhi(0xCD9E8D57u, c2);
        c0 = b_hi ^ c1 ^ k0;
        c1 = b_lo;
        c2 = a_hi ^ c3 ^ k1;
        c3 = a_lo;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return Philox4{c0, c1, c2, c3};
}

// Sampling threshold of a cumulative probability num/den (Sec. 2.1, Eq. map):
// min(2^32 - 1, floor(2^32 * fl(num / den))).  One IEEE division, an exact
// power-of-two scaling and a truncating conversion.
__device__ __forceinline__ uint32_t cumulative_threshold(double num, double den) {
    const double s = __dmul_rn(__ddiv_rn(num, den), 4294967296.0);
    return (s < 4294967295.0) ? __double2uint_rz(s) : 0xFFFFFFFFu;
}

// Relaxed (gpu-scope) accesses used for device-side hand-off between warps.
// The value itself is the signal (a single aligned store), so the loads need
// no ordering against other memory operations: no "memory" clobber, which
// lets independent loads around them be issued together.
__device__ __forceinline__ double ld_relaxed(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_relaxed(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void ld_relaxed_v2(const double* p, double& a, double& b) {
    asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p));
}
__device__ __forceinline__ void ld_relaxed_v4(const float* p, float& a, float& b, float& c, float& d) {
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(a), "=f"(b), "=f"(c), "=f"(d)
                 : "l"(p));
}
__device__ __forceinline__ void st_relaxed(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(int* p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bit patterns marking "not yet computed" in the sync-free triangular solves.
// They are NaN payloads that arithmetic never produces (GPU arithmetic returns
// the canonical NaN), and inputs are checked to be finite.
__device__ __forceinline__ double pending_value(double) {
    return __longlong_as_double(0x7FF4C0DEC0DE0001LL);
}
__device__ __forceinline__ float pending_value(float) { return __int_as_float(0x7FA0C0DE); }
__device__ __forceinline__ bool is_pending(double v) {
    return __double_as_longlong(v) == 0x7FF4C0DEC0DE0001LL;
}
__device__ __forceinline__ bool is_pending(float v) { return __float_as_int(v) == 0x7FA0C0DE; }

// Default upper bound on polls of one device-side wait before it gives up
// (about a second at L2 latency; rw_options.spin_limit overrides it, and the
// host passes the value in DevStatus::spin_limit).  Once any wait gives up, the
// others see the timeout flag within kAbortPoll polls and give up too, so a
// failing solve ends after about one wait limit in total.
constexpr unsigned kSpinLimit = 1u << 20;
constexpr unsigned kAbortPoll = 1024;

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One poll step of a bounded wait of at most `limit` polls: returns true when
// the wait must give up.
__device__ __forceinline__ bool wait_gives_up(unsigned& spins, unsigned limit, unsigned* timeout_flag) {
    ++spins;
    if (spins > limit) {
        atomicAdd(timeout_flag, 1u);
        return true;
    }
    return (spins % kAbortPoll) == 0 && ld_relaxed_u32(timeout_flag) != 0u;
}

// Software grid barrier for a co-resident (cooperatively launched) grid:
// *count (zero at launch) only grows; barrier number `epoch` (1, 2, ...) is
// passed once it reaches epoch * gridDim.x.  One thread per block arrives
// with a release atomic (cumulative over the block's stores, ordered by the
// preceding __syncthreads) and polls with acquire loads, so a barrier costs
// about two L2 round trips and no reset.  Every wait is bounded; returns false
// when it gave up (the timeout flag is then set).
__device__ __forceinline__ unsigned atom_add_release(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned epoch, DevStatus* st) {
    __shared__ int give_up;
    __syncthreads();
    if (threadIdx.x == 0) {
        give_up = 0;
        const unsigned target = epoch * gridDim.x;
        const unsigned limit = st->spin_limit;
        atom_add_release(count, 1u);
        unsigned spins = 0;
        while (ld_acquire_u32(count) < target) {
            if (wait_gives_up(spins, limit, &st->timeout)) {
                give_up = 1;
                break;
            }
        }
    }
    __syncthreads();
    return give_up == 0;
}

// Sums of NR per-lane values over the warp (NR a power of two, <= 16).  Each
// step hands half of the still-carried values to the partner lane, so NR = 4
// costs 7 shuffles instead of 4 x 5.  warp_sums_spread leaves the total of
// value j in lanes j * 32/NR ... j * 32/NR + 32/NR - 1; warp_sums moves it to
// lane j (j < NR).
template <typename T, int NR>
__device__ __forceinline__ T warp_sums_spread(T (&v)[NR]) {
    const unsigned lane = lane_id();
    int cnt = NR;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
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
    return v[0];
}

template <typename T, int NR>
__device__ __forceinline__ T warp_sums(T (&v)[NR]) {
    const T s = warp_sums_spread<T, NR>(v);
    constexpr int shift = NR >= 16 ? 1 : NR >= 8 ? 2 : NR >= 4 ? 3 : NR >= 2 ? 4 : 5;
    return __shfl_sync(kFull, s, ((int)lane_id() << shift) & 31);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

}  // namespace rw
