// Device-side building blocks of the SMC hot path (sm_103a).
//
// * Philox4x32-10 (Salmon et al., SC'11), written from its published
//   definition: per round, two 32x32->64 products of counter words 0 and 2
//   with M0 = 0xD2511F53 and M1 = 0xCD9E8D57, xor with the other counter words
//   and the key; the key advances by the Weyl constants 0x9E3779B9 and
//   0xBB67AE85 between rounds.  The paper gives each particle an independent
//   counter-based stream (Sec. 3.4); here the stream of a particle is its
//   counter (index, iteration, tag | stream_id << 16, draw).
// * uniform u = (j + 1) 2^-24 with j = x >> 8 (exact in float and double),
//   Box-Muller normals, warp/block reductions, 128-bit comparisons for the
//   fixed-point resampling targets.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "smc_layout.h"

namespace smc {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32 -> 64-bit product gives both halves
        const unsigned long long p0 = (unsigned long long)kPhiloxM0 * c.x;
        const unsigned long long p1 = (unsigned long long)kPhiloxM1 * c.z;
        const uint32_t kx = k.x + (uint32_t)r * kPhiloxW0, ky = k.y + (uint32_t)r * kPhiloxW1;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ kx, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ ky, (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint2 key, uint32_t index, uint32_t t, uint32_t tag,
                                      uint32_t stream, uint32_t d) {
    return philox4x32_10(make_uint4(index, t, (tag & 0xFFFFu) | (stream << 16), d), key);
}

__device__ __forceinline__ uint32_t u24(uint32_t x) { return x >> 8; }

template <typename R>
__device__ __forceinline__ R uniform01(uint32_t x) {
    return R((x >> 8) + 1u) * R(5.9604644775390625e-08);  // (j + 1) 2^-24
}

// ---- precision traits -------------------------------------------------------
template <typename R>
struct Math;

template <>
struct Math<float> {
    static __device__ __forceinline__ float exp(float x) { return expf(x); }
    static __device__ __forceinline__ float fast_exp(float x) { return __expf(x); }
    static __device__ __forceinline__ float fast_log(float x) { return __logf(x); }
    static __device__ __forceinline__ float log(float x) { return logf(x); }
    static __device__ __forceinline__ float log1p(float x) { return log1pf(x); }
    static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
    static __device__ __forceinline__ void sincospi(float x, float *s, float *c) { sincospif(x, s, c); }
    static __device__ __forceinline__ uint64_t fixed(float e, int frac) {
        // floor(e 2^frac) for e in [0, 1] (frac <= 61); NaN and negatives map
        // to 0.  Integer bit arithmetic on the float's fields: the value is
        // mant 2^(ex - 150), shifted by frac; no float-to-64-bit conversion
        // (that runs on the slow FP64 pipe).
        if (!(e > 0.0f)) return 0ull;
        const uint32_t bits = __float_as_uint(e);
        const int ex = (int)(bits >> 23);
        const uint64_t mant = (uint64_t)((bits & 0x7FFFFFu) | 0x800000u);
        const int sh = ex - 150 + frac;
        if (ex == 0) return 0ull;  // subnormal: below 2^-126, floor is 0 for frac <= 61
        if (sh >= 0) return mant << sh;
        return sh > -32 ? (mant >> (-sh)) : 0ull;
    }
    static __device__ __forceinline__ float neg_inf() { return -__int_as_float(0x7f800000); }
};

template <>
struct Math<double> {
    static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
    static __device__ __forceinline__ double fast_exp(double x) { return ::exp(x); }
    static __device__ __forceinline__ double fast_log(double x) { return ::log(x); }
    static __device__ __forceinline__ double log(double x) { return ::log(x); }
    static __device__ __forceinline__ double log1p(double x) { return ::log1p(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ void sincospi(double x, double *s, double *c) { ::sincospi(x, s, c); }
    static __device__ __forceinline__ uint64_t fixed(double e, int frac) {
        return (e > 0.0) ? __double2ull_rz(ldexp(e, frac)) : 0ull;
    }
    static __device__ __forceinline__ double neg_inf() { return -__longlong_as_double(0x7ff0000000000000ll); }
};

// 1 / x: the reciprocal-based float quotient (2 ulp; x within the normal
// range) on the FP32 path instead of the correctly rounded division
// routine, exact division in float64
template <typename R>
__device__ __forceinline__ R fast_rcp(R x) {
    if constexpr (sizeof(R) == 4) return __fdividef(1.0f, x);
    else return R(1) / x;
}

// Box-Muller pair from two uniforms in (0, 1]: z0 = r cos(2 pi u1),
// z1 = r sin(2 pi u1), r = sqrt(-2 ln u0).
template <typename R>
__device__ __forceinline__ void box_muller(R u0, R u1, R &z0, R &z1) {
    const R r = Math<R>::sqrt(R(-2) * Math<R>::log(u0));
    R s, c;
    Math<R>::sincospi(R(2) * u1, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// -2 ln u for u in [2^-24, 1] (the uniforms of uniform01): u = 2^e m with
// m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s), s = (m - 1) / (m + 1),
// |s| < 0.172, atanh s = s (1 + s^2/3 + s^4/5 + s^6/7) with a relative
// truncation error below 2^-25.  m - 1 is exact, so the result keeps a
// relative error of a few 2^-23 also near u = 1, where it is small and the
// hardware logarithm's absolute error would dominate sqrt(-2 ln u); no
// special cases arise on this domain.
__device__ __forceinline__ float neg2_log_unit(float u) {
    const int bits = __float_as_int(u);
    const int e = (bits - 0x3F3504F3) >> 23;  // 0x3F3504F3 = sqrt(1/2); arithmetic shift
    const float m = __int_as_float(bits - (e << 23));
    const float s = __fdividef(m - 1.0f, m + 1.0f);
    const float s2 = s * s;
    const float p = fmaf(s2, fmaf(s2, fmaf(s2, 1.0f / 7.0f, 1.0f / 5.0f), 1.0f / 3.0f), 1.0f);
    return fmaf(-1.38629436111989061883f, float(e), -4.0f * s * p);  // -2 (e ln 2 + 2 s p)
}

// FP32 Box-Muller on the MUFU pipe: the angle is taken in (-pi, pi], where
// the hardware sine/cosine are accurate to about 2^-21 absolute, using
// cos(2 pi u) = -cos(2 pi u - pi) and sin(2 pi u) = -sin(2 pi u - pi).
__device__ __forceinline__ void box_muller_fast(float u0, float u1, float &z0, float &z1) {
    const float r2 = neg2_log_unit(u0);
    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));  // sqrt on the MUFU pipe (r2 = 0 gives 0)
    const float th = fmaf(6.2831853071795864769f, u1, -3.14159265358979323846f);
    float s, c;
    __sincosf(th, &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}

// Four standard normals from one Philox call: (w0, w1) -> z0, z1; (w2, w3) -> z2, z3.
template <typename R>
__device__ __forceinline__ void normals4(uint4 w, R z[4]) {
    box_muller(uniform01<R>(w.x), uniform01<R>(w.y), z[0], z[1]);
    box_muller(uniform01<R>(w.z), uniform01<R>(w.w), z[2], z[3]);
}

// Same draws with the MUFU-pipe transforms for float (the hot loops).
template <typename R>
__device__ __forceinline__ void normals4_fast(uint4 w, R z[4]) {
    if constexpr (sizeof(R) == 4) {
        box_muller_fast(uniform01<float>(w.x), uniform01<float>(w.y), z[0], z[1]);
        box_muller_fast(uniform01<float>(w.z), uniform01<float>(w.w), z[2], z[3]);
    } else {
        normals4<R>(w, z);
    }
}

// ---- vector loads of K consecutive elements ----------------------------------
// Thread-contiguous items let every load be a 16-byte vector load; a partial
// group (the ragged tail) falls back to guarded scalar loads.  Loads go
// through L2 (ld.global.cg): the persistent iteration kernel reads data that
// other blocks wrote earlier in the same launch, which a per-SM L1 copy could
// hold stale.
template <typename R, int K>
__device__ __forceinline__ void load_k(const R *__restrict__ p, uint32_t i0, uint32_t n, R (&v)[K]) {
    static_assert((K * sizeof(R)) % 16 == 0, "vector width");
    if (i0 + K <= n) {
        const float4 *q = reinterpret_cast<const float4 *>(p + i0);
#pragma unroll
        for (int c = 0; c < (int)(K * sizeof(R) / 16); ++c) {
            const float4 w = __ldcg(q + c);
            reinterpret_cast<float4 *>(v)[c] = w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) v[j] = (i0 + j < n) ? __ldcg(p + i0 + j) : R(0);
    }
}

template <typename R, int K>
__device__ __forceinline__ void store_k(R *__restrict__ p, uint32_t i0, uint32_t n, const R (&v)[K]) {
    if (i0 + K <= n) {
        float4 *q = reinterpret_cast<float4 *>(p + i0);
#pragma unroll
        for (int c = 0; c < (int)(K * sizeof(R) / 16); ++c) q[c] = reinterpret_cast<const float4 *>(v)[c];
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (i0 + j < n) p[i0 + j] = v[j];
    }
}

__device__ __forceinline__ void load_idx4(const int32_t *__restrict__ p, uint32_t i0, uint32_t n, int32_t (&v)[4]) {
    if (i0 + 4 <= n) {
        const int4 w = __ldcg(reinterpret_cast<const int4 *>(p + i0));
        v[0] = w.x;
        v[1] = w.y;
        v[2] = w.z;
        v[3] = w.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (i0 + j < n) ? __ldcg(p + i0 + j) : 0;
    }
}

// ---- reductions -------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// inclusive warp scan of 64-bit unsigned values
__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// ---- 128-bit helpers for the rational resampling targets --------------------
struct U128 {
    uint64_t hi, lo;
};

__device__ __forceinline__ U128 mul64(uint64_t a, uint64_t b) { return U128{__umul64hi(a, b), a * b}; }

// a > b
__device__ __forceinline__ bool gt128(U128 a, U128 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }


// bit length of a 128-bit value
__device__ __forceinline__ int bitlen128(U128 a) {
    return a.hi ? 128 - __clzll((long long)a.hi) : (a.lo ? 64 - __clzll((long long)a.lo) : 0);
}

// ---- bounded spin (never waits forever: sets the error word and gives up) --
__device__ __forceinline__ void raise_error(DevState *st, int code) { atomicCAS(&st->error, 0, code); }

// Polls a bounded wait makes before it gives up (kSpinLimit unless
// smc_set_wait_limit changed it on this device).
__constant__ uint32_t c_wait_limit = kSpinLimit;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t atom_add_release_u32(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Barrier over the whole grid of a cooperative launch (every block resident
// at once).  Thread 0 publishes the block's writes and counts its arrival,
// then polls with acquire loads, at most c_wait_limit times; on timeout it
// raises SMC_E_TIMEOUT and the block gives up (returns false).  The k-th
// barrier of a launch waits for k * gridDim.x arrivals (target); the counter
// starts at zero and grid_depart() clears it at the end of the launch.
__device__ __forceinline__ bool grid_barrier(DevState *st, uint32_t target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        atom_add_release_u32(&st->grid_count, 1u);
        uint32_t it = 0;
        bool ok = true;
        while (ld_acquire_u32(&st->grid_count) < target) {
            if (++it >= c_wait_limit) {
                ok = false;
                break;
            }
            __nanosleep(32);
        }
        if (!ok) raise_error(st, SMC_E_TIMEOUT);
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    return s_ok != 0;
}
// After the barrier: the last block to leave clears the counters for the
// next launch (every block has passed its wait by then).
__device__ __forceinline__ void grid_depart(DevState *st) {
    __syncthreads();
    if (threadIdx.x == 0 && atom_add_release_u32(&st->grid_depart, 1u) == gridDim.x - 1) {
        st->grid_count = 0;
        st->grid_depart = 0;
    }
}

// Copy of the device state block in shared memory, read once per block:
// every block of a kernel reads the same few words, and letting every warp
// load them serialises on one L2 line.  Writes still go to the global block.
// Must be called by all threads of the block.
// first_use: the block takes no other snapshot in this launch (no barrier
// needed before the copy).
__device__ __forceinline__ const DevState *snapshot(const DevState *st, bool first_use = false) {
    __shared__ __align__(16) DevState s_st;
    constexpr int W = (int)(sizeof(DevState) / 4);
    static_assert(sizeof(DevState) % 4 == 0, "DevState size");
    if (!first_use) __syncthreads();  // a previous snapshot in the same block may still be read
    const uint32_t *src = reinterpret_cast<const uint32_t *>(st);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&s_st);
    for (int i = threadIdx.x; i < W; i += blockDim.x) dst[i] = __ldcg(src + i);
    __syncthreads();
    return &s_st;
}

}  // namespace smc
