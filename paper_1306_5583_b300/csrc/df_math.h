// Double-float ("DF") arithmetic: a value is the unevaluated sum hi + lo of
// two floats (|lo| <= ulp(hi) / 2), about 48 significant bits, computed on
// the FP32 pipe.  FP64 runs at 1/64 of the FP32 rate on B300 and a single
// dependent float64 operation costs tens of nanoseconds (measured on B300:
// a fused multiply-add 33 ns, a division 225 ns, a logarithm 1.1 us), so the
// FP32 path keeps its reductions and its per-iteration scalar work in DF.
//
// Error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum and the
// FMA-based TwoProduct.  The logarithm uses log x = e ln 2 + 2 atanh(s),
// s = (m - 1)/(m + 1), m = x 2^-e in [sqrt(1/2), sqrt(2)), with the atanh
// series in DF for its leading terms (absolute error below 1e-13 for the
// arguments used here).  Host and device.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace smc {

struct DF {
    float hi, lo;
};

DF_HD float df_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

DF_HD uint32_t df_f2u(float x) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
#endif
}

DF_HD float df_u2f(uint32_t u) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float x;
    std::memcpy(&x, &u, 4);
    return x;
#endif
}

DF_HD DF fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return DF{s, b - (s - a)};
}
DF_HD DF two_sum(float a, float b) {
    const float s = a + b;
    const float bp = s - a;
    return DF{s, (a - (s - bp)) + (b - bp)};
}
DF_HD DF two_prod(float a, float b) {
    const float p = a * b;
    return DF{p, df_fma(a, b, -p)};
}
DF_HD DF df_add(DF a, DF b) {
    const DF s = two_sum(a.hi, b.hi);
    const DF t = two_sum(a.lo, b.lo);
    DF r = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(r.hi, r.lo + t.lo);
}
DF_HD DF df_add_f(DF a, float b) {
    const DF s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}
DF_HD DF df_mul(DF a, DF b) {
    const DF p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, p.lo + (a.hi * b.lo + a.lo * b.hi));
}
DF_HD DF df_mul_f(DF a, float b) {
    const DF p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, df_fma(a.lo, b, p.lo));
}
// float quotient for df_div: on the device the reciprocal-based quotient
// (2 ulp, |y| < 2^126 in every use here) instead of the correctly rounded
// division routine; df_div's correction from the exact remainder makes the
// result accurate to about 2^-45 either way
DF_HD float df_quot(float x, float y) {
#if defined(__CUDA_ARCH__)
    return __fdividef(x, y);
#else
    return x / y;
#endif
}

// a / b: float quotient plus one correction from the exact remainder
DF_HD DF df_div(DF a, DF b) {
    const float q1 = df_quot(a.hi, b.hi);
    const DF r = df_add(a, df_mul_f(DF{-b.hi, -b.lo}, q1));
    const float q2 = df_quot(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}
DF_HD bool df_lt(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// x = hi + lo exactly for an integer 0 <= x < 2^31
DF_HD DF df_from_int(int64_t x) {
    const float h = float((uint32_t)(x >> 8)) * 256.0f;  // exact: below 2^23 times a power of two
    const float l = float((uint32_t)(x & 255));
    return two_sum(h, l);
}

DF_HD int df_clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// the top 24 bits of x (x >> sh < 2^24) as an exact float
DF_HD float df_top24(uint64_t x, int sh) {
    return float((uint32_t)(x >> sh)) * df_u2f((uint32_t)(127 + sh) << 23);
}

// 64-bit unsigned integer as a DF value (relative error below 2^-47), by
// integer arithmetic and exact 24-bit conversions
DF_HD DF df_from_u64(uint64_t x) {
    if (x == 0) return DF{0.0f, 0.0f};
    const int sh = 40 - df_clz64(x) > 0 ? 40 - df_clz64(x) : 0;
    const float hi = df_top24(x, sh);
    const uint64_t rest = x - ((x >> sh) << sh);  // below 2^sh
    if (rest == 0) return DF{hi, 0.0f};
    const int sh2 = 40 - df_clz64(rest) > 0 ? 40 - df_clz64(rest) : 0;
    return fast_two_sum(hi, df_top24(rest, sh2));
}

// natural logarithm of a DF value with 2^-125 <= hi < 2^126
DF_HD DF df_log(DF x) {
    constexpr double kLn2 = 0.693147180559945309417232121458;
    constexpr float kLn2Hi = (float)kLn2;
    constexpr float kLn2Lo = (float)(kLn2 - (double)kLn2Hi);
    constexpr float kThirdHi = (float)(1.0 / 3.0);
    constexpr float kThirdLo = (float)(1.0 / 3.0 - (double)kThirdHi);
    constexpr float kFifthHi = (float)(1.0 / 5.0);
    constexpr float kFifthLo = (float)(1.0 / 5.0 - (double)kFifthHi);
    // x = 2^e m with m in [sqrt(1/2), sqrt(2)); lo scaled by the same power
    const uint32_t bits = df_f2u(x.hi);
    int e = (int)((bits >> 23) & 0xFF) - 127;
    uint32_t mb = (bits & 0x7FFFFFu) | 0x3F800000u;  // [1, 2)
    if (mb > 0x3FB504F3u) {                            // above sqrt(2): halve
        mb -= 0x00800000u;
        ++e;
    }
    const float m = df_u2f(mb);
    const float ml = x.lo * df_u2f((uint32_t)(127 - e) << 23);  // lo 2^-e
    // s = (m - 1) / (m + 1) in DF; m - 1 is exact (Sterbenz)
    const DF s = df_div(two_sum(m - 1.0f, ml), df_add_f(two_sum(m, 1.0f), ml));
    const DF s2 = df_mul(s, s);
    // atanh(s) = s + s^3 P(s^2), P = 1/3 + s^2 (1/5 + s^2 Q), Q in float
    // (|s| < 0.172: the float part contributes below 1e-13)
    const float z = s2.hi;
    const float Q =
        1.0f / 7.0f +
        z * (1.0f / 9.0f + z * (1.0f / 11.0f + z * (1.0f / 13.0f + z * (1.0f / 15.0f + z * (1.0f / 17.0f)))));
    const DF inner = df_add_f(DF{kFifthHi, kFifthLo}, z * Q);
    const DF P = df_add(DF{kThirdHi, kThirdLo}, df_mul(s2, inner));
    const DF t = df_add(s, df_mul(df_mul(s, s2), P));
    const float fe = float(e);
    const DF el = df_add(two_prod(fe, kLn2Hi), DF{fe * kLn2Lo, 0.0f});
    return df_add(el, DF{2.0f * t.hi, 2.0f * t.lo});
}

// float -> double bit pattern without a conversion instruction (normal,
// zero, infinite and NaN inputs; subnormals flush to signed zero)
DF_HD uint64_t df_f2d_bits(float x) {
    const uint32_t u = df_f2u(x);
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    const uint32_t ex = (u >> 23) & 0xFF;
    const uint64_t mant = (uint64_t)(u & 0x7FFFFFu) << 29;
    if (ex == 0) return sign;
    if (ex == 0xFF) return sign | (0x7FFull << 52) | mant;
    return sign | ((uint64_t)(ex - 127 + 1023) << 52) | mant;
}

// hi + lo rounded to a double: two bit-pattern conversions and one addition
DF_HD double df_to_double(DF a) {
    const uint64_t h = df_f2d_bits(a.hi), l = df_f2d_bits(a.lo);
    double dh, dl;
#if defined(__CUDA_ARCH__)
    dh = __longlong_as_double((long long)h);
    dl = __longlong_as_double((long long)l);
#else
    std::memcpy(&dh, &h, 8);
    std::memcpy(&dl, &l, 8);
#endif
    return dh + dl;
}

}  // namespace smc
