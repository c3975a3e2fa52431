// Exact 64-bit thresholds of the grid targets of systematic and stratified
// resampling (host and device).
//
// Ancestor k is a_k = min{ i : Q_i D > Q_N P_k } with D = N 2^25 and
// P_k = 2^25 k + c_k (c_k = 2 j_k + 1 odd, below 2^25).  For an integer Q_i,
// Q_i D > X holds exactly when Q_i > floor(X / D), so the selection only needs
// the 64-bit threshold
//     tau_k = floor(Q_N (2^25 k + c_k) / (N 2^25)),
// which is computed here without 128-bit arithmetic.  With Q_N = a N + b,
// a c_k = H 2^25 + L and k b = u N + v (0 <= b, v < N, 0 <= L < 2^25):
//     tau_k = k a + H + u + floor((2^25 v + L N + c_k b) / (N 2^25)),
// and the last numerator is below 3 N 2^25, so that term is 0, 1 or 2.
// (u, v) advance from k to k + 1 by one addition of b and at most one
// carry; for a fixed c_k (systematic) tau itself advances with a remainder
// modulo D.  Bounds: N < 2^31, Q_N < 2^62.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define SMC_HD __host__ __device__ __forceinline__
#else
#define SMC_HD inline
#endif

namespace smc {

SMC_HD uint64_t umulhi64(uint64_t x, uint64_t y) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(x, y);
#else
    return (uint64_t)(((unsigned __int128)x * y) >> 64);
#endif
}

struct GridDiv {
    uint64_t n;     // N
    uint64_t a, b;  // Q_N = a N + b
    uint64_t mrec;  // floor((2^64 - 1) / N): floor(x / N) for x < 2^62 up to one correction
    uint64_t ah, al;  // a = ah 2^25 + al

    // mrec_ = floor((2^64 - 1) / N) (host-computed: no device division)
    SMC_HD void init(uint64_t qn, uint64_t n_, uint64_t mrec_) {
        n = n_;
        mrec = mrec_;
        a = umulhi64(qn, mrec);  // floor(qn / N) or one less
        b = qn - a * n;
        if (b >= n) {
            b -= n;
            ++a;
        }
        ah = a >> 25;
        al = a & ((1ull << 25) - 1);
    }
    // k b = u N + v
    SMC_HD void start(uint64_t k, uint64_t &u, uint64_t &v) const {
        const uint64_t kb = k * b;  // < 2^62
        u = umulhi64(kb, mrec);     // floor(kb / N) or one less
        v = kb - u * n;
        if (v >= n) {
            v -= n;
            ++u;
        }
    }
    // (u, v) of k -> (u, v) of k + 1
    SMC_HD void next(uint64_t &u, uint64_t &v) const {
        v += b;
        if (v >= n) {
            v -= n;
            ++u;
        }
    }
    // tau_k from (u, v) of k and c_k; *rem = Q_N P_k - tau_k D (in [0, D))
    SMC_HD uint64_t tau(uint64_t k, uint64_t c, uint64_t u, uint64_t v, uint64_t *rem = nullptr) const {
        const uint64_t alc = al * c;               // < 2^50
        const uint64_t H = ah * c + (alc >> 25);   // floor(a c / 2^25)
        const uint64_t L = alc & ((1ull << 25) - 1);
        const uint64_t D = n << 25;
        const uint64_t X = (v << 25) + L * n + c * b;  // < 3 D
        const uint64_t r = (X >= D ? 1ull : 0ull) + (X >= 2 * D ? 1ull : 0ull);
        if (rem) *rem = X - r * D;
        return k * a + H + u + r;
    }
    // Systematic targets (c fixed): Q_N P_{k+1} = Q_N P_k + a D + b 2^25, so
    // (tau, rem) advance by a and b 2^25 with at most one carry (b 2^25 < D).
    SMC_HD void advance(uint64_t &t, uint64_t &rem) const {
        const uint64_t D = n << 25;
        t += a;
        rem += b << 25;
        if (rem >= D) {
            rem -= D;
            ++t;
        }
    }
};

}  // namespace smc
