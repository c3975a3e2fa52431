// Block partials and the last-block grid combine shared by every kernel
// that produces new log-weights: online (max, sum e, sum e^2, sum e*h)
// with e = exp(lw - max), then log-normaliser, ESS, evidence increment,
// monitor and the resample decision (Sec. 2.1 ESS; Sec. 2.2 ratio of
// normalising constants; Sec. 4.1.5 Monitor; Sec. 4.1.3 threshold).
#pragma once

#include "df_math.h"
#include "smc_device.cuh"

namespace smc {

// Subtract a float64 scalar from a value of precision R with one rounding
// less than a plain conversion (hi/lo split of the scalar).
template <typename R>
struct Shift {
    R hi, lo;
    __device__ __forceinline__ explicit Shift(double v) : hi(R(v)), lo(R(v - double(R(v)))) {}
    __device__ __forceinline__ Shift(R h, R l) : hi(h), lo(l) {}
    __device__ __forceinline__ R sub_from(R x) const { return (x - hi) - lo; }
};

// The split of L_t kept in the state block (written once by the finalising
// thread), so per-thread code does no float64 arithmetic or conversion.
template <typename R>
__device__ __forceinline__ Shift<R> log_norm_shift(const DevState *sv) {
    if constexpr (sizeof(R) == 4) return Shift<R>(sv->log_norm_f[0], sv->log_norm_f[1]);
    else return Shift<R>(R(sv->log_norm), R(0));
}

// float split of a float64 value: hi + lo with hi = float(v)
__device__ __forceinline__ void split_float(double v, float *out) {
    out[0] = float(v);
    out[1] = float(v - double(out[0]));
}

// What the last block does with the combined sums.
struct FinalizeArgs {
    DevState *st;
    smc_record *rec;
    int32_t rec_cap;
    int32_t t;            // iteration whose weights were just computed
    int32_t mode;         // 0: new iteration (flip buffers), 1: reweight of iteration t in place
    int64_t n;
    double threshold;
    double alpha;         // GMM alpha_t (recorded)
    float thr_df[2];      // FP32 path: the threshold as a DF value
    int32_t thr_mode;     // FP32 path: 0 compare ESS < threshold N, 1 always, 2 never
    double log_evidence_prev;  // FP32 path, mode 0: log Z_{t-1} from the kernel's state snapshot
};

// ---- compensated float ("double-float") sums: see df_math.h ---------------
__device__ __forceinline__ DF df_shfl_xor(DF a, int o) {
    return DF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Per-block partial (max, sum e, sum e^2, sum e h0, sum e h1) with
// e = exp(lw - max): float64 fields for the FP64 path; for the FP32 path the
// (hi, lo) float pairs of the four sums in floats 0..7 (two 16-byte vectors)
// and the maximum in float 8, in the same 64 bytes.
constexpr int kSums = 4;

template <typename R>
struct PartialIO;

template <>
struct PartialIO<double> {
    static __device__ __forceinline__ void store(Partial *p, double m, const double (&s)[kSums]) {
        p->m = m;
        p->s1 = s[0];
        p->s2 = s[1];
        p->sx = s[2];
        p->sy = s[3];
        p->su = 0.0;
    }
};

template <>
struct PartialIO<float> {
    static __device__ __forceinline__ void store(Partial *p, float m, const DF (&s)[kSums]) {
        float4 *v = reinterpret_cast<float4 *>(p);
        v[0] = make_float4(s[0].hi, s[0].lo, s[1].hi, s[1].lo);
        v[1] = make_float4(s[2].hi, s[2].lo, s[3].hi, s[3].lo);
        reinterpret_cast<float *>(p)[8] = m;
    }
    static __device__ __forceinline__ float m(const Partial *p) { return __ldcg(reinterpret_cast<const float *>(p) + 8); }
    static __device__ __forceinline__ DF s(const Partial *p, int j) {
        const float *f = reinterpret_cast<const float *>(p);
        return DF{__ldcg(f + 2 * j), __ldcg(f + 2 * j + 1)};
    }
};

// Explicitly rounded multiply, add and fused multiply-add: the reductions
// spell out which products are fused, so every kernel that inlines them
// (a plain filter, the batched filters) rounds the same way.
template <typename R>
__device__ __forceinline__ R fma_x(R a, R b, R c) {
    if constexpr (sizeof(R) == 4) return __fmaf_rn(a, b, c);
    else return __fma_rn(a, b, c);
}
template <typename R>
__device__ __forceinline__ R mul_x(R a, R b) {
    if constexpr (sizeof(R) == 4) return __fmul_rn(a, b);
    else return __dmul_rn(a, b);
}
template <typename R>
__device__ __forceinline__ R add_x(R a, R b) {
    if constexpr (sizeof(R) == 4) return __fadd_rn(a, b);
    else return __dadd_rn(a, b);
}

// Four warp sums at once: at the first two butterfly levels each lane keeps
// half of its values and adds its partner's copy of that half (a transpose
// reduce), so 6 shuffles replace 20; lane 8q (q < 4) ends with the sum of
// value q.
template <typename R>
__device__ __forceinline__ R warp_sum4(R v0, R v1, R v2, R v3) {
    const int lane = threadIdx.x & 31;
    const bool up = lane & 16, hi8 = lane & 8;
    const R a = (up ? v2 : v0) + __shfl_xor_sync(0xffffffffu, up ? v0 : v2, 16);
    const R b = (up ? v3 : v1) + __shfl_xor_sync(0xffffffffu, up ? v1 : v3, 16);
    R x = (hi8 ? b : a) + __shfl_xor_sync(0xffffffffu, hi8 ? a : b, 8);
    x += __shfl_xor_sync(0xffffffffu, x, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    return x;
}

// The same transpose reduce for four double-float sums: lanes 8q .. 8q + 7
// end with the warp total of sum q (six double-float additions per lane
// instead of twenty for four separate trees).
__device__ __forceinline__ DF df_warp_sum4(DF v0, DF v1, DF v2, DF v3) {
    const int lane = threadIdx.x & 31;
    const bool up = lane & 16, hi8 = lane & 8;
    const DF a = df_add(up ? v2 : v0, df_shfl_xor(up ? v0 : v2, 16));
    const DF b = df_add(up ? v3 : v1, df_shfl_xor(up ? v1 : v3, 16));
    DF x = df_add(hi8 ? b : a, df_shfl_xor(hi8 ? a : b, 8));
    x = df_add(x, df_shfl_xor(x, 4));
    x = df_add(x, df_shfl_xor(x, 2));
    x = df_add(x, df_shfl_xor(x, 1));
    return x;
}

// Block-level partial of E items per thread.  lw = -inf marks inactive
// items.  Each warp reduces its own maximum m_w and its sums of
// e = exp(lw - m_w) in R (no block barrier), then one barrier hands the
// warp partials to warp 0, which rescales them by exp(m_w - M) to the block
// maximum M and adds them, in R: the per-warp sums already carry R's
// rounding, so wider arithmetic across the eight warps adds nothing (the
// FP32 partial's low words are zero; the grid combine is compensated).
// Warp 0 stores the partial (lane 0), so a grid ticket taken right after by
// thread 0 follows the partial in program order and the block's other
// writes through the barrier.
template <typename R, int E, int NH = 2>
__device__ __forceinline__ void block_partial(const R (&lw)[E], const R (&h0)[E], const R (&h1)[E],
                                              const R (&h2)[E], Partial *out) {
    // NH: how many of h0, h1 are monitored (the rest is reported as 0; h2 is unused)
    static_assert(NH >= 0 && NH <= 2, "at most two monitored values");
    constexpr int NW = kBlock / 32;
    __shared__ R s_max[NW];
    __shared__ R s_sum[NW][kSums];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    R m = Math<R>::neg_inf();
#pragma unroll
    for (int j = 0; j < E; ++j) m = fmax(m, lw[j]);
    m = warp_max(m);
    R v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    if (m > Math<R>::neg_inf()) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const R e = (lw[j] > Math<R>::neg_inf()) ? Math<R>::fast_exp(lw[j] - m) : R(0);
            v0 = add_x(v0, e);
            v1 = fma_x(e, e, v1);
            if (NH > 0) v2 = fma_x(e, h0[j], v2);
            if (NH > 1) v3 = fma_x(e, h1[j], v3);
        }
    }
    const R x = warp_sum4(v0, v1, v2, v3);
    if ((lane & 7) == 0) s_sum[warp][lane >> 3] = x;
    if (lane == 0) s_max[warp] = m;
    __syncthreads();
    if (warp != 0) return;
    const R mw = lane < NW ? s_max[lane] : Math<R>::neg_inf();
    R M = mw;
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) M = fmax(M, __shfl_xor_sync(0xffffffffu, M, o));
    const R sc = (mw > Math<R>::neg_inf()) ? Math<R>::fast_exp(mw - M) : R(0);
    R t[kSums];
#pragma unroll
    for (int q = 0; q < kSums; ++q) {
        const R w = lane < NW ? s_sum[lane][q] : R(0);
        t[q] = (q == 1) ? mul_x(mul_x(w, sc), sc) : mul_x(w, sc);
    }
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < kSums; ++q) t[q] += __shfl_xor_sync(0xffffffffu, t[q], o);
    if (lane == 0) {
        if constexpr (sizeof(R) == 8) {
            PartialIO<double>::store(out, M, t);
        } else {
            const DF d[kSums] = {DF{t[0], 0.0f}, DF{t[1], 0.0f}, DF{t[2], 0.0f}, DF{t[3], 0.0f}};
            PartialIO<float>::store(out, M, d);
        }
    }
}

// Returns true in the one block that arrives last; that block then holds
// the grid-wide sums in *out (thread 0 only).
struct Combined {
    double M, S1, S2, Sa, Sb, Sc;
};

// Block-level "am I the last of `count` arrivals" on a counter (the
// counter is reset by the caller's finalisation).  The block barrier orders
// the block's writes before thread 0's arrival, an acquire-release atomic
// (no sequentially consistent fence) publishes them, and the last arrival's
// acquire plus the barrier make every block's writes visible to the whole
// last block (which reads them through L2).
__device__ __forceinline__ unsigned atomic_add_acq_rel(uint32_t *p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ bool last_arrival(uint32_t *counter, uint32_t count) {
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomic_add_acq_rel(counter, 1u) == count - 1);
    __syncthreads();
    return s_last;
}

template <typename R>
__device__ __forceinline__ bool take_ticket(DevState *st) {
    return last_arrival(&st->ticket, gridDim.x);
}

// last_arrival for a block that has just run block_partial: that function's
// barrier already orders the block's writes before thread 0, which stored
// the partial itself, so thread 0 arrives at once and one barrier
// broadcasts the answer.
__device__ __forceinline__ bool last_arrival_after_partial(uint32_t *counter, uint32_t count) {
    __shared__ bool s_last;
    if (threadIdx.x == 0) s_last = (atomic_add_acq_rel(counter, 1u) == count - 1);
    __syncthreads();
    return s_last;
}

// FP32 path: grid-wide sums of nb block partials in compensated float, by
// the whole calling block (every thread receives the result).  Each thread
// fetches its partials (b = tid + r kBlock: two 16-byte vectors and the
// maximum each) in one round trip when nb <= PT kBlock, the block maximum
// rescales them, and fixed shuffle trees add them, so the result does not
// depend on arrival order (nor on PT).
struct CombinedDF {
    float M;
    DF S[kSums];
};

// PT: partials fetched per thread in the single round trip (9 registers
// each); the result does not depend on PT.
template <int PT = 4>
__device__ __forceinline__ void combine_partials_df(const Partial *part, int nb, CombinedDF *out) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ float s_m[kBlock / 32];
    __shared__ DF s_df[kBlock / 32][kSums];
    __shared__ CombinedDF s_out;
    const bool one_pass = nb <= PT * kBlock;
    float mm[PT];
    float4 va[PT], vb[PT];
    float M = -INFINITY;
    if (one_pass) {
#pragma unroll
        for (int r = 0; r < PT; ++r) {
            const int b = r * kBlock + tid;
            if (b < nb) {
                const float4 *src = reinterpret_cast<const float4 *>(&part[b]);
                va[r] = __ldcg(src);
                vb[r] = __ldcg(src + 1);
                mm[r] = PartialIO<float>::m(&part[b]);
            } else {
                va[r] = vb[r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                mm[r] = -INFINITY;
            }
            M = fmaxf(M, mm[r]);
        }
    } else {
        for (int b = tid; b < nb; b += kBlock) M = fmaxf(M, PartialIO<float>::m(&part[b]));
    }
    M = warp_maxf(M);
    if (lane == 0) s_m[warp] = M;
    __syncthreads();
    M = s_m[0];
#pragma unroll
    for (int w = 1; w < kBlock / 32; ++w) M = fmaxf(M, s_m[w]);
    DF S[kSums];
#pragma unroll
    for (int q = 0; q < kSums; ++q) S[q] = DF{0.0f, 0.0f};
    if (M > -INFINITY) {
        if (one_pass) {
#pragma unroll
            for (int r = 0; r < PT; ++r) {
                const float sc = (mm[r] > -INFINITY) ? expf(mm[r] - M) : 0.0f;
                S[0] = df_add(S[0], df_mul_f(DF{va[r].x, va[r].y}, sc));
                S[1] = df_add(S[1], df_mul_f(df_mul_f(DF{va[r].z, va[r].w}, sc), sc));
                S[2] = df_add(S[2], df_mul_f(DF{vb[r].x, vb[r].y}, sc));
                S[3] = df_add(S[3], df_mul_f(DF{vb[r].z, vb[r].w}, sc));
            }
        } else {
            for (int b = tid; b < nb; b += kBlock) {
                const float mb = PartialIO<float>::m(&part[b]);
                const float sc = (mb > -INFINITY) ? expf(mb - M) : 0.0f;
                S[0] = df_add(S[0], df_mul_f(PartialIO<float>::s(&part[b], 0), sc));
                S[1] = df_add(S[1], df_mul_f(df_mul_f(PartialIO<float>::s(&part[b], 1), sc), sc));
#pragma unroll
                for (int q = 2; q < kSums; ++q) S[q] = df_add(S[q], df_mul_f(PartialIO<float>::s(&part[b], q), sc));
            }
        }
    }
    // the warp's four sums by a transpose reduce: lanes 8q .. 8q + 7 hold sum q
    static_assert(kSums == 4 && kBlock / 32 == 8, "four sums, eight warps");
    const DF x = df_warp_sum4(S[0], S[1], S[2], S[3]);
    if ((lane & 7) == 0) s_df[warp][lane >> 3] = x;
    __syncthreads();
    if (warp == 0) {
        // one value per lane (lane 8q + w: sum q of warp w), reduced within
        // each group of eight lanes
        DF y = s_df[lane & 7][lane >> 3];
        y = df_add(y, df_shfl_xor(y, 4));
        y = df_add(y, df_shfl_xor(y, 2));
        y = df_add(y, df_shfl_xor(y, 1));
        if ((lane & 7) == 0) s_out.S[lane >> 3] = y;
        if (lane == 0) s_out.M = M;
    }
    __syncthreads();
    *out = s_out;
}

// Grid-wide sums of nb block partials, by the whole calling block (thread 0
// receives the result).  The same order of operations for every caller, so
// a filter gets bit-identical results alone or inside a batch.
template <typename R>
__device__ __forceinline__ void combine_partials(const Partial *part, int nb, Combined *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (sizeof(R) == 8) {
        __shared__ double s_red[kBlock / 32][6];
        double M = -INFINITY;
        for (int b = threadIdx.x; b < nb; b += kBlock) M = fmax(M, __ldcg(&part[b].m));
        M = warp_max(M);
        if (lane == 0) s_red[warp][0] = M;
        __syncthreads();
        M = s_red[0][0];
        for (int w = 1; w < kBlock / 32; ++w) M = fmax(M, s_red[w][0]);
        __syncthreads();
        double S[5] = {0, 0, 0, 0, 0};
        if (M > -INFINITY) {
            for (int b = threadIdx.x; b < nb; b += kBlock) {
                const double mb = __ldcg(&part[b].m);
                const double sc = (mb > -INFINITY) ? exp(mb - M) : 0.0;
                S[0] = fma_x(__ldcg(&part[b].s1), sc, S[0]);
                S[1] = fma_x(mul_x(__ldcg(&part[b].s2), sc), sc, S[1]);
                S[2] = fma_x(__ldcg(&part[b].sx), sc, S[2]);
                S[3] = fma_x(__ldcg(&part[b].sy), sc, S[3]);
                S[4] = fma_x(__ldcg(&part[b].su), sc, S[4]);
            }
        }
        for (int q = 0; q < 5; ++q) S[q] = warp_sum(S[q]);
        if (lane == 0)
            for (int q = 0; q < 5; ++q) s_red[warp][1 + q] = S[q];
        __syncthreads();
        if (threadIdx.x == 0) {
            Combined c{M, 0, 0, 0, 0, 0};
            for (int w = 0; w < kBlock / 32; ++w) {
                c.S1 += s_red[w][1];
                c.S2 += s_red[w][2];
                c.Sa += s_red[w][3];
                c.Sb += s_red[w][4];
                c.Sc += s_red[w][5];
            }
            *out = c;
        }
    } else {
        CombinedDF d;
        combine_partials_df<4>(part, nb, &d);
        if (threadIdx.x == 0)
            *out = Combined{df_to_double(DF{d.M, 0.0f}), df_to_double(d.S[0]), df_to_double(d.S[1]),
                            df_to_double(d.S[2]), df_to_double(d.S[3]), 0.0};
    }
    __syncthreads();
}

template <typename R>
__device__ __forceinline__ bool last_block_combine(DevState *st, const Partial *part, Combined *out) {
    if (!take_ticket<R>(st)) return false;
    combine_partials<R>(part, gridDim.x, out);
    return true;
}

__device__ __forceinline__ bool resample_decision(double ess, int64_t n, double threshold) {
    if (threshold >= 1.0) return true;
    if (threshold <= 0.0) return false;
    return ess < threshold * double(n);
}

// Thread 0 of the last block: write the record of iteration f.t and update
// the device state.  Returns false (and raises SMC_E_NONFINITE) when the
// weights are all zero or NaN; the buffers are then left as they were.
__device__ __forceinline__ bool finalize_weights(const FinalizeArgs &f, const Combined &c, double *L_out) {
    DevState *st = f.st;
    smc_record *r = &f.rec[f.t % f.rec_cap];
    const bool ok = (c.M > -INFINITY) && (c.M < INFINITY) && (c.S1 > 0.0) && (c.S1 < INFINITY) &&
                    (c.S2 > 0.0);
    st->ticket = 0;
    if (!ok) {
        r->t = f.t;
        r->status = SMC_E_NONFINITE;
        raise_error(st, SMC_E_NONFINITE);
        return false;
    }
    const double L = c.M + log(c.S1);
    const double ess = c.S1 * c.S1 / c.S2;
    const bool due = resample_decision(ess, f.n, f.threshold);
    const double prev_logz = (f.mode == 0) ? (f.t == 0 ? 0.0 : st->log_evidence) : st->log_evidence - st->log_norm;
    // mode 1 (reweighting the same iteration): replace the old increment L_t
    // by the new one, i.e. log Z += L'_t - L_t
    const double logz = prev_logz + L;
    r->log_norm = L;
    r->log_evidence = logz;
    r->ess = ess;
    r->mean[0] = c.Sa / c.S1;
    r->mean[1] = c.Sb / c.S1;
    r->mean_post[0] = r->mean_post[1] = __longlong_as_double(0x7ff8000000000000ll);  // set by post_mean_kernel
    r->max_lw = c.M;
    r->t = f.t;
    r->resampled = due ? 1 : 0;
    r->status = SMC_OK;
    r->alpha = f.alpha;
    st->max_lw = c.M;
    st->max_lw_f = float(c.M);
    st->log_norm = L;
    split_float(L, st->log_norm_f);
    st->log_evidence = logz;
    st->ess = ess;
    st->due = due ? 1 : 0;
    *L_out = L;
    return true;
}

// FP32 path of finalize_weights: the same record and state updates with the
// per-iteration scalars in compensated float (no float64 logarithm or
// division; doubles only for the stored values: bit-pattern conversions and
// the float64 evidence sum).  Called by the whole last block; lane 0 of
// warps 0-3 share the work so that the logarithm, the ESS division and the
// means run at the same time:
//   warp 0: L_t = M + log S1, log Z_t, the status of a failed iteration
//   warp 1: ESS and the resample decision
//   warp 2: filtered means
//   warp 3: maximum, record header, ticket reset
// Returns ok (every thread).  With L_dst set, warp 0 also stores L_t there.
__device__ __forceinline__ bool finalize_weights_df(const FinalizeArgs &f, const CombinedDF &c,
                                                    double *L_dst = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const DF S1 = c.S[0], S2 = c.S[1];
    const bool ok = (c.M > -INFINITY) && (c.M < INFINITY) && (S1.hi > 0.0f) && (S1.hi < INFINITY) && (S2.hi > 0.0f);
    if (lane != 0 || warp >= 4) return ok;
    DevState *st = f.st;
    smc_record *r = &f.rec[f.t % f.rec_cap];
    if (warp == 0) {
        if (!ok) {
            r->t = f.t;
            r->status = SMC_E_NONFINITE;
            raise_error(st, SMC_E_NONFINITE);
            return ok;
        }
        const DF L = df_add_f(df_log(S1), c.M);
        const double Ld = df_to_double(L);
        // mode 1 (reweighting the same iteration): replace the old increment
        // L_t by the new one, i.e. log Z += L'_t - L_t
        const double prev_logz =
            (f.mode == 0) ? (f.t == 0 ? 0.0 : f.log_evidence_prev) : st->log_evidence - st->log_norm;
        const double logz = prev_logz + Ld;
        r->log_norm = Ld;
        r->log_evidence = logz;
        st->log_norm = Ld;
        st->log_norm_f[0] = L.hi;
        st->log_norm_f[1] = L.lo;
        st->log_evidence = logz;
        if (L_dst) *L_dst = Ld;
    } else if (warp == 3) {
        st->ticket = 0;
        if (ok) {
            const double Md = df_to_double(DF{c.M, 0.0f});
            r->max_lw = Md;
            r->t = f.t;
            r->status = SMC_OK;
            r->alpha = f.alpha;
            st->max_lw = Md;
            st->max_lw_f = c.M;
        }
    } else if (ok && warp == 1) {
        const DF ess = df_div(df_mul(S1, S1), S2);
        const bool due = f.thr_mode == 1   ? true
                         : f.thr_mode == 2 ? false
                                           : df_lt(ess, df_mul(DF{f.thr_df[0], f.thr_df[1]}, df_from_int(f.n)));
        const double essd = df_to_double(ess);
        r->ess = essd;
        r->resampled = due ? 1 : 0;
        st->ess = essd;
        st->due = due ? 1 : 0;
    } else if (ok) {
        r->mean[0] = df_to_double(df_div(c.S[2], S1));
        r->mean[1] = df_to_double(df_div(c.S[3], S1));
        r->mean_post[0] = r->mean_post[1] = __longlong_as_double(0x7ff8000000000000ll);  // set by post_mean_kernel
    }
    return ok;
}

}  // namespace smc
