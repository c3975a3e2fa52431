// Resampling (Sec. 2.1, eq:resample; Douc et al. 2005 schemes; copy_from
// convention of Sec. 4.1.2) on exact 64-bit fixed-point weights.
//
// Weights: q_i = floor(exp(lw_i - M) 2^F), F = 61 - ceil(log2 N), so every
// prefix sum Q_i is an exact integer below 2^62: the CDF is order-independent
// and bit-reproducible.
// Targets are rationals P_k / D (u = (2j + 1) / 2^25):
//   systematic  P_k = 2^25 k + 2j + 1        D = N 2^25  (one j per iteration)
//   stratified  P_k = 2^25 k + 2j_k + 1      D = N 2^25  (j_k independent)
//   multinomial P_k = m (2 j_(k) + 1)        D = m 2^25  (j_(k) the sorted iid j's)
// and a_k = min{ i : Q_i D > Q_N P_k }.  Residual resampling takes the
// multinomial targets on its residual weights (m = R draws) and puts the
// deterministic copies in front of each particle's draws.
//
// Every scheme runs as one cooperative kernel (a grid barrier between the
// scan of the weights and the selection) in which particle i writes its own
// outputs [K(Q_{i-1}), K(Q_i)), K from a closed form (systematic,
// stratified) or from a histogram of the draws (multinomial, residual).
// The reduce-then-scan kernels with a merge-path search per output serve the
// allocation-free systematic entry and the batched filters.
#pragma once

#include "grid_threshold.h"
#include "weight_reduce.cuh"

namespace smc {

// ----------------------------------------------------------- generators --

// q_i = floor(exp(lw_i - M) 2^F) from the current log-weights.
template <typename R>
struct QGen {
    const R *lw[2];
    int frac;
    const R *cur_lw;
    R m;
    __device__ __forceinline__ void prepare(const DevState *st) {
        cur_lw = st->cur_lw ? lw[1] : lw[0];
        if constexpr (sizeof(R) == 4) m = st->max_lw_f;
        else m = R(st->max_lw);
    }
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const {
        return Math<R>::fixed(Math<R>::fast_exp(__ldcg(cur_lw + i) - m), frac);
    }
    // kScanItems consecutive values from 16-byte vector loads
    static constexpr bool kVec = true;
    __device__ __forceinline__ void load8(uint32_t i0, uint32_t n, unsigned long long (&v)[kScanItems]) const {
        R w[kScanItems];
        load_k<R, kScanItems>(cur_lw, i0, n, w);
#pragma unroll
        for (int j = 0; j < kScanItems; ++j)
            v[j] = (i0 + j < n) ? Math<R>::fixed(Math<R>::fast_exp(w[j] - m), frac) : 0ull;
    }
};

// kScanItems consecutive generator values starting at i0 (0 past n)
template <class Gen, typename = void>
struct HasVec {
    static constexpr bool value = false;
};
template <class Gen>
struct HasVec<Gen, decltype((void)Gen::kVec, void())> {
    static constexpr bool value = Gen::kVec;
};

template <class Gen>
__device__ __forceinline__ void gen_items(const Gen &g, int64_t i0, int64_t n, unsigned long long (&v)[kScanItems]) {
    if constexpr (HasVec<Gen>::value) {
        g.load8((uint32_t)i0, (uint32_t)n, v);
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) v[j] = (i0 + j < n) ? g(i0 + j) : 0ull;
    }
}

// A 64-bit integer as a float from its 32-bit halves: the 64-bit
// integer <-> float conversions run on the FP64 pipe (1/64 of the FP32
// rate on B300); the result is within a few float ulps, for estimates.
__device__ __forceinline__ float u64_to_float(unsigned long long x) {
    return fmaf(__uint2float_rn((uint32_t)(x >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)x));
}

// floor(n q / qn) for q <= qn < 2^62, n < 2^31 (exact: float estimate from
// inv_qn ~ 1 / qn, then integer correction with 128-bit products)
__device__ __forceinline__ unsigned long long floor_nq_over(unsigned long long n, unsigned long long q,
                                                            unsigned long long qn, float inv_qn) {
    if (qn == 0 || q > qn) return 0;
    const U128 num = mul64(n, q);
    const float est = u64_to_float(n) * u64_to_float(q) * inv_qn;  // below 2^31 + rounding
    unsigned long long d = (unsigned long long)__float2uint_rz(fminf(fmaxf(est, 0.0f), 4294967040.0f));
    if (d > n) d = n;
    while (d > 0 && gt128(mul64(d, qn), num)) --d;
    while (!gt128(mul64(d + 1, qn), num)) ++d;
    return d;
}

// ---------------------------------------------------------------- sinks --

struct NoSink {
    static constexpr bool kActive = false;
    __device__ __forceinline__ void operator()(int64_t, unsigned long long, DevState *) const {}
};

struct StoreSink {  // inclusive prefix sums to an array (the fixed-point CDF)
    static constexpr bool kActive = true;
    unsigned long long *dst;
    __device__ __forceinline__ void operator()(int64_t i, unsigned long long v, DevState *) const {
        if (dst) dst[i] = v;
    }
};

// --------------------------------------------------------------- targets --
//
// A target set gives, per block: prepare(state) and setup(Q_N) (run by one
// thread, then broadcast), count(), first_at_least(X, Q_N) = the first k
// with Q_N P_k >= X D (the tile's output range), and thresholds(k0, tau):
// tau_j = floor(Q_N P_{k0+j} / D) for j < kScanItems (k0 a multiple of
// kScanItems; entries past count() are never used), so that
// a_k = min{ i : Q_i > tau_k } with 64-bit comparisons only.

struct NoTargets {
    static constexpr bool kActive = false;
    __device__ __forceinline__ void prepare(const DevState *) {}
    __device__ __forceinline__ void setup(unsigned long long) {}
    __device__ __forceinline__ int64_t count() const { return 0; }
    __device__ __forceinline__ int64_t first_at_least(unsigned long long, unsigned long long) const { return 0; }
    __device__ __forceinline__ void thresholds(int64_t, unsigned long long (&)[kScanItems]) const {}
};

__device__ __forceinline__ uint4 resample_words(uint2 key, uint32_t stream, uint32_t t, int64_t k4) {
    return draw(key, (uint32_t)(k4 >> 2), t, TAG_RESAMPLE, stream, 0u);
}

// j_k of resampling draw k at iteration t (word k % 4 of call k / 4)
__device__ __forceinline__ uint32_t resample_u24_at(uint2 key, uint32_t stream, uint32_t t, int64_t k) {
    const uint4 w = resample_words(key, stream, t, k & ~3ll);
    const uint32_t ww = ((k & 3) == 0) ? w.x : ((k & 3) == 1) ? w.y : ((k & 3) == 2) ? w.z : w.w;
    return u24(ww);
}

// Systematic (one u per iteration) and stratified (u_k per output) targets,
// P_k = 2^25 k + c_k, D = N 2^25; thresholds from GridDiv.
template <bool kStratified>
struct GridTargets {
    static constexpr bool kActive = true;
    int64_t n;
    uint2 key;
    uint32_t stream;
    uint32_t t;
    unsigned long long c;  // 2j + 1 (systematic)
    unsigned long long mrec;  // floor((2^64 - 1) / n), from the host
    unsigned long long c_fixed;  // nonzero: c itself instead of a draw (the multinomial value thresholds)
    GridDiv dv;
    __device__ __forceinline__ void prepare(const DevState *st) { prepare_at((uint32_t)st->t); }
    __device__ __forceinline__ void prepare_at(uint32_t tt) {
        t = tt;
        c = c_fixed ? c_fixed : 2ull * u24(draw(key, 0u, t, TAG_RESAMPLE, stream, 0u).x) + 1ull;
    }
    // closed form: z(X) = X N / Q_N - c 2^-25 (systematic) or X N / Q_N
    // (stratified) in double-float, with its absolute error bound (relative
    // error below 2^-42 of z <= N)
    DF sN, ncc;
    float margin;
    unsigned long long qn;
    __device__ __forceinline__ void setup(unsigned long long QN) {
        dv.init(QN, (unsigned long long)n, mrec);
        qn = QN;
        if (QN) sN = df_div(df_from_int(n), df_from_u64(QN));
        const DF cd = df_from_int(kStratified ? 0 : (int64_t)c);
        ncc = DF{-cd.hi * 0x1p-25f, -cd.lo * 0x1p-25f};
        margin = fmaxf(float(n) * 0x1p-40f, 0x1p-20f);
    }
    __device__ __forceinline__ int64_t count() const { return n; }
    // K(X) = #{k : tau_k < X} = the first k with Q_N P_k >= X D, i.e. with
    // k + c_k 2^-25 >= y = X N / Q_N.  Systematic (c fixed): K = ceil z,
    // z = y - c 2^-25.  Stratified (c_k in (0, 2^25)): K = k0 = floor y when
    // c_k0 >= frac(y) 2^25, else k0 + 1.  z is carried as floor zi, fraction
    // zf and an error bound err; whenever a float decision lies within its
    // error bound, exact 64-bit / 128-bit thresholds decide.
    struct ZPos {
        int64_t zi;
        float zf, err;
    };
    // z(X) from the double-float estimate
    __device__ __forceinline__ ZPos z_at(unsigned long long X) const {
        const DF z = df_add(df_mul(df_from_u64(X), sN), ncc);  // > -1
        const float fh = floorf(z.hi);                         // integer in [-1, 2^31]
        float fr = (z.hi - fh) + z.lo;
        const float adj = floorf(fr);  // lo may exceed one unit when hi >= 2^24
        fr -= adj;
        ZPos p;
        p.zi = (fh < 0.0f ? -1ll : (int64_t)__float2uint_rn(fh)) + (int64_t)__float2int_rn(adj);
        p.zf = fr;
        p.err = margin;
        return p;
    }
    // z(X + q) from z(X) for a fixed-point weight q: a float increment with
    // relative error below 2^-22, the rounding of the fraction added to err
    __device__ __forceinline__ void z_advance(ZPos &p, unsigned long long q) const {
        const float qf = fmaf(__uint2float_rn((uint32_t)(q >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)q));
        const float d = qf * sN.hi;
        const float f = p.zf + d;
        const float w = floorf(f);
        p.zi += (int64_t)__float2uint_rn(w);
        p.zf = f - w;
        p.err += fmaf(d, 0x1p-21f, 0x1p-21f);
    }
    // stratified draws: a block's table of 2j + 1 for the outputs
    // [kb, kb + cnt) in shared memory, in two pieces of kScanTile entries;
    // past it (a tile with still more outputs) one Philox call per boundary
    struct DrawCache {
        const uint32_t *tab0 = nullptr, *tab1 = nullptr;
        int64_t kb = 0;
        int cnt = 0;
    };
    __device__ __forceinline__ unsigned long long c_at(int64_t k, DrawCache &dc) const {
        const int64_t i = k - dc.kb;
        if (i >= 0 && i < dc.cnt) return i < kScanTile ? dc.tab0[i] : dc.tab1[i - kScanTile];
        return 2ull * resample_u24_at(key, stream, t, k) + 1ull;
    }
    __device__ __forceinline__ int64_t k_from(const ZPos &p, unsigned long long X, DrawCache &dc) const {
        if constexpr (kStratified) {
            if (!(p.zf > p.err && p.zf < 1.0f - p.err)) return first_at_least(X, qn);  // floor y uncertain
            const int64_t k0 = p.zi;
            if (k0 >= n) return n;
            const unsigned long long ck = c_at(k0, dc);
            // frac(y) 2^25 with the bound of zf, the product's rounding (2) and
            // the float conversion of ck < 2^25 (1)
            const float thr = p.zf * 33554432.0f, tol = fmaf(p.err, 33554432.0f, 4.0f);
            const float cf = __uint2float_rn((uint32_t)ck);  // ck < 2^25
            int64_t k;
            if (cf > thr + tol) k = k0;
            else if (cf < thr - tol) k = k0 + 1;
            else {
                uint64_t u, v;
                dv.start((uint64_t)k0, u, v);
                k = dv.tau((uint64_t)k0, ck, u, v) >= X ? k0 : k0 + 1;
            }
            return k > n ? n : k;
        }
        int64_t k;
        if (p.zf > p.err && p.zf < 1.0f - p.err) {
            k = p.zi + 1;
        } else {
            const int64_t m = (p.zf <= p.err) ? p.zi : p.zi + 1;  // z within err of m
            if (m < 0) k = 0;
            else if (m >= n) k = n;
            else {
                uint64_t u, v;
                dv.start((uint64_t)m, u, v);
                k = dv.tau((uint64_t)m, c, u, v) >= X ? m : m + 1;
            }
        }
        return k < 0 ? 0 : (k > n ? n : k);
    }
    __device__ __forceinline__ unsigned long long P(int64_t k) const {
        const unsigned long long ck = kStratified ? 2ull * resample_u24_at(key, stream, t, k) + 1ull : c;
        return ((unsigned long long)k << 25) + ck;
    }
    // first k in [0, n] with QN P_k >= X D.  With k0 = floor(X N / QN) the
    // answer is k0 or k0 + 1 (P_k / 2^25 lies in (k, k + 1)); k0 comes from a
    // double-float estimate (error far below 1) corrected with exact 128-bit
    // products.
    __device__ __forceinline__ int64_t first_at_least(unsigned long long X, unsigned long long QN) const {
        const unsigned long long N = (unsigned long long)n;
        const DF e = df_mul(df_div(df_from_u64(X), df_from_u64(QN)), df_from_int(n));
        int64_t k0 = (int64_t)__float2uint_rd(fmaxf(e.hi, 0.0f));
        if (k0 > n) k0 = n;
        const U128 xn = mul64(X, N);
        while (k0 > 0 && gt128(mul64((unsigned long long)k0, QN), xn)) --k0;  // k0 QN <= X N
        while (k0 < n && !gt128(mul64((unsigned long long)k0 + 1, QN), xn)) ++k0;  // X N < (k0 + 1) QN
        if (k0 >= n) return n;
        return gt128(mul64(X, N << 25), mul64(QN, P(k0))) ? k0 + 1 : k0;
    }
    __device__ __forceinline__ void thresholds(int64_t k0, unsigned long long (&tau)[kScanItems]) const {
        static_assert(kScanItems == 8, "two Philox calls per thread");
        unsigned long long cw[kScanItems];
        if (kStratified) {
            const uint4 w0 = resample_words(key, stream, t, k0), w1 = resample_words(key, stream, t, k0 + 4);
            const uint32_t ww[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) cw[j] = 2ull * u24(ww[j]) + 1ull;
        }
        uint64_t u, v;
        dv.start((uint64_t)k0, u, v);
        if (kStratified) {
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) {
                if (j > 0) dv.next(u, v);
                tau[j] = dv.tau((uint64_t)(k0 + j), cw[j], u, v);
            }
        } else {
            uint64_t rem;
            uint64_t t = dv.tau((uint64_t)k0, c, u, v, &rem);
            tau[0] = t;
#pragma unroll
            for (int j = 1; j < kScanItems; ++j) {
                dv.advance(t, rem);
                tau[j] = t;
            }
        }
    }
};

// ----------------------------------------------------------------- outputs --

struct AncOut {
    int32_t *anc;
    int32_t *host_err = nullptr;  // smc_iterate_host's graph: the mapped staging's error word
    __device__ __forceinline__ void operator()(int64_t k, int32_t a) const { anc[k] = a; }
    // after a failure in this kernel: the device error word to the staging
    __device__ __forceinline__ void report(const DevState *st) const {
        if (host_err && threadIdx.x == 0)
            *reinterpret_cast<volatile int32_t *>(host_err) = *reinterpret_cast<const volatile int32_t *>(&st->error);
    }
};

// ---------------------------------------------------------------- kernels --

// sv: the block's snapshot of the state block
__device__ __forceinline__ bool gated_out(const DevState *sv, int gate) {
    if (sv->error) return true;
    return gate && !sv->due;
}

// Sum of gen(i) over tile `tile` (kScanTile elements), returned to thread 0.
template <class Gen>
__device__ __forceinline__ unsigned long long tile_sum(const Gen &g, int64_t n, int tile) {
    __shared__ unsigned long long s_w[kBlock / 32];
    const int64_t i0 = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    unsigned long long v[kScanItems];
    gen_items(g, i0, n, v);
    unsigned long long acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) acc += v[j];
    acc = warp_sum(acc);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    unsigned long long s = 0;
    if (threadIdx.x == 0)
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) s += s_w[w];
    return s;
}

// Exact sum of nt tile sums by the whole block (thread 0 receives it).
__device__ __forceinline__ unsigned long long sum_tiles(const unsigned long long *tsum, int nt) {
    __shared__ unsigned long long s_w[kBlock / 32];
    unsigned long long tot = 0;
    for (int b = threadIdx.x; b < nt; b += kBlock) tot += __ldcg(&tsum[b]);
    tot = warp_sum(tot);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = tot;
    __syncthreads();
    unsigned long long s = 0;
    if (threadIdx.x == 0)
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) s += s_w[w];
    return s;
}

// Sum of gen(i) over each tile of kScanTile elements -> tsum[tile]; the last
// block writes the exact total to *total.
template <class Gen>
__global__ void __launch_bounds__(kBlock) tile_reduce_kernel(Gen gen, int64_t n, unsigned long long *tsum,
                                                             unsigned long long *total, uint32_t *ticket,
                                                             DevState *st, int gate) {
    const DevState *sv = snapshot(st);
    if (gated_out(sv, gate)) return;
    Gen g = gen;
    g.prepare(sv);
    const unsigned long long s = tile_sum(g, n, blockIdx.x);
    if (threadIdx.x == 0) tsum[blockIdx.x] = s;
    if (!total) return;  // the consumer sums the tiles itself
    if (!last_arrival(ticket, gridDim.x)) return;
    const unsigned long long tot = sum_tiles(tsum, gridDim.x);
    if (threadIdx.x == 0) {
        *total = tot;
        *ticket = 0;
    }
}

// Sum of one value per thread, returned to every thread.
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v) {
    __shared__ unsigned long long s_w[kBlock / 32];
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) t += s_w[w];
    return t;
}

// Exclusive prefix (tiles before `tile`) and total of nt tile sums, by the
// whole block in one pass; every thread receives both.
__device__ __forceinline__ void tile_prefix_total(const unsigned long long *tsum, int tile, int nt,
                                                  unsigned long long *pre_out, unsigned long long *tot_out) {
    __shared__ unsigned long long s_p[kBlock / 32], s_t[kBlock / 32];
    unsigned long long pre = 0, tot = 0;
    for (int b = threadIdx.x; b < nt; b += kBlock) {
        const unsigned long long v = __ldcg(&tsum[b]);
        tot += v;
        if (b < tile) pre += v;
    }
    pre = warp_sum(pre);
    tot = warp_sum(tot);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        s_p[threadIdx.x >> 5] = pre;
        s_t[threadIdx.x >> 5] = tot;
    }
    __syncthreads();
    pre = 0;
    tot = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) {
        pre += s_p[w];
        tot += s_t[w];
    }
    *pre_out = pre;
    *tot_out = tot;
}

// The block's target set: prepared (and set up for Q_N) by one thread and
// broadcast, so per-block constants (a Philox draw, 64-bit divisions) are
// computed once.
template <class Tgt>
__device__ __forceinline__ const Tgt &block_targets_ref(const Tgt &proto, const DevState *sv, unsigned long long QN) {
    __shared__ Tgt s_tg;
    __syncthreads();
    if (threadIdx.x == 0) {
        Tgt t = proto;
        t.prepare(sv);
        t.setup(QN);
        s_tg = t;
    }
    __syncthreads();
    return s_tg;
}
template <class Tgt>
__device__ __forceinline__ Tgt block_targets(const Tgt &proto, const DevState *sv, unsigned long long QN) {
    return block_targets_ref(proto, sv, QN);
}

// Shared-memory buffers of one scan tile (declared once per kernel).  The
// 64-bit arrays have one pad word after every kScanItems entries and the
// ancestor array one after every 32: a thread owns kScanItems consecutive
// entries, and without padding the 64-byte stride between threads would put
// 16 threads of a warp on the same banks.
__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

struct TileBufs {
    unsigned long long q[kScanTile + kScanTile / 8];    // tile-relative inclusive prefix sums (pad8)
    unsigned long long tau[kScanTile + kScanTile / 8];  // thresholds of one round, relative to the tile (pad8)
    int32_t a[kScanTile + kScanTile / 32];              // ancestors of one round (pad32)
    unsigned long long w[kBlock / 32];
    int64_t k[2];                                       // the tile's output range
};

// Inclusive scan of kScanItems values per thread (thread t owns the tile
// entries t kScanItems + j) into tb.q; returns the total to every thread.
__device__ __forceinline__ unsigned long long scan_items_q(unsigned long long (&loc)[kScanItems], TileBufs &tb) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        acc += loc[j];
        loc[j] = acc;
    }
    const unsigned long long winc = warp_incl_scan(acc);
    __syncthreads();  // tb may still be read by a previous round
    if (lane == 31) tb.w[warp] = winc;
    __syncthreads();
    unsigned long long wpre = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w)
        if (w < warp) wpre += tb.w[w];
    const unsigned long long base = wpre + (winc - acc);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) tb.q[pad8(tid * kScanItems + j)] = base + loc[j];
    __syncthreads();
    return tb.q[pad8(kScanTile - 1)];
}

// Inclusive scan of the tile's values into tb.q (tile-relative; zeros past
// n); returns the tile's total to every thread.
template <class Gen>
__device__ __forceinline__ unsigned long long scan_tile_local(const Gen &g, int64_t n, int tile, TileBufs &tb) {
    unsigned long long loc[kScanItems];
    gen_items(g, (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems, n, loc);
    return scan_items_q(loc, tb);
}

// Selection for one scanned tile (tb.q holds its tile-relative prefix sums,
// pre the exclusive prefix before it, total its sum): the CDF is optionally
// stored through `sink`, then every output k in the tile's range
// [k_lo, k_hi) gets a_k = t0 + #{i : Q_i <= tau_k} (Q_i = pre + q_i).
// Outputs go in rounds of kScanTile; a round merges its sorted thresholds
// with the tile's sorted prefix sums along the merge path, so every thread
// takes the same number of merge steps whatever the weights look like.
template <class Tgt, class Out, class Sink>
__device__ __forceinline__ void select_tile(const Tgt &tg, const Out &out, const Sink &sink, int64_t n, int tile,
                                            unsigned long long pre, unsigned long long total,
                                            unsigned long long QN, DevState *st, TileBufs &tb) {
    constexpr int kSteps = 2 * kScanItems;  // merge steps per thread: (outputs + inputs) / threads
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t0 = (int64_t)tile * kScanTile;
    const int len = (int)min((int64_t)kScanTile, n - t0);
    if (Sink::kActive) {
#pragma unroll
        for (int r = 0; r < kScanItems; ++r) {
            const int idx = r * kBlock + tid;
            if (idx < len) sink(t0 + idx, pre + tb.q[pad8(idx)], st);
        }
    }
    if (!Tgt::kActive || QN == 0) return;
    if (lane == 0 && warp < 2) {  // the two ends of the output range, one warp each
        const int64_t cnt = tg.count();
        if (warp == 0) tb.k[0] = min(tg.first_at_least(pre, QN), cnt);
        else tb.k[1] = (t0 + len >= n) ? cnt : min(tg.first_at_least(pre + total, QN), cnt);
    }
    __syncthreads();
    const int64_t k_lo = tb.k[0], k_hi = tb.k[1];
    for (int64_t kb = k_lo & ~(int64_t)(kScanItems - 1); kb < k_hi; kb += kScanTile) {
        const int m = (int)min((int64_t)kScanTile, k_hi - kb);
        const int j0 = tid * kScanItems;
        if (j0 < m) {
            unsigned long long tau[kScanItems];
            tg.thresholds(kb + j0, tau);
#pragma unroll
            for (int j = 0; j < kScanItems; ++j)  // outputs before k_lo clamp to 0 (merged, never written)
                tb.tau[pad8(j0 + j)] = tau[j] >= pre ? tau[j] - pre : 0ull;
        }
        __syncthreads();
        const int tot = m + len;
        const int d0 = tid * kSteps;
        if (d0 < tot) {
            // split of diagonal d0: k outputs and d0 - k inputs come first
            int lo = max(0, d0 - len), hi = min(d0, m);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (tb.tau[pad8(mid)] < tb.q[pad8(d0 - mid - 1)]) lo = mid + 1;
                else hi = mid;
            }
            int k = lo, i = d0 - lo;
            unsigned long long av = k < m ? tb.tau[pad8(k)] : ~0ull;
            unsigned long long bv = i < len ? tb.q[pad8(i)] : ~0ull;
#pragma unroll
            for (int s = 0; s < kSteps; ++s) {
                if (d0 + s >= tot) break;
                if (k < m && (i >= len || av < bv)) {  // output k: inputs 0..i-1 have Q <= tau_k < Q_i
                    tb.a[pad32(k)] = (int32_t)(t0 + min(i, len - 1));
                    ++k;
                    av = k < m ? tb.tau[pad8(k)] : ~0ull;
                } else {
                    ++i;
                    bv = i < len ? tb.q[pad8(i)] : ~0ull;
                }
            }
        }
        __syncthreads();
        for (int j = tid; j < m; j += kBlock)
            if (kb + j >= k_lo) out(kb + j, tb.a[pad32(j)]);
        __syncthreads();
    }
}

// Selection of one scanned tile (systematic, stratified) from the
// closed-form offspring ranges: particle i receives the outputs k in [K(Q_{i-1}), K(Q_i)).  Each
// thread finds K at the boundaries of its kScanItems particles (no search,
// no merge; z moves by q_i N / Q_N from one boundary to the next); a particle with offspring marks the first of its outputs in a
// shared window of kScanTile outputs, and an inclusive max-scan over the
// window gives every output its ancestor (the marked particles increase
// with the position).  A tile owning more outputs than one window takes
// several windows (a degenerate weight), carrying the last ancestor over.
// tb.q holds the tile's scan (tile-relative), pre the prefix before it.
// The closed form gives an index K0(X) into the targets' own count; kmap
// turns it into the output count K(X) (the identity for systematic and
// stratified targets; the draw histogram for multinomial value thresholds).
struct KIdentity {
    static constexpr bool kActive = false;
    __device__ __forceinline__ int64_t operator()(int64_t k) const { return k; }
    __device__ __forceinline__ void map_block(int32_t *, int64_t *) const {}
};

template <bool kStratified, class Out, class KMap = KIdentity>
__device__ __forceinline__ void select_tile_closed(const GridTargets<kStratified> &tg, const Out &out, int64_t n,
                                                   int tile, unsigned long long pre, unsigned long long QN,
                                                   TileBufs &tb, const KMap &kmap = KMap{}) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int base = tid * kScanItems;
    const int64_t t0 = (int64_t)tile * kScanTile;
    if (QN == 0) return;
    // K(Q_i) for the thread's particles i: z at the left boundary from the
    // double-float estimate, the rest by increments (re-anchored if the
    // bound grows); kept in shared memory (the tile's threshold buffer,
    // unused here) as K[i] = the end of particle i's outputs, so particle
    // i's outputs are [K[i - 1], K[i]) and K[-1] = K(pre) = the tile's first
    // output
    int32_t *Kend = reinterpret_cast<int32_t *>(tb.tau);  // pad32 layout, K <= N < 2^31
    typename GridTargets<kStratified>::DrawCache dc;
    if constexpr (kStratified) {
        // the draws of the tile's outputs, from about its first one
        // (floor(Q_pre N / Q_N), rounded down to a Philox call) to past its
        // last, at most 2 kScanTile of them: uniform Philox calls into the
        // ancestor buffer (unused until the windows) and the threshold buffer
        // past the offspring ends, so that no thread calls Philox for a
        // boundary inside that range
        constexpr int kTab1 = kScanTile + kScanTile / 32 + 1;  // 32-bit words: past Kend
        static_assert(kTab1 + kScanTile <= 2 * (kScanTile + kScanTile / 8), "inside the threshold buffer");
        const int64_t kb = max(tg.z_at(pre).zi, (int64_t)0) & ~int64_t(3);
        const int64_t ke = min(tg.z_at(pre + tb.q[pad8(kScanTile - 1)]).zi + 2, n);  // past the last output
        const int calls = (int)min((ke - kb + 3) >> 2, (int64_t)(2 * kScanTile / 4));
        uint32_t *tab0 = reinterpret_cast<uint32_t *>(tb.a);
        uint32_t *tab1 = reinterpret_cast<uint32_t *>(tb.tau) + kTab1;
        for (int c = tid; c < calls; c += kBlock) {
            const uint4 w = resample_words(tg.key, tg.stream, tg.t, kb + 4 * (int64_t)c);
            uint32_t *d = (4 * c < kScanTile) ? tab0 + 4 * c : tab1 + (4 * c - kScanTile);
            d[0] = 2u * u24(w.x) + 1u;
            d[1] = 2u * u24(w.y) + 1u;
            d[2] = 2u * u24(w.z) + 1u;
            d[3] = 2u * u24(w.w) + 1u;
        }
        __syncthreads();
        dc.tab0 = tab0;
        dc.tab1 = tab1;
        dc.kb = kb;
        dc.cnt = 4 * max(calls, 0);
    }
    {
        unsigned long long qprev = base ? tb.q[pad8(base - 1)] : 0ull;
        typename GridTargets<kStratified>::ZPos zp = tg.z_at(pre + qprev);
        if (tid == 0) tb.k[0] = tg.k_from(zp, pre, dc);  // mapped with the thread's own entries
#pragma unroll 1
        for (int j = 0; j < kScanItems; ++j) {
            const unsigned long long qj = tb.q[pad8(base + j)];
            tg.z_advance(zp, qj - qprev);
            if (zp.err > 0x1p-8f) zp = tg.z_at(pre + qj);
            Kend[pad32(base + j)] = (int32_t)tg.k_from(zp, pre + qj, dc);
            qprev = qj;
        }
    }
    if constexpr (KMap::kActive) {  // the count map over the tile's entries, thread t taking t + r kBlock
        __syncthreads();
        kmap.map_block(Kend, &tb.k[0]);
    }
    __syncthreads();
    const int64_t k_lo = tb.k[0], k_hi = Kend[pad32(kScanTile - 1)];
    int32_t carry = -1;
    for (int64_t w0 = k_lo; w0 < k_hi; w0 += kScanTile) {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) tb.a[pad32(base + j)] = -1;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int64_t ks = (base + j) ? Kend[pad32(base + j - 1)] : k_lo, ke = Kend[pad32(base + j)];
            if (ke > ks && ks >= w0 && ks < w0 + kScanTile) tb.a[pad32((int)(ks - w0))] = base + j;
        }
        __syncthreads();
        int32_t v[kScanItems];
        int32_t run = -1;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            run = max(run, tb.a[pad32(base + j)]);
            v[j] = run;
        }
        int32_t inc = run;  // inclusive warp max-scan of the thread maxima
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = max(inc, y);
        }
        __shared__ int32_t s_wmax[kBlock / 32];
        if (lane == 31) s_wmax[warp] = inc;
        int32_t before = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) before = -1;
        __syncthreads();
        before = max(before, carry);
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w)
            if (w < warp) before = max(before, s_wmax[w]);
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) tb.a[pad32(base + j)] = max(v[j], before);
        __syncthreads();
        const int m = (int)min((int64_t)kScanTile, k_hi - w0);
        for (int j = tid; j < m; j += kBlock) out(w0 + j, (int32_t)(t0 + tb.a[pad32(j)]));
        carry = tb.a[pad32(kScanTile - 1)];
        __syncthreads();
    }
}

// Selection of one scanned tile for the grid targets: the CDF sink, then
// the closed-form pass.
template <bool kStratified, class Out, class Sink, class KMap = KIdentity>
__device__ __forceinline__ void select_tile_grid(const GridTargets<kStratified> &tg, const Out &out, const Sink &sink,
                                                 int64_t n, int tile, unsigned long long pre, unsigned long long total,
                                                 unsigned long long QN, DevState *st, TileBufs &tb,
                                                 const KMap &kmap = KMap{}) {
    if (Sink::kActive) select_tile(NoTargets{}, out, sink, n, tile, pre, total, QN, st, tb);
    select_tile_closed(tg, out, n, tile, pre, QN, tb, kmap);
}
// Scan (+ selection) pass: one block per tile.  Q_N is the exact total of
// the tile sums (every block sums them), or a given total.
template <class Gen, class Tgt, class Out, class Sink>
__global__ void __launch_bounds__(kBlock) scan_select_kernel(Gen gen, Tgt tgt, Out out, Sink sink, int64_t n,
                                                             const unsigned long long *tsum,
                                                             const unsigned long long *total, DevState *st, int gate,
                                                             int set_ready) {
    const DevState *sv = snapshot(st);
    if (gated_out(sv, gate)) return;
    if (set_ready && blockIdx.x == 0 && threadIdx.x == 0) st->ready = 1;
    Gen g = gen;
    g.prepare(sv);
    unsigned long long pre, QN;
    tile_prefix_total(tsum, blockIdx.x, gridDim.x, &pre, &QN);
    if (total) QN = __ldcg(total);
    const Tgt tg = block_targets(tgt, sv, QN);
    __shared__ TileBufs tb;
    const unsigned long long ts = scan_tile_local(g, n, blockIdx.x, tb);
    select_tile(tg, out, sink, n, blockIdx.x, pre, ts, QN, st, tb);
}

// One-pass resampling for grid targets (systematic, stratified): a
// cooperative launch of at most one wave, each block owning a contiguous
// range of scan tiles.  Phase 1 scans its tiles and publishes the tile sums
// and the block's sum; after a grid barrier phase 2 takes the block's prefix
// and Q_N from the block sums and selects, starting with the last tile whose
// scan is still in shared memory (a block with one tile never rescans).
template <class Gen, bool kStratified, class Sink>
__global__ void __launch_bounds__(kBlock, 4) grid_resample_kernel(Gen gen, GridTargets<kStratified> tgt, AncOut out,
                                                               Sink sink, int64_t n, unsigned long long *tsum,
                                                               unsigned long long *bsum, DevState *st, int gate) {
    __shared__ TileBufs tb;
    // launched as a programmatic dependent of the move kernel: wait until
    // that grid has completed and its writes are visible (returns at once
    // for an ordinary launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const DevState *sv = snapshot(st, true);
    if (gated_out(sv, gate)) return;  // the same decision in every block
    Gen g = gen;
    g.prepare(sv);
    const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
    const int G = gridDim.x, b = blockIdx.x;
    const int t_lo = (int)((int64_t)ntiles * b / G), t_hi = (int)((int64_t)ntiles * (b + 1) / G);
    // tile sums (the last tile scanned, its scan kept for phase 2)
    unsigned long long bs = 0;
    for (int tile = t_lo; tile < t_hi - 1; ++tile) {
        const unsigned long long s = tile_sum(g, n, tile);  // to thread 0
        if (threadIdx.x == 0) {
            tsum[tile] = s;
            bs += s;
        }
    }
    const unsigned long long last = scan_tile_local(g, n, t_hi - 1, tb);
    if (threadIdx.x == 0) {
        tsum[t_hi - 1] = last;
        bsum[b] = bs + last;
    }
    if (!grid_barrier(st, gridDim.x)) return out.report(st);
    if (b == 0 && threadIdx.x == 0) st->ready = 1;
    unsigned long long pre, QN;
    tile_prefix_total(bsum, b, G, &pre, &QN);
    const GridTargets<kStratified> tg = block_targets(tgt, sv, QN);
    // the last tile first (its scan is in tb), then the others rescanned
    unsigned long long before_last = 0;  // sum of the block's other tiles
    if (t_hi - 1 > t_lo) {  // the same branch in the whole block
        for (int tile = t_lo + (int)threadIdx.x; tile < t_hi - 1; tile += kBlock) before_last += __ldcg(&tsum[tile]);
        before_last = block_sum_u64(before_last);
    }
    select_tile_grid(tg, out, sink, n, t_hi - 1, pre + before_last, last, QN, st, tb);
    for (int tile = t_lo; tile < t_hi - 1; ++tile) {
        const unsigned long long ts = scan_tile_local(g, n, tile, tb);
        select_tile_grid(tg, out, sink, n, tile, pre, ts, QN, st, tb);
        pre += ts;
    }
    grid_depart(st);
}

// ------------------------------------------- multinomial by a histogram --
//
// Multinomial selection (P_k = m (2 j_(k) + 1), D = m 2^25, j_(k) the sorted
// draws) without a sort: output k goes to the first i with
// Q_i 2^25 > Q_N (2 j_(k) + 1), so particle i receives the outputs
// [H(v(Q_{i-1})), H(v(Q_i))), where H(v) = #{k : j_k < v} and v(X) is the
// smallest s with Q_N (2 s + 1) >= X 2^25, i.e. v(X) = ceil(X 2^24 / Q_N - 1/2):
// the systematic closed form with n = 2^24 and c = 2^24 (GridTargets with
// c_fixed).  H comes from a histogram of the draws, one byte per value.

// the sum of the four bytes of x
__device__ __forceinline__ uint32_t byte_sum(uint32_t x) {
    x = (x & 0x00FF00FFu) + ((x >> 8) & 0x00FF00FFu);
    return (x & 0xFFFFu) + (x >> 16);
}
// the bytes of x with index below p (p may lie outside 0..4)
__device__ __forceinline__ uint32_t bytes_below(uint32_t x, int p) {
    return p >= 4 ? x : (p <= 0 ? 0u : x & ((1u << (8 * p)) - 1u));
}

// Bucket record written by the histogram scan: x = the bucket's prefix within
// its histogram tile, bit 31 set when a value of the bucket was drawn more
// than 3 times; y = the bucket's 16 counts as 2-bit fields (valid without
// that bit).  One 8-byte load then serves a lookup, and the count below a
// value is two population counts.
struct HistArgs {
    uint32_t *hist;  // [kHistWords]: byte counts of the values (cleared by each use)
    uint2 *hrec;     // [kHistBuckets] bucket records
    uint32_t *htot;  // [kHistTiles] histogram tile totals
};

// the four byte counts of x (each at most 3) as 2-bit fields
__device__ __forceinline__ uint32_t pack2(uint32_t x) {
    return (x & 0x3u) | ((x >> 6) & 0xCu) | ((x >> 12) & 0x30u) | ((x >> 18) & 0xC0u);
}

// Offset (32-bit words) of the histogram tile prefix in the tile's threshold
// buffer, past the offspring ends of select_tile_closed.
constexpr int kHistTpreOffset = kScanTile + kScanTile / 8;
static_assert(kHistTpreOffset >= kScanTile + kScanTile / 32, "clear of the offspring ends");
static_assert(kHistTpreOffset + kHistTiles <= 2 * (kScanTile + kScanTile / 8), "inside the threshold buffer");

// H(v) for v in [0, 2^24]: the tile prefix (shared memory), the bucket
// prefix and the draws below v in its bucket (from the record, or from the
// byte counts of a bucket with a value drawn more than 3 times)
struct HistMap {
    const uint4 *hist;
    const uint2 *hrec;
    const uint32_t *tpre;
    int64_t m;  // number of draws
    __device__ __forceinline__ int64_t bucket(int64_t v) const {
        return min(v, (int64_t(1) << kHistValueBits) - 1) >> 4;
    }
    __device__ __forceinline__ int64_t finish(int64_t v, uint2 r) const {
        if (v >= (int64_t(1) << kHistValueBits)) return m;
        const int64_t bk = v >> 4;
        const int p = (int)(v & 15);
        uint32_t in;
        if (r.x >> 31) {
            const uint4 w = hist[bk];
            in = byte_sum(bytes_below(w.x, p)) + byte_sum(bytes_below(w.y, p - 4)) +
                 byte_sum(bytes_below(w.z, p - 8)) + byte_sum(bytes_below(w.w, p - 12));
        } else {
            const uint32_t f = r.y & ((1u << (2 * p)) - 1u);  // the fields below p (2p <= 30)
            in = (uint32_t)__popc(f & 0x55555555u) + 2u * (uint32_t)__popc(f & 0xAAAAAAAAu);
        }
        return (int64_t)tpre[bk / kScanTile] + (int64_t)(r.x & 0x7FFFFFFFu) + (int64_t)in;
    }
    // Loads through L1: neighbouring boundaries of a thread and a warp share
    // records, and no SM loads these lines before the grid barrier whose
    // acquire orders them after the writes.
    __device__ __forceinline__ int64_t operator()(int64_t v) const { return finish(v, hrec[bucket(v)]); }
    // K[e] = H(K[e]) for the tile's entries e = threadIdx.x + j kBlock (a
    // warp's loads then cover neighbouring particles, whose records are
    // neighbours) and, in thread 0, *k0 = H(*k0): every record load issued
    // first
    static constexpr bool kActive = true;
    __device__ __forceinline__ void map_block(int32_t *K, int64_t *k0) const {
        int32_t v[kScanItems];
        uint2 r[kScanItems];
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            v[j] = K[pad32((int)threadIdx.x + j * kBlock)];
            r[j] = hrec[bucket(v[j])];
        }
        int64_t v0 = 0;
        uint2 r0 = make_uint2(0u, 0u);
        if (threadIdx.x == 0) {
            v0 = *k0;
            r0 = hrec[bucket(v0)];
        }
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) K[pad32((int)threadIdx.x + j * kBlock)] = (int32_t)finish(v[j], r[j]);
        if (threadIdx.x == 0) *k0 = finish(v0, r0);
    }
};

// The block's share of the draws k in [0, m) of iteration t (Philox calls
// [calls b / G, calls (b + 1) / G)) counted into the histogram.  A byte that
// wraps lowers the histogram's total by 255 or 256, which the selection
// phase detects.
__device__ __forceinline__ void hist_draws(uint2 key, uint32_t stream, uint32_t t, int64_t m, uint32_t *hist, int b,
                                           int G) {
    const int64_t calls = (m + 3) >> 2;
    const int64_t c_lo = calls * b / G, c_hi = calls * (b + 1) / G;
    for (int64_t cc = c_lo + threadIdx.x; cc < c_hi; cc += kBlock) {
        const uint4 w = resample_words(key, stream, t, 4 * cc);
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (4 * cc + j < m) {
                const uint32_t v = u24(ww[j]);
                atomicAdd(&hist[v >> 2], 1u << (8u * (v & 3u)));
            }
        }
    }
}

// Bucket prefixes of histogram tile ht within the tile (thread t takes the
// buckets r kBlock + t, coalesced) and the tile's total.
__device__ __forceinline__ void hist_scan_tile(const uint4 *h, uint2 *hrec, uint32_t *htot, int ht) {
    __shared__ uint32_t s_w[kScanItems][kBlock / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t b0 = (int64_t)ht * kScanTile;
    // c: the bucket's count (at most 16 * 255) with the record's bit 31
    uint32_t c[kScanItems], inc[kScanItems], f2[kScanItems];
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const uint4 w = __ldcg(&h[b0 + r * kBlock + tid]);
        inc[r] = byte_sum(w.x) + byte_sum(w.y) + byte_sum(w.z) + byte_sum(w.w);
        c[r] = inc[r] | (((w.x | w.y | w.z | w.w) & 0xFCFCFCFCu) ? 0x80000000u : 0u);
        f2[r] = pack2(w.x) | (pack2(w.y) << 8) | (pack2(w.z) << 16) | (pack2(w.w) << 24);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int r = 0; r < kScanItems; ++r) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc[r], o);
            if (lane >= o) inc[r] += y;
        }
    }
    __syncthreads();  // s_w may still be read for the previous tile
    if (lane == 31)
#pragma unroll
        for (int r = 0; r < kScanItems; ++r) s_w[r][warp] = inc[r];
    __syncthreads();
    uint32_t row = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        uint32_t wpre = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) {
            const uint32_t x = s_w[r][w];
            tot += x;
            wpre += (w < warp) ? x : 0u;
        }
        const uint32_t prefix = row + wpre + inc[r] - (c[r] & 0x7FFFFFFFu);
        hrec[b0 + r * kBlock + tid] = make_uint2(prefix | (c[r] & 0x80000000u), f2[r]);
        row += tot;
    }
    if (tid == 0) htot[ht] = row;
}

// Exclusive prefix of the histogram tile totals into tpre (shared memory),
// by the whole block; returns the histogram's total to every thread.
__device__ __forceinline__ uint32_t hist_tile_prefix(const uint32_t *htot, uint32_t *tpre) {
    static_assert(kHistTiles == 2 * kBlock, "two histogram tiles per thread");
    __shared__ uint32_t s_w[kBlock / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t a = __ldcg(&htot[2 * tid]), b = __ldcg(&htot[2 * tid + 1]);
    uint32_t inc = a + b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) {
        const uint32_t x = s_w[w];
        tot += x;
        wpre += (w < warp) ? x : 0u;
    }
    const uint32_t ex = wpre + inc - (a + b);
    tpre[2 * tid] = ex;
    tpre[2 * tid + 1] = ex + a;
    __syncthreads();
    return tot;
}

// One-pass multinomial resampling: a cooperative launch of one full wave.
// Phase 1: the block's share of the histogram cleared (full-line stores: the
// lines are allocated in L2 without a DRAM read) and the tile sums of its
// weight tiles (the last tile's scan kept); grid barrier; phase 2: the
// block's share of the N draws counted into the histogram (L2 atomics), then
// its weight prefix and targets; grid barrier; phase 3: the bucket records
// of its histogram tiles; grid barrier; phase 4: selection of its weight
// tiles with K(X) = H(v(X)).  A block may own no weight tile or no
// histogram tile.
template <typename R, class Sink>
__global__ void __launch_bounds__(kBlock, 4) grid_multinomial_kernel(QGen<R> gen, GridTargets<false> tgt, AncOut out,
                                                                  Sink sink, int64_t n, unsigned long long *tsum,
                                                                  unsigned long long *bsum, HistArgs h, DevState *st,
                                                                  int gate) {
    __shared__ TileBufs tb;
    asm volatile("griddepcontrol.wait;" ::: "memory");  // as in grid_resample_kernel
    const DevState *sv = snapshot(st, true);
    if (gated_out(sv, gate)) return;
    QGen<R> g = gen;
    g.prepare(sv);
    const int G = gridDim.x, b = blockIdx.x;
    {
        uint4 *h4 = reinterpret_cast<uint4 *>(h.hist);
        const int64_t z_hi = kHistBuckets * (b + 1) / G;
        for (int64_t i = kHistBuckets * b / G + threadIdx.x; i < z_hi; i += kBlock) h4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
    const int t_lo = (int)((int64_t)ntiles * b / G), t_hi = (int)((int64_t)ntiles * (b + 1) / G);
    unsigned long long bs = 0, last = 0;
    for (int tile = t_lo; tile < t_hi - 1; ++tile) {
        const unsigned long long s = tile_sum(g, n, tile);  // to thread 0
        if (threadIdx.x == 0) {
            tsum[tile] = s;
            bs += s;
        }
    }
    if (t_hi > t_lo) last = scan_tile_local(g, n, t_hi - 1, tb);
    if (threadIdx.x == 0) {
        if (t_hi > t_lo) tsum[t_hi - 1] = last;
        bsum[b] = bs + last;
    }
    if (!grid_barrier(st, G)) return out.report(st);
    if (b == 0 && threadIdx.x == 0) st->ready = 1;
    hist_draws(tgt.key, tgt.stream, (uint32_t)sv->t, n, h.hist, b, G);
    // the block's weight prefix and targets (the block sums are complete)
    // while the other blocks' atomics drain
    unsigned long long pre = 0, QN = 0, before_last = 0;  // before_last: sum of the block's other tiles
    const GridTargets<false> *tg = nullptr;  // the block's copy in shared memory (no registers across phases)
    if (t_hi > t_lo) {  // the same branch in the whole block
        tile_prefix_total(bsum, b, G, &pre, &QN);
        tg = &block_targets_ref(tgt, sv, QN);
        if (t_hi - 1 > t_lo) {
            for (int tile = t_lo + (int)threadIdx.x; tile < t_hi - 1; tile += kBlock)
                before_last += __ldcg(&tsum[tile]);
            before_last = block_sum_u64(before_last);
        }
    }
    if (!grid_barrier(st, 2 * G)) return out.report(st);
    const int h_lo = (int)((int64_t)kHistTiles * b / G), h_hi = (int)((int64_t)kHistTiles * (b + 1) / G);
    for (int ht = h_lo; ht < h_hi; ++ht) hist_scan_tile(reinterpret_cast<const uint4 *>(h.hist), h.hrec, h.htot, ht);
    if (!grid_barrier(st, 3 * G)) return out.report(st);
    if (t_hi > t_lo) {
        uint32_t *tpre = reinterpret_cast<uint32_t *>(tb.tau) + kHistTpreOffset;
        const uint32_t total = hist_tile_prefix(h.htot, tpre);
        if (total != (uint32_t)n && threadIdx.x == 0) {  // a wrapped count
            raise_error(st, SMC_E_RANGE);
            out.report(st);
        }
        const HistMap km{reinterpret_cast<const uint4 *>(h.hist), h.hrec, tpre, n};
        select_tile_grid(*tg, out, sink, n, t_hi - 1, pre + before_last, last, QN, st, tb, km);
        for (int tile = t_lo; tile < t_hi - 1; ++tile) {
            const unsigned long long ts = scan_tile_local(g, n, tile, tb);
            select_tile_grid(*tg, out, sink, n, tile, pre, ts, QN, st, tb, km);
            pre += ts;
        }
    }
    grid_depart(st);
}

// ------------------------------------- in-place ("j stays j") ancestors --
//
// The copy(N, copy_from) convention of Sec. 4.1.2 lets copy_from[k] name the
// parent of new particle k in any arrangement of the ancestor multiset.  The
// in-place arrangement keeps every particle with offspring in its own slot
// (copy_from[j] = j) and fills the slots of particles without offspring with
// the extra copies, both in increasing order, so that a gather reads almost
// only its own slot.  From the sorted ancestors a_k: output k is a first copy
// when k = 0 or a_k != a_{k-1}; the extra copies in increasing k are the
// extras in increasing parent order; with F_k the first copies up to k and
// S_j the survivors below slot j,
//     extra[k - F_k] = a_k (k not a first copy),   surv[a_k] = 1 (first copy),
//     copy_from[j] = j if surv[j], else extra[j - S_j].
// One cooperative wave over tiles of kScanTile outputs, three grid barriers.

// Exclusive block scan of one count per thread; *total receives the sum.
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *total) {
    __shared__ uint32_t s_w[kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) {
        if (w < warp) pre += s_w[w];
        tot += s_w[w];
    }
    *total = tot;
    return pre + inc - v;
}

struct InplaceArgs {
    int32_t *anc;
    int32_t *extra;   // [N] extra copies in order
    int32_t *surv;    // [N] 1 where the particle has offspring
    unsigned long long *tf, *ts;  // per-tile counts of first copies and of survivors
    unsigned long long *bf, *bs;  // per-block counts
};

__global__ void __launch_bounds__(kBlock, 4) inplace_kernel(InplaceArgs ia, int64_t n, DevState *st) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const DevState *sv = snapshot(st, true);
    if (sv->error || !sv->ready) return;  // nothing was resampled
    const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
    const int G = gridDim.x, b = blockIdx.x;
    const int t_lo = (int)((int64_t)ntiles * b / G), t_hi = (int)((int64_t)ntiles * (b + 1) / G);
    const int base = threadIdx.x * kScanItems;
    // phase 1: first copies per tile; the survivor flags of the tile cleared
    unsigned long long bf = 0;
    for (int tile = t_lo; tile < t_hi; ++tile) {
        const int64_t k0 = (int64_t)tile * kScanTile + base;
        uint32_t f = 0;
        int32_t prev = (k0 > 0 && k0 - 1 < n) ? __ldcg(ia.anc + k0 - 1) : -1;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int64_t k = k0 + j;
            if (k < n) {
                const int32_t a = __ldcg(ia.anc + k);
                f += (a != prev) ? 1u : 0u;
                prev = a;
                ia.surv[k] = 0;
            }
        }
        uint32_t tot;
        block_excl_scan_u32(f, &tot);
        if (threadIdx.x == 0) ia.tf[tile] = tot;
        bf += tot;
    }
    if (threadIdx.x == 0) ia.bf[b] = bf;
    if (!grid_barrier(st, G)) return;
    // phase 2: extras to their rank, survivor flags
    unsigned long long pre, total;
    tile_prefix_total(ia.bf, b, G, &pre, &total);
    for (int tile = t_lo; tile < t_hi; ++tile) {
        const int64_t k0 = (int64_t)tile * kScanTile + base;
        int32_t a[kScanItems];
        bool first[kScanItems];
        uint32_t f = 0;
        int32_t prev = (k0 > 0 && k0 - 1 < n) ? __ldcg(ia.anc + k0 - 1) : -1;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int64_t k = k0 + j;
            a[j] = (k < n) ? __ldcg(ia.anc + k) : -1;
            first[j] = (k < n) && (a[j] != prev);
            f += first[j] ? 1u : 0u;
            prev = a[j];
        }
        uint32_t tot;
        unsigned long long F = pre + block_excl_scan_u32(f, &tot);  // first copies before the thread's items
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int64_t k = k0 + j;
            if (k >= n) break;
            if (first[j]) {
                ++F;
                ia.surv[a[j]] = 1;
            } else {
                ia.extra[k - (int64_t)F] = a[j];
            }
        }
        pre += tot;
    }
    if (!grid_barrier(st, 2 * G)) return;
    // phase 3: survivors per tile
    unsigned long long bs = 0;
    for (int tile = t_lo; tile < t_hi; ++tile) {
        const int64_t j0 = (int64_t)tile * kScanTile + base;
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j)
            if (j0 + j < n) c += (uint32_t)__ldcg(ia.surv + j0 + j);
        uint32_t tot;
        block_excl_scan_u32(c, &tot);
        if (threadIdx.x == 0) ia.ts[tile] = tot;
        bs += tot;
    }
    if (threadIdx.x == 0) ia.bs[b] = bs;
    if (!grid_barrier(st, 3 * G)) return;
    // phase 4: the arrangement
    tile_prefix_total(ia.bs, b, G, &pre, &total);
    for (int tile = t_lo; tile < t_hi; ++tile) {
        const int64_t j0 = (int64_t)tile * kScanTile + base;
        int32_t sv8[kScanItems];
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            sv8[j] = (j0 + j < n) ? __ldcg(ia.surv + j0 + j) : 0;
            c += (uint32_t)sv8[j];
        }
        uint32_t tot;
        unsigned long long S = pre + block_excl_scan_u32(c, &tot);  // survivors before the thread's slots
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int64_t jj = j0 + j;
            if (jj >= n) break;
            if (sv8[j]) {
                ia.anc[jj] = (int32_t)jj;
                ++S;
            } else {
                ia.anc[jj] = __ldcg(ia.extra + (jj - (int64_t)S));
            }
        }
        pre += tot;
    }
    grid_depart(st);
}

// ------------------------------------------------- residual, one pass --
//
// Residual resampling (deterministic copies d_i = floor(N q_i / Q_N), then
// R = N - sum d multinomial draws on the residual weights
// r_i = (N q_i - d_i Q_N) >> s, s = max(0, bitlen(R Q_N) - 62)) with the
// offspring in particle order: particle i owns the outputs [O_{i-1}, O_i),
// O_i = D_i + H_R(v(RQ_i)), D and RQ the prefix sums of d and r, H_R the
// histogram count of the R draws below a value and v the multinomial value
// threshold taken on RQ_N.

// per-tile and per-block sums of the three passes (q, d, r)
struct ResidualSums {
    unsigned long long *tq, *td, *tr;  // [ntiles]
    unsigned long long *bq, *bd, *br;  // [gridDim.x]
};

// d_i and r_i of the thread's kScanItems particles from the tile's q scan in
// tb.q (zeros past n give zeros)
__device__ __forceinline__ void residual_items(const TileBufs &tb, unsigned long long N, unsigned long long QN,
                                               int shift, unsigned long long (&d)[kScanItems],
                                               unsigned long long (&r)[kScanItems]) {
    const int base = threadIdx.x * kScanItems;
    unsigned long long prev = base ? tb.q[pad8(base - 1)] : 0ull;
    const float inv_qn = QN ? __fdividef(1.0f, u64_to_float(QN)) : 0.0f;  // the estimate's error is corrected exactly
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const unsigned long long qc = tb.q[pad8(base + j)];
        const unsigned long long qi = qc - prev;
        prev = qc;
        d[j] = floor_nq_over(N, qi, QN, inv_qn);
        r[j] = (N * qi - d[j] * QN) >> shift;  // the remainder is below Q_N: exact modulo 2^64
    }
}

// The residual count map: O = H_R(v) + the deterministic copies up to the
// boundary (d0 before the tile, dloc[j] the tile-relative inclusive prefix)
struct ResidualMap {
    static constexpr bool kActive = true;
    HistMap hm;
    int64_t d0;
    const int32_t *dloc;  // pad32 layout
    __device__ __forceinline__ void map_block(int32_t *K, int64_t *k0) const {
        hm.map_block(K, k0);  // the same entries per thread as below
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int e = pad32((int)threadIdx.x + j * kBlock);
            K[e] += (int32_t)(d0 + dloc[e]);
        }
        if (threadIdx.x == 0) *k0 += d0;
    }
};

// q, d and r of one tile into the tile buffers for the selection: the q scan
// in tb.q on entry (kept or rescanned); on exit tb.q holds the r scan and
// tb.a the d scan (tile-relative, int32: at most N).  d_known: the thread's
// own entries of tb.a already hold its d_i (kept from the d-sum pass).
__device__ __forceinline__ void residual_tile_scans(TileBufs &tb, unsigned long long N, unsigned long long QN,
                                                    int shift, bool d_known = false) {
    unsigned long long d[kScanItems], r[kScanItems];
    if (d_known) {
        const int b0 = threadIdx.x * kScanItems;
        unsigned long long prev = b0 ? tb.q[pad8(b0 - 1)] : 0ull;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const unsigned long long qc = tb.q[pad8(b0 + j)];
            d[j] = (unsigned long long)(uint32_t)tb.a[pad32(b0 + j)];
            r[j] = (N * (qc - prev) - d[j] * QN) >> shift;
            prev = qc;
        }
    } else {
        residual_items(tb, N, QN, shift, d, r);
    }
    scan_items_q(d, tb);  // d scan (every thread has read its q entries before the first barrier inside)
    const int base = threadIdx.x * kScanItems;
    int32_t *dl = tb.a;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) dl[pad32(base + j)] = (int32_t)tb.q[pad8(base + j)];
    scan_items_q(r, tb);
}

// The residual count map of the systematic and stratified residual steps:
// O = K_R(RQ) from the closed form over the R residual outputs, plus the
// deterministic copies up to the boundary (d0 before the tile, dl[j] the
// tile-relative inclusive prefix of the entries the thread maps).  The
// entries are taken into registers before the selection: the stratified
// selection stages its draw table in the buffer that held them.
struct DPrefixMap {
    static constexpr bool kActive = true;
    int64_t d0;
    int32_t dl[kScanItems];
    // from the d scan (pad32 layout); the caller synchronises the block
    // before anything overwrites dloc
    __device__ __forceinline__ void load(const int32_t *dloc) {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) dl[j] = dloc[pad32((int)threadIdx.x + j * kBlock)];
    }
    __device__ __forceinline__ void map_block(int32_t *K, int64_t *k0) const {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) K[pad32((int)threadIdx.x + j * kBlock)] += (int32_t)(d0 + dl[j]);
        if (threadIdx.x == 0) *k0 += d0;
    }
};

// Residual steps: the R residual outputs drawn multinomially (a histogram
// of R iid draws, as for multinomial resampling), systematically (one
// uniform, targets (k + u) / R) or stratified (targets (k + u_k) / R).
constexpr int kResMultinomial = 0, kResSystematic = 1, kResStratified = 2;

template <int kMode>
using ResidualTargets = GridTargets<kMode == kResStratified>;

// One-pass residual resampling: a cooperative launch of one full wave.
// Phase 1: histogram share cleared, q tile sums (a block with one tile keeps
// its q scan until phase 3); barrier; phase 2: Q_N, d sums (a block with one
// tile keeps its d_i until phase 3; the stored CDF); barrier; phase 3: R and
// s, the R draws into the histogram, r sums (a kept tile gets its d and r
// scans); barrier; phase 4: the bucket records of the block's histogram
// tiles, its r prefix and targets; barrier; phase 5: selection.  Blocks with
// several tiles rescan the q of every tile in every phase.  The systematic
// and stratified residual steps use no histogram: their targets are the
// closed form over R outputs (set up on the device once R is known).
template <typename R, class Sink, int kMode = kResMultinomial>
__global__ void __launch_bounds__(kBlock, 4) grid_residual_kernel(QGen<R> gen, ResidualTargets<kMode> tgt, AncOut out,
                                                               Sink sink, int64_t n, ResidualSums rs, HistArgs h,
                                                               DevState *st, int gate) {
    constexpr bool kHist = (kMode == kResMultinomial);
    __shared__ TileBufs tb;
    asm volatile("griddepcontrol.wait;" ::: "memory");  // as in grid_resample_kernel
    const DevState *sv = snapshot(st, true);
    if (gated_out(sv, gate)) return;
    QGen<R> g = gen;
    g.prepare(sv);
    const int G = gridDim.x, b = blockIdx.x;
    const unsigned long long N = (unsigned long long)n;
    if constexpr (kHist) {
        uint4 *h4 = reinterpret_cast<uint4 *>(h.hist);
        const int64_t z_hi = kHistBuckets * (b + 1) / G;
        for (int64_t i = kHistBuckets * b / G + threadIdx.x; i < z_hi; i += kBlock) h4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
    const int t_lo = (int)((int64_t)ntiles * b / G), t_hi = (int)((int64_t)ntiles * (b + 1) / G);
    const bool keep = (t_hi - t_lo == 1);  // the one tile's q scan stays in tb.q
    // phase 1: q tile sums
    unsigned long long bq = 0;
    for (int tile = t_lo; tile < t_hi; ++tile) {
        const unsigned long long s = scan_tile_local(g, n, tile, tb);
        if (threadIdx.x == 0) rs.tq[tile] = s;
        bq += s;
    }
    if (threadIdx.x == 0) rs.bq[b] = bq;
    if (!grid_barrier(st, G)) return out.report(st);
    if (b == 0 && threadIdx.x == 0) st->ready = 1;
    // phase 2: d sums; the CDF of q where it is stored
    unsigned long long pre_q, QN;
    tile_prefix_total(rs.bq, b, G, &pre_q, &QN);
    unsigned long long bd = 0;
    for (int tile = t_lo; tile < t_hi; ++tile) {
        const unsigned long long ts = keep ? bq : scan_tile_local(g, n, tile, tb);
        unsigned long long d[kScanItems], r[kScanItems];
        residual_items(tb, N, QN, 0, d, r);
        unsigned long long sd = 0;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            sd += d[j];
            if (keep) tb.a[pad32((int)threadIdx.x * kScanItems + j)] = (int32_t)d[j];  // kept for phase 3
        }
        sd = block_sum_u64(sd);
        if (threadIdx.x == 0) rs.td[tile] = sd;
        bd += sd;
        if (Sink::kActive) select_tile(NoTargets{}, out, sink, n, tile, pre_q, ts, QN, st, tb);
        pre_q += ts;
    }
    if (threadIdx.x == 0) rs.bd[b] = bd;
    if (!grid_barrier(st, 2 * G)) return out.report(st);
    // phase 3: R, s, the draws; r sums (a kept tile also gets its d and r scans)
    unsigned long long pre_d, Dtot;
    tile_prefix_total(rs.bd, b, G, &pre_d, &Dtot);
    const unsigned long long Rn = Dtot < N ? N - Dtot : 0ull;
    const int shift = max(0, bitlen128(mul64(Rn, QN)) - 62);
    if constexpr (kHist) hist_draws(tgt.key, tgt.stream, (uint32_t)sv->t, (int64_t)Rn, h.hist, b, G);
    unsigned long long br = 0;
    for (int tile = t_lo; tile < t_hi; ++tile) {
        unsigned long long sr;
        if (keep) {
            residual_tile_scans(tb, N, QN, shift, true);
            sr = tb.q[pad8(kScanTile - 1)];
        } else {
            scan_tile_local(g, n, tile, tb);
            unsigned long long d[kScanItems], r[kScanItems];
            residual_items(tb, N, QN, shift, d, r);
            sr = 0;
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) sr += r[j];
            sr = block_sum_u64(sr);
        }
        if (threadIdx.x == 0) rs.tr[tile] = sr;
        br += sr;
    }
    if (threadIdx.x == 0) rs.br[b] = br;
    if (!grid_barrier(st, 3 * G)) return out.report(st);
    // phase 4: histogram tiles; the r prefix and the targets on RQ_N
    if constexpr (kHist) {
        const int h_lo = (int)((int64_t)kHistTiles * b / G), h_hi = (int)((int64_t)kHistTiles * (b + 1) / G);
        for (int ht = h_lo; ht < h_hi; ++ht)
            hist_scan_tile(reinterpret_cast<const uint4 *>(h.hist), h.hrec, h.htot, ht);
    }
    unsigned long long pre_r, RQN;
    tile_prefix_total(rs.br, b, G, &pre_r, &RQN);
    // RQ_N = 0 exactly when R = 0: any positive total then gives v = 0 and H = 0
    // (and for the closed form over R = 0 outputs, K = 0 everywhere)
    ResidualTargets<kMode> proto = tgt;
    if constexpr (!kHist) {
        proto.n = (int64_t)Rn;
        proto.mrec = Rn ? ~0ull / Rn : 0ull;
    }
    const ResidualTargets<kMode> tg = block_targets(proto, sv, RQN ? RQN : 1ull);
    if constexpr (kHist) {
        if (!grid_barrier(st, 4 * G)) return out.report(st);
    }
    // phase 5: selection
    if (t_hi > t_lo) {  // the same branch in the whole block
        unsigned long long d0 = pre_d, r0 = pre_r;
        if constexpr (kHist) {
            uint32_t *tpre = reinterpret_cast<uint32_t *>(tb.tau) + kHistTpreOffset;
            const uint32_t total = hist_tile_prefix(h.htot, tpre);
            if (total != (uint32_t)Rn && threadIdx.x == 0) {  // a wrapped count
                raise_error(st, SMC_E_RANGE);
                out.report(st);
            }
            const HistMap hm{reinterpret_cast<const uint4 *>(h.hist), h.hrec, tpre, (int64_t)Rn};
            for (int tile = t_lo; tile < t_hi; ++tile) {
                if (!keep) {
                    scan_tile_local(g, n, tile, tb);
                    residual_tile_scans(tb, N, QN, shift);
                }
                const ResidualMap km{hm, (int64_t)d0, tb.a};
                select_tile_closed(tg, out, n, tile, r0, RQN ? RQN : 1ull, tb, km);
                d0 += __ldcg(&rs.td[tile]);
                r0 += __ldcg(&rs.tr[tile]);
            }
        } else {
            for (int tile = t_lo; tile < t_hi; ++tile) {
                if (!keep) {
                    scan_tile_local(g, n, tile, tb);
                    residual_tile_scans(tb, N, QN, shift);
                }
                DPrefixMap km;
                km.d0 = (int64_t)d0;
                km.load(tb.a);
                __syncthreads();  // every thread holds its d prefix before tb.a is reused
                select_tile_closed(tg, out, n, tile, r0, RQN ? RQN : 1ull, tb, km);
                d0 += __ldcg(&rs.td[tile]);
                r0 += __ldcg(&rs.tr[tile]);
            }
        }
    }
    grid_depart(st);
}

}  // namespace smc
