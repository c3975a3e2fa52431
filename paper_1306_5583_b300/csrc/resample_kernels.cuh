// Resampling (Sec. 2.1, eq:resample; Douc et al. 2005 schemes; copy_from
// convention of Sec. 4.1.2) on exact 64-bit fixed-point weights.
//
// Weights: q_i = floor(exp(lw_i - M) 2^F), F = 61 - ceil(log2 N), so the
// inclusive prefix sums Q_i are exact integers below 2^62: the CDF is
// order-independent and bit-reproducible, and the decoupled look-back scan
// may add either predecessor aggregates or inclusive prefixes.
// Targets are rationals P_k / D (D = N 2^25, u = (2j + 1) / 2^25):
//   systematic  P_k = 2^25 k + 2j + 1         (one j per iteration)
//   stratified  P_k = 2^25 k + 2j_k + 1       (j_k independent)
//   multinomial P_k = N (2 j_(k) + 1)         (j_(k) sorted iid j's)
// and a_k = min{ i : Q_i D > Q_N P_k }, found by binary search over CDF
// tiles staged in shared memory.  Residual resampling keeps
// floor(N q_i / Q_N) copies and draws the rest multinomially from the
// remainders (multinomial residual step).
#pragma once

#include "smc_device.cuh"

namespace smc {

// ---------------------------------------------------------------- scans --

__device__ __forceinline__ unsigned long long ld_status(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void st_status(unsigned long long *p, unsigned long long v) {
    *(volatile unsigned long long *)p = v;
}

// Warp 0: exclusive prefix of tile `tile` from its predecessors' status
// words.  Waits are bounded; on timeout the error word is set and the
// missing predecessor counts as zero.
__device__ __forceinline__ unsigned long long lookback(const unsigned long long *status, int tile,
                                                       DevState *st) {
    const int lane = threadIdx.x & 31;
    unsigned long long prefix = 0;
    int pred = tile - 1;
    while (true) {
        const int idx = pred - lane;
        unsigned long long s = kStatIncl;  // before tile 0: an inclusive zero
        if (idx >= 0) {
            uint32_t spins = 0;
            s = ld_status(&status[idx]);
            while ((s & kStatMask) == 0) {
                if (++spins > kSpinLimit) {
                    raise_error(st, SMC_E_TIMEOUT);
                    s = kStatIncl;
                    break;
                }
                if (spins > 64) __nanosleep(64);
                s = ld_status(&status[idx]);
            }
        }
        const unsigned incl = __ballot_sync(0xffffffffu, (s & kStatMask) == kStatIncl);
        const int stop = incl ? __ffs(incl) - 1 : 32;
        const unsigned long long v = (lane <= stop) ? (s & ~kStatMask) : 0ull;
        prefix += warp_sum(v);
        if (incl) break;
        pred -= 32;
    }
    return prefix;
}

// Exact inclusive scan out(i, sum_{j <= i} gen(j)), i < n, one tile of
// kScanTile elements per block, tiles taken in launch order from a
// per-slot counter (so every predecessor has started: the look-back always
// finishes).  Each launch clears its tiles' entries of the other status
// array and the last block to finish flips the slot's parity.
template <class Gen, class Out>
__global__ void __launch_bounds__(kBlock) scan_kernel(Gen gen, Out out, int64_t n, ScanSlot slot, int slot_id,
                                                      DevState *st, int gate) {
    __shared__ unsigned long long s_v[kScanTile];
    __shared__ unsigned long long s_warp[kBlock / 32];
    __shared__ unsigned long long s_prefix;
    __shared__ int s_tile;
    if (*(volatile int32_t *)&st->error) return;
    if (gate && !*(volatile int32_t *)&st->due) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        const unsigned tile = atomicAdd(&st->scan_counter[slot_id], 1u);
        if (tile == gridDim.x - 1) st->scan_counter[slot_id] = 0;
        s_tile = (int)tile;
    }
    __syncthreads();
    const int tile = s_tile;
    const int parity = (int)(*(volatile uint32_t *)&st->scan_parity[slot_id] & 1u);
    unsigned long long *status = slot.status[parity];
    unsigned long long *other = slot.status[parity ^ 1];
    Gen g = gen;
    g.prepare(st);
    const int64_t t0 = (int64_t)tile * kScanTile;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const int64_t i = t0 + r * kBlock + tid;
        s_v[r * kBlock + tid] = (i < n) ? g(i) : 0ull;
    }
    __syncthreads();
    unsigned long long loc[kScanItems];
    unsigned long long acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        acc += s_v[tid * kScanItems + j];
        loc[j] = acc;
    }
    const unsigned long long winc = warp_incl_scan(acc);
    if (lane == 31) s_warp[warp] = winc;
    __syncthreads();
    unsigned long long wpre = 0, agg = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) {
        const unsigned long long v = s_warp[w];
        if (w < warp) wpre += v;
        agg += v;
    }
    const unsigned long long texcl = wpre + (winc - acc);
    if (warp == 0) {
        unsigned long long prefix = 0;
        if (tile == 0) {
            if (lane == 0) st_status(&status[0], kStatIncl | agg);
        } else {
            if (lane == 0) st_status(&status[tile], kStatAgg | agg);
            prefix = lookback(status, tile, st);
            if (lane == 0) st_status(&status[tile], kStatIncl | (prefix + agg));
        }
        if (lane == 0) {
            other[tile] = 0ull;
            s_prefix = prefix;
        }
    }
    __syncthreads();
    const unsigned long long pre = s_prefix + texcl;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) s_v[tid * kScanItems + j] = pre + loc[j];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const int64_t i = t0 + r * kBlock + tid;
        if (i < n) out(i, s_v[r * kBlock + tid], st);
    }
    // the last block to finish flips the parity of this slot
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&st->scan_done[slot_id], 1u);
        if (done == gridDim.x - 1) {
            st->scan_done[slot_id] = 0;
            st->scan_parity[slot_id] ^= 1u;
        }
    }
}

// ----------------------------------------------------------- generators --

// q_i = floor(exp(lw_i - M) 2^F) from the current log-weights.
template <typename R>
struct QGen {
    const R *lw[2];
    int frac;
    const R *cur_lw;
    R m;
    __device__ __forceinline__ void prepare(const DevState *st) {
        cur_lw = lw[*(const volatile int32_t *)&st->cur];
        m = R(*(const volatile double *)&st->max_lw);
    }
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const {
        return Math<R>::fixed(Math<R>::exp(cur_lw[i] - m), frac);
    }
};

struct QOut {
    unsigned long long *Q;
    int64_t n;
    __device__ __forceinline__ void operator()(int64_t i, unsigned long long v, DevState *st) const {
        Q[i] = v;
        if (i == n - 1) st->qn = v;
    }
};

// values read from an array (bucket counts)
struct CountGen {
    const uint32_t *cnt;
    __device__ __forceinline__ void prepare(const DevState *) {}
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const { return cnt[i]; }
};

struct StoreOut {
    unsigned long long *dst;
    __device__ __forceinline__ void operator()(int64_t i, unsigned long long v, DevState *) const { dst[i] = v; }
};

// floor(n q / qn) for q <= qn < 2^62, n < 2^31 (exact: float estimate, then
// integer correction with 128-bit products)
__device__ __forceinline__ unsigned long long floor_nq_over(unsigned long long n, unsigned long long q,
                                                            unsigned long long qn) {
    if (qn == 0 || q > qn) return 0;
    const U128 num = mul64(n, q);
    float est = (float(n) * float(q)) / float(qn);
    unsigned long long d = (unsigned long long)fmaxf(est, 0.0f);
    if (d > n) d = n;
    // d * qn <= num < (d + 1) * qn
    while (d > 0 && gt128(mul64(d, qn), num)) --d;
    while (!gt128(mul64(d + 1, qn), num)) ++d;
    return d;
}

// residual: deterministic copies d_i and remainders rem_i = n q_i - d_i Q_N
struct ResidualParts {
    const unsigned long long *Q;
    int64_t n;
    unsigned long long qn;
    __device__ __forceinline__ void prepare(const DevState *st) { qn = *(const volatile unsigned long long *)&st->qn; }
    __device__ __forceinline__ unsigned long long q(int64_t i) const { return i ? Q[i] - Q[i - 1] : Q[0]; }
    __device__ __forceinline__ unsigned long long d(int64_t i) const {
        return floor_nq_over((unsigned long long)n, q(i), qn);
    }
};

// residual weights r_i = rem_i >> s, s = max(0, bitlen(R Q_N) - 62)
struct ResidualRGen {
    ResidualParts p;
    int shift;
    __device__ __forceinline__ void prepare(const DevState *st) {
        p.prepare(st);
        const unsigned long long sd = *(const volatile unsigned long long *)&st->sum_d;
        const unsigned long long R = sd < (unsigned long long)p.n ? (unsigned long long)p.n - sd : 0ull;
        shift = max(0, bitlen128(mul64(R, p.qn)) - 62);
    }
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const {
        const unsigned long long qi = p.q(i);
        const unsigned long long di = floor_nq_over((unsigned long long)p.n, qi, p.qn);
        const unsigned long long rem = (unsigned long long)p.n * qi - di * p.qn;  // < Q_N, exact mod 2^64
        return rem >> shift;
    }
};

// final offspring o_i = d_i + (residual draws of i)
struct ResidualOGen {
    ResidualParts p;
    const uint32_t *extra;
    __device__ __forceinline__ void prepare(const DevState *st) { p.prepare(st); }
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const { return p.d(i) + extra[i]; }
};

// --------------------------------------------------------------- targets --

// P_k numerators for 4 consecutive outputs k4..k4+3 (k4 % 4 == 0), common
// denominator D, and the number of outputs.
struct SystematicTargets {
    int64_t n;
    uint2 key;
    uint32_t stream;
    unsigned long long j2p1;
    __device__ __forceinline__ void prepare(const DevState *st) {
        const uint32_t t = (uint32_t)*(const volatile int32_t *)&st->t;
        j2p1 = 2ull * u24(draw(key, 0u, t, TAG_RESAMPLE, stream, 0u).x) + 1ull;
    }
    __device__ __forceinline__ int64_t count(const DevState *) const { return n; }
    __device__ __forceinline__ unsigned long long denom(const DevState *) const { return (unsigned long long)n << 25; }
    __device__ __forceinline__ void get4(int64_t k4, unsigned long long P[4]) const {
#pragma unroll
        for (int j = 0; j < 4; ++j) P[j] = ((unsigned long long)(k4 + j) << 25) + j2p1;
    }
};

__device__ __forceinline__ uint4 resample_words(uint2 key, uint32_t stream, uint32_t t, int64_t k4) {
    return draw(key, (uint32_t)(k4 >> 2), t, TAG_RESAMPLE, stream, 0u);
}

struct StratifiedTargets {
    int64_t n;
    uint2 key;
    uint32_t stream;
    uint32_t t;
    __device__ __forceinline__ void prepare(const DevState *st) { t = (uint32_t)*(const volatile int32_t *)&st->t; }
    __device__ __forceinline__ int64_t count(const DevState *) const { return n; }
    __device__ __forceinline__ unsigned long long denom(const DevState *) const { return (unsigned long long)n << 25; }
    __device__ __forceinline__ void get4(int64_t k4, unsigned long long P[4]) const {
        const uint4 w = resample_words(key, stream, t, k4);
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) P[j] = ((unsigned long long)(k4 + j) << 25) + 2ull * u24(ww[j]) + 1ull;
    }
};

// sorted j's; m = number of draws (N, or R for the residual step)
struct SortedTargets {
    const uint32_t *sorted;
    int64_t n;        // used when from_residual == 0
    int64_t n_total;  // N (for R = N - sum_d)
    int from_residual;
    unsigned long long m;
    __device__ __forceinline__ void prepare(const DevState *st) {
        const unsigned long long sd = *(const volatile unsigned long long *)&st->sum_d;
        m = from_residual ? (sd < (unsigned long long)n_total ? (unsigned long long)n_total - sd : 0ull)
                          : (unsigned long long)n;
    }
    __device__ __forceinline__ int64_t count(const DevState *) const { return (int64_t)m; }
    __device__ __forceinline__ unsigned long long denom(const DevState *) const { return m << 25; }
    __device__ __forceinline__ void get4(int64_t k4, unsigned long long P[4]) const {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t k = k4 + j;
            P[j] = (k < (int64_t)m) ? m * (2ull * sorted[k] + 1ull) : 0ull;
        }
    }
};

// expansion of an offspring CDF O (O_N = n): a_k = min{i : O_i > k}
struct ExpandTargets {
    int64_t n;
    __device__ __forceinline__ void prepare(const DevState *) {}
    __device__ __forceinline__ int64_t count(const DevState *) const { return n; }
    __device__ __forceinline__ unsigned long long denom(const DevState *) const { return (unsigned long long)n; }
    __device__ __forceinline__ void get4(int64_t k4, unsigned long long P[4]) const {
#pragma unroll
        for (int j = 0; j < 4; ++j) P[j] = (unsigned long long)(k4 + j);
    }
};

// ------------------------------------------------------------ selection --

struct AncOut {
    int32_t *anc;
    __device__ __forceinline__ void operator()(int64_t k, int64_t a) const { anc[k] = (int32_t)a; }
};

struct CountOut {  // residual draws: histogram of the selected particles
    uint32_t *extra;
    __device__ __forceinline__ void operator()(int64_t, int64_t a) const { atomicAdd(&extra[a], 1u); }
};

// first i in [lo, hi) with Q_i D > target (hi when none)
__device__ __forceinline__ int64_t upper_bound_global(const unsigned long long *Q, int64_t lo, int64_t hi,
                                                      unsigned long long D, U128 target) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (gt128(mul64(__ldcg(&Q[mid]), D), target)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ int upper_bound_smem(const unsigned long long *s, int lo, int hi, unsigned long long D,
                                                U128 target) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (gt128(mul64(s[mid], D), target)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// a_k = min{ i : Q_i D > Q_N P_k } for k < count.  Block b handles outputs
// [b kSelTile, (b + 1) kSelTile); the tile ends of the CDF scan (its
// inclusive status words) locate the CDF tiles that hold the block's
// ancestors, which are staged in shared memory when they fit (at most
// kSelCap entries), else searched in global memory.
template <class Tgt, class Out>
__global__ void __launch_bounds__(kBlock) select_kernel(Tgt tgt, Out out, const unsigned long long *Q, int64_t n_cdf,
                                                        ScanSlot cdf_slot, int cdf_slot_id, DevState *st, int gate,
                                                        int set_ready, int spl_cap) {
    extern __shared__ unsigned long long s_dyn[];
    unsigned long long *s_spl = s_dyn;                   // [spl_cap] CDF tile ends
    unsigned long long *s_q = s_dyn + spl_cap;           // [kSelCap] staged CDF entries
    __shared__ int s_range[2];
    if (*(volatile int32_t *)&st->error) return;
    if (gate && !*(volatile int32_t *)&st->due) return;
    Tgt tg = tgt;
    tg.prepare(st);
    const int64_t count = tg.count(st);
    const int64_t k0 = (int64_t)blockIdx.x * kSelTile;
    if (set_ready && blockIdx.x == 0 && threadIdx.x == 0) st->ready = 1;
    if (k0 >= count) return;
    const unsigned long long D = tg.denom(st);
    const unsigned long long QN = __ldcg(&Q[n_cdf - 1]);
    const int ntiles = (int)((n_cdf + kScanTile - 1) / kScanTile);
    // the scan's parity was flipped when it finished: its status words are
    // in the other array
    const int parity = (int)((*(volatile uint32_t *)&st->scan_parity[cdf_slot_id] & 1u) ^ 1u);
    const unsigned long long *spl = cdf_slot.status[parity];
    const bool use_spl = ntiles <= spl_cap;
    if (use_spl) {
        for (int i = threadIdx.x; i < ntiles; i += kBlock) s_spl[i] = __ldcg(&spl[i]) & ~kStatMask;
    }
    // this thread's targets
    const int64_t k4 = k0 + 4 * (int64_t)threadIdx.x;
    unsigned long long P[4];
    tg.get4(k4, P);
    U128 T[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) T[j] = mul64(QN, P[j]);
    __syncthreads();
    // CDF range of the block: tiles holding a_{k0} and a_{last}
    const int64_t k_last = min(k0 + kSelTile, count) - 1;
    if (threadIdx.x == 0 || threadIdx.x == kBlock - 1) {
        const int64_t k = (threadIdx.x == 0) ? k0 : k_last;
        unsigned long long Pk[4];
        tg.get4(k & ~3ll, Pk);
        const U128 Tk = mul64(QN, Pk[k & 3]);
        int tl = 0;
        if (use_spl) tl = upper_bound_smem(s_spl, 0, ntiles, D, Tk);
        else tl = (threadIdx.x == 0) ? 0 : ntiles - 1;
        if (tl > ntiles - 1) tl = ntiles - 1;
        s_range[threadIdx.x == 0 ? 0 : 1] = tl;
    }
    __syncthreads();
    const int64_t lo = (int64_t)s_range[0] * kScanTile;
    const int64_t hi = min((int64_t)(s_range[1] + 1) * kScanTile, n_cdf);
    const bool staged = use_spl && (hi - lo) <= kSelCap;
    if (staged) {
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBlock) s_q[i - lo] = __ldcg(&Q[i]);
    }
    __syncthreads();
    int64_t prev = lo;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t k = k4 + j;
        if (k >= count) break;
        int64_t a;
        if (staged) a = lo + upper_bound_smem(s_q, (int)(prev - lo), (int)(hi - lo), D, T[j]);
        else a = upper_bound_global(Q, prev, n_cdf, D, T[j]);
        if (a >= n_cdf) a = n_cdf - 1;  // unreachable in exact arithmetic (P_k < D)
        out(k, a);
        prev = a;
    }
}

// ------------------------------------------------- sorting iid uniforms --

// j_k of resampling draw k at iteration t (word k % 4 of call k / 4)
__device__ __forceinline__ uint32_t resample_u24_at(uint2 key, uint32_t stream, uint32_t t, int64_t k) {
    const uint4 w = resample_words(key, stream, t, k & ~3ll);
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
    return u24(ww[k & 3]);
}

struct UniformSortArgs {
    uint2 key;
    uint32_t stream;
    int64_t n_total;      // N
    int from_residual;    // count = N - sum_d (residual step) or N
    int bucket_shift;     // bucket = j >> bucket_shift
    uint32_t *cnt;        // [nbuckets], zero on entry
    uint32_t *fill;       // [nbuckets], zero on entry
    unsigned long long *boff;  // [nbuckets] inclusive bucket ends
    uint32_t *sorted;     // [N]
    int64_t nbuckets;
};

__device__ __forceinline__ int64_t draw_count(const UniformSortArgs &a, const DevState *st) {
    if (!a.from_residual) return a.n_total;
    const unsigned long long sd = *(const volatile unsigned long long *)&st->sum_d;
    return sd < (unsigned long long)a.n_total ? a.n_total - (int64_t)sd : 0;
}

__global__ void __launch_bounds__(kBlock) bucket_count_kernel(UniformSortArgs a, DevState *st, int gate) {
    if (*(volatile int32_t *)&st->error) return;
    if (gate && !*(volatile int32_t *)&st->due) return;
    const int64_t count = draw_count(a, st);
    const uint32_t t = (uint32_t)st->t;
    const int64_t k4 = 4 * ((int64_t)blockIdx.x * kBlock + threadIdx.x);
    if (k4 >= count) return;
    const uint4 w = resample_words(a.key, a.stream, t, k4);
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (k4 + j < count) atomicAdd(&a.cnt[u24(ww[j]) >> a.bucket_shift], 1u);
}

__global__ void __launch_bounds__(kBlock) bucket_scatter_kernel(UniformSortArgs a, DevState *st, int gate) {
    if (*(volatile int32_t *)&st->error) return;
    if (gate && !*(volatile int32_t *)&st->due) return;
    const int64_t count = draw_count(a, st);
    const uint32_t t = (uint32_t)st->t;
    const int64_t k4 = 4 * ((int64_t)blockIdx.x * kBlock + threadIdx.x);
    if (k4 >= count) return;
    const uint4 w = resample_words(a.key, a.stream, t, k4);
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (k4 + j < count) {
            const uint32_t jj = u24(ww[j]);
            const int64_t b = jj >> a.bucket_shift;
            const unsigned long long start = a.boff[b] - a.cnt[b];
            const uint32_t pos = atomicAdd(&a.fill[b], 1u);
            a.sorted[start + pos] = jj;
        }
    }
}

// one thread per bucket: insertion sort of the (few) values in the bucket,
// then clear the counters for the next use
__global__ void __launch_bounds__(kBlock) bucket_sort_kernel(UniformSortArgs a, DevState *st, int gate) {
    if (*(volatile int32_t *)&st->error) return;
    if (gate && !*(volatile int32_t *)&st->due) return;
    const int64_t b = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (b >= a.nbuckets) return;
    const uint32_t c = a.cnt[b];
    if (c > 1) {
        const unsigned long long lo = a.boff[b] - c;
        for (uint32_t i = 1; i < c; ++i) {
            const uint32_t v = a.sorted[lo + i];
            uint32_t j = i;
            while (j > 0 && a.sorted[lo + j - 1] > v) {
                a.sorted[lo + j] = a.sorted[lo + j - 1];
                --j;
            }
            a.sorted[lo + j] = v;
        }
    }
    a.cnt[b] = 0;
    a.fill[b] = 0;
}

// ----------------------------------------------------------- residual ----

// sum_i d_i -> st->sum_d (zeroed by the weighting kernel); clears the
// residual draw histogram
__global__ void __launch_bounds__(kBlock) residual_d_kernel(ResidualParts p, uint32_t *extra, DevState *st, int gate) {
    __shared__ unsigned long long s_w[kBlock / 32];
    if (*(volatile int32_t *)&st->error) return;
    if (gate && !*(volatile int32_t *)&st->due) return;
    ResidualParts pp = p;
    pp.prepare(st);
    const int64_t i0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    unsigned long long acc = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const int64_t i = i0 + r * kBlock;
        if (i < pp.n) {
            acc += pp.d(i);
            extra[i] = 0u;
        }
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kBlock / 32; ++w) s += s_w[w];
        atomicAdd(&st->sum_d, s);
    }
}

}  // namespace smc
