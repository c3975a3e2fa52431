// Block partials and the last-block grid combine shared by every kernel
// that produces new log-weights: online (max, sum e, sum e^2, sum e*h)
// with e = exp(lw - max), then log-normaliser, ESS, evidence increment,
// monitor and the resample decision (Sec. 2.1 ESS; Sec. 2.2 ratio of
// normalising constants; Sec. 4.1.5 Monitor; Sec. 4.1.3 threshold).
#pragma once

#include "smc_device.cuh"

namespace smc {

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
};

// Block-level partial of E items per thread.  lw = -inf marks inactive
// items.  Per-thread and per-warp sums run in R; the 8 warp sums are
// combined in float64.
template <typename R, int E>
__device__ __forceinline__ void block_partial(const R (&lw)[E], const R (&h0)[E], const R (&h1)[E],
                                              const R (&h2)[E], Partial *out) {
    __shared__ R s_max[kBlock / 32];
    __shared__ double s_sum[kBlock / 32][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    R m = Math<R>::neg_inf();
#pragma unroll
    for (int j = 0; j < E; ++j) m = fmax(m, lw[j]);
    m = warp_max(m);
    if (lane == 0) s_max[warp] = m;
    __syncthreads();
    m = s_max[0];
#pragma unroll
    for (int w = 1; w < kBlock / 32; ++w) m = fmax(m, s_max[w]);

    R s1 = 0, s2 = 0, sa = 0, sb = 0, sc = 0;
    if (m > Math<R>::neg_inf()) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const R e = (lw[j] > Math<R>::neg_inf()) ? Math<R>::exp(lw[j] - m) : R(0);
            s1 += e;
            s2 += e * e;
            sa += e * h0[j];
            sb += e * h1[j];
            sc += e * h2[j];
        }
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    sc = warp_sum(sc);
    if (lane == 0) {
        s_sum[warp][0] = double(s1);
        s_sum[warp][1] = double(s2);
        s_sum[warp][2] = double(sa);
        s_sum[warp][3] = double(sb);
        s_sum[warp][4] = double(sc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0, t2 = 0, ta = 0, tb = 0, tc = 0;
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) {
            t1 += s_sum[w][0];
            t2 += s_sum[w][1];
            ta += s_sum[w][2];
            tb += s_sum[w][3];
            tc += s_sum[w][4];
        }
        Partial p;
        p.m = double(m);
        p.s1 = t1;
        p.s2 = t2;
        p.sx = ta;
        p.sy = tb;
        p.su = tc;
        p.pad[0] = p.pad[1] = 0;
        *out = p;
    }
}

// Scale factor exp(mb - M) in the kernel's precision.
template <typename R>
__device__ __forceinline__ double partial_scale(double mb, double M) {
    if (!(mb > -INFINITY)) return 0.0;
    return double(Math<R>::exp(R(mb - M)));
}

// Returns true in the one block that arrives last; that block then holds
// the grid-wide sums in *out (thread 0 only).
struct Combined {
    double M, S1, S2, Sa, Sb, Sc;
};

template <typename R>
__device__ __forceinline__ bool last_block_combine(DevState *st, const Partial *part, Combined *out) {
    __shared__ bool s_last;
    __shared__ double s_red[kBlock / 32][6];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&st->ticket, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int nb = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double M = -INFINITY;
    for (int b = threadIdx.x; b < nb; b += kBlock) M = fmax(M, __ldcg(&part[b].m));
    M = warp_max(M);
    if (lane == 0) s_red[warp][0] = M;
    __syncthreads();
    M = s_red[0][0];
#pragma unroll
    for (int w = 1; w < kBlock / 32; ++w) M = fmax(M, s_red[w][0]);
    __syncthreads();
    double S1 = 0, S2 = 0, Sa = 0, Sb = 0, Sc = 0;
    if (M > -INFINITY) {
        for (int b = threadIdx.x; b < nb; b += kBlock) {
            const double sc = partial_scale<R>(__ldcg(&part[b].m), M);
            const double sc2 = sc * sc;
            S1 += __ldcg(&part[b].s1) * sc;
            S2 += __ldcg(&part[b].s2) * sc2;
            Sa += __ldcg(&part[b].sx) * sc;
            Sb += __ldcg(&part[b].sy) * sc;
            Sc += __ldcg(&part[b].su) * sc;
        }
    }
    S1 = warp_sum(S1);
    S2 = warp_sum(S2);
    Sa = warp_sum(Sa);
    Sb = warp_sum(Sb);
    Sc = warp_sum(Sc);
    if (lane == 0) {
        s_red[warp][1] = S1;
        s_red[warp][2] = S2;
        s_red[warp][3] = Sa;
        s_red[warp][4] = Sb;
        s_red[warp][5] = Sc;
    }
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
    r->max_lw = c.M;
    r->t = f.t;
    r->resampled = due ? 1 : 0;
    r->status = SMC_OK;
    r->alpha = f.alpha;
    st->max_lw = c.M;
    st->log_norm = L;
    st->log_evidence = logz;
    st->ess = ess;
    st->due = due ? 1 : 0;
    *L_out = L;
    return true;
}

}  // namespace smc
