// WeightSet::add_log_weight (Sec. 4.1.6): multiply the current weights by
// exp(incw_i), i.e. lw_t,i += incw_i, then the normaliser, ESS, monitor and
// resample decision of the same iteration again (finalisation mode 1: the
// evidence increment L_t is replaced by the new one).  The new log-weights
// go to the other buffer, so a failure leaves the previous ones in place.
#pragma once

#include "weight_reduce.cuh"

namespace smc {

template <typename R>
struct AddArgs {
    int64_t n;
    const R *lw[2];     // log-weight buffers
    R *lw_w[2];
    const R *incw;      // n increments
    const R *h[2][2];   // [buffer][row] monitored rows (CV: x_pos, y_pos), or null (GMM)
    smc_record *rec;
    int32_t rec_cap;
    DevState *st;
    Partial *part;
    double threshold;
    float thr_df[2];
    int32_t thr_mode;
    int32_t gmm;        // GMM: keep the running shift base_shift = L_t
};

template <typename R>
__global__ void __launch_bounds__(kBlock) add_log_weight_kernel(AddArgs<R> a) {
    constexpr int E = kPfItems;
    DevState *st = a.st;
    const DevState *sv = snapshot(st);
    if (sv->error) return;
    const int cur = sv->cur, cur_lw = sv->cur_lw;
    const R *lw_in = a.lw[cur_lw];
    R *lw_out = a.lw_w[cur_lw ^ 1];
    const R *h0 = a.h[cur][0], *h1 = a.h[cur][1];
    const uint32_t n = (uint32_t)a.n;
    const uint32_t i0 = (blockIdx.x * (uint32_t)kBlock + threadIdx.x) * (uint32_t)E;
    R lw[E], inc[E], x0[E], x1[E], zero[E];
    load_k<R, E>(lw_in, i0, n, lw);
    load_k<R, E>(a.incw, i0, n, inc);
    if (h0) {
        load_k<R, E>(h0, i0, n, x0);
        load_k<R, E>(h1, i0, n, x1);
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
        lw[j] = (i0 + j < n) ? lw[j] + inc[j] : Math<R>::neg_inf();
        zero[j] = R(0);
        if (!h0) x0[j] = x1[j] = R(0);
    }
    store_k<R, E>(lw_out, i0, n, lw);
    block_partial<R, E, 2>(lw, x0, x1, zero, &a.part[blockIdx.x]);
    if (!take_ticket<R>(st)) return;
    FinalizeArgs f{st,  a.rec, a.rec_cap, sv->t, 1, a.n, a.threshold, sv->alpha, {a.thr_df[0], a.thr_df[1]},
                   a.thr_mode, sv->log_evidence};
    bool done = false;
    if constexpr (sizeof(R) == 4) {
        CombinedDF c;
        combine_partials_df<4>(a.part, gridDim.x, &c);
        // every thread; warp 0 also stores L_t as the GMM base shift
        done = finalize_weights_df(f, c, a.gmm ? &st->base_shift : nullptr);
    } else {
        Combined c;
        combine_partials<R>(a.part, gridDim.x, &c);
        double L = 0.0;
        if (threadIdx.x == 0) done = finalize_weights(f, c, &L);
        if (threadIdx.x == 0 && done && a.gmm) st->base_shift = L;
    }
    if (threadIdx.x == 0 && done) st->cur_lw = cur_lw ^ 1;
}

}  // namespace smc
