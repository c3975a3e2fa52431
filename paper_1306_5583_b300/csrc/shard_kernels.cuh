// One shard of a particle filter partitioned over ranks (Sec. 3.1 MPI
// module: the weight set normalised across ranks).
#pragma once

#include "pf_kernels.cuh"
#include "resample_kernels.cuh"

namespace smc {

// ---- one shard of a filter partitioned over ranks (the sharded filter) ------
// The particles of a filter of N_g particles are split in blocks over
// ranks; rank r holds the particles [offset, offset + N_r) under their
// global Philox indices.  Per iteration: the shard moves and weighs its
// particles and reduces them to one partial (pf_shard_move_kernel); the
// partials of every rank, gathered in rank order, are combined and
// finalised identically on every rank (pf_finalize on the gathered array:
// global normaliser, ESS, evidence increment, means, decision); when the
// ESS test asks, the shard's fixed-point total (with the global maximum
// and F of N_g) is gathered, every rank selects the outputs of its own
// particles on the global CDF (shard_select_kernel) and the copies move to
// the ranks that own their output slots (shard_pack_kernel, an all-to-all,
// shard_unpack_kernel).

// Move + weight of the shard; the last block reduces its partials to one
// partial of the shard (FP32: the double-float sums and the float maximum
// in the partial layout; FP64: float64 fields) and leaves the state as it
// is for the combine of every rank's partials.
template <typename R>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 5 : 4) pf_shard_move_kernel(PfArgs<R> a, Partial *out) {
    DevState *st = a.st;
    int32_t src[kPfItems];
    load_idx4(a.anc, (blockIdx.x * (uint32_t)kBlock + threadIdx.x) * (uint32_t)kPfItems, (uint32_t)a.n, src);
    const DevState *sv = snapshot(st, true);
    if (sv->error) return;
    const int32_t t = sv->t + 1;
    const bool gather = (t > 0) && (sv->ready != 0);
    pf_tile<R>(a, blockIdx.x, t, sv->cur, sv->cur_lw, gather, log_norm_shift<R>(sv), a.part, src);
    if (!last_arrival_after_partial(&st->ticket, gridDim.x)) return;
    if constexpr (sizeof(R) == 4) {
        CombinedDF c;
        combine_partials_df<4>(a.part, gridDim.x, &c);
        if (threadIdx.x == 0) {
            PartialIO<float>::store(out, c.M, c.S);
            st->ticket = 0;
        }
    } else {
        Combined c;
        combine_partials<R>(a.part, gridDim.x, &c);
        if (threadIdx.x == 0) {
            const double s4[kSums] = {c.S1, c.S2, c.Sa, c.Sb};
            PartialIO<double>::store(out, c.M, s4);
            st->ticket = 0;
        }
    }
}

// The gathered partials of every rank (rank order) combined and finalised:
// the same finalisation as a whole filter's, on world partials.
// n_global: the filter's N (the ESS threshold is on the whole filter).
template <typename R>
__global__ void __launch_bounds__(kBlock) pf_shard_finalize_kernel(PfArgs<R> a, const Partial *parts, int world,
                                                                   int64_t n_global) {
    DevState *st = a.st;
    const DevState *sv = snapshot(st, true);
    if (sv->error) return;
    PfArgs<R> g = a;
    g.part = const_cast<Partial *>(parts);
    g.n = n_global;
    pf_finalize<R>(g, st, sv, world, sv->t + 1, sv->cur, sv->cur_lw);
}

// After the resampling decision: the outputs of the shard's particles on
// the global fixed-point CDF.  Q_before: the totals of the ranks before
// this one, Q_N: every rank's; tsum: the shard's scan-tile sums.  Output k
// (global) gets its local source particle in src[k]; range[0..1] receives
// the shard's first and past-the-last outputs.
template <typename R, bool kStratified>
__global__ void __launch_bounds__(kBlock) shard_select_kernel(QGen<R> gen, GridTargets<kStratified> tgt,
                                                              int64_t n, const unsigned long long *tsum,
                                                              const unsigned long long *totals, int rank, int world,
                                                              int32_t *src, int64_t *range, DevState *st) {
    const DevState *sv = snapshot(st, true);
    if (sv->error || !sv->due) return;
    QGen<R> g = gen;
    g.prepare(sv);
    __shared__ unsigned long long s_q[2];
    if (threadIdx.x == 0) {
        unsigned long long qb = 0, qn = 0;
        for (int r = 0; r < world; ++r) {
            const unsigned long long v = __ldcg(&totals[r]);
            if (r < rank) qb += v;
            qn += v;
        }
        s_q[0] = qb;
        s_q[1] = qn;
    }
    __syncthreads();
    const unsigned long long Qb = s_q[0], QN = s_q[1];
    unsigned long long pre, tot;
    tile_prefix_total(tsum, blockIdx.x, gridDim.x, &pre, &tot);
    const GridTargets<kStratified> tg = block_targets(tgt, sv, QN);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        range[0] = tg.first_at_least(Qb, QN);
        range[1] = (rank == world - 1) ? tg.count() : tg.first_at_least(Qb + tot, QN);
    }
    __shared__ TileBufs tb;
    const unsigned long long ts = scan_tile_local(g, n, blockIdx.x, tb);
    select_tile_closed(tg, AncOut{src}, n, blockIdx.x, Qb + pre, QN, tb);
}

// The state rows of the shard's outputs [k_lo, k_lo + count) packed in
// output order (four values per output) for the exchange.
template <typename R>
__global__ void __launch_bounds__(kBlock) shard_pack_kernel(PfArgs<R> a, const int32_t *src, int64_t k_lo,
                                                            int64_t count, R *send) {
    const int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (j >= count) return;
    const DevState *st = a.st;
    const int cur = *reinterpret_cast<const volatile int32_t *>(&st->cur);
    const int32_t s = src[k_lo + j];
#pragma unroll
    for (int d = 0; d < 4; ++d) send[4 * j + d] = (cur ? a.x[1][d] : a.x[0][d])[s];
}

// The received copies become the shard's particles (in output order, which
// is the shard's slot order) with equal log-weights -log N_g; the running
// shift L is cleared so that the next move starts from log W = -log N_g.
template <typename R>
__global__ void __launch_bounds__(kBlock) shard_unpack_kernel(PfArgs<R> a, const R *recv) {
    const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    DevState *st = a.st;
    const int cur = *reinterpret_cast<const volatile int32_t *>(&st->cur);
    const int cur_lw = *reinterpret_cast<const volatile int32_t *>(&st->cur_lw);
    if (i < a.n) {
#pragma unroll
        for (int d = 0; d < 4; ++d) (cur ? a.x[1][d] : a.x[0][d])[i] = recv[4 * i + d];
        (cur_lw ? a.lw[1] : a.lw[0])[i] = a.neg_log_n;
    }
    if (i == 0) {
        st->log_norm = 0.0;
        st->log_norm_f[0] = st->log_norm_f[1] = 0.0f;
    }
}

// The same for d state rows of pitch ld (the mixture sampler's rows:
// parameters, log-prior, log-likelihood and, for Langevin moves, the cached
// gradient).
template <typename R>
__global__ void __launch_bounds__(kBlock) shard_pack_rows_kernel(const R *x0, const R *x1, int64_t ld, int d,
                                                                 const DevState *st, const int32_t *src, int64_t k_lo,
                                                                 int64_t count, R *send) {
    const int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (j >= count) return;
    const int cur = *reinterpret_cast<const volatile int32_t *>(&st->cur);
    const R *x = cur ? x1 : x0;
    const int32_t s = src[k_lo + j];
    for (int r = 0; r < d; ++r) send[(int64_t)d * j + r] = x[(int64_t)r * ld + s];
}

// The received copies become the shard's particles with log-weights -log N_g
// and no pending shift (the next reweighting starts from log W = -log N_g).
template <typename R>
__global__ void __launch_bounds__(kBlock) shard_unpack_rows_kernel(R *x0, R *x1, R *lw0, R *lw1, int64_t ld, int d,
                                                                   int64_t n, R neg_log_n, DevState *st,
                                                                   const R *recv) {
    const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    const int cur = *reinterpret_cast<const volatile int32_t *>(&st->cur);
    const int cur_lw = *reinterpret_cast<const volatile int32_t *>(&st->cur_lw);
    if (i < n) {
        R *x = cur ? x1 : x0;
        for (int r = 0; r < d; ++r) x[(int64_t)r * ld + i] = recv[(int64_t)d * i + r];
        (cur_lw ? lw1 : lw0)[i] = neg_log_n;
    }
    if (i == 0) st->base_shift = 0.0;
}

}  // namespace smc
