// Batched form: many independent constant-velocity particle filters of
// uneven N and T advanced by one launch per kernel per iteration.
//
// Filters are ordered by decreasing length, so the filters still running
// at iteration t are a prefix and so are their tiles; a persistent grid
// walks the active tiles (tile -> filter by a lookup table).  Each filter
// keeps its own device state block, records, tile partials and tile sums,
// and the tile bodies are the plain path's (pf_tile, tile_sum,
// scan_select_tile), so every filter computes exactly what a plain run with
// the same Philox stream computes.  The last tile of a filter to arrive
// finalises that filter (normaliser, ESS, evidence, resample decision).
#pragma once

#include "pf_kernels.cuh"
#include "resample_kernels.cuh"

namespace smc {

struct BatchState {
    int32_t t;        // last completed iteration, -1 before initialize
    uint32_t ticket;  // grid-level ticket of the move/weight kernel
    int32_t pad[2];
};

template <typename R>
struct BatchArgs {
    PfArgs<R> proto;              // model constants; per-filter pointers are set per tile
    R *x[2][4];                   // concatenated state rows (filter b at offset off[b])
    R *lw[2];
    int32_t *anc;
    const double *obs;
    const R *obs_r;               // observations in R (converted after each smc_batch_set_data)
    smc_record *rec;
    Partial *part;
    unsigned long long *tsum;
    DevState *fst;                // per-filter state blocks
    BatchState *bs;
    const int64_t *n;             // particles per filter
    const int64_t *off;           // particle offset (multiple of 64)
    const int32_t *tfirst;        // first weighting tile of each filter, [nf + 1]
    const int32_t *sfirst;        // first scan tile of each filter, [nf + 1]
    const int32_t *tile_filter;   // weighting tile -> filter
    const int32_t *stile_filter;  // scan tile -> filter
    const int32_t *act_tiles;     // active weighting tiles at iteration t
    const int32_t *act_stiles;    // active scan tiles at iteration t
    const int64_t *obs_off;       // first observation row of each filter
    const int64_t *rec_off;       // first record of each filter
    const int32_t *n_iter;        // iterations of each filter (= its observations)
    const uint32_t *stream_of;    // Philox stream of each filter
    const unsigned long long *mrec;  // floor((2^64 - 1) / N) of each filter
    const double *log_n;          // log N of each filter
    const R *neg_log_n;           // -log N of each filter in R
    const int32_t *frac;          // fixed-point fraction bits of each filter
    int32_t tmax;
    int32_t stratified;
    int32_t chunk;                // consecutive tiles a block takes per step of its grid-stride walk
};

template <typename R>
__device__ __forceinline__ PfArgs<R> filter_args(const BatchArgs<R> &B, int b) {
    PfArgs<R> a = B.proto;
    const int64_t o = B.off[b];
    for (int k = 0; k < 2; ++k) {
        for (int r = 0; r < 4; ++r) a.x[k][r] = B.x[k][r] + o;
        a.lw[k] = B.lw[k] + o;
    }
    a.n = B.n[b];
    a.anc = B.anc + o;
    a.obs = B.obs + 2 * B.obs_off[b];
    a.obs_r = B.obs_r + 2 * B.obs_off[b];
    a.neg_log_n = B.neg_log_n[b];
    a.rec = B.rec + B.rec_off[b];
    a.rec_cap = B.n_iter[b];
    a.st = &B.fst[b];
    a.part = B.part + B.tfirst[b];
    a.log_n = B.log_n[b];
    a.stream = B.stream_of[b];
    return a;
}

template <typename R>
__global__ void __launch_bounds__(kBlock, 3) batch_pf_kernel(BatchArgs<R> B) {
    const int32_t t = B.bs->t + 1;
    if (t >= B.tmax) return;
    const int nact = B.act_tiles[t];
    for (int item = blockIdx.x; item * B.chunk < nact; item += gridDim.x)
        for (int tile = item * B.chunk; tile < min(nact, (item + 1) * B.chunk); ++tile) {
            const int b = B.tile_filter[tile];
            DevState *st = &B.fst[b];
            const DevState *sv = snapshot(st);
            if (sv->error) continue;
            const PfArgs<R> a = filter_args(B, b);
            const int cur = sv->cur, cur_lw = sv->cur_lw;
            const bool gather = (t > 0) && (sv->ready != 0);
            const int nblk = B.tfirst[b + 1] - B.tfirst[b];
            if constexpr (sizeof(R) == 8)  // the plain double-precision move tiles: one particle per thread
                pf_tile<R, 1>(a, (uint32_t)(tile - B.tfirst[b]), t, cur, cur_lw, gather, log_norm_shift<R>(sv), a.part,
                              nullptr, (uint32_t)pf64_move_threads(a.n));
            else
                pf_tile<R>(a, (uint32_t)(tile - B.tfirst[b]), t, cur, cur_lw, gather, log_norm_shift<R>(sv), a.part);
            if (last_arrival_after_partial(&st->ticket, (uint32_t)nblk)) pf_finalize<R, 1>(a, st, sv, nblk, t, cur, cur_lw);
        }
    if (last_arrival(&B.bs->ticket, gridDim.x) && threadIdx.x == 0) {
        B.bs->t = t;
        B.bs->ticket = 0;
    }
}

template <typename R>
__device__ __forceinline__ QGen<R> filter_qgen(const BatchArgs<R> &B, int b, const DevState *st) {
    QGen<R> g;
    g.lw[0] = B.lw[0] + B.off[b];
    g.lw[1] = B.lw[1] + B.off[b];
    g.frac = B.frac[b];
    g.prepare(st);
    return g;
}

// tile sums of the fixed-point weights of every filter whose ESS test asked
// for resampling; the filter's last tile writes its exact total
template <typename R>
__global__ void __launch_bounds__(kBlock) batch_reduce_kernel(BatchArgs<R> B) {
    const int32_t t = B.bs->t;
    if (t < 0 || t >= B.tmax) return;
    const int nact = B.act_stiles[t];
    for (int item = blockIdx.x; item * B.chunk < nact; item += gridDim.x)
        for (int tile = item * B.chunk; tile < min(nact, (item + 1) * B.chunk); ++tile) {
            const int b = B.stile_filter[tile];
            DevState *st = &B.fst[b];
            const DevState *sv = snapshot(st);
            if (gated_out(sv, 1)) continue;
            const QGen<R> g = filter_qgen(B, b, sv);
            const int ns = B.sfirst[b + 1] - B.sfirst[b];
            const unsigned long long s = tile_sum(g, B.n[b], tile - B.sfirst[b]);
            if (threadIdx.x == 0) B.tsum[tile] = s;
            if (last_arrival(&st->scan_ticket[SLOT_CDF], (uint32_t)ns)) {
                const unsigned long long tot = sum_tiles(B.tsum + B.sfirst[b], ns);
                if (threadIdx.x == 0) {
                    st->scan_total[SLOT_CDF] = tot;
                    st->scan_ticket[SLOT_CDF] = 0;
                }
            }
        }
}

template <typename R, bool kStratified>
__device__ __forceinline__ void batch_select_tile(const BatchArgs<R> &B, int tile, int b, DevState *st,
                                                  const DevState *sv) {
    const QGen<R> g = filter_qgen(B, b, sv);
    const int lt = tile - B.sfirst[b];
    if (lt == 0 && threadIdx.x == 0) st->ready = 1;
    unsigned long long pre, QN;
    tile_prefix_total(B.tsum + B.sfirst[b], lt, lt, &pre, &QN);
    QN = sv->scan_total[SLOT_CDF];
    GridTargets<kStratified> proto{};
    proto.n = B.n[b];
    proto.key = B.proto.key;
    proto.stream = B.stream_of[b];
    proto.mrec = B.mrec[b];
    const GridTargets<kStratified> tg = block_targets(proto, sv, QN);
    __shared__ TileBufs tb;
    const unsigned long long ts = scan_tile_local(g, B.n[b], lt, tb);
    select_tile_grid(tg, AncOut{B.anc + B.off[b]}, NoSink{}, B.n[b], lt, pre, ts, QN, st, tb);
}

template <typename R, bool kStratified>
__global__ void __launch_bounds__(kBlock) batch_select_kernel(BatchArgs<R> B) {
    const int32_t t = B.bs->t;
    if (t < 0 || t >= B.tmax) return;
    const int nact = B.act_stiles[t];
    for (int item = blockIdx.x; item * B.chunk < nact; item += gridDim.x)
        for (int tile = item * B.chunk; tile < min(nact, (item + 1) * B.chunk); ++tile) {
            const int b = B.stile_filter[tile];
            DevState *st = &B.fst[b];
            const DevState *sv = snapshot(st);
            if (gated_out(sv, 1)) continue;
            batch_select_tile<R, kStratified>(B, tile, b, st, sv);
        }
}

__global__ void batch_reset_kernel(DevState *fst, int nf, BatchState *bs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) {
        bs->t = -1;
        bs->ticket = 0;
    }
    if (b >= nf) return;
    DevState *st = &fst[b];
    st->t = -1;
    st->cur = 0;
    st->cur_lw = 0;
    st->due = 0;
    st->ready = 0;
    st->error = 0;
    st->ticket = 0;
    st->log_norm = 0;
    st->log_evidence = 0;
    st->ess = 0;
    st->max_lw = 0;
    st->max_lw_f = 0;
    st->log_norm_f[0] = st->log_norm_f[1] = 0;
    for (int k = 0; k < kScanSlots; ++k) {
        st->scan_ticket[k] = 0;
        st->scan_total[k] = 0;
    }
}

}  // namespace smc
