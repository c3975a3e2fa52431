// Particle filter for the almost-constant-velocity model (Sec. 5.1,
// Algorithm 1), one fused kernel per iteration:
//   gather by the pending ancestors (copy_from convention, Sec. 4.1.2)
//   -> propagate X_t = A X_{t-1} + V_t with Philox/Box-Muller noise
//   -> add log g(Y_t | X_t) (full Student-t, or Gaussian, density)
//   -> block partials of (max, sum e, sum e^2, sum e x_pos, sum e y_pos)
//   -> last block: normaliser, ESS, evidence increment, filtered means,
//      resample decision.
// State is structure-of-arrays, double-buffered (read buffer cur, write
// buffer cur ^ 1); log-weights are double-buffered the same way so a
// failed iteration leaves the previous particle system untouched.
#pragma once

#include "weight_reduce.cuh"

namespace smc {

template <typename R>
struct PfArgs {
    int64_t n;
    R *x[2][4];          // [buffer][row] rows: x_pos, y_pos, x_vel, y_vel
    R *lw[2];            // [buffer]
    const int32_t *anc;  // ancestors of the pending resampling step
    const double *obs;   // (n_obs, 2) observations
    const R *obs_r;      // the same in R (read by every thread: no conversion in the kernel)
    R neg_log_n;         // -log N in R
    smc_record *rec;
    int32_t rec_cap;
    DevState *st;
    Partial *part;
    double log_n;
    double threshold;
    float thr_df[2];   // threshold as a DF value (FP32 finalize)
    int32_t thr_mode;  // 0 compare, 1 always, 2 never
    R delta, sd_pos, sd_vel, sd_pos0, sd_vel0;
    R inv_scale, inv_nu, half_nu1, ll_const;  // ll_const = 2 log(density constant)
    int32_t gaussian;
    uint2 key;
    uint32_t stream;
    uint32_t index0;     // Philox index of particle 0 (a shard of a larger filter: its first global index)
    // smc_iterate_host's graph (zero / null otherwise): the kernel is a
    // programmatic dependent of the kernel that stores the step's observation
    // (it waits for that grid just before reading y_t), and the record and
    // error word go to the staging in mapped host memory
    int32_t obs_after_wait;
    HostIO *hio_out;
    // rows of the observation buffer: an iteration past it (a caller's graph
    // replayed more often than the data allow) raises SMC_E_RANGE
    int32_t obs_cap;
    // active threads per block of the double-precision move kernel (one
    // particle each); the float kernel uses every thread, four particles each
    uint32_t tile_threads;
};

// E consecutive elements from i0 (zeros past n): 16-byte vectors where E
// elements fill them, else guarded scalar loads; the same for stores.
template <typename R, int E>
__device__ __forceinline__ void load_e(const R *__restrict__ p, uint32_t i0, uint32_t n, R (&v)[E]) {
    if constexpr ((E * sizeof(R)) % 16 == 0) {
        load_k<R, E>(p, i0, n, v);
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = (i0 + j < n) ? __ldcg(p + i0 + j) : R(0);
    }
}
template <typename R, int E>
__device__ __forceinline__ void store_e(R *__restrict__ p, uint32_t i0, uint32_t n, const R (&v)[E]) {
    if constexpr ((E * sizeof(R)) % 16 == 0) {
        store_k<R, E>(p, i0, n, v);
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (i0 + j < n) p[i0 + j] = v[j];
    }
}
template <int E>
__device__ __forceinline__ void load_idx_e(const int32_t *__restrict__ p, uint32_t i0, uint32_t n, int32_t (&v)[E]) {
    if constexpr (E == 4) {
        load_idx4(p, i0, n, v);
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = (i0 + j < n) ? __ldcg(p + i0 + j) : 0;
    }
}

// First particle of a thread: E per thread, tile_threads active threads per
// block (the others get n: no particle).
template <int E>
__device__ __forceinline__ uint32_t tile_first(uint32_t blk, uint32_t tile_threads, uint32_t n) {
    return (threadIdx.x < tile_threads) ? (blk * tile_threads + threadIdx.x) * (uint32_t)E : n;
}

// log g(Y_t | X_t): full Student-t (or Gaussian) density of both position
// coordinates.  FP32 uses log(1 + a) on the MUFU pipe (absolute error of a
// few 1e-7, well inside the 1e-5 tolerance of the FP32 path).
template <typename R>
__device__ __forceinline__ R cv_loglik(const PfArgs<R> &a, R yx, R yy, R px, R py) {
    const R zx = (yx - px) * a.inv_scale, zy = (yy - py) * a.inv_scale;
    if (a.gaussian) return a.ll_const - R(0.5) * (zx * zx + zy * zy);
    if constexpr (sizeof(R) == 4)  // one logarithm of the product (1 + zx^2/nu)(1 + zy^2/nu)
        return a.ll_const - a.half_nu1 * __logf((1.0f + zx * zx * a.inv_nu) * (1.0f + zy * zy * a.inv_nu));
    else
        return a.ll_const - a.half_nu1 * (Math<R>::log1p(zx * zx * a.inv_nu) + Math<R>::log1p(zy * zy * a.inv_nu));
}

// One tile (E tile_threads particles, block-local index blk) of the fused
// gather + move + weight step, ending in the tile's block partial.  One
// thread owns E consecutive particles: every input is fetched with
// 16-byte vector loads (or, after resampling, as independent gathers
// through one vector load of ancestor indices) before any arithmetic, so
// the memory system sees all of a thread's requests at once.
// pre_src: the tile's ancestor indices when the caller has fetched them
// already (the same load_idx4 of the same i0), else null.
// E particles per thread and tile_threads active threads per block (the
// move kernel's double-precision tiles: E = 1, 64 or 256 threads; every
// other caller: E = 4, all 256 threads, i.e. 1024-particle tiles).  The
// arithmetic of a particle does not depend on the tiling.
template <typename R, int E = kPfItems>
__device__ __forceinline__ void pf_tile(const PfArgs<R> &a, uint32_t blk, int32_t t, int cur, int cur_lw,
                                        bool gather, Shift<R> Lprev, Partial *part,
                                        const int32_t *pre_src = nullptr, uint32_t tile_threads = kBlock) {
    const uint32_t n = (uint32_t)a.n;
    const uint32_t i0 = tile_first<E>(blk, tile_threads, n);
    // buffer selection by value (no dynamic indexing of the pointer table)
    const R *xs0 = cur ? a.x[1][0] : a.x[0][0], *xs1 = cur ? a.x[1][1] : a.x[0][1];
    const R *xs2 = cur ? a.x[1][2] : a.x[0][2], *xs3 = cur ? a.x[1][3] : a.x[0][3];
    R *xd0 = cur ? a.x[0][0] : a.x[1][0], *xd1 = cur ? a.x[0][1] : a.x[1][1];
    R *xd2 = cur ? a.x[0][2] : a.x[1][2], *xd3 = cur ? a.x[0][3] : a.x[1][3];
    const R *lws = cur_lw ? a.lw[1] : a.lw[0];
    R *lwd = cur_lw ? a.lw[0] : a.lw[1];
    R v0[E], v1[E], v2[E], v3[E], lwin[E];
    if (t > 0) {
        if (gather) {
            // sorted ancestors: a thread's four sources are mostly the same
            // or adjacent elements, so the gathers go through L1 (the read
            // buffer was written by an earlier launch) instead of asking L2
            // once per item for the same sectors
            int32_t src[E];
            if (pre_src) {
#pragma unroll
                for (int j = 0; j < E; ++j) src[j] = pre_src[j];
            } else {
                load_idx_e<E>(a.anc, i0, n, src);
            }
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const uint32_t sidx = (i0 + j < n) ? (uint32_t)src[j] : 0u;
                v0[j] = __ldg(xs0 + sidx);
                v1[j] = __ldg(xs1 + sidx);
                v2[j] = __ldg(xs2 + sidx);
                v3[j] = __ldg(xs3 + sidx);
            }
        } else {
            load_e<R, E>(xs0, i0, n, v0);
            load_e<R, E>(xs1, i0, n, v1);
            load_e<R, E>(xs2, i0, n, v2);
            load_e<R, E>(xs3, i0, n, v3);
            load_e<R, E>(lws, i0, n, lwin);
        }
    }
    // observation y_t (one broadcast load) and -log N, already in R
    R yx = R(0), yy = R(0);
    if (!a.obs_after_wait) {
        yx = __ldcg(a.obs_r + 2 * t);
        yy = __ldcg(a.obs_r + 2 * t + 1);
    }
    const R base_eq = a.neg_log_n;
    R s0[E], s1[E], s2[E], s3[E], lwv[E], zero[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        R z[4];
        zero[j] = R(0);
        if (t == 0) {
            normals4_fast<R>(draw(a.key, a.index0 + i0 + j, 0u, TAG_INIT, a.stream, 0u), z);
            s0[j] = a.sd_pos0 * z[0];
            s1[j] = a.sd_pos0 * z[1];
            s2[j] = a.sd_vel0 * z[2];
            s3[j] = a.sd_vel0 * z[3];
        } else {
            normals4_fast<R>(draw(a.key, a.index0 + i0 + j, (uint32_t)t, TAG_MOVE, a.stream, 0u), z);
            s0[j] = v0[j] + a.delta * v2[j] + a.sd_pos * z[0];
            s1[j] = v1[j] + a.delta * v3[j] + a.sd_pos * z[1];
            s2[j] = v2[j] + a.sd_vel * z[2];
            s3[j] = v3[j] + a.sd_vel * z[3];
        }
    }
    if (a.obs_after_wait) {  // the move above overlapped the grid that stores y_t
        asm volatile("griddepcontrol.wait;" ::: "memory");
        yx = __ldcg(a.obs_r + 2 * t);
        yy = __ldcg(a.obs_r + 2 * t + 1);
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const R b = (t == 0 || gather) ? base_eq : Lprev.sub_from(lwin[j]);
        lwv[j] = (i0 + j < n) ? b + cv_loglik(a, yx, yy, s0[j], s1[j]) : Math<R>::neg_inf();
    }
    store_e<R, E>(xd0, i0, n, s0);
    store_e<R, E>(xd1, i0, n, s1);
    store_e<R, E>(xd2, i0, n, s2);
    store_e<R, E>(xd3, i0, n, s3);
    store_e<R, E>(lwd, i0, n, lwv);
    block_partial<R, E, 2>(lwv, s0, s1, zero, &part[blk]);
}

// Last tile of a filter: combine its nblk partials, write the record of
// iteration t and advance the filter's state.
// PT: partials per thread of the single-round-trip combine (register budget
// of the caller; the result does not depend on it).
template <typename R, int PT = 4>
__device__ __forceinline__ void pf_finalize(const PfArgs<R> &a, DevState *st, const DevState *sv, int nblk,
                                            int32_t t, int cur, int cur_lw) {
    FinalizeArgs f{st,  a.rec,   a.rec_cap, t, 0, a.n, a.threshold, 0.0, {a.thr_df[0], a.thr_df[1]}, a.thr_mode,
                   sv->log_evidence};
    bool done = false;
    int flipper = 0;  // the thread that advances the state
    if constexpr (sizeof(R) == 4) {
        CombinedDF c;
        combine_partials_df<PT>(a.part, nblk, &c);
        done = finalize_weights_df(f, c);  // every thread; warps 0-3 write
        flipper = 3 * 32;                  // the warp with the shortest share
    } else {
        Combined c;
        combine_partials<R>(a.part, nblk, &c);
        double L;
        if (threadIdx.x == 0) done = finalize_weights(f, c, &L);
    }
    if (threadIdx.x == flipper && done) {
        st->t = t;
        st->cur = cur ^ 1;
        st->cur_lw = cur_lw ^ 1;
        st->ready = 0;
    }
    if (a.hio_out) {  // smc_iterate_host: the record and the error word to the mapped staging
        __syncthreads();
        if (threadIdx.x < 32) {
            static_assert(sizeof(smc_record) % 4 == 0, "record words");
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&a.rec[t % a.rec_cap]);
            volatile uint32_t *dst = reinterpret_cast<volatile uint32_t *>(&a.hio_out->rec);
            for (int i = threadIdx.x; i < (int)(sizeof(smc_record) / 4); i += 32) dst[i] = __ldcg(src + i);
            if (threadIdx.x == 0) {
                const int32_t e = *reinterpret_cast<volatile int32_t *>(&st->error);
                if (e) a.hio_out->status = e;
            }
        }
    }
}

// Five blocks per SM for FP32 (48 registers, no spills; six spill), four
// for FP64.  FP32: four particles per thread, 1024-particle tiles; FP64: one
// particle per thread, a.tile_threads per block.
template <typename R, bool kChain = false>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 5 : 4) pf_iterate_kernel(PfArgs<R> a) {
    constexpr int E = (sizeof(R) == 4) ? kPfItems : 1;
    const uint32_t tt = (sizeof(R) == 4) ? (uint32_t)kBlock : a.tile_threads;
    // kChain: a later iteration of a captured chain, launched as a
    // programmatic dependent of the previous iteration's last kernel; it
    // waits for that grid before it reads anything
    if constexpr (kChain) asm volatile("griddepcontrol.wait;" ::: "memory");
    DevState *st = a.st;
    // the ancestor indices do not depend on the state block: their load is
    // in flight while the snapshot is read (unused when nothing is gathered)
    int32_t src[E];
    load_idx_e<E>(a.anc, tile_first<E>(blockIdx.x, tt, (uint32_t)a.n), (uint32_t)a.n, src);
    const DevState *sv = snapshot(st, true);
    if (sv->error) {  // an earlier step failed: nothing runs, the error goes back to smc_iterate_host
        if (a.hio_out && blockIdx.x == 0 && threadIdx.x == 0) a.hio_out->status = sv->error;
        return;
    }
    const int32_t t = sv->t + 1;
    if (t >= a.obs_cap) {  // the same in every block: nothing runs
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            raise_error(st, SMC_E_RANGE);
            if (a.hio_out) a.hio_out->status = SMC_E_RANGE;
        }
        return;
    }
    const int cur = sv->cur, cur_lw = sv->cur_lw;
    const bool gather = (t > 0) && (sv->ready != 0);
    pf_tile<R, E>(a, blockIdx.x, t, cur, cur_lw, gather, log_norm_shift<R>(sv), a.part, src, tt);
    if (!last_arrival_after_partial(&st->ticket, gridDim.x)) return;
    // every other block has finished: a programmatic dependent (the one-pass
    // resampler) may start its launch while this block combines
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    pf_finalize<R>(a, st, sv, gridDim.x, t, cur, cur_lw);
}

// Post-resampling filtered mean (SMC_FLAG_POST_MEAN), after the resampling
// step of iteration t: the mean of the two positions over the particle
// system that ends the iteration (Sec. 4.1.5 evaluates monitors after the
// whole iteration), i.e. (1/N) sum_k pos_{a_k} over the pending ancestors
// when the iteration resampled, else the weighted mean already in the
// record.  Per-thread and per-block sums in R, the block sums added by the
// last block in a fixed order (double-float on the FP32 path, float64 on
// the FP64 path): deterministic.
template <typename R>
__global__ void __launch_bounds__(kBlock) post_mean_kernel(PfArgs<R> a) {
    DevState *st = a.st;
    const DevState *sv = snapshot(st, true);
    if (sv->error || sv->t < 0) return;
    smc_record *r = &a.rec[sv->t % a.rec_cap];
    // the result also goes to smc_iterate_host's staging (whose record the
    // move kernel has already written)
    volatile double *hmp = a.hio_out ? a.hio_out->rec.mean_post : nullptr;
    if (!sv->ready) {  // no resampling: the weighted system ends the iteration
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            r->mean_post[0] = r->mean[0];
            r->mean_post[1] = r->mean[1];
            if (hmp) {
                hmp[0] = r->mean[0];
                hmp[1] = r->mean[1];
            }
        }
        return;
    }
    const uint32_t n = (uint32_t)a.n;
    const R *x0 = sv->cur ? a.x[1][0] : a.x[0][0], *x1 = sv->cur ? a.x[1][1] : a.x[0][1];
    const uint32_t i0 = (blockIdx.x * (uint32_t)kBlock + threadIdx.x) * (uint32_t)kPfItems;
    int32_t src[kPfItems];
    load_idx4(a.anc, i0, n, src);
    R sx = R(0), sy = R(0);
#pragma unroll
    for (int j = 0; j < kPfItems; ++j)
        if (i0 + j < n) {
            sx += __ldg(x0 + src[j]);
            sy += __ldg(x1 + src[j]);
        }
    __shared__ R s_w[2][kBlock / 32];
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_w[0][warp] = sx;
        s_w[1][warp] = sy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        R bx = R(0), by = R(0);
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) {
            bx += s_w[0][w];
            by += s_w[1][w];
        }
        R *pp = reinterpret_cast<R *>(&a.part[blockIdx.x]);
        pp[0] = bx;
        pp[1] = by;
    }
    if (!last_arrival(&st->ticket, gridDim.x)) return;
    // the last block: the block sums in a fixed order
    const int nb = (int)gridDim.x;
    if constexpr (sizeof(R) == 4) {
        DF tx{0.0f, 0.0f}, ty{0.0f, 0.0f};
        for (int b = threadIdx.x; b < nb; b += kBlock) {
            const float *pp = reinterpret_cast<const float *>(&a.part[b]);
            tx = df_add_f(tx, __ldcg(pp));
            ty = df_add_f(ty, __ldcg(pp + 1));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tx = df_add(tx, df_shfl_xor(tx, o));
            ty = df_add(ty, df_shfl_xor(ty, o));
        }
        __shared__ DF s_df[2][kBlock / 32];
        if (lane == 0) {
            s_df[0][warp] = tx;
            s_df[1][warp] = ty;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            DF X = s_df[0][0], Y = s_df[1][0];
#pragma unroll
            for (int w = 1; w < kBlock / 32; ++w) {
                X = df_add(X, s_df[0][w]);
                Y = df_add(Y, s_df[1][w]);
            }
            r->mean_post[0] = df_to_double(X) / (double)a.n;
            r->mean_post[1] = df_to_double(Y) / (double)a.n;
            if (hmp) {
                hmp[0] = r->mean_post[0];
                hmp[1] = r->mean_post[1];
            }
            st->ticket = 0;
        }
    } else {
        double tx = 0.0, ty = 0.0;
        for (int b = threadIdx.x; b < nb; b += kBlock) {
            const double *pp = reinterpret_cast<const double *>(&a.part[b]);
            tx += __ldcg(pp);
            ty += __ldcg(pp + 1);
        }
        tx = warp_sum(tx);
        ty = warp_sum(ty);
        __shared__ double s_d[2][kBlock / 32];
        if (lane == 0) {
            s_d[0][warp] = tx;
            s_d[1][warp] = ty;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double X = 0.0, Y = 0.0;
#pragma unroll
            for (int w = 0; w < kBlock / 32; ++w) {
                X += s_d[0][w];
                Y += s_d[1][w];
            }
            r->mean_post[0] = X / (double)a.n;
            r->mean_post[1] = Y / (double)a.n;
            if (hmp) {
                hmp[0] = r->mean_post[0];
                hmp[1] = r->mean_post[1];
            }
            st->ticket = 0;
        }
    }
}

}  // namespace smc
