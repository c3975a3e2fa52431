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
    smc_record *rec;
    int32_t rec_cap;
    DevState *st;
    Partial *part;
    double log_n;
    double threshold;
    R delta, sd_pos, sd_vel, sd_pos0, sd_vel0;
    R inv_scale, inv_nu, half_nu1, ll_const;  // ll_const = 2 log(density constant)
    int32_t gaussian;
    uint2 key;
    uint32_t stream;
};

// log g(Y_t | X_t): full Student-t (or Gaussian) density of both position
// coordinates.  FP32 uses log(1 + a) on the MUFU pipe (absolute error of a
// few 1e-7, well inside the 1e-5 tolerance of the FP32 path).
template <typename R>
__device__ __forceinline__ R cv_loglik(const PfArgs<R> &a, R yx, R yy, R px, R py) {
    const R zx = (yx - px) * a.inv_scale, zy = (yy - py) * a.inv_scale;
    if (a.gaussian) return a.ll_const - R(0.5) * (zx * zx + zy * zy);
    if constexpr (sizeof(R) == 4)
        return a.ll_const - a.half_nu1 * (__logf(1.0f + zx * zx * a.inv_nu) + __logf(1.0f + zy * zy * a.inv_nu));
    else
        return a.ll_const - a.half_nu1 * (Math<R>::log1p(zx * zx * a.inv_nu) + Math<R>::log1p(zy * zy * a.inv_nu));
}

template <typename R>
__global__ void __launch_bounds__(kBlock) pf_iterate_kernel(PfArgs<R> a) {
    DevState *st = a.st;
    if (*(volatile int32_t *)&st->error) return;
    const int32_t t = st->t + 1;
    const int cur = st->cur;
    const bool gather = (t > 0) && (st->ready != 0);
    const Shift<R> Lprev(st->log_norm);
    const R yx = R(a.obs[2 * t]), yy = R(a.obs[2 * t + 1]);
    const R base_eq = R(-a.log_n);
    const int cur_lw = st->cur_lw;
    const R *__restrict__ lw_in = a.lw[cur_lw];
    R *__restrict__ lw_out = a.lw[cur_lw ^ 1];
    const R *__restrict__ x0s = a.x[cur][0];
    const R *__restrict__ x1s = a.x[cur][1];
    const R *__restrict__ x2s = a.x[cur][2];
    const R *__restrict__ x3s = a.x[cur][3];
    R *__restrict__ x0d = a.x[cur ^ 1][0];
    R *__restrict__ x1d = a.x[cur ^ 1][1];
    R *__restrict__ x2d = a.x[cur ^ 1][2];
    R *__restrict__ x3d = a.x[cur ^ 1][3];
    const uint32_t n = (uint32_t)a.n;

    R lwv[kPfItems], px[kPfItems], py[kPfItems], zero[kPfItems];
    const uint32_t base = blockIdx.x * (uint32_t)kPfTile + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kPfItems; ++j) {
        const uint32_t i = base + (uint32_t)(j * kBlock);
        lwv[j] = Math<R>::neg_inf();
        px[j] = py[j] = zero[j] = R(0);
        if (i < n) {
            R s0, s1, s2, s3, z[4];
            if (t == 0) {
                normals4_fast<R>(draw(a.key, i, 0u, TAG_INIT, a.stream, 0u), z);
                s0 = a.sd_pos0 * z[0];
                s1 = a.sd_pos0 * z[1];
                s2 = a.sd_vel0 * z[2];
                s3 = a.sd_vel0 * z[3];
            } else {
                const uint32_t src = gather ? (uint32_t)__ldg(&a.anc[i]) : i;
                const R v0 = x0s[src], v1 = x1s[src], v2 = x2s[src], v3 = x3s[src];
                normals4_fast<R>(draw(a.key, i, (uint32_t)t, TAG_MOVE, a.stream, 0u), z);
                s0 = v0 + a.delta * v2 + a.sd_pos * z[0];
                s1 = v1 + a.delta * v3 + a.sd_pos * z[1];
                s2 = v2 + a.sd_vel * z[2];
                s3 = v3 + a.sd_vel * z[3];
            }
            x0d[i] = s0;
            x1d[i] = s1;
            x2d[i] = s2;
            x3d[i] = s3;
            const R b = (t == 0 || gather) ? base_eq : Lprev.sub_from(lw_in[i]);
            lwv[j] = b + cv_loglik(a, yx, yy, s0, s1);
            lw_out[i] = lwv[j];
            px[j] = s0;
            py[j] = s1;
        }
    }
    block_partial<R, kPfItems>(lwv, px, py, zero, &a.part[blockIdx.x]);
    Combined c;
    if (!last_block_combine<R>(st, a.part, &c)) return;
    if (threadIdx.x == 0) {
        FinalizeArgs f{st, a.rec, a.rec_cap, t, 0, a.n, a.threshold, 0.0};
        double L;
        if (finalize_weights(f, c, &L)) {
            st->t = t;
            st->cur = cur ^ 1;
            st->cur_lw = cur_lw ^ 1;
            st->ready = 0;
        }
    }
}

}  // namespace smc
