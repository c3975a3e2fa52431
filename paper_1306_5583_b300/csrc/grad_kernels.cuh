// Gradient of the particle filter's log-likelihood estimate with respect to
// theta = (sd_pos, sd_vel, obs_scale, obs_df), with the resampling of a
// recorded forward run held fixed (stop-gradient resampling) and the move
// noise reparameterised through its Philox counters.
//
// * pf_replay_kernel: one iteration with given theta, recorded ancestors and
//   recorded resampling decisions (the forward tile body pf_tile, unchanged);
//   used to recompute the trajectory between checkpoints and to evaluate the
//   estimate at other theta (finite differences).
// * pf_adjoint_kernel: one reverse step t: weight adjoint
//   gbar_t = W_t (+ gbar_{t+1} - W_t sum gbar_{t+1} when t did not resample),
//   position adjoint from the observation density, theta partial sums, and
//   A^T xbar_t for the parents.
// * pf_parent_gather_kernel: each parent collects A^T xbar of its children
//   (children of a parent are contiguous in the sorted ancestor array), in a
//   fixed order, so the gradient is deterministic.
#pragma once

#include "pf_kernels.cuh"

namespace smc {

// last block of a replay step: L_t from the tile partials, running log Z
template <typename R>
__global__ void __launch_bounds__(kBlock) pf_replay_kernel(PfArgs<R> a, int32_t t, int gather,
                                                           const double *L_prev, double *L_out, double *logz,
                                                           uint32_t *ticket) {
    // L_{t-1} split once per block (hi + lo in R)
    __shared__ R s_lprev[2];
    if (threadIdx.x == 0) {
        const double lp = (t > 0 && !gather) ? __ldcg(L_prev) : 0.0;
        s_lprev[0] = R(lp);
        s_lprev[1] = R(lp - double(s_lprev[0]));
    }
    __syncthreads();
    pf_tile<R>(a, blockIdx.x, t, 0, 0, gather != 0, Shift<R>(s_lprev[0], s_lprev[1]), a.part);
    if (!last_arrival(ticket, gridDim.x)) return;
    // L_t as the forward kernels compute it (compensated float on the FP32 path)
    double L;
    if constexpr (sizeof(R) == 4) {
        CombinedDF d;
        combine_partials_df<1>(a.part, gridDim.x, &d);
        L = df_to_double(df_add_f(df_log(d.S[0]), d.M));
    } else {
        Combined c;
        combine_partials<R>(a.part, gridDim.x, &c);
        L = c.M + log(c.S1);
    }
    if (threadIdx.x == 0) {
        *L_out = L;
        *logz = (t == 0 ? 0.0 : *logz) + L;
        *ticket = 0;
    }
}

// Five block sums (result to thread 0, as float64).  FP64 path: float64
// warp sums.  FP32 path: DF warp trees from the per-thread float sums; the
// partial keeps (hi, lo) pairs in the same 64 bytes.
template <typename R>
__device__ __forceinline__ void block_sum5(const R (&v)[5], double (&out)[5]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (sizeof(R) == 8) {
        __shared__ double s_red[kBlock / 32][5];
        double u[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) u[q] = warp_sum(v[q]);
        __syncthreads();
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 5; ++q) s_red[warp][q] = u[q];
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                out[q] = 0.0;
                for (int k = 0; k < kBlock / 32; ++k) out[q] += s_red[k][q];
            }
        }
    } else {
        __shared__ DF s_red[kBlock / 32][5];
        DF u[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) u[q] = DF{v[q], 0.0f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 5; ++q) u[q] = df_add(u[q], df_shfl_xor(u[q], o));
        __syncthreads();
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 5; ++q) s_red[warp][q] = u[q];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < 5; ++q) u[q] = lane < kBlock / 32 ? s_red[lane][q] : DF{0.0f, 0.0f};
#pragma unroll
            for (int o = (kBlock / 32) / 2; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 5; ++q) u[q] = df_add(u[q], df_shfl_xor(u[q], o));
            if (lane == 0) {
                float *f = reinterpret_cast<float *>(out);  // packed (hi, lo) pairs for store_sum5
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    f[2 * q] = u[q].hi;
                    f[2 * q + 1] = u[q].lo;
                }
            }
        }
    }
}

template <typename R>
__device__ __forceinline__ void store_sum5(Partial *p, const double (&w)[5]) {
    if constexpr (sizeof(R) == 8) {
        p->m = 0;
        p->s1 = w[0];
        p->s2 = w[1];
        p->sx = w[2];
        p->sy = w[3];
        p->su = w[4];
    } else {
        const float *f = reinterpret_cast<const float *>(w);
        float *d = reinterpret_cast<float *>(p);
#pragma unroll
        for (int k = 0; k < 10; ++k) d[k] = f[k];
    }
}

// grid sums of nb partials of store_sum5 (thread 0 receives float64 values)
template <typename R>
__device__ __forceinline__ void combine_sum5(const Partial *part, int nb, double (&out)[5]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (sizeof(R) == 8) {
        double u[5] = {0, 0, 0, 0, 0};
        for (int b = threadIdx.x; b < nb; b += kBlock) {
            u[0] += __ldcg(&part[b].s1);
            u[1] += __ldcg(&part[b].s2);
            u[2] += __ldcg(&part[b].sx);
            u[3] += __ldcg(&part[b].sy);
            u[4] += __ldcg(&part[b].su);
        }
        block_sum5<double>(u, out);
    } else {
        __shared__ DF s_red[kBlock / 32][5];
        DF u[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) u[q] = DF{0.0f, 0.0f};
        for (int b = threadIdx.x; b < nb; b += kBlock) {
            const float *f = reinterpret_cast<const float *>(&part[b]);
#pragma unroll
            for (int q = 0; q < 5; ++q) u[q] = df_add(u[q], DF{__ldcg(f + 2 * q), __ldcg(f + 2 * q + 1)});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 5; ++q) u[q] = df_add(u[q], df_shfl_xor(u[q], o));
        __syncthreads();
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 5; ++q) s_red[warp][q] = u[q];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < 5; ++q) u[q] = lane < kBlock / 32 ? s_red[lane][q] : DF{0.0f, 0.0f};
#pragma unroll
            for (int o = (kBlock / 32) / 2; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 5; ++q) u[q] = df_add(u[q], df_shfl_xor(u[q], o));
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 5; ++q) out[q] = df_to_double(u[q]);
        }
    }
}

template <typename R>
struct AdjArgs {
    int64_t n;
    int64_t ld;
    const R *x;          // x_t rows (pitch ld)
    const R *lw;         // lw_t
    const float *gbar_next;
    float *gbar;         // gbar_t (out)
    const R *xbar_f;     // adjoint of x_t from iteration t+1 (4 rows), or null at the last iteration
    R *at;               // A^T xbar_t (4 rows, out)
    const double *obs;
    const smc_record *rec;  // records of the recorded run
    int32_t rec_cap;
    double *S_next_in;   // sum gbar_{t+1}
    double *S_out;       // sum gbar_t
    double *grad;        // accumulated dJ/dtheta (4)
    Partial *part;
    uint32_t *ticket;
    int32_t t, last;
    R delta, inv_scale, scale, nu, inv_nu, half_nu1, dnu_const;  // dnu_const = (psi((nu+1)/2) - psi(nu/2))/2 - 1/(2 nu)
    int32_t gaussian;
    uint2 key;
    uint32_t stream;
};

template <typename R>
__global__ void __launch_bounds__(kBlock) pf_adjoint_kernel(AdjArgs<R> a) {
    constexpr int E = kPfItems;
    // per-block scalars converted once by thread 0 (no per-thread float64)
    __shared__ R s_L[2], s_S;
    __shared__ int s_res;
    const uint32_t n = (uint32_t)a.n;
    if (threadIdx.x == 0) {
        const smc_record *r = &a.rec[a.t % a.rec_cap];
        const double L = r->log_norm;
        s_L[0] = R(L);
        s_L[1] = R(L - double(s_L[0]));
        s_res = r->resampled;
        s_S = R(a.last ? 0.0 : __ldcg(a.S_next_in));
    }
    __syncthreads();
    const bool chain = !(a.last || s_res);  // lw_{t+1} depends on lw_t
    const Shift<R> Lt(s_L[0], s_L[1]);
    const R S_next = s_S;
    const uint32_t i0 = (blockIdx.x * (uint32_t)kBlock + threadIdx.x) * (uint32_t)E;
    R x0[E], x1[E], x2[E], x3[E], lw[E], f0[E], f1[E], f2[E], f3[E];
    float gn[E];
    load_k<R, E>(a.x, i0, n, x0);
    load_k<R, E>(a.x + a.ld, i0, n, x1);
    load_k<R, E>(a.x + 2 * a.ld, i0, n, x2);
    load_k<R, E>(a.x + 3 * a.ld, i0, n, x3);
    load_k<R, E>(a.lw, i0, n, lw);
    if (a.xbar_f) {
        load_k<R, E>(a.xbar_f, i0, n, f0);
        load_k<R, E>(a.xbar_f + a.ld, i0, n, f1);
        load_k<R, E>(a.xbar_f + 2 * a.ld, i0, n, f2);
        load_k<R, E>(a.xbar_f + 3 * a.ld, i0, n, f3);
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) f0[j] = f1[j] = f2[j] = f3[j] = R(0);
    }
    if (chain) load_k<float, E>(a.gbar_next, i0, n, gn);
    __shared__ R s_y[2];
    if (threadIdx.x == 0) {
        s_y[0] = R(a.obs[2 * a.t]);
        s_y[1] = R(a.obs[2 * a.t + 1]);
    }
    __syncthreads();
    const R yx = s_y[0], yy = s_y[1];
    R sg[E], sds[E], sdn[E], sp[E], sv[E], a0[E], a1[E], a2[E], a3[E];
    float gout[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const bool ok = i0 + j < n;
        const R W = ok ? Math<R>::exp(Lt.sub_from(lw[j])) : R(0);
        const R g = chain ? W + R(gn[j]) - W * S_next : W;
        const R zx = (yx - x0[j]) * a.inv_scale, zy = (yy - x1[j]) * a.inv_scale;
        R gx, gy, ds, dn;
        if (a.gaussian) {
            gx = zx * a.inv_scale;
            gy = zy * a.inv_scale;
            ds = (zx * zx + zy * zy - R(2)) * a.inv_scale;
            dn = R(0);
        } else {
            const R qx = fast_rcp(a.nu + zx * zx), qy = fast_rcp(a.nu + zy * zy);
            gx = (a.nu + R(1)) * zx * qx * a.inv_scale;
            gy = (a.nu + R(1)) * zy * qy * a.inv_scale;
            ds = (R(-2) + (a.nu + R(1)) * (zx * zx * qx + zy * zy * qy)) * a.inv_scale;
            dn = R(2) * a.dnu_const - R(0.5) * (Math<R>::log1p(zx * zx * a.inv_nu) + Math<R>::log1p(zy * zy * a.inv_nu)) +
                 a.half_nu1 * a.inv_nu * (zx * zx * qx + zy * zy * qy);
        }
        const R b0 = f0[j] + g * gx, b1 = f1[j] + g * gy, b2 = f2[j], b3 = f3[j];
        R e[4] = {0, 0, 0, 0};
        // the forward move's own noise (the same transform as pf_tile)
        if (a.t > 0) normals4_fast<R>(draw(a.key, i0 + j, (uint32_t)a.t, TAG_MOVE, a.stream, 0u), e);
        sg[j] = ok ? g : R(0);
        sds[j] = ok ? g * ds : R(0);
        sdn[j] = ok ? g * dn : R(0);
        sp[j] = ok ? b0 * e[0] + b1 * e[1] : R(0);
        sv[j] = ok ? b2 * e[2] + b3 * e[3] : R(0);
        a0[j] = b0;
        a1[j] = b1;
        a2[j] = b2 + a.delta * b0;
        a3[j] = b3 + a.delta * b1;
        gout[j] = float(g);
    }
    store_k<float, E>(a.gbar, i0, n, gout);
    store_k<R, E>(a.at, i0, n, a0);
    store_k<R, E>(a.at + a.ld, i0, n, a1);
    store_k<R, E>(a.at + 2 * a.ld, i0, n, a2);
    store_k<R, E>(a.at + 3 * a.ld, i0, n, a3);
    // block sums of (gbar, gbar ds, gbar dnu, d sd_pos, d sd_vel): float64 on
    // the FP64 path, compensated float (per-thread float sums) on the FP32 path
    R v[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < E; ++j) {
        v[0] += sg[j];
        v[1] += sds[j];
        v[2] += sdn[j];
        v[3] += sp[j];
        v[4] += sv[j];
    }
    double w[5];
    block_sum5<R>(v, w);
    if (threadIdx.x == 0) store_sum5<R>(&a.part[blockIdx.x], w);
    if (!last_arrival(a.ticket, gridDim.x)) return;
    combine_sum5<R>(a.part, (int)gridDim.x, w);
    if (threadIdx.x == 0) {
        *a.S_out = w[0];
        a.grad[2] += w[1];
        a.grad[3] += w[2];
        if (a.t > 0) {
            a.grad[0] += w[3];
            a.grad[1] += w[4];
        }
        *a.ticket = 0;
    }
}

// xbar_f[j] = sum over children k of parent j (anc sorted) of at[k]
template <typename R>
__global__ void __launch_bounds__(kBlock) pf_parent_gather_kernel(const int32_t *anc, const R *at, R *xbar_f,
                                                                  int64_t n, int64_t ld) {
    const int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (j >= n) return;
    int64_t lo = 0, hi = n;  // first k with anc[k] >= j
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (__ldg(&anc[m]) < j) lo = m + 1;
        else hi = m;
    }
    R s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int64_t k = lo; k < n && __ldg(&anc[k]) == j; ++k) {
        s0 += at[k];
        s1 += at[ld + k];
        s2 += at[2 * ld + k];
        s3 += at[3 * ld + k];
    }
    xbar_f[j] = s0;
    xbar_f[ld + j] = s1;
    xbar_f[2 * ld + j] = s2;
    xbar_f[3 * ld + j] = s3;
}

}  // namespace smc
