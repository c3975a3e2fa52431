// Tempered SMC sampler for the Bayesian Gaussian mixture (Sec. 5.2,
// Algorithm 2).
//
// Kernels per iteration t:
//   gmm_reweight_kernel  lw_t = log W_{t-1} + (alpha_t - alpha_{t-1}) l(theta_{t-1})
//                        (eq:inc_weight_mcmc), normaliser = standard evidence
//                        increment (eq:smc-ds in Algorithm 2's form), ESS test;
//   resampling           the shared fixed-point CDF / selection kernels;
//   gmm_mcmc_kernel      gather by the ancestors, then the three random-walk
//                        Metropolis blocks on mu, log lambda and the weights'
//                        log-ratios at alpha_t (Sec. 5.2.1 list), then the
//                        path-sampling integrand U_t = sum_i W_t,i l(theta_t,i)
//                        (eq:path_import) and the trapezoid update (eq:path_est).
//
// The likelihood l(theta) = sum_k log sum_j omega_j sqrt(lambda_j / 2 pi)
// exp(-lambda_j (y_k - mu_j)^2 / 2) is the hot loop: the data tile is staged in
// shared memory by a bulk (TMA) copy, four lanes share one particle (each
// takes every fourth datum), each datum is a log-sum-exp over the components
// in base 2 (MUFU ex2), and the per-datum logs are folded into one lg2 per
// group of 8 data (the sum of logs is the log of the product; every factor
// is in [1, r]).  Group sums are accumulated with Kahan compensation in
// float, the quad's partial sums in float64.
#pragma once

#include "weight_reduce.cuh"

namespace smc {

constexpr bool kGmmEnabled = true;
constexpr int kGmmMaxComp = 8;
constexpr int64_t kGmmMaxData = 8192;
constexpr int kQuad = 4;                      // lanes per particle in the likelihood loop
constexpr int kGmmGroup = 8;                  // data per lg2
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2e = 1.44269504088896340736;

template <typename R>
struct GmmArgs {
    int64_t n;
    int64_t ld;             // row pitch of the state and log-weight arrays
    int32_t nd;             // data points
    const R *y;             // data (16-byte aligned, padded to a multiple of 16 bytes)
    R *x[2];                // state buffers; row j at x[b] + j * ld
    R *lw[2];
    const int32_t *anc;
    const double *alpha;    // alpha_t, t = 0..T
    int32_t T;
    smc_record *rec;
    int32_t rec_cap;
    DevState *st;
    Partial *part;
    double log_n;
    double threshold;
    // prior: lp = lp_const + sum_j [-(mu_j - mu0)^2 / (2 sd0^2) + (a - 1) log lambda_j - b lambda_j]
    double mu0, sd0, inv_sd0, lp_const, shape_m1, rate;
    double half_nd_log2pi;  // nd log(2 pi) / 2
    double mala_eps;        // Langevin step size
    // the same constants in float for the FP32 instantiation (no per-thread float64)
    float mu0_f, inv_sd0_f, lp_const_f, shape_m1_f, rate_f, mala_eps_f;
    float hnl_f[2];         // half_nd_log2pi as a double-float value
    uint2 key;
    uint32_t stream;
    // a shard of a sampler partitioned over ranks: the Philox index of
    // particle 0 (its global index), and where the init, reweight and mcmc
    // kernels put the shard's combined partial instead of finalising (null:
    // a whole sampler)
    uint32_t index0;
    Partial *shard_out;
};

// Model constants in the kernel's precision R (the FP64 instantiation keeps
// its float64 values; the FP32 one uses the float copies).
template <typename R>
struct GmmC {
    R mu0, inv_sd0, lp_const, shape_m1, rate, eps;
};
template <typename R>
__device__ __forceinline__ GmmC<R> gmm_c(const GmmArgs<R> &a) {
    if constexpr (sizeof(R) == 8) return GmmC<R>{a.mu0, a.inv_sd0, a.lp_const, a.shape_m1, a.rate, a.mala_eps};
    else return GmmC<R>{a.mu0_f, a.inv_sd0_f, a.lp_const_f, a.shape_m1_f, a.rate_f, a.mala_eps_f};
}

// Metropolis log-ratio of the tempered target from (log-prior, log-likelihood)
// pairs.  FP64: as written; FP32: grouped so that the nearly equal
// log-likelihoods cancel exactly (Sterbenz) before the multiplication by alpha.
template <typename R>
__device__ __forceinline__ R mh_delta(R lp2, R lp, R ll2, R ll, R a_t) {
    if constexpr (sizeof(R) == 8) return (lp2 + a_t * ll2) - (lp + a_t * ll);
    else return (lp2 - lp) + a_t * (ll2 - ll);
}

// moves of the mcmc kernel
constexpr int kMoveRW = 0;
constexpr int kMoveMALA = 1;
constexpr int kMoveRWMALA = 2;

// ---- per-datum math in base 2 ---------------------------------------------
template <typename R>
struct Base2;

template <>
struct Base2<float> {
    static __device__ __forceinline__ float ex2(float x) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float lg2(float x) {
        float y;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
};

template <>
struct Base2<double> {
    static __device__ __forceinline__ double ex2(double x) { return ::exp2(x); }
    static __device__ __forceinline__ double lg2(double x) { return ::log2(x); }
};

// Kahan-compensated accumulator
template <typename R>
struct Kahan {
    R s = 0, c = 0;
    __device__ __forceinline__ void add(R v) {
        const R y = v - c;
        const R t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// The quad's four partial sums (Kahan pairs s - c) added up and converted
// from log2 to log, minus nd log(2 pi) / 2: float64 on the FP64 path,
// double-float (rounded to float at the end) on the FP32 path.
template <typename R>
__device__ __forceinline__ R quad_log_sum(R s, R c, const GmmArgs<R> &a) {
    if constexpr (sizeof(R) == 8) {
        double v = double(s) - double(c);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        return v * kLn2 - a.half_nd_log2pi;
    } else {
        constexpr float kLn2Hi = (float)kLn2;
        constexpr float kLn2Lo = (float)(kLn2 - (double)kLn2Hi);
        DF v = two_sum(s, -c);
        v = df_add(v, df_shfl_xor(v, 1));
        v = df_add(v, df_shfl_xor(v, 2));
        const DF r = df_add(df_mul(v, DF{kLn2Hi, kLn2Lo}), DF{-a.hnl_f[0], -a.hnl_f[1]});
        return r.hi + r.lo;
    }
}

// One datum of the likelihood loop: log2 of sum_j omega_j sqrt(lambda_j)
// exp(-lambda_j (y - mu_j)^2 / 2) as m + log2(s), s in [1, NC] after the
// shift by the largest term; the group accumulates m and the product of s.
template <typename R, int NC>
__device__ __forceinline__ void gmm_datum(R yk, const R (&mu)[NC], const R (&c2)[NC], const R (&h2)[NC], R &msum,
                                          R &prod) {
    R a[NC];
    R m = -INFINITY;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const R d = yk - mu[j];
        a[j] = c2[j] - h2[j] * d * d;
        m = fmax(m, a[j]);
    }
    R s = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) s += Base2<R>::ex2(a[j] - m);
    msum += m;
    prod *= s;
}

// One datum of the likelihood-and-gradient loop: gmm_datum plus the
// responsibilities' sums sd, sl, sr.
template <typename R, int NC>
__device__ __forceinline__ void gmm_datum_grad(R yk, const R (&mu)[NC], const R (&c2)[NC], const R (&h2)[NC],
                                               R &msum, R &prod, R (&sd)[NC], R (&sl)[NC], R (&sr)[NC]) {
    R a[NC], d[NC], dd[NC];
    R m = -INFINITY;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        d[j] = yk - mu[j];
        dd[j] = d[j] * d[j];  // shared by the exponent and the second-moment sum
        a[j] = c2[j] - h2[j] * dd[j];
        m = fmax(m, a[j]);
    }
    R e[NC], s = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        e[j] = Base2<R>::ex2(a[j] - m);
        s += e[j];
    }
    const R inv = fast_rcp(s);  // s in [1, NC]: the division routine would cost more than the datum
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const R rho = e[j] * inv;
        sd[j] += rho * d[j];
        sl[j] += rho * dd[j];
        sr[j] += rho;
    }
    msum += m;
    prod *= s;
}

// Log-likelihood of one particle, the data split over the kQuad lanes of
// its quad (lane q takes y_q, y_{q+4}, ...; the full l(theta) is returned
// in all four lanes): groups of kGmmGroup data share one lg2 of the product
// of their sums.  Full groups are unrolled; the ragged end takes a rolled
// loop (the same groups either way).
template <typename R, int NC>
__device__ __forceinline__ R gmm_loglik_quad(const R (&mu)[NC], const R (&lam)[NC], const R (&om)[NC],
                                             const R *__restrict__ ys, int nd, int q, const GmmArgs<R> &ga) {
    R c2[NC], h2[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        // log2(omega_j sqrt(lambda_j)) and lambda_j log2(e) / 2
        c2[j] = Base2<R>::lg2(om[j]) + R(0.5) * Base2<R>::lg2(lam[j]);
        h2[j] = R(0.5 * kLog2e) * lam[j];
    }
    Kahan<R> acc;
    const int cnt = nd > q ? (nd - q + kQuad - 1) / kQuad : 0;  // data of this lane
    int k = q;
#pragma unroll 1
    for (int gi = cnt / kGmmGroup; gi > 0; --gi, k += kQuad * kGmmGroup) {
        R msum = 0, prod = 1;
#pragma unroll
        for (int g = 0; g < kGmmGroup; ++g) gmm_datum<R, NC>(ys[k + g * kQuad], mu, c2, h2, msum, prod);
        acc.add(msum + Base2<R>::lg2(prod));
    }
    if (k < nd) {
        R msum = 0, prod = 1;
#pragma unroll 1
        for (; k < nd; k += kQuad) gmm_datum<R, NC>(ys[k], mu, c2, h2, msum, prod);
        acc.add(msum + Base2<R>::lg2(prod));
    }
    return quad_log_sum<R>(acc.s, acc.c, ga);
}

// Log-likelihood and its gradient in (mu, log lambda, log(omega_j / omega_r))
// for one particle (quad-split data as above).  gm, gl, gz receive
// sum_k rho_kj lambda_j (y_k - mu_j), sum_k rho_kj (1 - lambda_j (y_k - mu_j)^2) / 2
// and sum_k (rho_kj - omega_j), with rho the responsibilities.
template <typename R, int NC>
__device__ __forceinline__ R gmm_loglik_grad_quad(const R (&mu)[NC], const R (&lam)[NC], const R (&om)[NC],
                                                  const R *__restrict__ ys, int nd, int q, const GmmArgs<R> &ga,
                                                  R (&gm)[NC], R (&gl)[NC], R (&gz)[NC]) {
    R c2[NC], h2[NC], sd[NC], sl[NC], sr[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        c2[j] = Base2<R>::lg2(om[j]) + R(0.5) * Base2<R>::lg2(lam[j]);
        h2[j] = R(0.5 * kLog2e) * lam[j];
        sd[j] = sl[j] = sr[j] = R(0);
    }
    Kahan<R> acc;
    const int cnt = nd > q ? (nd - q + kQuad - 1) / kQuad : 0;
    int k = q;
#pragma unroll 1
    for (int gi = cnt / kGmmGroup; gi > 0; --gi, k += kQuad * kGmmGroup) {
        R msum = 0, prod = 1;
#pragma unroll
        for (int g = 0; g < kGmmGroup; ++g)
            gmm_datum_grad<R, NC>(ys[k + g * kQuad], mu, c2, h2, msum, prod, sd, sl, sr);
        acc.add(msum + Base2<R>::lg2(prod));
    }
    if (k < nd) {
        R msum = 0, prod = 1;
#pragma unroll 1
        for (; k < nd; k += kQuad) gmm_datum_grad<R, NC>(ys[k], mu, c2, h2, msum, prod, sd, sl, sr);
        acc.add(msum + Base2<R>::lg2(prod));
    }
    const R total = quad_log_sum<R>(acc.s, acc.c, ga);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        sd[j] += __shfl_xor_sync(0xffffffffu, sd[j], 1);
        sd[j] += __shfl_xor_sync(0xffffffffu, sd[j], 2);
        sl[j] += __shfl_xor_sync(0xffffffffu, sl[j], 1);
        sl[j] += __shfl_xor_sync(0xffffffffu, sl[j], 2);
        sr[j] += __shfl_xor_sync(0xffffffffu, sr[j], 1);
        sr[j] += __shfl_xor_sync(0xffffffffu, sr[j], 2);
        gm[j] = lam[j] * sd[j];
        gl[j] = R(0.5) * (sr[j] - lam[j] * sl[j]);
        gz[j] = sr[j] - R(nd) * om[j];
    }
    return total;
}

template <typename R, int NC>
__device__ __forceinline__ R gmm_log_prior(const GmmArgs<R> &a, const R (&mu)[NC], const R (&lam)[NC],
                                           const R (&om)[NC]) {
    const GmmC<R> k = gmm_c<R>(a);
    R lp = k.lp_const;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const R z = (mu[j] - k.mu0) * k.inv_sd0;
        lp += R(-0.5) * z * z - k.rate * lam[j];
        if (k.shape_m1 != R(0)) lp += k.shape_m1 * Math<R>::log(lam[j]);
        bad |= !(lam[j] > R(0)) || !(om[j] >= R(0));
    }
    return bad ? Math<R>::neg_inf() : lp;
}

// r standard normals from draws 0 and 1 of (index, t, tag)
template <typename R, int NC>
__device__ __forceinline__ void gmm_normals(uint2 key, uint32_t i, uint32_t t, uint32_t tag, uint32_t stream,
                                            R (&z)[NC]) {
    R w[8];
    normals4<R>(draw(key, i, t, tag, stream, 0u), w);
    if (NC > 4) normals4<R>(draw(key, i, t, tag, stream, 1u), w + 4);
#pragma unroll
    for (int j = 0; j < NC; ++j) z[j] = w[j];
}

template <typename R>
__device__ __forceinline__ R mh_log_uniform(uint2 key, uint32_t i, uint32_t t, uint32_t tag, uint32_t stream) {
    return Math<R>::log(uniform01<R>(draw(key, i, t, tag, stream, DRAW_MH_UNIFORM).x));
}

// Bulk-copy (TMA) the data into shared memory; bounded wait on the mbarrier.
// Returns false to every thread when the copy did not complete within the
// wait limit (SMC_E_TIMEOUT raised): the caller must not read the tile.
__device__ __forceinline__ bool stage_data(void *smem_dst, const void *gsrc, uint32_t bytes, DevState *st) {
    __shared__ alignas(8) unsigned long long s_mbar;
    __shared__ uint32_t s_done;
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem_dst);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
            "l"(gsrc), "r"(bytes), "r"(mbar)
            : "memory");
    }
    uint32_t done = 0;
    for (uint32_t it = 0; it < c_wait_limit && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mbar)
            : "memory");
    }
    if (!done) {
        // the copy did not complete in time: raise the error, then wait once
        // more (bounded) so that a late copy does not land in the shared
        // memory of a later block; the caller skips its compute either way
        raise_error(st, SMC_E_TIMEOUT);
        uint32_t late = 0;
        for (uint32_t it = 0; it < c_wait_limit && !late; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(late)
                : "r"(mbar)
                : "memory");
        }
    }
    if (threadIdx.x == 0) s_done = 1u;
    __syncthreads();
    if (!done) atomicAnd(&s_done, 0u);  // any thread that gave up
    __syncthreads();
    return s_done != 0u;
}

// ---- state rows -------------------------------------------------------------
template <typename R, int NC>
struct Theta {
    R mu[NC], lam[NC], om[NC];
    R lp, ll;
    R gm[NC], gl[NC], gz[NC];  // cached likelihood gradient (Langevin moves)
};

// rows: mu (NC), lambda (NC), omega (NC), log-prior, log-likelihood, then
// with G the gradient: d/dmu (NC), d/dlog lambda (NC), d/dz (NC - 1)
template <typename R, int NC, bool G>
__device__ __forceinline__ void load_theta(const R *x, int64_t ld, int64_t i, Theta<R, NC> &th) {
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        th.mu[j] = x[(int64_t)j * ld + i];
        th.lam[j] = x[(int64_t)(NC + j) * ld + i];
        th.om[j] = x[(int64_t)(2 * NC + j) * ld + i];
    }
    th.lp = x[(int64_t)(3 * NC) * ld + i];
    th.ll = x[(int64_t)(3 * NC + 1) * ld + i];
    if (G) {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            th.gm[j] = x[(int64_t)(3 * NC + 2 + j) * ld + i];
            th.gl[j] = x[(int64_t)(4 * NC + 2 + j) * ld + i];
            th.gz[j] = (j < NC - 1) ? x[(int64_t)(5 * NC + 2 + j) * ld + i] : R(0);
        }
    }
}

template <typename R, int NC, bool G>
__device__ __forceinline__ void store_theta(R *x, int64_t ld, int64_t i, const Theta<R, NC> &th) {
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        x[(int64_t)j * ld + i] = th.mu[j];
        x[(int64_t)(NC + j) * ld + i] = th.lam[j];
        x[(int64_t)(2 * NC + j) * ld + i] = th.om[j];
    }
    x[(int64_t)(3 * NC) * ld + i] = th.lp;
    x[(int64_t)(3 * NC + 1) * ld + i] = th.ll;
    if (G) {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            x[(int64_t)(3 * NC + 2 + j) * ld + i] = th.gm[j];
            x[(int64_t)(4 * NC + 2 + j) * ld + i] = th.gl[j];
            if (j < NC - 1) x[(int64_t)(5 * NC + 2 + j) * ld + i] = th.gz[j];
        }
    }
}

// One Metropolis-adjusted Langevin move on u = (mu, log lambda, z), z_j =
// log(omega_j / omega_r), targeting gamma = log-prior + alpha l + sum log lambda
// + sum log omega, from the cached likelihood gradient at the current point.
// Returns 1 when accepted.  All four lanes of a quad take the same decision.
// Arithmetic in R (float64 on the FP64 path).
template <typename R, int NC>
__device__ __forceinline__ uint32_t mala_move(const GmmArgs<R> &a, Theta<R, NC> &th, R &lp, R &ll, R a_t,
                                              uint32_t ii, uint32_t t, const R *ys, int q) {
    constexpr int D = 3 * NC - 1;
    const GmmC<R> k = gmm_c<R>(a);
    const R eps = k.eps, h = R(0.5) * eps * eps;
    // gradient of gamma at the current point
    R u[D], g[D], xi[D];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        u[j] = th.mu[j];
        u[NC + j] = Math<R>::log(th.lam[j]);
        g[j] = -(th.mu[j] - k.mu0) * k.inv_sd0 * k.inv_sd0 + a_t * th.gm[j];
        g[NC + j] = k.shape_m1 - k.rate * th.lam[j] + R(1) + a_t * th.gl[j];
        if (j < NC - 1) {
            u[2 * NC + j] = Math<R>::log(th.om[j] / th.om[NC - 1]);
            g[2 * NC + j] = R(1) - R(NC) * th.om[j] + a_t * th.gz[j];
        }
    }
    // 3r - 1 normals from draws 0, 1, 2, ... of TAG_MALA
#pragma unroll
    for (int c = 0; c < (D + 3) / 4; ++c) {
        R z4[4];
        normals4<R>(draw(a.key, ii, t, TAG_MALA, a.stream, (uint32_t)c), z4);
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (4 * c + m < D) xi[4 * c + m] = z4[m];
    }
    R up[D];
    R xi2 = 0;
#pragma unroll
    for (int kk = 0; kk < D; ++kk) {
        up[kk] = u[kk] + h * g[kk] + eps * xi[kk];
        xi2 += xi[kk] * xi[kk];
    }
    Theta<R, NC> p2;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        p2.mu[j] = up[j];
        p2.lam[j] = Math<R>::exp(up[NC + j]);
    }
    R vmax = 0;
#pragma unroll
    for (int j = 0; j < NC - 1; ++j) vmax = fmax(vmax, up[2 * NC + j]);
    R sum = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        p2.om[j] = Math<R>::exp(((j < NC - 1) ? up[2 * NC + j] : R(0)) - vmax);
        sum += p2.om[j];
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) p2.om[j] = p2.om[j] / sum;
    const R lp2 = gmm_log_prior<R, NC>(a, p2.mu, p2.lam, p2.om);
    const R ll2 = gmm_loglik_grad_quad<R, NC>(p2.mu, p2.lam, p2.om, ys, a.nd, q, a, p2.gm, p2.gl, p2.gz);
    R jac = 0, jac2 = 0, bwd = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        jac += u[NC + j] + Math<R>::log(th.om[j]);
        jac2 += up[NC + j] + Math<R>::log(p2.om[j]);
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const R gpm = -(p2.mu[j] - k.mu0) * k.inv_sd0 * k.inv_sd0 + a_t * p2.gm[j];
        const R gpl = k.shape_m1 - k.rate * p2.lam[j] + R(1) + a_t * p2.gl[j];
        const R rm = u[j] - up[j] - h * gpm;
        const R rl = u[NC + j] - up[NC + j] - h * gpl;
        bwd += rm * rm + rl * rl;
        if (j < NC - 1) {
            const R gpz = R(1) - R(NC) * p2.om[j] + a_t * p2.gz[j];
            const R rz = u[2 * NC + j] - up[2 * NC + j] - h * gpz;
            bwd += rz * rz;
        }
    }
    R delta;
    if constexpr (sizeof(R) == 8)
        delta = (lp2 + a_t * ll2 + jac2) - (lp + a_t * ll + jac) - bwd / (2.0 * eps * eps) + 0.5 * xi2;
    else
        delta = mh_delta<R>(lp2, lp, ll2, ll, a_t) + (jac2 - jac) - bwd / (R(2) * eps * eps) + R(0.5) * xi2;
    const R lu = mh_log_uniform<R>(a.key, ii, t, TAG_MALA, a.stream);
    if (lu <= delta) {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            th.mu[j] = p2.mu[j];
            th.lam[j] = p2.lam[j];
            th.om[j] = p2.om[j];
            th.gm[j] = p2.gm[j];
            th.gl[j] = p2.gl[j];
            th.gz[j] = p2.gz[j];
        }
        lp = lp2;
        ll = ll2;
        return 1u;
    }
    return 0u;
}

// ---- tempered log-target and its gradient at given points -------------------
// gamma_alpha(u) = log-prior(theta(u)) + alpha l(theta(u)) + log |d theta / d u|
// in u = (mu, log lambda, z), z_j = log(omega_j / omega_r): the target of the
// Langevin move, with the same expressions (Sec. 5.2 model; the gradient is
// the hand-written adjoint through the per-datum log-sum-exp).  One quad of
// lanes per point; u and grad are (3r - 1) rows of pitch ldu.
template <typename R, int NC>
__global__ void __launch_bounds__(kBlock) gmm_log_target_kernel(GmmArgs<R> a, const R *u, int64_t count,
                                                                int64_t ldu, double alpha, R *logt, R *grad) {
    constexpr int D = 3 * NC - 1;
    extern __shared__ __align__(16) unsigned char s_raw[];
    const R *ys = reinterpret_cast<const R *>(s_raw);
    if (!stage_data(s_raw, a.y, (uint32_t)(((size_t)a.nd * sizeof(R) + 15) & ~size_t(15)), a.st)) return;
    const int q = threadIdx.x & (kQuad - 1);
    const int64_t i = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / kQuad;
    const bool active = i < count;
    const int64_t ii = active ? i : count - 1;
    R uu[D];
#pragma unroll
    for (int k = 0; k < D; ++k) uu[k] = u[(int64_t)k * ldu + ii];
    Theta<R, NC> th;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        th.mu[j] = uu[j];
        th.lam[j] = Math<R>::exp(uu[NC + j]);
    }
    R vmax = 0;
#pragma unroll
    for (int j = 0; j < NC - 1; ++j) vmax = fmax(vmax, uu[2 * NC + j]);
    R sum = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        th.om[j] = Math<R>::exp(((j < NC - 1) ? uu[2 * NC + j] : R(0)) - vmax);
        sum += th.om[j];
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) th.om[j] = th.om[j] / sum;
    const double lp = double(gmm_log_prior<R, NC>(a, th.mu, th.lam, th.om));
    const double ll = double(gmm_loglik_grad_quad<R, NC>(th.mu, th.lam, th.om, ys, a.nd, q, a, th.gm, th.gl, th.gz));
    if (!active || q != 0) return;
    double jac = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) jac += double(uu[NC + j]) + double(Math<R>::log(th.om[j]));
    logt[ii] = R(lp + alpha * ll + jac);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        grad[(int64_t)j * ldu + ii] =
            R(-(double(th.mu[j]) - a.mu0) * a.inv_sd0 * a.inv_sd0 + alpha * double(th.gm[j]));
        grad[(int64_t)(NC + j) * ldu + ii] = R(a.shape_m1 - a.rate * double(th.lam[j]) + 1.0 + alpha * double(th.gl[j]));
        if (j < NC - 1)
            grad[(int64_t)(2 * NC + j) * ldu + ii] = R(1.0 - NC * double(th.om[j]) + alpha * double(th.gz[j]));
    }
}

// ---- init: theta ~ prior, equal weights, U_0 --------------------------------
// ---- finalisation of the init, reweight and mcmc kernels (thread 0 of
// the last block, or of gmm_shard_finalize_kernel on every rank's partials
// of a partitioned sampler) ---------------------------------------------------
template <typename R>
__device__ __forceinline__ void gmm_init_finish(const GmmArgs<R> &a, DevState *st, const Combined &c, int cur,
                                                int cur_lw) {
    FinalizeArgs f{st, a.rec, a.rec_cap, 0, 0, a.n, a.threshold, 0.0};
    double L;
    if (finalize_weights(f, c, &L)) {
        const double U0 = c.Sa / c.S1;
        smc_record *r = &a.rec[0];
        r->path_u = U0;
        r->path_log_z = 0.0;
        r->log_evidence = 0.0;  // the prior is normalised: log Z_0 = 0
        st->log_evidence = 0.0;
        st->path_u = U0;
        st->path_log_z = 0.0;
        st->alpha = 0.0;
        st->base_shift = L;
        st->t = 0;
        st->cur = cur ^ 1;
        st->cur_lw = cur_lw ^ 1;
        st->ready = 0;
        st->gathered = 0;
        st->accept[0] = st->accept[1] = st->accept[2] = st->accept[3] = 0;
    }
}

template <typename R>
__device__ __forceinline__ void gmm_reweight_finish(const GmmArgs<R> &a, DevState *st, const Combined &c, int32_t t,
                                                    int cur_lw, double a_t) {
    FinalizeArgs f{st, a.rec, a.rec_cap, t, 0, a.n, a.threshold, a_t};
    double L;
    if (finalize_weights(f, c, &L)) {
        smc_record *r = &a.rec[t % a.rec_cap];
        r->path_u = st->path_u;
        r->path_log_z = st->path_log_z;
        st->alpha = a_t;
        st->base_shift = L;
        st->t = t;
        st->cur_lw = cur_lw ^ 1;
        st->accept[0] = st->accept[1] = st->accept[2] = st->accept[3] = 0;
    }
}

// accepted moves per block in st->accept (summed over the ranks for a
// partitioned sampler); rates over a.n particles
template <typename R, int MOVE>
__device__ __forceinline__ void gmm_mcmc_finish(const GmmArgs<R> &a, DevState *st, const Combined &c, int32_t t,
                                                int cur, bool gather) {
    constexpr bool G = (MOVE != kMoveRW);
    smc_record *r = &a.rec[t % a.rec_cap];
    if (!(c.S1 > 0.0)) {
        raise_error(st, SMC_E_NONFINITE);
        r->status = SMC_E_NONFINITE;
        st->ticket = 0;
        return;
    }
    st->ticket = 0;
    const double a_t = a.alpha[t], a_p = (t > 0) ? a.alpha[t - 1] : 0.0;
    const double U = c.Sa / c.S1;
    const double plz = st->path_log_z + 0.5 * (a_t - a_p) * (U + st->path_u);
    r->path_u = U;
    r->path_log_z = plz;
    for (int b = 0; b < 3; ++b)
        r->accept[b] = (MOVE == kMoveMALA) ? 0.0 : double(*(volatile uint32_t *)&st->accept[b]) / double(a.n);
    r->accept_mala = G ? double(*(volatile uint32_t *)&st->accept[3]) / double(a.n) : 0.0;
    st->path_u = U;
    st->path_log_z = plz;
    st->cur = cur ^ 1;
    if (gather) st->base_shift = 0.0;
    st->gathered = gather ? 1 : 0;
    st->ready = 0;
}

// A shard's partial (the last block, whole block): its blocks' partials
// combined in a fixed order into one partial of the partial layout (FP32:
// double-float sums and the float maximum; FP64: float64 fields); with
// accept, bytes 48..63 (unused by both layouts) carry the shard's four
// accepted-move counts.
constexpr int kShardAcceptOffset = 48;
template <typename R>
__device__ __forceinline__ void gmm_shard_partial_out(DevState *st, const Partial *part, int nb, Partial *out,
                                                      bool accept) {
    if constexpr (sizeof(R) == 4) {
        CombinedDF c;
        combine_partials_df<4>(part, nb, &c);
        if (threadIdx.x == 0) PartialIO<float>::store(out, c.M, c.S);
    } else {
        Combined c;
        combine_partials<R>(part, nb, &c);
        if (threadIdx.x == 0) {
            const double s4[kSums] = {c.S1, c.S2, c.Sa, c.Sb};
            PartialIO<double>::store(out, c.M, s4);
        }
    }
    if (threadIdx.x == 0) {
        uint32_t *w = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(out) + kShardAcceptOffset);
        for (int k = 0; k < 4; ++k) w[k] = accept ? *(volatile uint32_t *)&st->accept[k] : 0u;
        st->ticket = 0;
    }
}

template <typename R, int NC, bool G>
__global__ void __launch_bounds__(kBlock) gmm_init_kernel(GmmArgs<R> a) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    const R *ys = reinterpret_cast<const R *>(s_raw);
    DevState *st = a.st;
    const DevState *sv = snapshot(st);
    if (sv->error) return;
    if (!stage_data(s_raw, a.y, (uint32_t)(((size_t)a.nd * sizeof(R) + 15) & ~size_t(15)), st)) return;
    const int q = threadIdx.x & (kQuad - 1);
    const int64_t i = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / kQuad;
    const bool active = i < a.n;
    const int64_t ii = active ? i : a.n - 1;  // inactive lanes compute a copy, keep the shuffles full
    Theta<R, NC> th;
    {
        R z[NC];
        gmm_normals<R, NC>(a.key, (a.index0 + (uint32_t)ii), 0u, TAG_INIT, a.stream, z);
#pragma unroll
        for (int j = 0; j < NC; ++j) th.mu[j] = R(a.mu0) + R(a.sd0) * z[j];
        const int shape = (int)a.shape_m1 + 1;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            R e = 0;
            for (int m = 0; m < shape; ++m) {
                const int idx = j * shape + m;
                const uint4 w = draw(a.key, (a.index0 + (uint32_t)ii), 0u, TAG_INIT, a.stream, 8u + (uint32_t)(idx >> 2));
                const uint32_t ww = (idx & 3) == 0 ? w.x : (idx & 3) == 1 ? w.y : (idx & 3) == 2 ? w.z : w.w;
                e -= Math<R>::log(uniform01<R>(ww));
            }
            th.lam[j] = e / R(a.rate);
        }
        R E[NC], sum = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const uint4 w = draw(a.key, (a.index0 + (uint32_t)ii), 0u, TAG_INIT, a.stream, 64u + (uint32_t)(j >> 2));
            const uint32_t ww = (j & 3) == 0 ? w.x : (j & 3) == 1 ? w.y : (j & 3) == 2 ? w.z : w.w;
            E[j] = -Math<R>::log(uniform01<R>(ww));
            sum += E[j];
        }
#pragma unroll
        for (int j = 0; j < NC; ++j) th.om[j] = E[j] / sum;
    }
    th.lp = gmm_log_prior<R, NC>(a, th.mu, th.lam, th.om);
    th.ll = G ? gmm_loglik_grad_quad<R, NC>(th.mu, th.lam, th.om, ys, a.nd, q, a, th.gm, th.gl, th.gz)
              : gmm_loglik_quad<R, NC>(th.mu, th.lam, th.om, ys, a.nd, q, a);
    const int cur = sv->cur, cur_lw = sv->cur_lw;
    const R lw0 = R(-a.log_n);
    if (active && q == 0) {
        store_theta<R, NC, G>(a.x[cur ^ 1], a.ld, i, th);
        a.lw[cur_lw ^ 1][i] = lw0;
    }
    R lwv[1] = {(active && q == 0) ? lw0 : Math<R>::neg_inf()};
    R h0[1] = {th.ll}, zero[1] = {R(0)};
    block_partial<R, 1, 1>(lwv, h0, zero, zero, &a.part[blockIdx.x]);
    if (a.shard_out) {  // a shard: its combined partial, finalised with every rank's (gmm_shard_finalize_kernel)
        if (take_ticket<R>(st)) gmm_shard_partial_out<R>(st, a.part, gridDim.x, a.shard_out, false);
        return;
    }
    Combined c;
    if (!last_block_combine<R>(st, a.part, &c)) return;
    if (threadIdx.x == 0) gmm_init_finish<R>(a, st, c, cur, cur_lw);
}

// ---- reweight: lw_t = log W_{t-1} + dalpha l ---------------------------------
template <typename R, int NC>
__global__ void __launch_bounds__(kBlock) gmm_reweight_kernel(GmmArgs<R> a) {
    DevState *st = a.st;
    const DevState *sv = snapshot(st);
    if (sv->error) return;
    const int32_t t = sv->t + 1;
    const double a_t = a.alpha[t], a_p = a.alpha[t - 1];
    // per-block constants converted once: alpha_t - alpha_{t-1} and the
    // running shift as a split (hi, lo) in R
    __shared__ R s_k[3];
    if (threadIdx.x == 0) {
        s_k[0] = R(a_t - a_p);
        s_k[1] = R(sv->base_shift);
        s_k[2] = R(sv->base_shift - double(s_k[1]));
    }
    __syncthreads();
    const R dal = s_k[0];
    const Shift<R> base(s_k[1], s_k[2]);
    const int cur = sv->cur, cur_lw = sv->cur_lw;
    const R *lw_in = a.lw[cur_lw];
    R *lw_out = a.lw[cur_lw ^ 1];
    const R *ll = a.x[cur] + (int64_t)(3 * NC + 1) * a.ld;
    R lwv[kPfItems], zero[kPfItems];
    const int64_t b0 = (int64_t)blockIdx.x * kPfTile + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kPfItems; ++j) {
        const int64_t i = b0 + j * kBlock;
        lwv[j] = Math<R>::neg_inf();
        zero[j] = R(0);
        if (i < a.n) {
            lwv[j] = base.sub_from(lw_in[i]) + dal * ll[i];
            lw_out[i] = lwv[j];
        }
    }
    block_partial<R, kPfItems, 0>(lwv, zero, zero, zero, &a.part[blockIdx.x]);
    if (a.shard_out) {
        if (take_ticket<R>(st)) gmm_shard_partial_out<R>(st, a.part, gridDim.x, a.shard_out, false);
        return;
    }
    Combined c;
    if (!last_block_combine<R>(st, a.part, &c)) return;
    if (threadIdx.x == 0) gmm_reweight_finish<R>(a, st, c, t, cur_lw, a_t);
}

// ---- mcmc: gather, three Metropolis blocks, path sampling -------------------
template <typename R, int NC, int MOVE>
__global__ void __launch_bounds__(kBlock) gmm_mcmc_kernel(GmmArgs<R> a) {
    constexpr bool G = (MOVE != kMoveRW);
    extern __shared__ __align__(16) unsigned char s_raw[];
    __shared__ uint32_t s_acc[4];
    const R *ys = reinterpret_cast<const R *>(s_raw);
    DevState *st = a.st;
    const DevState *sv = snapshot(st);
    if (sv->error) return;
    if (threadIdx.x < 4) s_acc[threadIdx.x] = 0;
    const int32_t t = sv->t;
    // per-block constants, computed once in float64: alpha_t and the
    // proposal scales from max(alpha_t, 0.02)
    __shared__ R s_k[4];
    if (threadIdx.x == 0) {
        const double at = a.alpha[t];
        const double aclamp = fmax(at, 0.02);
        s_k[0] = R(at);
        s_k[1] = R(0.15 / aclamp);
        s_k[2] = R((1.0 + sqrt(1.0 / aclamp)) * 0.15);
        s_k[3] = R((1.0 + sqrt(1.0 / aclamp)) * 0.2);
    }
    // (its barriers publish s_k); a copy that timed out leaves the data tile
    // unread: the block stops and the error word invalidates the step
    if (!stage_data(s_raw, a.y, (uint32_t)(((size_t)a.nd * sizeof(R) + 15) & ~size_t(15)), st)) return;
    const R a_t = s_k[0], s_mu = s_k[1], s_lam = s_k[2], s_om = s_k[3];
    const bool gather = sv->ready != 0;
    const int cur = sv->cur, cur_lw = sv->cur_lw;
    const int q = threadIdx.x & (kQuad - 1);
    const int64_t i = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / kQuad;
    const bool active = i < a.n;
    const int64_t ii = active ? i : a.n - 1;
    const int64_t src = gather ? (int64_t)__ldg(&a.anc[ii]) : ii;
    Theta<R, NC> th;
    load_theta<R, NC, G>(a.x[cur], a.ld, src, th);
    R ll = th.ll, lp = th.lp;
    uint32_t acc_mask = 0;
    if (MOVE != kMoveMALA) {
    // block 1: mu
    {
        R z[NC], mu2[NC];
        gmm_normals<R, NC>(a.key, (a.index0 + (uint32_t)ii), (uint32_t)t, TAG_MH_MU, a.stream, z);
#pragma unroll
        for (int j = 0; j < NC; ++j) mu2[j] = th.mu[j] + s_mu * z[j];
        const R lp2 = gmm_log_prior<R, NC>(a, mu2, th.lam, th.om);
        const R ll2 = gmm_loglik_quad<R, NC>(mu2, th.lam, th.om, ys, a.nd, q, a);
        const R delta = mh_delta<R>(lp2, lp, ll2, ll, a_t);
        const R lu = mh_log_uniform<R>(a.key, (a.index0 + (uint32_t)ii), (uint32_t)t, TAG_MH_MU, a.stream);
        if (lu <= delta) {
#pragma unroll
            for (int j = 0; j < NC; ++j) th.mu[j] = mu2[j];
            lp = lp2;
            ll = ll2;
            acc_mask |= 1u;
        }
    }
    // block 2: log lambda
    {
        R z[NC], lam2[NC];
        gmm_normals<R, NC>(a.key, (a.index0 + (uint32_t)ii), (uint32_t)t, TAG_MH_LAMBDA, a.stream, z);
        R jac = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const R dz = s_lam * z[j];
            lam2[j] = Math<R>::exp(Math<R>::log(th.lam[j]) + dz);
            jac += dz;
        }
        const R lp2 = gmm_log_prior<R, NC>(a, th.mu, lam2, th.om);
        const R ll2 = gmm_loglik_quad<R, NC>(th.mu, lam2, th.om, ys, a.nd, q, a);
        const R delta = mh_delta<R>(lp2, lp, ll2, ll, a_t) + jac;
        const R lu = mh_log_uniform<R>(a.key, (a.index0 + (uint32_t)ii), (uint32_t)t, TAG_MH_LAMBDA, a.stream);
        if (lu <= delta) {
#pragma unroll
            for (int j = 0; j < NC; ++j) th.lam[j] = lam2[j];
            lp = lp2;
            ll = ll2;
            acc_mask |= 2u;
        }
    }
    // block 3: additive log-ratios of the weights
    if (NC > 1) {
        R z[NC], om2[NC];
        gmm_normals<R, NC>(a.key, (a.index0 + (uint32_t)ii), (uint32_t)t, TAG_MH_WEIGHT, a.stream, z);
        R v[NC];
        R vmax = 0;  // the last log-ratio is 0
#pragma unroll
        for (int j = 0; j < NC - 1; ++j) {
            v[j] = Math<R>::log(th.om[j] / th.om[NC - 1]) + s_om * z[j];
            vmax = fmax(vmax, v[j]);
        }
        v[NC - 1] = 0;
        R sum = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            om2[j] = Math<R>::exp(v[j] - vmax);
            sum += om2[j];
        }
        R jac = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            om2[j] = om2[j] / sum;
            jac += Math<R>::log(om2[j]) - Math<R>::log(th.om[j]);
        }
        const R lp2 = gmm_log_prior<R, NC>(a, th.mu, th.lam, om2);
        const R ll2 = gmm_loglik_quad<R, NC>(th.mu, th.lam, om2, ys, a.nd, q, a);
        const R delta = mh_delta<R>(lp2, lp, ll2, ll, a_t) + jac;
        const R lu = mh_log_uniform<R>(a.key, (a.index0 + (uint32_t)ii), (uint32_t)t, TAG_MH_WEIGHT, a.stream);
        if (lu <= delta) {
#pragma unroll
            for (int j = 0; j < NC; ++j) th.om[j] = om2[j];
            lp = lp2;
            ll = ll2;
            acc_mask |= 4u;
        }
    } else {
        acc_mask |= 4u;
    }
    }  // random-walk blocks
    if (MOVE == kMoveRWMALA) {
        // the blocks moved theta: refresh the cached gradient at the current point
        ll = gmm_loglik_grad_quad<R, NC>(th.mu, th.lam, th.om, ys, a.nd, q, a, th.gm, th.gl, th.gz);
    }
    if (G) acc_mask |= mala_move<R, NC>(a, th, lp, ll, a_t, (a.index0 + (uint32_t)ii), (uint32_t)t, ys, q) << 3;
    th.lp = lp;
    th.ll = ll;
    R lwi = R(-a.log_n);
    if (active && q == 0) {
        store_theta<R, NC, G>(a.x[cur ^ 1], a.ld, i, th);
        if (gather) a.lw[cur_lw][i] = lwi;  // equal weights after resampling
        else lwi = a.lw[cur_lw][i];
        atomicAdd(&s_acc[0], acc_mask & 1u);
        atomicAdd(&s_acc[1], (acc_mask >> 1) & 1u);
        atomicAdd(&s_acc[2], (acc_mask >> 2) & 1u);
        atomicAdd(&s_acc[3], (acc_mask >> 3) & 1u);
    }
    __syncthreads();
    if (threadIdx.x < 4 && s_acc[threadIdx.x]) atomicAdd(&st->accept[threadIdx.x], s_acc[threadIdx.x]);
    R lwv[1] = {(active && q == 0) ? lwi : Math<R>::neg_inf()};
    R h0[1] = {th.ll}, zero[1] = {R(0)};
    block_partial<R, 1, 1>(lwv, h0, zero, zero, &a.part[blockIdx.x]);
    if (a.shard_out) {
        if (take_ticket<R>(st)) gmm_shard_partial_out<R>(st, a.part, gridDim.x, a.shard_out, true);
        return;
    }
    Combined c;
    if (!last_block_combine<R>(st, a.part, &c)) return;
    if (threadIdx.x == 0) gmm_mcmc_finish<R, MOVE>(a, st, c, t, cur, gather);
}

// A partitioned sampler's finalisation on every rank's shard partials (rank
// order, gathered): kind 0 after the init kernels (t = 0), 1 after the
// reweight kernels, 2 after the mcmc kernels (the ranks' accepted-move
// counts summed into st->accept first).  a.n is the sampler's N.  The same
// finalisation functions as a whole sampler's, on the combined partials.
template <typename R, int MOVE>
__global__ void __launch_bounds__(kBlock) gmm_shard_finalize_kernel(GmmArgs<R> a, const Partial *parts, int world,
                                                                    int kind) {
    DevState *st = a.st;
    const DevState *sv = snapshot(st, true);
    if (sv->error) return;
    Combined c;
    combine_partials<R>(parts, world, &c);  // every thread; thread 0 holds the result
    if (threadIdx.x != 0) return;
    if (kind == 0) {
        gmm_init_finish<R>(a, st, c, sv->cur, sv->cur_lw);
    } else if (kind == 1) {
        const int32_t t = sv->t + 1;
        gmm_reweight_finish<R>(a, st, c, t, sv->cur_lw, a.alpha[t]);
    } else {
        for (int k = 0; k < 4; ++k) {
            uint32_t v = 0;
            for (int r = 0; r < world; ++r)
                v += *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(&parts[r]) +
                                                         kShardAcceptOffset + 4 * k);
            st->accept[k] = v;
        }
        gmm_mcmc_finish<R, MOVE>(a, st, c, sv->t, sv->cur, false);
    }
}

// ---- adaptive tempering (SMC_ALPHA_ADAPTIVE) ---------------------------------
// alpha_t such that the conditional ESS of the incremental weights
// w_i = exp(delta l_i), delta = alpha_t - alpha_{t-1}, under the current
// normalised weights W_i,
//     CESS(delta) = N (sum_i W_i w_i)^2 / sum_i W_i w_i^2   (Sec. 2.1 ESS),
// equals rho N (the annealing schemes of Sec. 5.2.3 made adaptive):
// alpha_t = 1 when CESS(1 - alpha_{t-1}) >= rho N, else kAdaptSteps halvings
// of [0, 1 - alpha_{t-1}] keeping the lower end.  One cooperative wave; each
// block keeps its particles' (log W_i, l_i), and every evaluation is a block
// partial (max and sum of exp for x = log W + delta l and y = log W +
// 2 delta l), a grid barrier, and the same fixed-order combine in every
// block, so that every block takes the same decision and the midpoints are
// float64 values computed identically everywhere.
constexpr int kAdaptSteps = 40;  // halvings

template <typename R>
struct AlphaPartial {  // one per block and evaluation
    R mx, sx, my, sy;
};

// log CESS - log(rho N) >= 0 from the block partials, by one warp (lane 0
// receives the answer): float64 on the FP64 path, double-float sums and
// logarithms on the FP32 path (no float64 arithmetic there).
// ln_rel = log N - log(rho N) as a double-float (hi, lo) value
template <typename R>
__device__ __forceinline__ bool alpha_cess_ge(const AlphaPartial<R> *part, int G, double log_n, double log_target,
                                              DF ln_rel) {
    const int lane = threadIdx.x & 31;
    R MX = Math<R>::neg_inf(), MY = Math<R>::neg_inf();
    for (int q = lane; q < G; q += 32) {
        MX = fmax(MX, __ldcg(&part[q].mx));
        MY = fmax(MY, __ldcg(&part[q].my));
    }
    MX = warp_max(MX);
    MY = warp_max(MY);
    if constexpr (sizeof(R) == 8) {
        double ax = 0.0, ay = 0.0;
        for (int q = lane; q < G; q += 32) {
            const double pmx = __ldcg(&part[q].mx), pmy = __ldcg(&part[q].my);
            if (pmx > -INFINITY) ax += __ldcg(&part[q].sx) * exp(pmx - MX);
            if (pmy > -INFINITY) ay += __ldcg(&part[q].sy) * exp(pmy - MY);
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        if (!(ax > 0.0) || !(ay > 0.0)) return false;
        return 2.0 * (MX + log(ax)) - (MY + log(ay)) + log_n >= log_target;
    } else {
        DF ax{0.0f, 0.0f}, ay{0.0f, 0.0f};
        for (int q = lane; q < G; q += 32) {
            const float pmx = __ldcg(&part[q].mx), pmy = __ldcg(&part[q].my);
            if (pmx > -INFINITY) ax = df_add(ax, two_prod(__ldcg(&part[q].sx), __expf(pmx - MX)));
            if (pmy > -INFINITY) ay = df_add(ay, two_prod(__ldcg(&part[q].sy), __expf(pmy - MY)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ax = df_add(ax, df_shfl_xor(ax, o));
            ay = df_add(ay, df_shfl_xor(ay, o));
        }
        if (!(ax.hi > 0.0f) || !(ay.hi > 0.0f)) return false;
        // 2 (MX + log A) - (MY + log B) + log N - log(rho N), in double-float
        DF v = df_add(df_add_f(df_add(df_log(ax), df_log(ax)), 2.0f * MX), DF{-MY, 0.0f});
        const DF lb = df_log(ay);
        v = df_add(v, DF{-lb.hi, -lb.lo});
        v = df_add(v, ln_rel);
        return v.hi >= 0.0f;
    }
}

// Candidates per grid barrier: the upper end of the interval (first round
// only) and the seven midpoints of the next three halvings, evaluated
// together; the walk down that subtree takes exactly the decisions that
// three sequential halvings would take, on the same float64 midpoints.
constexpr int kAdaptLevels = 3;
constexpr int kAdaptCand = (1 << kAdaptLevels);  // 7 midpoints + the upper end

template <typename R>
__global__ void __launch_bounds__(kBlock, 4) gmm_alpha_kernel(GmmArgs<R> a, int32_t ll_row, double log_target,
                                                              double *alpha_out, AlphaPartial<R> *part) {
    DevState *st = a.st;
    const DevState *sv = snapshot(st, true);
    if (sv->error) return;
    const int32_t t = sv->t + 1;
    const double a_prev = a.alpha[t - 1];
    const int G = gridDim.x, b = blockIdx.x;
    const int64_t i_lo = a.n * b / G, i_hi = a.n * (b + 1) / G;
    const int cur = sv->cur, cur_lw = sv->cur_lw;
    const R *lw_in = a.lw[cur_lw];
    const R *ll = a.x[cur] + (int64_t)ll_row * a.ld;
    __shared__ R s_k[2];
    if (threadIdx.x == 0) {  // the reweighting kernel's split of the running shift
        s_k[0] = R(sv->base_shift);
        s_k[1] = R(sv->base_shift - double(s_k[0]));
    }
    __syncthreads();
    const Shift<R> base(s_k[0], s_k[1]);
    // the thread's first kMax particles kept in registers, the rest read
    // again at every round
    constexpr int kMax = 4;
    R lwk[kMax], llk[kMax];
#pragma unroll
    for (int j = 0; j < kMax; ++j) {
        const int64_t i = i_lo + threadIdx.x + (int64_t)j * kBlock;
        lwk[j] = (i < i_hi) ? base.sub_from(lw_in[i]) : Math<R>::neg_inf();
        llk[j] = (i < i_hi) ? ll[i] : R(0);
    }
    const int64_t i_rest = i_lo + threadIdx.x + (int64_t)kMax * kBlock;
    __shared__ double s_d[kAdaptCand];       // the round's candidates
    __shared__ R s_dr[2][kAdaptCand];          // and their float conversions (d, 2d), made once per block
    __shared__ R s_red[4][kAdaptCand][kBlock / 32];
    __shared__ int s_ge[kAdaptCand];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // float64 constants computed once per block (float64 is 1/64 of the
    // FP32 rate on B300)
    __shared__ DF s_ln;
    __shared__ double s_logn;
    if (threadIdx.x == 0) {
        s_logn = log(double(a.n));
        const float h = float(s_logn - log_target);
        s_ln = DF{h, float((s_logn - log_target) - double(h))};
    }
    __syncthreads();
    const double log_n = s_logn;
    const DF ln_rel = s_ln;
    double lo = 0.0, hi = 1.0 - a_prev, delta = 0.0;
    bool done = !(hi > 0.0);
    int levels = 0;  // halvings taken
    uint32_t barriers = 0;
    while (!done && levels < kAdaptSteps) {
        const bool first = (barriers == 0);
        // candidates: the subtree's midpoints in heap order (0; 1, 2; 3..6),
        // each the midpoint of its interval as a sequential halving computes
        // it; slot 7 the upper end in the first round
        if (threadIdx.x == 0) {
            double m[7];
            m[0] = 0.5 * (lo + hi);
            m[1] = 0.5 * (lo + m[0]);
            m[2] = 0.5 * (m[0] + hi);
            m[3] = 0.5 * (lo + m[1]);
            m[4] = 0.5 * (m[1] + m[0]);
            m[5] = 0.5 * (m[0] + m[2]);
            m[6] = 0.5 * (m[2] + hi);
            for (int c = 0; c < 7; ++c) s_d[c] = m[c];
            s_d[7] = hi;
            for (int c = 0; c < kAdaptCand; ++c) {
                s_dr[0][c] = R(s_d[c]);
                s_dr[1][c] = R(2.0 * s_d[c]);
            }
        }
        __syncthreads();
        AlphaPartial<R> *pe = part + (size_t)(barriers & 1u) * kAdaptCand * (size_t)G;
#pragma unroll 1
        for (int c = 0; c < kAdaptCand; ++c) {
            if (c == 7 && !first) break;
            const R dr = s_dr[0][c], d2 = s_dr[1][c];
            R mx = Math<R>::neg_inf(), my = Math<R>::neg_inf();
#pragma unroll
            for (int j = 0; j < kMax; ++j) {
                mx = fmax(mx, lwk[j] + dr * llk[j]);
                my = fmax(my, lwk[j] + d2 * llk[j]);
            }
            for (int64_t i = i_rest; i < i_hi; i += kBlock) {
                const R w = base.sub_from(lw_in[i]), l = ll[i];
                mx = fmax(mx, w + dr * l);
                my = fmax(my, w + d2 * l);
            }
            mx = warp_max(mx);
            my = warp_max(my);
            if (lane == 0) {
                s_red[0][c][warp] = mx;
                s_red[1][c][warp] = my;
            }
            __syncthreads();
            mx = s_red[0][c][0];
            my = s_red[1][c][0];
#pragma unroll
            for (int w = 1; w < kBlock / 32; ++w) {
                mx = fmax(mx, s_red[0][c][w]);
                my = fmax(my, s_red[1][c][w]);
            }
            R sx = R(0), sy = R(0);
            if (mx > Math<R>::neg_inf()) {
#pragma unroll
                for (int j = 0; j < kMax; ++j)
                    if (lwk[j] > Math<R>::neg_inf()) {
                        sx += Math<R>::fast_exp(lwk[j] + dr * llk[j] - mx);
                        sy += Math<R>::fast_exp(lwk[j] + d2 * llk[j] - my);
                    }
                for (int64_t i = i_rest; i < i_hi; i += kBlock) {
                    const R w = base.sub_from(lw_in[i]), l = ll[i];
                    if (w > Math<R>::neg_inf()) {
                        sx += Math<R>::fast_exp(w + dr * l - mx);
                        sy += Math<R>::fast_exp(w + d2 * l - my);
                    }
                }
            }
            sx = warp_sum(sx);
            sy = warp_sum(sy);
            if (lane == 0) {
                s_red[2][c][warp] = sx;
                s_red[3][c][warp] = sy;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                R tx = R(0), ty = R(0);
#pragma unroll
                for (int w = 0; w < kBlock / 32; ++w) {
                    tx += s_red[2][c][w];
                    ty += s_red[3][c][w];
                }
                // partials of consecutive rounds alternate between two
                // halves: a block writing round e + 2 has passed the barrier
                // of e + 1, reached by every block after it read round e
                pe[(size_t)c * G + b] = AlphaPartial<R>{mx, tx, my, ty};
            }
        }
        ++barriers;
        if (!grid_barrier(st, barriers * (uint32_t)G)) return;
        // every block: the same combines in the same order, one warp per candidate
        if (warp < kAdaptCand && (warp < 7 || first)) {
            const bool ge = alpha_cess_ge<R>(pe + (size_t)warp * G, G, log_n, log_target, ln_rel);
            if (lane == 0) s_ge[warp] = ge ? 1 : 0;
        }
        __syncthreads();
        if (first && s_ge[7]) {
            delta = hi;
            done = true;
        } else {
            // walk the subtree: at node k the answer sends the interval to
            // [mid, hi] (CESS still at least the target) or [lo, mid]
            int k = 0;
            for (int l = 0; l < kAdaptLevels && levels < kAdaptSteps; ++l, ++levels) {
                const double mid = s_d[k];
                const bool ge = s_ge[k] != 0;
                if (ge) lo = mid;
                else hi = mid;
                k = 2 * k + (ge ? 2 : 1);
            }
        }
        __syncthreads();  // s_d, s_red and s_ge are reused by the next round
    }
    if (!done) delta = lo;
    if (b == 0 && threadIdx.x == 0) alpha_out[t] = fmin(1.0, a_prev + delta);
    if (barriers) grid_depart(st);
}

}  // namespace smc
