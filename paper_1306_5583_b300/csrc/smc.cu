// C ABI of the SMC hot path (include/smc.h): context, workspace carving and
// the launch sequence of each call.  Device kernels live in the included
// headers; this file only marshals arguments and orders launches.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <chrono>
#include <atomic>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "pf_kernels.cuh"
#include "resample_kernels.cuh"
#include "shard_kernels.cuh"
#include "gmm_kernels.cuh"
#include "batch_kernels.cuh"
#include "grad_kernels.cuh"
#include "weight_kernels.cuh"

using namespace smc;

struct smc_ctx;

namespace {

// Gaussian-mixture sampler (Sec. 5.2); defined after the context.
int gmm_move(smc_ctx *c);
int gmm_mcmc(smc_ctx *c);
int gmm_initialize(smc_ctx *c);
int gmm_on_data(smc_ctx *c);
int gmm_setup(smc_ctx *c);
void gmm_release(smc_ctx *c);
int gmm_launch_reweight(smc_ctx *c);
int gmm_launch_mcmc(smc_ctx *c);
int gmm_log_target_any(smc_ctx *c, const void *u, int64_t count, double alpha, void *logt, void *grad);
// a mixture shard: kernel kind 0 init, 1 reweight, 2 mcmc, its partial to d_partial; and the
// finalisation of a kind on every rank's partials
int gmm_shard_launch(smc_ctx *c, int kind, void *d_partial);
int gmm_shard_finalize_any(smc_ctx *c, const void *d_partials, int32_t world, int kind);

constexpr size_t kAlign = 256;

// float copy of observations / data for the FP32 kernels
__global__ void to_float_kernel(const double *src, float *dst, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}
constexpr int kMaxCoopGrid = 2048;  // blocks of a cooperative launch (B300: at most 148 x 8)
constexpr int kIterChunk = 8;       // iterations per graph launch of smc_iterate (n >= kIterChunk)

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

int ceil_log2(int64_t n) {
    int b = 0;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

struct Layout {
    size_t st, rec, part, x, lw, anc, Q, tsum, bsum, inc, obs, obs_f, alpha;
    size_t dhist, drec, dtot;  // multinomial / residual draw histogram, bucket records, tile totals
    size_t hist, ckpt, seg, gbar, xbar, at, rep, rep_part, scal, inpl, adapt, done, total;
    int ck;           // steps between checkpoints (record mode)
    int64_t nck;      // checkpoints
    int d;            // state rows
    int64_t ld;       // row pitch in elements (N rounded up to 64: 16-byte aligned rows)
    int64_t nbw;      // blocks of the weighting kernels
    int64_t nbw_move; // blocks of the particle filter's move kernel
    int32_t move_threads;  // active threads per block of that kernel
    int64_t ntiles;   // scan tiles of an N-element scan
    size_t rsize;
};

bool valid_config(const smc_config *c) {
    if (!c) return false;
    if (c->model != SMC_MODEL_CV && c->model != SMC_MODEL_CV_GAUSS && c->model != SMC_MODEL_GMM) return false;
    if (c->precision != 32 && c->precision != 64) return false;
    if (c->n_particles < 1 || c->n_particles > (int64_t(1) << 30)) return false;
    if (c->max_records < 2) return false;
    if (c->scheme < SMC_MULTINOMIAL || c->scheme > SMC_RESIDUAL_STRATIFIED) return false;
    if (!(c->threshold == c->threshold)) return false;
    if (c->max_data < 1) return false;
    if ((c->flags & SMC_FLAG_INPLACE) && (c->flags & SMC_FLAG_RECORD)) return false;  // the gradient needs sorted ancestors
    if (c->model == SMC_MODEL_GMM) {
        if (!kGmmEnabled) return false;
        if (c->gmm.n_comp < 1 || c->gmm.n_comp > kGmmMaxComp) return false;
        if (c->gmm.n_iter < 1 || c->gmm.shape0 < 1 || !(c->gmm.rate0 > 0) || !(c->gmm.sd0 > 0)) return false;
        if (c->gmm.move < SMC_GMM_RW || c->gmm.move > SMC_GMM_RW_MALA) return false;
        if (c->gmm.move != SMC_GMM_RW && !(c->gmm.mala_step > 0)) return false;
        if (c->gmm.schedule < SMC_ALPHA_LINEAR || c->gmm.schedule > SMC_ALPHA_ADAPTIVE) return false;
        if (c->gmm.schedule == SMC_ALPHA_ADAPTIVE && !(c->gmm.ess_target > 0.0 && c->gmm.ess_target < 1.0))
            return false;
        if (c->max_data > kGmmMaxData) return false;
    } else {
        if (!(c->cv.obs_scale > 0) || !(c->cv.obs_df > 0)) return false;
    }
    return true;
}

Layout make_layout(const smc_config *c) {
    Layout L{};
    const int64_t n = c->n_particles;
    const size_t rs = (c->precision == 32) ? 4 : 8;
    L.rsize = rs;
    L.d = (c->model == SMC_MODEL_GMM)
              ? 3 * c->gmm.n_comp + 2 + ((c->gmm.move != SMC_GMM_RW) ? 3 * c->gmm.n_comp - 1 : 0)
              : 4;
    L.ld = (n + 63) & ~int64_t(63);
    L.nbw = (n + kPfTile - 1) / kPfTile;
    // the double-precision particle filter's move kernel: one particle per
    // thread in tiles of 64 (N <= 2^16) or 256 threads, so that a small
    // filter's float64 work (Box-Muller, Student-t, exponentials) spreads over
    // many SMs instead of one SM's float64 units
    const bool pf64 = c->model != SMC_MODEL_GMM && c->precision == 64;
    L.move_threads = pf64 ? pf64_move_threads(n) : kBlock;
    L.nbw_move = pf64 ? (n + L.move_threads - 1) / L.move_threads : L.nbw;
    L.ntiles = (n + kScanTile - 1) / kScanTile;
    const bool hists = (c->scheme == SMC_MULTINOMIAL || c->scheme == SMC_RESIDUAL);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    L.st = take(sizeof(DevState));
    L.rec = take(sizeof(smc_record) * (size_t)c->max_records);
    const int64_t nblk = (c->model == SMC_MODEL_GMM) ? std::max<int64_t>(L.nbw, (kQuad * n + kBlock - 1) / kBlock)
                                                     : std::max<int64_t>(L.nbw, L.nbw_move);
    L.part = take(sizeof(Partial) * (size_t)std::max<int64_t>(nblk, 1));
    L.x = take(2 * (size_t)L.d * L.ld * rs);
    L.lw = take(2 * (size_t)L.ld * rs);
    L.anc = take((size_t)L.ld * 4);
    L.Q = take((size_t)n * 8);
    L.tsum = take((size_t)kScanSlots * L.ntiles * 8);
    L.bsum = take((size_t)3 * kMaxCoopGrid * 8);  // block sums of the cooperative kernels (three for residual)
    L.inc = take((size_t)L.ld * rs);            // staged increments of smc_add_log_weight
    const int64_t obs_vals = (c->model == SMC_MODEL_GMM) ? c->max_data : 2 * c->max_data;
    L.obs = take((size_t)obs_vals * 8);
    L.obs_f = take((size_t)obs_vals * 4);
    L.alpha = take((c->model == SMC_MODEL_GMM) ? ((size_t)c->gmm.n_iter + 1) * 8 : 0);
    L.dhist = take(hists ? (size_t)kHistWords * 4 : 0);
    L.drec = take(hists ? (size_t)kHistBuckets * 8 : 0);
    L.dtot = take(hists ? (size_t)kHistTiles * 4 : 0);
    const bool rec = (c->flags & SMC_FLAG_RECORD) && c->model != SMC_MODEL_GMM;
    L.ck = (c->checkpoint_every > 0) ? c->checkpoint_every : 16;
    L.nck = rec ? (c->max_data + L.ck - 1) / L.ck : 0;
    const size_t row = (size_t)L.ld * rs;
    L.hist = take(rec ? (size_t)c->max_data * L.ld * 4 : 0);
    L.ckpt = take((size_t)L.nck * 5 * row);
    L.seg = take(rec ? (size_t)L.ck * 5 * row : 0);
    L.gbar = take(rec ? 2 * (size_t)L.ld * 4 : 0);
    L.xbar = take(rec ? 4 * row : 0);
    L.at = take(rec ? 4 * row : 0);
    L.rep = take(rec ? 2 * 5 * row : 0);
    L.rep_part = take(rec ? sizeof(Partial) * (size_t)std::max<int64_t>(L.nbw, 1) : 0);
    L.scal = take(rec ? 256 : 0);
    L.inpl = take((c->flags & SMC_FLAG_INPLACE) ? 2 * (size_t)L.ld * 4 : 0);  // extras and survivor flags
    // adaptive tempering: two rounds of candidate partials per block
    L.adapt = take((c->model == SMC_MODEL_GMM && c->gmm.schedule == SMC_ALPHA_ADAPTIVE)
                       ? 2 * (size_t)kAdaptCand * kMaxCoopGrid * sizeof(AlphaPartial<double>)
                       : 0);
    L.done = take(sizeof(uint32_t));  // smc_iterate_host's sequence counter
    L.total = off;
    return L;
}

}  // namespace

struct smc_ctx {
    smc_config cfg;
    Layout L;
    char *ws;
    cudaStream_t stream;
    DevState *st;
    smc_record *rec;
    Partial *part;
    void *x[2];
    void *lw[2];
    int32_t *anc;
    unsigned long long *Q;
    unsigned long long *tsum;
    unsigned long long *bsum;  // block sums of the cooperative kernels (kMaxCoopGrid)
    uint32_t *sorted;
    uint32_t *dhist;  // multinomial draw histogram: byte counts (cleared by each use)
    uint2 *drec;
    uint32_t *dtot;
    double *obs;
    float *obs_f;
    double *alpha;
    int64_t n_obs;
    int32_t t_host;       // last iteration queued, -1 before initialize
    int initialized;
    int device;
    DevState host_st;     // last state read back
    cudaGraphExec_t graph;  // one captured iteration (move, resampling, mcmc)
    HostIO *hio;            // smc_iterate_host's staging: pinned, mapped (host address)
    HostIO *hio_d;          // the same buffer's device address
    cudaGraphExec_t graph_host;  // one iteration reading and writing the staging (smc_iterate_host)
    cudaGraphExec_t graph_chunk; // kIterChunk iterations in one graph (smc_iterate with n >= kIterChunk)
    int capture_host_io;    // while capturing graph_host: the kernels get the staging's addresses
    cudaEvent_t ev_move[2]; // profiling: recorded around the move kernel in the iteration graph
    int dependent_launch;   // while capturing: launch the one-pass resampler as a programmatic dependent
    int no_dependent;       // the CUDA driver refused the programmatic dependent launch once: capture without
    int chain_move;         // while capturing a later iteration of a chain: the move kernel is a
                            // programmatic dependent of the previous iteration's last kernel
    int no_chain;           // the CUDA driver refused that once: chains capture ordinary edges
    int64_t shard_n;        // a shard of a partitioned filter: the filter's N (0: not a shard)
    int64_t shard_off;      // and the global index of the shard's first particle
    void *shard_out;        // while launching a mixture shard's kernel: where its partial goes
    int shard_pending;      // the mixture shard's partial awaiting smc_shard_finalize: 0 init, 1 reweight
    uint32_t *done_seq = nullptr;  // smc_iterate_host's device counter (the workspace's last word)
    uint32_t done_want = 0;        // and the host's count of its launches
};

namespace {

int cuda_check(cudaError_t e) { return e == cudaSuccess ? SMC_OK : SMC_E_CUDA; }

uint2 key_of(const smc_ctx *c) { return make_uint2((uint32_t)(c->cfg.seed & 0xffffffffu), (uint32_t)(c->cfg.seed >> 32)); }

__global__ void reset_state_kernel(DevState *st) {
    st->t = -1;
    st->cur = 0;
    st->cur_lw = 0;
    st->base_shift = 0;
    st->gathered = 0;
    st->due = 0;
    st->ready = 0;
    st->error = 0;
    st->ticket = 0;
    st->max_lw = 0;
    st->log_norm = 0;
    st->max_lw_f = 0;
    st->log_norm_f[0] = st->log_norm_f[1] = 0;
    st->log_evidence = 0;
    st->ess = 0;
    st->alpha = 0;
    st->path_u = 0;
    st->path_log_z = 0;
    st->grid_count = 0;
    st->grid_depart = 0;
    for (int i = 0; i < 4; ++i) st->accept[i] = 0;
}

// Self-test of the bounded device waits: one block runs the grid barrier of
// the cooperative kernels for a grid of two blocks, so the second arrival
// never comes; the wait gives up after c_wait_limit polls and raises
// SMC_E_TIMEOUT.  The barrier counters are cleared afterwards (as the last
// departure of a real launch does).  Nothing else in the state changes.
__global__ void wait_selftest_kernel(DevState *st) {
    const bool ok = grid_barrier(st, 2u);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->grid_count = 0;
        st->grid_depart = 0;
        if (ok) raise_error(st, SMC_E_STATE);  // cannot happen: nothing else arrives
    }
}

// smc_iterate_host, last node of its graph: the call's sequence number
// (a device counter, advanced here) into the mapped staging, after every
// earlier kernel of the call has completed; the host waits on it instead of
// synchronising the stream
__global__ void host_done_kernel(HostIO *io, uint32_t *seq) {
    const uint32_t v = *seq + 1u;
    *seq = v;
    __threadfence_system();
    reinterpret_cast<volatile HostIO *>(io)->done = v;
}

// smc_iterate_host on a particle filter, first node of its graph: the
// observation of iteration t + 1 from the mapped staging into the workspace
// (and its float copy, rounded as on the host).  The move kernel, its
// programmatic dependent, starts at once and waits for this grid only
// before it reads y_t.
__global__ void host_obs_kernel(const HostIO *io, const DevState *st, double *obs, float *obs_f) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (threadIdx.x != 0 || st->error) return;
    const volatile HostIO *v = io;
    if (!v->has_obs) return;
    const int64_t t = (int64_t)st->t + 1;
    const double x = v->obs[0], y = v->obs[1];
    obs[2 * t] = x;
    obs[2 * t + 1] = y;
    obs_f[2 * t] = __double2float_rn(x);
    obs_f[2 * t + 1] = __double2float_rn(y);
}

// smc_iterate_host on a GMM sampler, last node of its graph: the record of
// iteration t and the device error word into the mapped staging (one warp;
// the particle filters' move kernel writes them itself)
__global__ void host_rec_kernel(HostIO *io, const DevState *st, const smc_record *rec, int32_t max_records) {
    const int32_t t = st->t;
    static_assert(sizeof(smc_record) % 4 == 0, "record words");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(rec + (t >= 0 ? t % max_records : 0));
    volatile uint32_t *dst = reinterpret_cast<volatile uint32_t *>(&io->rec);
    for (int i = threadIdx.x; i < (int)(sizeof(smc_record) / 4); i += 32) dst[i] = src[i];
    if (threadIdx.x == 0) io->status = st->error;
}

// the resampling threshold for the FP32 finalize: a DF value and a mode
// (always at >= 1, never at <= 0, otherwise compare ESS < threshold N)
template <class A>
void set_threshold_df(A &a, double thr) {
    a.thr_mode = thr >= 1.0 ? 1 : (thr <= 0.0 ? 2 : 0);
    a.thr_df[0] = (float)thr;
    a.thr_df[1] = (float)(thr - (double)a.thr_df[0]);
}

// observation-density constants of the constant-velocity model
template <typename R>
void set_obs_params(PfArgs<R> &a, double s, double nu, bool gaussian) {
    a.inv_scale = R(1.0 / s);
    a.inv_nu = R(1.0 / nu);
    a.half_nu1 = R(0.5 * (nu + 1.0));
    a.gaussian = gaussian ? 1 : 0;
    double cst;
    if (gaussian) cst = -0.5 * std::log(2.0 * M_PI) - std::log(s);
    else cst = std::lgamma(0.5 * (nu + 1.0)) - std::lgamma(0.5 * nu) - 0.5 * std::log(nu * M_PI) - std::log(s);
    a.ll_const = R(2.0 * cst);
}

template <typename R>
PfArgs<R> pf_args(smc_ctx *c) {
    PfArgs<R> a;
    const smc_config &g = c->cfg;
    const int64_t n = g.n_particles;
    a.n = n;
    for (int b = 0; b < 2; ++b) {
        R *base = static_cast<R *>(c->x[b]);
        for (int r = 0; r < 4; ++r) a.x[b][r] = base + (size_t)r * c->L.ld;
        a.lw[b] = static_cast<R *>(c->lw[b]);
    }
    a.anc = c->anc;
    a.obs = c->obs;
    a.obs_r = (sizeof(R) == 4) ? reinterpret_cast<const R *>(c->obs_f) : reinterpret_cast<const R *>(c->obs);
    a.neg_log_n = R(-std::log((double)n));
    a.rec = c->rec;
    a.rec_cap = g.max_records;
    a.st = c->st;
    a.part = c->part;
    a.log_n = std::log((double)n);
    a.threshold = g.threshold;
    set_threshold_df(a, g.threshold);
    a.delta = R(g.cv.delta);
    a.sd_pos = R(g.cv.sd_pos);
    a.sd_vel = R(g.cv.sd_vel);
    a.sd_pos0 = R(g.cv.sd_pos0);
    a.sd_vel0 = R(g.cv.sd_vel0);
    set_obs_params(a, g.cv.obs_scale, g.cv.obs_df, g.model == SMC_MODEL_CV_GAUSS);
    a.key = key_of(c);
    a.stream = g.stream_id;
    a.index0 = (uint32_t)c->shard_off;
    if (c->shard_n) {  // equal weights after resampling are 1 / N of the whole filter
        a.neg_log_n = R(-std::log((double)c->shard_n));
        a.log_n = std::log((double)c->shard_n);
    }
    a.obs_after_wait = 0;
    a.hio_out = c->capture_host_io ? c->hio_d : nullptr;
    a.obs_cap = (int32_t)c->cfg.max_data;
    a.tile_threads = (uint32_t)c->L.move_threads;
    return a;
}

template <typename R>
int launch_pf(smc_ctx *c) {
    PfArgs<R> a = pf_args<R>(c);
    if (c->chain_move) {
        // a later iteration of a captured chain: its blocks launch while the
        // previous iteration's last kernel completes and wait for it first
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)c->L.nbw_move);
        lc.blockDim = dim3(kBlock);
        lc.stream = c->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        return cuda_check(cudaLaunchKernelEx(&lc, pf_iterate_kernel<R, true>, a));
    }
    if (c->capture_host_io && c->dependent_launch) {
        // smc_iterate_host's graph: a programmatic dependent of host_obs_kernel
        a.obs_after_wait = 1;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)c->L.nbw_move);
        lc.blockDim = dim3(kBlock);
        lc.stream = c->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        return cuda_check(cudaLaunchKernelEx(&lc, pf_iterate_kernel<R>, a));
    }
    pf_iterate_kernel<R><<<(unsigned)c->L.nbw_move, kBlock, 0, c->stream>>>(a);
    return cuda_check(cudaGetLastError());
}

// SMC_FLAG_POST_MEAN (particle filters): the post-resampling mean of the
// iteration just resampled, into its record
int launch_post_mean(smc_ctx *c) {
    if (!(c->cfg.flags & SMC_FLAG_POST_MEAN) || c->cfg.model == SMC_MODEL_GMM) return SMC_OK;
    if (c->cfg.precision == 32)
        post_mean_kernel<float><<<(unsigned)c->L.nbw, kBlock, 0, c->stream>>>(pf_args<float>(c));
    else
        post_mean_kernel<double><<<(unsigned)c->L.nbw, kBlock, 0, c->stream>>>(pf_args<double>(c));
    return cuda_check(cudaGetLastError());
}

unsigned long long *tsum_of(smc_ctx *c, int slot) { return c->tsum + (size_t)slot * c->L.ntiles; }

// SMC_FLAG_INPLACE: the step's sorted ancestors rearranged in place
// (inplace_kernel), one cooperative wave after each resampling step
int launch_inplace(smc_ctx *c);

// The ancestor output of the resampling kernels (and, while graph_host is
// captured, the staging's error word for their failures).
AncOut anc_out(smc_ctx *c) {
    AncOut o{c->anc};
    o.host_err = c->capture_host_io ? &c->hio_d->status : nullptr;
    return o;
}

// Resident blocks of a cooperative kernel on the current device (cached per
// kernel by the caller's arrays, indexed by device).
int coop_capacity(const void *kern, int (&per_sm)[64], int (&sms)[64], int *slots) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SMC_E_CUDA;
    if (!per_sm[dev]) {
        int b = 0, m = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kBlock, 0) != cudaSuccess || b < 1)
            return SMC_E_CUDA;
        if (cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || m < 1)
            return SMC_E_CUDA;
        sms[dev] = m;
        per_sm[dev] = b;
    }
    *slots = per_sm[dev] * sms[dev];
    return SMC_OK;
}

// Cooperative launch on the context's stream; while capturing the iteration
// graph, also a programmatic dependent of the move kernel: the blocks become
// resident while the move kernel's last block combines the partials and wait
// (griddepcontrol.wait) for its completion.
template <class... KArgs, class... Args>
int launch_coop(smc_ctx *c, int grid, void (*kern)(KArgs...), Args... args) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(kBlock);
    lc.dynamicSmemBytes = 0;
    lc.stream = c->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = c->dependent_launch ? 2 : 1;
    return cuda_check(cudaLaunchKernelEx(&lc, kern, args...));
}

// One-pass systematic / stratified resampling (grid_resample_kernel): at
// most one block per scan tile.
template <typename R, bool kS, class Sink>
int launch_grid_resample(smc_ctx *c, const QGen<R> &qg, Sink sk, int gate) {
    const int64_t n = c->cfg.n_particles;
    const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
    auto kern = grid_resample_kernel<QGen<R>, kS, Sink>;
    static int per_sm[64] = {}, sms[64] = {};  // this instantiation
    int slots = 0;
    if (int rc = coop_capacity(reinterpret_cast<const void *>(kern), per_sm, sms, &slots)) return rc;
    const int grid = std::max(1, std::min({ntiles, slots, kMaxCoopGrid}));
    GridTargets<kS> tg{};
    tg.n = n;
    tg.key = key_of(c);
    tg.stream = c->cfg.stream_id;
    tg.mrec = ~0ull / (unsigned long long)n;
    return launch_coop(c, grid, kern, qg, tg, anc_out(c), sk, n, tsum_of(c, SLOT_CDF), c->bsum, c->st, gate);
}

// One-pass multinomial resampling (grid_multinomial_kernel): one full wave
// (blocks without a weight tile still count draws and scan the histogram).
// The value thresholds v(X) = ceil(X 2^24 / Q_N - 1/2) are the systematic
// closed form with n = 2^24 and c = 2^24.
template <typename R, class Sink>
int launch_grid_multinomial(smc_ctx *c, const QGen<R> &qg, Sink sk, int gate) {
    const int64_t n = c->cfg.n_particles;
    auto kern = grid_multinomial_kernel<R, Sink>;
    static int per_sm[64] = {}, sms[64] = {};
    int slots = 0;
    if (int rc = coop_capacity(reinterpret_cast<const void *>(kern), per_sm, sms, &slots)) return rc;
    const int grid = std::max(1, std::min(slots, kMaxCoopGrid));
    GridTargets<false> tg{};
    tg.n = int64_t(1) << kHistValueBits;
    tg.key = key_of(c);
    tg.stream = c->cfg.stream_id;
    tg.c_fixed = 1ull << kHistValueBits;
    tg.mrec = ~0ull >> kHistValueBits;  // floor((2^64 - 1) / 2^24)
    HistArgs h;
    h.hist = c->dhist;
    h.hrec = c->drec;
    h.htot = c->dtot;
    return launch_coop(c, grid, kern, qg, tg, anc_out(c), sk, n, tsum_of(c, SLOT_CDF), c->bsum, h, c->st, gate);
}

// One-pass residual resampling (grid_residual_kernel): one full wave; the
// q, d and r tile sums in three scan slots, the block sums in three rows.
// kMode: the residual step (multinomial draws through the histogram, or the
// systematic / stratified closed form over the R residual outputs).
template <typename R, class Sink, int kMode = kResMultinomial>
int launch_grid_residual(smc_ctx *c, const QGen<R> &qg, Sink sk, int gate) {
    const int64_t n = c->cfg.n_particles;
    auto kern = grid_residual_kernel<R, Sink, kMode>;
    static int per_sm[64] = {}, sms[64] = {};
    int slots = 0;
    if (int rc = coop_capacity(reinterpret_cast<const void *>(kern), per_sm, sms, &slots)) return rc;
    const int grid = std::max(1, std::min(slots, kMaxCoopGrid));
    ResidualTargets<kMode> tg{};
    tg.key = key_of(c);
    tg.stream = c->cfg.stream_id;
    if (kMode == kResMultinomial) {
        tg.n = int64_t(1) << kHistValueBits;
        tg.c_fixed = 1ull << kHistValueBits;
        tg.mrec = ~0ull >> kHistValueBits;
    } else {
        tg.n = n;  // replaced by R on the device
        tg.c_fixed = 0;
        tg.mrec = ~0ull / (unsigned long long)n;
    }
    HistArgs h;
    h.hist = c->dhist;
    h.hrec = c->drec;
    h.htot = c->dtot;
    ResidualSums rs;
    rs.tq = tsum_of(c, SLOT_CDF);
    rs.td = tsum_of(c, SLOT_RES_D);
    rs.tr = tsum_of(c, SLOT_RES_R);
    rs.bq = c->bsum;
    rs.bd = c->bsum + kMaxCoopGrid;
    rs.br = c->bsum + 2 * kMaxCoopGrid;
    return launch_coop(c, grid, kern, qg, tg, anc_out(c), sk, n, rs, h, c->st, gate);
}

// q_i = floor(exp(lw_i - M) 2^F) over the context's log-weight buffers
template <typename R>
QGen<R> qgen_of(const smc_ctx *c) {
    QGen<R> qg;
    qg.lw[0] = static_cast<const R *>(c->lw[0]);
    qg.lw[1] = static_cast<const R *>(c->lw[1]);
    qg.frac = 61 - ceil_log2(c->cfg.n_particles);
    qg.cur_lw = nullptr;
    qg.m = 0;
    return qg;
}

// the global outputs of a shard's particles (smc_shard_select)
template <typename R, bool kS>
int shard_select_t(smc_ctx *c, const uint64_t *d_totals, int32_t rank, int32_t world, int32_t *d_src,
                   int64_t *d_range) {
    const int64_t n = c->cfg.n_particles;
    const unsigned tiles = (unsigned)((n + kScanTile - 1) / kScanTile);
    QGen<R> qg = qgen_of<R>(c);
    qg.frac = 61 - ceil_log2(c->shard_n);
    GridTargets<kS> tg{};
    tg.n = c->shard_n;
    tg.key = key_of(c);
    tg.stream = c->cfg.stream_id;
    tg.mrec = ~0ull / (unsigned long long)c->shard_n;
    shard_select_kernel<R, kS><<<tiles, kBlock, 0, c->stream>>>(
        qg, tg, n, tsum_of(c, SLOT_CDF), reinterpret_cast<const unsigned long long *>(d_totals), rank, world, d_src,
        d_range, c->st);
    return cuda_check(cudaGetLastError());
}

int launch_inplace(smc_ctx *c) {
    if (!(c->cfg.flags & SMC_FLAG_INPLACE)) return SMC_OK;
    const int64_t n = c->cfg.n_particles;
    const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
    static int per_sm[64] = {}, sms[64] = {};
    int slots = 0;
    if (int rc = coop_capacity(reinterpret_cast<const void *>(inplace_kernel), per_sm, sms, &slots)) return rc;
    const int grid = std::max(1, std::min({ntiles, slots, kMaxCoopGrid}));
    InplaceArgs ia;
    ia.anc = c->anc;
    ia.extra = reinterpret_cast<int32_t *>(c->ws + c->L.inpl);
    ia.surv = ia.extra + c->L.ld;
    ia.tf = tsum_of(c, 4);
    ia.ts = tsum_of(c, 5);
    ia.bf = c->bsum;
    ia.bs = c->bsum + kMaxCoopGrid;
    const int dep = c->dependent_launch;
    c->dependent_launch = 0;  // an ordinary node after the resampler
    const int rc = launch_coop(c, grid, inplace_kernel, ia, n, c->st);
    c->dependent_launch = dep;
    return rc;
}

template <typename R>
int launch_resample(smc_ctx *c, int gate) {
    const int64_t n = c->cfg.n_particles;
    const bool keep = (c->cfg.flags & SMC_FLAG_KEEP_CDF) != 0;
    QGen<R> qg;
    qg.lw[0] = static_cast<const R *>(c->lw[0]);
    qg.lw[1] = static_cast<const R *>(c->lw[1]);
    qg.frac = 61 - ceil_log2(n);
    qg.cur_lw = nullptr;
    qg.m = 0;
    const StoreSink qsink{keep ? c->Q : nullptr};
    switch (c->cfg.scheme) {  // one cooperative pass each
        case SMC_SYSTEMATIC:
            return keep ? launch_grid_resample<R, false>(c, qg, qsink, gate)
                        : launch_grid_resample<R, false>(c, qg, NoSink{}, gate);
        case SMC_STRATIFIED:
            return keep ? launch_grid_resample<R, true>(c, qg, qsink, gate)
                        : launch_grid_resample<R, true>(c, qg, NoSink{}, gate);
        case SMC_MULTINOMIAL:
            return keep ? launch_grid_multinomial<R>(c, qg, qsink, gate)
                        : launch_grid_multinomial<R>(c, qg, NoSink{}, gate);
        case SMC_RESIDUAL:
            return keep ? launch_grid_residual<R>(c, qg, qsink, gate) : launch_grid_residual<R>(c, qg, NoSink{}, gate);
        case SMC_RESIDUAL_SYSTEMATIC:
            return keep ? launch_grid_residual<R, StoreSink, kResSystematic>(c, qg, qsink, gate)
                        : launch_grid_residual<R, NoSink, kResSystematic>(c, qg, NoSink{}, gate);
        case SMC_RESIDUAL_STRATIFIED:
            return keep ? launch_grid_residual<R, StoreSink, kResStratified>(c, qg, qsink, gate)
                        : launch_grid_residual<R, NoSink, kResStratified>(c, qg, NoSink{}, gate);
        default:
            break;
    }
    return SMC_E_ARG;
}

int resample_any(smc_ctx *c, int gate) {
    return (c->cfg.precision == 32) ? launch_resample<float>(c, gate) : launch_resample<double>(c, gate);
}

// lw += (staged increments in c->inc), normaliser and decision again
template <typename R>
int launch_add_log_weight(smc_ctx *c) {
    AddArgs<R> a{};
    a.n = c->cfg.n_particles;
    const bool gmm = c->cfg.model == SMC_MODEL_GMM;
    for (int b = 0; b < 2; ++b) {
        a.lw[b] = static_cast<const R *>(c->lw[b]);
        a.lw_w[b] = static_cast<R *>(c->lw[b]);
        const R *base = static_cast<const R *>(c->x[b]);
        a.h[b][0] = gmm ? nullptr : base;
        a.h[b][1] = gmm ? nullptr : base + c->L.ld;
    }
    a.incw = reinterpret_cast<const R *>(c->ws + c->L.inc);
    a.rec = c->rec;
    a.rec_cap = c->cfg.max_records;
    a.st = c->st;
    a.part = c->part;
    a.threshold = c->cfg.threshold;
    set_threshold_df(a, c->cfg.threshold);
    a.gmm = gmm ? 1 : 0;
    add_log_weight_kernel<R><<<(unsigned)c->L.nbw, kBlock, 0, c->stream>>>(a);
    return cuda_check(cudaGetLastError());
}

int add_log_weight_any(smc_ctx *c) {
    return (c->cfg.precision == 32) ? launch_add_log_weight<float>(c) : launch_add_log_weight<double>(c);
}

int read_state(smc_ctx *c) {
    cudaError_t e = cudaMemcpyAsync(&c->host_st, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return SMC_E_CUDA;
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return SMC_E_CUDA;
    return c->host_st.error;
}

// ---- recording for the gradient (SMC_FLAG_RECORD, CV models) ----
bool recording(const smc_ctx *c) { return (c->cfg.flags & SMC_FLAG_RECORD) && c->cfg.model != SMC_MODEL_GMM; }

size_t row_bytes(const smc_ctx *c) { return (size_t)c->L.ld * c->L.rsize; }

char *ckpt_slot(smc_ctx *c, int64_t k) { return c->ws + c->L.ckpt + (size_t)k * 5 * row_bytes(c); }

// after the move of iteration t_host: state checkpoint every ck iterations
// (the PF kernels flip both buffers each iteration: after iteration t the
// current buffers have parity (t + 1) & 1)
int record_after_move(smc_ctx *c) {
    if (!recording(c)) return SMC_OK;
    const int32_t t = c->t_host;
    if (t % c->L.ck) return SMC_OK;
    const int par = (t + 1) & 1;
    char *dst = ckpt_slot(c, t / c->L.ck);
    int rc = cuda_check(cudaMemcpyAsync(dst, c->x[par], 4 * row_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
    if (!rc)
        rc = cuda_check(
            cudaMemcpyAsync(dst + 4 * row_bytes(c), c->lw[par], row_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
    return rc;
}

// after the resampling step of iteration t_host: keep its ancestors
int record_after_resample(smc_ctx *c) {
    if (!recording(c)) return SMC_OK;
    int32_t *dst = reinterpret_cast<int32_t *>(c->ws + c->L.hist) + (size_t)c->t_host * c->L.ld;
    return cuda_check(cudaMemcpyAsync(dst, c->anc, (size_t)c->cfg.n_particles * 4, cudaMemcpyDeviceToDevice,
                                      c->stream));
}

int move_any(smc_ctx *c) {
    if (!c->initialized || c->shard_n) return SMC_E_STATE;
    if (c->cfg.model == SMC_MODEL_GMM) return gmm_move(c);
    if (c->t_host + 1 >= c->n_obs) return SMC_E_ARG;
    const int rc = (c->cfg.precision == 32) ? launch_pf<float>(c) : launch_pf<double>(c);
    if (rc != SMC_OK) return rc;
    c->t_host += 1;
    return record_after_move(c);
}

// The kernels of one iteration, without host bookkeeping (capturable).
int launch_iteration(smc_ctx *c) {
    int rc;
    if (c->cfg.model == SMC_MODEL_GMM) {
        rc = gmm_launch_reweight(c);
        if (!rc) rc = resample_any(c, 1);
        if (!rc) rc = launch_inplace(c);
        if (!rc) rc = gmm_launch_mcmc(c);
    } else {
        // external event records: captured as event-record nodes of the graph
        // (a plain record during capture only orders the captured work)
        if (c->ev_move[0] &&
            (rc = cuda_check(cudaEventRecordWithFlags(c->ev_move[0], c->stream, cudaEventRecordExternal))))
            return rc;
        rc = (c->cfg.precision == 32) ? launch_pf<float>(c) : launch_pf<double>(c);
        if (!rc && c->ev_move[1])
            rc = cuda_check(cudaEventRecordWithFlags(c->ev_move[1], c->stream, cudaEventRecordExternal));
        if (!rc) rc = resample_any(c, 1);
        if (!rc) rc = launch_inplace(c);
        if (!rc) rc = launch_post_mean(c);
    }
    return rc;
}

// one iteration; host_io: smc_iterate_host's, which reads the observation
// from the mapped staging (a one-warp first kernel, overlapped with the move)
// and writes the record and error word back there (the particle filters'
// kernels themselves; a GMM sampler through a last one-warp kernel)
int launch_iteration_io(smc_ctx *c, bool host_io) {
    if (!host_io) return launch_iteration(c);
    if (c->cfg.model == SMC_MODEL_GMM) {
        if (int rc = launch_iteration(c)) return rc;
        host_rec_kernel<<<1, 32, 0, c->stream>>>(c->hio_d, c->st, c->rec, c->cfg.max_records);
    } else {
        host_obs_kernel<<<1, 32, 0, c->stream>>>(c->hio_d, c->st, c->obs, c->obs_f);
        if (int rc = cuda_check(cudaGetLastError())) return rc;
        c->capture_host_io = 1;
        const int rc = launch_iteration(c);
        c->capture_host_io = 0;
        if (rc) return rc;
    }
    if (int rc = cuda_check(cudaGetLastError())) return rc;
    host_done_kernel<<<1, 1, 0, c->stream>>>(c->hio_d, c->done_seq);
    return cuda_check(cudaGetLastError());
}

void drop_graphs(smc_ctx *c) {
    for (cudaGraphExec_t *g : {&c->graph, &c->graph_host, &c->graph_chunk})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
}

// iterations: how many consecutive iterations the graph holds (host_io: 1)
// chain: the move kernels after the first as programmatic dependents (PF)
int build_graph_once(smc_ctx *c, cudaGraphExec_t *dst, bool host_io, int iterations = 1, bool chain = false) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SMC_E_CUDA;
    int rc = SMC_OK;
    for (int i = 0; i < iterations && !rc; ++i) {
        c->chain_move = (i > 0 && chain) ? 1 : 0;
        rc = launch_iteration_io(c, host_io);
    }
    c->chain_move = 0;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : SMC_E_CUDA;
    }
    const cudaError_t e2 = cudaGraphInstantiate(dst, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return SMC_E_CUDA;
    }
    return SMC_OK;
}

// One iteration captured as a graph (host_io: the graph of smc_iterate_host).
// The one-pass resampler is captured as a programmatic dependent of the move
// kernel where the CUDA driver accepts that for a cooperative launch; otherwise
// (one refusal) as an ordinary node.
int build_graph(smc_ctx *c, bool host_io = false) {
    cudaGraphExec_t *dst = host_io ? &c->graph_host : &c->graph;
    if (*dst) return SMC_OK;
    if (!c->no_dependent && !c->ev_move[1]) {
        c->dependent_launch = 1;
        const int rc = build_graph_once(c, dst, host_io);
        c->dependent_launch = 0;
        if (rc == SMC_OK) return SMC_OK;
        c->no_dependent = 1;
    }
    return build_graph_once(c, dst, host_io);
}

// kIterChunk iterations in one graph, with the launch form the one-iteration
// graph settled on (build_graph first)
int build_graph_chunk(smc_ctx *c) {
    if (c->graph_chunk) return SMC_OK;
    if (int rc = build_graph(c)) return rc;
    c->dependent_launch = (!c->no_dependent && !c->ev_move[1]) ? 1 : 0;
    // the particle filters' move kernels after the first wait for the
    // previous iteration as programmatic dependents (no event node between)
    const bool chain = c->dependent_launch && !c->no_chain && c->cfg.model != SMC_MODEL_GMM && !c->ev_move[0];
    int rc = build_graph_once(c, &c->graph_chunk, false, kIterChunk, chain);
    if (rc != SMC_OK && chain) {  // refused once: ordinary edges from now on
        c->no_chain = 1;
        rc = build_graph_once(c, &c->graph_chunk, false, kIterChunk);
    }
    c->dependent_launch = 0;
    return rc;
}

int mcmc_any(smc_ctx *c) {
    if (!c->initialized) return SMC_E_STATE;
    if (c->cfg.model == SMC_MODEL_GMM) return gmm_mcmc(c);
    return SMC_OK;
}

}  // namespace

// ------------------------------------------------------------------ ABI --

extern "C" {

size_t smc_workspace_bytes(const smc_config *cfg) {
    if (!valid_config(cfg)) return 0;
    return make_layout(cfg).total;
}

int smc_create(smc_ctx **out, const smc_config *cfg, void *d_workspace, size_t bytes, void *cuda_stream) {
    if (!out) return SMC_E_ARG;
    *out = nullptr;
    if (!valid_config(cfg)) return SMC_E_ARG;
    const Layout L = make_layout(cfg);
    if (!d_workspace || bytes < L.total || ((uintptr_t)d_workspace & (kAlign - 1))) return SMC_E_WORKSPACE;
    smc_ctx *c = new (std::nothrow) smc_ctx();
    if (!c) return SMC_E_ARG;
    c->cfg = *cfg;
    c->L = L;
    c->ws = static_cast<char *>(d_workspace);
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->st = reinterpret_cast<DevState *>(c->ws + L.st);
    c->rec = reinterpret_cast<smc_record *>(c->ws + L.rec);
    c->part = reinterpret_cast<Partial *>(c->ws + L.part);
    const size_t half_x = (size_t)L.d * L.ld * L.rsize;
    c->x[0] = c->ws + L.x;
    c->x[1] = c->ws + L.x + half_x;
    c->lw[0] = c->ws + L.lw;
    c->lw[1] = c->ws + L.lw + (size_t)L.ld * L.rsize;
    c->anc = reinterpret_cast<int32_t *>(c->ws + L.anc);
    c->Q = reinterpret_cast<unsigned long long *>(c->ws + L.Q);
    c->tsum = reinterpret_cast<unsigned long long *>(c->ws + L.tsum);
    c->bsum = reinterpret_cast<unsigned long long *>(c->ws + L.bsum);
    c->dhist = reinterpret_cast<uint32_t *>(c->ws + L.dhist);
    c->drec = reinterpret_cast<uint2 *>(c->ws + L.drec);
    c->dtot = reinterpret_cast<uint32_t *>(c->ws + L.dtot);
    c->obs = reinterpret_cast<double *>(c->ws + L.obs);
    c->obs_f = reinterpret_cast<float *>(c->ws + L.obs_f);
    c->alpha = reinterpret_cast<double *>(c->ws + L.alpha);
    c->done_seq = reinterpret_cast<uint32_t *>(c->ws + L.done);
    c->n_obs = 0;
    c->t_host = -1;
    c->initialized = 0;
    c->graph = nullptr;
    c->graph_host = nullptr;
    c->graph_chunk = nullptr;
    c->capture_host_io = 0;
    c->hio = nullptr;
    c->hio_d = nullptr;
    cudaGetDevice(&c->device);
    // zero the state block, records, scan status words and block sums
    int rc = cuda_check(cudaMemsetAsync(c->ws, 0, L.part, c->stream));
    if (!rc) rc = cuda_check(cudaMemsetAsync(c->ws + L.tsum, 0, L.inc - L.tsum, c->stream));
    if (!rc) rc = cuda_check(cudaMemsetAsync(c->done_seq, 0, sizeof(uint32_t), c->stream));
    if (!rc) {
        reset_state_kernel<<<1, 1, 0, c->stream>>>(c->st);
        rc = cuda_check(cudaGetLastError());
    }
    if (!rc && cfg->model == SMC_MODEL_GMM) rc = gmm_setup(c);
    // smc_iterate_host's staging: pinned and mapped into the device's address space
    if (!rc) rc = cuda_check(cudaHostAlloc(reinterpret_cast<void **>(&c->hio), sizeof(HostIO), cudaHostAllocMapped));
    if (!rc) rc = cuda_check(cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->hio_d), c->hio, 0));
    if (rc) {
        if (c->hio) cudaFreeHost(c->hio);
        delete c;
        return rc;
    }
    std::memset(c->hio, 0, sizeof(HostIO));
    *out = c;
    return SMC_OK;
}

int smc_destroy(smc_ctx *c) {
    if (!c) return SMC_E_ARG;
    drop_graphs(c);
    if (c->hio) cudaFreeHost(c->hio);
    gmm_release(c);
    delete c;
    return SMC_OK;
}

int smc_set_data(smc_ctx *c, const double *obs, int64_t count, int on_device) {
    if (!c || !obs || count < 1 || count > c->cfg.max_data) return SMC_E_ARG;
    const int64_t vals = (c->cfg.model == SMC_MODEL_GMM) ? count : 2 * count;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int rc = cuda_check(cudaMemcpyAsync(c->obs, obs, (size_t)vals * 8, k, c->stream));
    if (rc) return rc;
    if (!on_device) rc = cuda_check(cudaStreamSynchronize(c->stream));  // the host buffer may go away
    if (rc) return rc;
    c->n_obs = count;
    return gmm_on_data(c);
}

int smc_initialize(smc_ctx *c) {
    if (!c) return SMC_E_ARG;
    if (c->n_obs < 1) return SMC_E_STATE;
    reset_state_kernel<<<1, 1, 0, c->stream>>>(c->st);
    int rc = cuda_check(cudaGetLastError());
    if (rc) return rc;
    c->initialized = 1;
    c->t_host = -1;
    if (c->shard_n) return SMC_OK;  // a shard's first step (t = 0) is smc_shard_move and the rest of the exchange
    if (c->cfg.model == SMC_MODEL_GMM) {
        rc = gmm_initialize(c);
    } else {
        rc = (c->cfg.precision == 32) ? launch_pf<float>(c) : launch_pf<double>(c);
        if (!rc) c->t_host = 0;
        if (!rc) rc = record_after_move(c);
    }
    if (rc) return rc;
    rc = resample_any(c, 1);
    if (!rc) rc = launch_inplace(c);
    if (!rc) rc = launch_post_mean(c);
    if (!rc) rc = record_after_resample(c);
    return rc;
}

int smc_move(smc_ctx *c) {
    if (!c) return SMC_E_ARG;
    return move_any(c);
}

int smc_resample(smc_ctx *c, int force) {
    if (!c) return SMC_E_ARG;
    if (!c->initialized || c->shard_n) return SMC_E_STATE;
    int rc = resample_any(c, force ? 0 : 1);
    if (!rc) rc = launch_inplace(c);
    if (!rc) rc = launch_post_mean(c);
    return rc ? rc : record_after_resample(c);
}

int smc_mcmc(smc_ctx *c) {
    if (!c) return SMC_E_ARG;
    return mcmc_any(c);
}

int smc_iterate(smc_ctx *c, int32_t n) {
    if (!c || n < 0) return SMC_E_ARG;
    if (!c->initialized || c->shard_n) return SMC_E_STATE;
    // graph replay: every kernel reads the iteration index from the device
    // state, so one captured iteration serves every t (host bookkeeping and
    // the recording copies are not captured)
    const int64_t limit = (c->cfg.model == SMC_MODEL_GMM) ? c->cfg.gmm.n_iter : c->n_obs - 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (c->stream != nullptr && cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess) return SMC_E_CUDA;
    if (cs != cudaStreamCaptureStatusNone) {
        // the caller is capturing the context's stream: the n iterations'
        // kernels go into the caller's graph (particle filters; the launch
        // form of the context's own iteration graph, which must exist)
        if (cs != cudaStreamCaptureStatusActive || c->cfg.model == SMC_MODEL_GMM || recording(c) || !c->graph)
            return SMC_E_STATE;
        if (c->t_host + (int64_t)n > limit) return SMC_E_ARG;
        c->dependent_launch = (!c->no_dependent && !c->ev_move[1]) ? 1 : 0;
        int rc = SMC_OK;
        for (int32_t i = 0; i < n && !rc; ++i) rc = launch_iteration(c);
        c->dependent_launch = 0;
        if (rc) return rc;
        c->t_host += n;
        return SMC_OK;
    }
    if (c->stream != nullptr && !recording(c) && n > 0) {
        if (c->t_host + (int64_t)n > limit) return SMC_E_ARG;
        int rc = build_graph(c);
        if (rc) return rc;
        int32_t i = 0;
        if (n >= kIterChunk) {  // whole chunks of iterations per graph launch
            if ((rc = build_graph_chunk(c))) return rc;
            for (; i + kIterChunk <= n; i += kIterChunk)
                if (cudaGraphLaunch(c->graph_chunk, c->stream) != cudaSuccess) return SMC_E_CUDA;
        }
        for (; i < n; ++i)
            if (cudaGraphLaunch(c->graph, c->stream) != cudaSuccess) return SMC_E_CUDA;
        c->t_host += n;
        return SMC_OK;
    }
    for (int32_t i = 0; i < n; ++i) {
        int rc = move_any(c);
        if (!rc) rc = resample_any(c, 1);
        if (!rc) rc = launch_inplace(c);
        if (!rc) rc = launch_post_mean(c);
        if (!rc) rc = record_after_resample(c);
        if (!rc) rc = mcmc_any(c);
        if (rc) return rc;
    }
    return SMC_OK;
}

int smc_iterate_host(smc_ctx *c, const double *h_obs_t, smc_record *h_record) {
    if (!c || !h_record) return SMC_E_ARG;
    if (!c->initialized || c->shard_n) return SMC_E_STATE;
    const int32_t t = c->t_host + 1;
    const bool with_obs = h_obs_t && c->cfg.model != SMC_MODEL_GMM;
    if (with_obs && t >= c->cfg.max_data) return SMC_E_ARG;
    const int64_t limit = (c->cfg.model == SMC_MODEL_GMM)
                              ? c->cfg.gmm.n_iter
                              : std::max<int64_t>(c->n_obs, with_obs ? t + 1 : 0) - 1;
    if (t > limit) return SMC_E_ARG;
    int rc;
    if (c->stream != nullptr && !recording(c)) {
        // one graph launch: the observation goes in and the record comes out
        // through the mapped staging, read and written by the graph's kernels
        if ((rc = build_graph(c, true))) return rc;
        c->hio->status = SMC_OK;
        c->hio->has_obs = with_obs ? 1 : 0;
        if (with_obs) {
            c->hio->obs[0] = h_obs_t[0];
            c->hio->obs[1] = h_obs_t[1];
        }
        if (cudaGraphLaunch(c->graph_host, c->stream) != cudaSuccess) return SMC_E_CUDA;
        // the graph's last kernel writes the call's sequence number once the
        // record and the error word are in the staging: wait for it (a
        // second bounded by the clock, then a synchronise, which also
        // surfaces a fault)
        const uint32_t want = ++c->done_want;
        const volatile uint32_t *done = &c->hio->done;
        const auto t0 = std::chrono::steady_clock::now();
        for (uint32_t spin = 1; *done != want; ++spin)
            if (!(spin & 0xFFFFu) && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(1)) break;
        if (*done != want && (rc = cuda_check(cudaStreamSynchronize(c->stream)))) return rc;
        if (with_obs && c->n_obs < t + 1) c->n_obs = t + 1;
        c->t_host = t;
        std::memcpy(h_record, &c->hio->rec, sizeof(smc_record));
        return c->hio->status;
    }
    if (with_obs) {
        rc = cuda_check(cudaMemcpyAsync(c->obs + 2 * (size_t)t, h_obs_t, 16, cudaMemcpyHostToDevice, c->stream));
        if (rc) return rc;
        if (c->cfg.precision == 32) {
            // the FP32 kernels read the float copy: rounded here (as the device
            // conversion does) and sent from the context's pinned staging,
            // which this synchronising call leaves free for the next one
            c->hio->obs_f[0] = (float)h_obs_t[0];
            c->hio->obs_f[1] = (float)h_obs_t[1];
            rc = cuda_check(cudaMemcpyAsync(c->obs_f + 2 * (size_t)t, c->hio->obs_f, 2 * sizeof(float),
                                            cudaMemcpyHostToDevice, c->stream));
            if (rc) return rc;
        }
        if (c->n_obs < t + 1) c->n_obs = t + 1;
    }
    rc = smc_iterate(c, 1);
    if (rc) return rc;
    rc = cuda_check(cudaMemcpyAsync(h_record, c->rec + (t % c->cfg.max_records), sizeof(smc_record),
                                    cudaMemcpyDeviceToHost, c->stream));
    if (rc) return rc;
    return read_state(c);
}

int smc_ess(smc_ctx *c, double *h_ess) {
    if (!c) return SMC_E_ARG;
    if (!h_ess) return SMC_OK;
    const int rc = read_state(c);
    *h_ess = c->host_st.ess;
    return rc;
}

int smc_log_evidence(smc_ctx *c, double *h_out) {
    if (!c || !h_out) return SMC_E_ARG;
    const int rc = read_state(c);
    *h_out = c->host_st.log_evidence;
    return rc;
}

int smc_path_sampling(smc_ctx *c, double *h_out) {
    if (!c || !h_out) return SMC_E_ARG;
    if (c->cfg.model != SMC_MODEL_GMM) return SMC_E_ARG;
    const int rc = read_state(c);
    *h_out = c->host_st.path_log_z;
    return rc;
}

int smc_iteration(const smc_ctx *c, int32_t *t) {
    if (!c || !t) return SMC_E_ARG;
    *t = c->t_host;
    return SMC_OK;
}

int smc_state_dim(const smc_ctx *c, int32_t *d) {
    if (!c || !d) return SMC_E_ARG;
    *d = c->L.d;
    return SMC_OK;
}

static int copy_out(smc_ctx *c, void *dst, const void *src, size_t bytes, int on_device) {
    if (!dst) return SMC_E_ARG;
    int rc = read_state(c);  // also surfaces device errors
    if (rc == SMC_E_CUDA) return rc;  // a device error word still lets the data be read
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    int rc2 = cuda_check(cudaMemcpyAsync(dst, src, bytes, k, c->stream));
    if (!rc2) rc2 = cuda_check(cudaStreamSynchronize(c->stream));
    return rc2 ? rc2 : rc;
}

// One copy per row: pitched copies are specified for pitches up to
// cudaDevAttrMaxPitch (2^31 - 1 bytes), which rows of more than 2^29
// floats exceed.
static int copy_pitched(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, int rows,
                        cudaMemcpyKind k, cudaStream_t stream) {
    for (int r = 0; r < rows; ++r) {
        const int rc = cuda_check(cudaMemcpyAsync(static_cast<char *>(dst) + (size_t)r * dpitch,
                                                  static_cast<const char *>(src) + (size_t)r * spitch, width, k, stream));
        if (rc) return rc;
    }
    return SMC_OK;
}

// state rows are stored with a pitch of ld elements; callers see d x N packed
static int copy_rows(smc_ctx *c, void *dst, const void *src, int rows, bool to_caller, int on_device) {
    const size_t w = (size_t)c->cfg.n_particles * c->L.rsize, pitch = (size_t)c->L.ld * c->L.rsize;
    cudaMemcpyKind k;
    if (to_caller) k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    else k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t dpitch = to_caller ? w : pitch, spitch = to_caller ? pitch : w;
    int rc = copy_pitched(dst, dpitch, src, spitch, w, rows, k, c->stream);
    if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream));
    return rc;
}

int smc_read_state(smc_ctx *c, void *dst, int on_device) {
    if (!c || !dst) return SMC_E_ARG;
    int rc = read_state(c);
    if (rc == SMC_E_CUDA) return rc;  // a device error word still lets the data be read
    const int rc2 = copy_rows(c, dst, c->x[c->host_st.cur & 1], c->L.d, true, on_device);
    return rc2 ? rc2 : rc;
}

int smc_read_log_weight(smc_ctx *c, void *dst, int on_device) {
    if (!c) return SMC_E_ARG;
    int rc = read_state(c);
    if (rc == SMC_E_CUDA) return rc;  // a device error word still lets the data be read
    return copy_out(c, dst, c->lw[c->host_st.cur_lw & 1], (size_t)c->cfg.n_particles * c->L.rsize, on_device);
}

int smc_read_ancestors(smc_ctx *c, int32_t *dst, int on_device) {
    if (!c) return SMC_E_ARG;
    return copy_out(c, dst, c->anc, (size_t)c->cfg.n_particles * 4, on_device);
}

int smc_read_cdf(smc_ctx *c, uint64_t *dst, int on_device) {
    if (!c) return SMC_E_ARG;
    if (!(c->cfg.flags & SMC_FLAG_KEEP_CDF)) return SMC_E_STATE;
    return copy_out(c, dst, c->Q, (size_t)c->cfg.n_particles * 8, on_device);
}

int smc_read_history(smc_ctx *c, smc_record *h, int32_t count, int32_t *n_written) {
    if (!c || !h || count < 0) return SMC_E_ARG;
    int rc = read_state(c);
    if (rc == SMC_E_CUDA) return rc;  // a device error word still lets the data be read
    const int32_t last = c->host_st.t;
    const int32_t avail = (last < 0) ? 0 : std::min<int32_t>(last + 1, c->cfg.max_records);
    const int32_t m = std::min(count, avail);
    const int32_t cap = c->cfg.max_records;
    for (int32_t i = 0; i < m;) {  // at most two contiguous pieces of the ring
        const int32_t t = last - m + 1 + i;
        const int32_t slot = t % cap;
        const int32_t len = std::min(m - i, cap - slot);
        int rc2 = cuda_check(cudaMemcpyAsync(h + i, c->rec + slot, sizeof(smc_record) * (size_t)len,
                                             cudaMemcpyDeviceToHost, c->stream));
        if (rc2) return rc2;
        i += len;
    }
    int rc2 = cuda_check(cudaStreamSynchronize(c->stream));
    if (n_written) *n_written = m;
    return rc2 ? rc2 : rc;
}

int smc_write_state(smc_ctx *c, const void *src, int on_device) {
    if (!c || !src) return SMC_E_ARG;
    int rc = read_state(c);
    if (rc) return rc;
    return copy_rows(c, c->x[c->host_st.cur & 1], src, c->L.d, false, on_device);
}

int smc_write_log_weight(smc_ctx *c, const void *src, int on_device) {
    if (!c || !src) return SMC_E_ARG;
    if (!c->initialized) return SMC_E_STATE;
    int rc = read_state(c);
    if (rc) return rc;
    if (c->host_st.ready) return SMC_E_STATE;  // a resampling is pending
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t bytes = (size_t)c->cfg.n_particles * c->L.rsize;
    rc = cuda_check(cudaMemcpyAsync(c->lw[c->host_st.cur_lw & 1], src, bytes, k, c->stream));
    // then the normaliser, ESS, evidence increment and decision of the new weights (a zero increment)
    if (!rc) rc = cuda_check(cudaMemsetAsync(c->ws + c->L.inc, 0, bytes, c->stream));
    if (!rc) rc = add_log_weight_any(c);
    if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream));
    return rc;
}

int smc_add_log_weight(smc_ctx *c, const void *incw, int on_device) {
    if (!c || !incw) return SMC_E_ARG;
    if (!c->initialized) return SMC_E_STATE;
    int rc = read_state(c);
    if (rc) return rc;
    if (c->host_st.ready) return SMC_E_STATE;  // a resampling is pending
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    rc = cuda_check(cudaMemcpyAsync(c->ws + c->L.inc, incw, (size_t)c->cfg.n_particles * c->L.rsize, k, c->stream));
    if (!rc) rc = add_log_weight_any(c);
    if (!rc && !on_device) rc = cuda_check(cudaStreamSynchronize(c->stream));  // the host buffer may go away
    return rc;
}

// ---- checkpoint / restore ----
struct CkptHeader {
    char magic[8];  // "SMCCKPT1"
    int32_t model, precision, scheme, d;
    int64_t n;
    int32_t max_records, t_host;
    uint64_t seed;
    uint32_t stream_id, state_size;
    uint64_t total;
};

static size_t ckpt_bytes(const smc_ctx *c) {
    const size_t n = (size_t)c->cfg.n_particles, rs = c->L.rsize;
    return sizeof(CkptHeader) + sizeof(DevState) + sizeof(smc_record) * (size_t)c->cfg.max_records +
           (size_t)c->L.d * n * rs + n * rs + n * 4;
}

int smc_checkpoint(smc_ctx *c, void *h_blob, size_t *bytes) {
    if (!c || !bytes) return SMC_E_ARG;
    if (!c->initialized) return SMC_E_STATE;
    if (recording(c)) return SMC_E_ARG;
    const size_t need = ckpt_bytes(c);
    if (!h_blob) {
        *bytes = need;
        return SMC_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return SMC_E_ARG;
    }
    int rc = read_state(c);
    if (rc) return rc;
    char *p = static_cast<char *>(h_blob);
    CkptHeader h{};
    std::memcpy(h.magic, "SMCCKPT1", 8);
    h.model = c->cfg.model;
    h.precision = c->cfg.precision;
    h.scheme = c->cfg.scheme;
    h.d = c->L.d;
    h.n = c->cfg.n_particles;
    h.max_records = c->cfg.max_records;
    h.t_host = c->t_host;
    h.seed = c->cfg.seed;
    h.stream_id = c->cfg.stream_id;
    h.state_size = (uint32_t)sizeof(DevState);
    h.total = need;
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    std::memcpy(p, &c->host_st, sizeof(DevState));
    p += sizeof(DevState);
    const size_t n = (size_t)c->cfg.n_particles, rs = c->L.rsize;
    rc = cuda_check(cudaMemcpyAsync(p, c->rec, sizeof(smc_record) * (size_t)c->cfg.max_records,
                                    cudaMemcpyDeviceToHost, c->stream));
    p += sizeof(smc_record) * (size_t)c->cfg.max_records;
    if (!rc) rc = copy_rows(c, p, c->x[c->host_st.cur & 1], c->L.d, true, 0);
    p += (size_t)c->L.d * n * rs;
    if (!rc) rc = copy_out(c, p, c->lw[c->host_st.cur_lw & 1], n * rs, 0);
    p += n * rs;
    if (!rc) rc = copy_out(c, p, c->anc, n * 4, 0);
    if (!rc) *bytes = need;
    return rc;
}

int smc_restore(smc_ctx *c, const void *h_blob, size_t bytes) {
    if (!c || !h_blob) return SMC_E_ARG;
    if (recording(c)) return SMC_E_ARG;
    if (bytes < sizeof(CkptHeader)) return SMC_E_ARG;
    CkptHeader h;
    std::memcpy(&h, h_blob, sizeof(h));
    if (std::memcmp(h.magic, "SMCCKPT1", 8) != 0 || h.model != c->cfg.model || h.precision != c->cfg.precision ||
        h.scheme != c->cfg.scheme || h.d != c->L.d || h.n != c->cfg.n_particles ||
        h.max_records != c->cfg.max_records || h.seed != c->cfg.seed || h.stream_id != c->cfg.stream_id ||
        h.state_size != sizeof(DevState) || h.total != ckpt_bytes(c) || bytes < h.total)
        return SMC_E_ARG;
    if (c->cfg.model != SMC_MODEL_GMM && h.t_host >= c->n_obs) return SMC_E_STATE;  // data first
    const char *p = static_cast<const char *>(h_blob) + sizeof(h);
    DevState s;
    std::memcpy(&s, p, sizeof(s));
    p += sizeof(s);
    // counters of kernels in flight are idle at a checkpoint; start them clean
    s.error = 0;
    s.ticket = 0;
    s.grid_count = 0;
    s.grid_depart = 0;
    for (int k = 0; k < kScanSlots; ++k) s.scan_ticket[k] = 0;
    const size_t n = (size_t)c->cfg.n_particles, rs = c->L.rsize;
    int rc = cuda_check(cudaMemcpyAsync(c->st, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream));
    if (!rc) rc = cuda_check(cudaMemcpyAsync(c->rec, p, sizeof(smc_record) * (size_t)c->cfg.max_records,
                                             cudaMemcpyHostToDevice, c->stream));
    p += sizeof(smc_record) * (size_t)c->cfg.max_records;
    if (!rc) rc = copy_rows(c, c->x[s.cur & 1], p, c->L.d, false, 0);
    p += (size_t)c->L.d * n * rs;
    if (!rc) rc = cuda_check(cudaMemcpyAsync(c->lw[s.cur_lw & 1], p, n * rs, cudaMemcpyHostToDevice, c->stream));
    p += n * rs;
    if (!rc) rc = cuda_check(cudaMemcpyAsync(c->anc, p, n * 4, cudaMemcpyHostToDevice, c->stream));
    // an adaptive schedule lives on the device: its current alpha (kept in
    // the state block) goes back into the schedule for the next iteration
    if (!rc && c->cfg.model == SMC_MODEL_GMM && c->cfg.gmm.schedule == SMC_ALPHA_ADAPTIVE && h.t_host >= 0)
        rc = cuda_check(cudaMemcpyAsync(c->alpha + h.t_host, &s.alpha, 8, cudaMemcpyHostToDevice, c->stream));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream));
    if (rc) return rc;
    c->t_host = h.t_host;
    c->initialized = 1;
    c->host_st = s;
    return SMC_OK;
}

int smc_gmm_log_target(smc_ctx *c, const void *d_u, int64_t count, double alpha, void *d_logt, void *d_grad) {
    if (!c || !d_u || !d_logt || !d_grad || count < 1 || !(alpha >= 0.0) || !(alpha <= 1.0)) return SMC_E_ARG;
    if (c->cfg.model != SMC_MODEL_GMM) return SMC_E_ARG;
    if (c->n_obs < 1) return SMC_E_STATE;
    return gmm_log_target_any(c, d_u, count, alpha, d_logt, d_grad);
}

int smc_set_move_events(smc_ctx *c, void *ev_before, void *ev_after) {
    if (!c) return SMC_E_ARG;
    c->ev_move[0] = static_cast<cudaEvent_t>(ev_before);
    c->ev_move[1] = static_cast<cudaEvent_t>(ev_after);
    drop_graphs(c);  // captured again, with or without the events, at the next smc_iterate
    return SMC_OK;
}

int smc_sync(smc_ctx *c) {
    if (!c) return SMC_E_ARG;
    return read_state(c);
}

int smc_set_wait_limit(uint32_t polls) {
    const uint32_t v = polls ? polls : kSpinLimit;
    return cuda_check(cudaMemcpyToSymbol(c_wait_limit, &v, sizeof(v)));
}

int smc_wait_selftest(smc_ctx *c) {
    if (!c) return SMC_E_ARG;
    wait_selftest_kernel<<<1, kBlock, 0, c->stream>>>(c->st);
    return cuda_check(cudaGetLastError());
}

// ---- one shard of a filter partitioned over ranks --------------------------

int smc_shard_configure(smc_ctx *c, int64_t n_global, int64_t offset) {
    if (!c) return SMC_E_ARG;
    const smc_config &g = c->cfg;
    if (g.scheme != SMC_SYSTEMATIC && g.scheme != SMC_STRATIFIED) return SMC_E_ARG;
    // a partitioned mixture sampler takes a fixed schedule (an adaptive
    // alpha would need a grid-wide search over every rank's particles)
    if (g.model == SMC_MODEL_GMM && g.gmm.schedule == SMC_ALPHA_ADAPTIVE) return SMC_E_ARG;
    if (g.flags & (SMC_FLAG_RECORD | SMC_FLAG_INPLACE | SMC_FLAG_POST_MEAN)) return SMC_E_ARG;
    if (offset < 0 || n_global < offset + g.n_particles || n_global > (int64_t(1) << 30)) return SMC_E_ARG;
    c->shard_n = n_global;
    c->shard_off = offset;
    c->initialized = 0;
    drop_graphs(c);
    return SMC_OK;
}

int smc_shard_move(smc_ctx *c, void *d_partial) {
    if (!c || !d_partial) return SMC_E_ARG;
    if (!c->shard_n || !c->initialized) return SMC_E_STATE;
    if (c->cfg.model == SMC_MODEL_GMM) {  // iteration 0: the prior draws; then the reweighting
        const int kind = (c->t_host < 0) ? 0 : 1;
        if (kind == 1 && c->t_host + 1 > c->cfg.gmm.n_iter) return SMC_E_ARG;
        const int rc = gmm_shard_launch(c, kind, d_partial);
        if (!rc) {
            c->t_host += 1;
            c->shard_pending = kind;
        }
        return rc;
    }
    if (c->t_host + 1 >= c->n_obs) return SMC_E_ARG;
    if (c->cfg.precision == 32)
        pf_shard_move_kernel<float><<<(unsigned)c->L.nbw, kBlock, 0, c->stream>>>(pf_args<float>(c),
                                                                                  static_cast<Partial *>(d_partial));
    else
        pf_shard_move_kernel<double><<<(unsigned)c->L.nbw, kBlock, 0, c->stream>>>(pf_args<double>(c),
                                                                                   static_cast<Partial *>(d_partial));
    const int rc = cuda_check(cudaGetLastError());
    if (!rc) c->t_host += 1;
    return rc;
}

int smc_shard_finalize(smc_ctx *c, const void *d_partials, int32_t world) {
    if (!c || !d_partials || world < 1) return SMC_E_ARG;
    if (!c->shard_n) return SMC_E_STATE;
    if (c->cfg.model == SMC_MODEL_GMM) return gmm_shard_finalize_any(c, d_partials, world, c->shard_pending);
    const Partial *p = static_cast<const Partial *>(d_partials);
    if (c->cfg.precision == 32)
        pf_shard_finalize_kernel<float><<<1, kBlock, 0, c->stream>>>(pf_args<float>(c), p, world, c->shard_n);
    else
        pf_shard_finalize_kernel<double><<<1, kBlock, 0, c->stream>>>(pf_args<double>(c), p, world, c->shard_n);
    return cuda_check(cudaGetLastError());
}

int smc_shard_total(smc_ctx *c, uint64_t *d_total) {
    if (!c || !d_total) return SMC_E_ARG;
    if (!c->shard_n) return SMC_E_STATE;
    const int64_t n = c->cfg.n_particles;
    const unsigned tiles = (unsigned)((n + kScanTile - 1) / kScanTile);
    const int frac = 61 - ceil_log2(c->shard_n);
    unsigned long long *tot = reinterpret_cast<unsigned long long *>(d_total);
    if (c->cfg.precision == 32) {
        QGen<float> qg = qgen_of<float>(c);
        qg.frac = frac;
        tile_reduce_kernel<QGen<float>><<<tiles, kBlock, 0, c->stream>>>(qg, n, tsum_of(c, SLOT_CDF), tot,
                                                                          &c->st->scan_ticket[SLOT_CDF], c->st, 1);
    } else {
        QGen<double> qg = qgen_of<double>(c);
        qg.frac = frac;
        tile_reduce_kernel<QGen<double>><<<tiles, kBlock, 0, c->stream>>>(qg, n, tsum_of(c, SLOT_CDF), tot,
                                                                           &c->st->scan_ticket[SLOT_CDF], c->st, 1);
    }
    return cuda_check(cudaGetLastError());
}


int smc_shard_select(smc_ctx *c, const uint64_t *d_totals, int32_t rank, int32_t world, int32_t *d_src,
                     int64_t *d_range) {
    if (!c || !d_totals || !d_src || !d_range || world < 1 || rank < 0 || rank >= world) return SMC_E_ARG;
    if (!c->shard_n) return SMC_E_STATE;
    const bool strat = c->cfg.scheme == SMC_STRATIFIED;
    if (c->cfg.precision == 32)
        return strat ? shard_select_t<float, true>(c, d_totals, rank, world, d_src, d_range)
                     : shard_select_t<float, false>(c, d_totals, rank, world, d_src, d_range);
    return strat ? shard_select_t<double, true>(c, d_totals, rank, world, d_src, d_range)
                 : shard_select_t<double, false>(c, d_totals, rank, world, d_src, d_range);
}

int smc_shard_mcmc(smc_ctx *c, void *d_partial) {
    if (!c || !d_partial) return SMC_E_ARG;
    if (!c->shard_n || !c->initialized) return SMC_E_STATE;
    if (c->cfg.model != SMC_MODEL_GMM || c->t_host < 1) return SMC_E_STATE;
    return gmm_shard_launch(c, 2, d_partial);
}

int smc_shard_mcmc_finalize(smc_ctx *c, const void *d_partials, int32_t world) {
    if (!c || !d_partials || world < 1) return SMC_E_ARG;
    if (!c->shard_n || c->cfg.model != SMC_MODEL_GMM || c->t_host < 1) return SMC_E_STATE;
    return gmm_shard_finalize_any(c, d_partials, world, 2);
}

int smc_shard_pack(smc_ctx *c, const int32_t *d_src, int64_t k_lo, int64_t count, void *d_send) {
    if (!c || !d_src || k_lo < 0 || count < 0 || (count && !d_send)) return SMC_E_ARG;
    if (!c->shard_n) return SMC_E_STATE;
    if (!count) return SMC_OK;
    const unsigned g = (unsigned)((count + kBlock - 1) / kBlock);
    if (c->cfg.model == SMC_MODEL_GMM) {  // every state row of the mixture sampler
        const int d = (int)c->L.d;
        if (c->cfg.precision == 32)
            shard_pack_rows_kernel<float><<<g, kBlock, 0, c->stream>>>(
                static_cast<const float *>(c->x[0]), static_cast<const float *>(c->x[1]), c->L.ld, d, c->st, d_src,
                k_lo, count, static_cast<float *>(d_send));
        else
            shard_pack_rows_kernel<double><<<g, kBlock, 0, c->stream>>>(
                static_cast<const double *>(c->x[0]), static_cast<const double *>(c->x[1]), c->L.ld, d, c->st,
                d_src, k_lo, count, static_cast<double *>(d_send));
        return cuda_check(cudaGetLastError());
    }
    if (c->cfg.precision == 32)
        shard_pack_kernel<float><<<g, kBlock, 0, c->stream>>>(pf_args<float>(c), d_src, k_lo, count,
                                                              static_cast<float *>(d_send));
    else
        shard_pack_kernel<double><<<g, kBlock, 0, c->stream>>>(pf_args<double>(c), d_src, k_lo, count,
                                                               static_cast<double *>(d_send));
    return cuda_check(cudaGetLastError());
}

int smc_shard_unpack(smc_ctx *c, const void *d_recv) {
    if (!c || !d_recv) return SMC_E_ARG;
    if (!c->shard_n) return SMC_E_STATE;
    const unsigned g = (unsigned)((c->cfg.n_particles + kBlock - 1) / kBlock);
    if (c->cfg.model == SMC_MODEL_GMM) {
        const int d = (int)c->L.d;
        const int64_t n = c->cfg.n_particles;
        const double nl = -std::log((double)c->shard_n);
        if (c->cfg.precision == 32)
            shard_unpack_rows_kernel<float><<<g, kBlock, 0, c->stream>>>(
                static_cast<float *>(c->x[0]), static_cast<float *>(c->x[1]), static_cast<float *>(c->lw[0]),
                static_cast<float *>(c->lw[1]), c->L.ld, d, n, (float)nl, c->st, static_cast<const float *>(d_recv));
        else
            shard_unpack_rows_kernel<double><<<g, kBlock, 0, c->stream>>>(
                static_cast<double *>(c->x[0]), static_cast<double *>(c->x[1]), static_cast<double *>(c->lw[0]),
                static_cast<double *>(c->lw[1]), c->L.ld, d, n, nl, c->st, static_cast<const double *>(d_recv));
        return cuda_check(cudaGetLastError());
    }
    if (c->cfg.precision == 32)
        shard_unpack_kernel<float><<<g, kBlock, 0, c->stream>>>(pf_args<float>(c), static_cast<const float *>(d_recv));
    else
        shard_unpack_kernel<double><<<g, kBlock, 0, c->stream>>>(pf_args<double>(c),
                                                                 static_cast<const double *>(d_recv));
    return cuda_check(cudaGetLastError());
}

const char *smc_error_string(int code) {
    switch (code) {
        case SMC_OK: return "ok";
        case SMC_E_ARG: return "invalid argument or configuration";
        case SMC_E_WORKSPACE: return "workspace too small or misaligned";
        case SMC_E_NONFINITE: return "all weights are zero or NaN";
        case SMC_E_TIMEOUT: return "a bounded device wait gave up";
        case SMC_E_CUDA: return "CUDA runtime error";
        case SMC_E_STATE: return "call out of order";
        case SMC_E_RANGE: return "a device counter left its range";
    }
    return "unknown error";
}

}  // extern "C"

// ------------------------------------------------------------ primitives --

namespace {
__global__ void philox_kernel(const uint4 *ctr, uint2 key, uint4 *out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}
}  // namespace

extern "C" int smc_philox4x32_10(const uint32_t *d_ctr, const uint32_t key[2], uint32_t *d_out, int64_t n,
                                 void *cuda_stream) {
    if (!d_ctr || !key || !d_out || n < 0) return SMC_E_ARG;
    if (((uintptr_t)d_ctr | (uintptr_t)d_out) & 15) return SMC_E_ARG;
    if (n == 0) return SMC_OK;
    const unsigned grid = (unsigned)((n + 255) / 256);
    philox_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        reinterpret_cast<const uint4 *>(d_ctr), make_uint2(key[0], key[1]), reinterpret_cast<uint4 *>(d_out), n);
    return cuda_check(cudaGetLastError());
}

// ------------------------------------------------------------------ GMM --
namespace {

double gmm_alpha(const smc_gmm_params &g, int32_t t) {
    if (g.schedule == SMC_ALPHA_ADAPTIVE) return 0.0;  // alpha_0; the rest is chosen on the device
    const double x = (double)t / (double)g.n_iter;
    double a = (g.schedule == SMC_ALPHA_LINEAR) ? x : std::pow(x, g.power);
    return std::min(1.0, std::max(0.0, a));
}

int gmm_setup(smc_ctx *c) {
    const smc_gmm_params &g = c->cfg.gmm;
    double *tab = new (std::nothrow) double[(size_t)g.n_iter + 1];
    if (!tab) return SMC_E_ARG;
    for (int32_t t = 0; t <= g.n_iter; ++t) tab[t] = gmm_alpha(g, t);
    int rc = cuda_check(cudaMemcpyAsync(c->alpha, tab, ((size_t)g.n_iter + 1) * 8, cudaMemcpyHostToDevice, c->stream));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream));
    delete[] tab;
    return rc;
}

int gmm_on_data(smc_ctx *c) {
    // float copy of the data for the FP32 kernels (every model)
    const int64_t n = (c->cfg.model == SMC_MODEL_GMM) ? c->n_obs : 2 * c->n_obs;
    to_float_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->obs, c->obs_f, n);
    return cuda_check(cudaGetLastError());
}

void gmm_release(smc_ctx *) {}

template <typename R>
GmmArgs<R> gmm_args(smc_ctx *c) {
    GmmArgs<R> a;
    const smc_config &cfg = c->cfg;
    const smc_gmm_params &g = cfg.gmm;
    const int64_t n = cfg.n_particles;
    a.n = n;
    a.ld = c->L.ld;
    a.nd = (int32_t)c->n_obs;
    a.y = (sizeof(R) == 4) ? reinterpret_cast<const R *>(c->obs_f) : reinterpret_cast<const R *>(c->obs);
    for (int b = 0; b < 2; ++b) {
        a.x[b] = static_cast<R *>(c->x[b]);
        a.lw[b] = static_cast<R *>(c->lw[b]);
    }
    a.anc = c->anc;
    a.alpha = c->alpha;
    a.T = g.n_iter;
    a.rec = c->rec;
    a.rec_cap = cfg.max_records;
    a.st = c->st;
    a.part = c->part;
    a.log_n = std::log((double)n);
    a.threshold = cfg.threshold;
    const int r = g.n_comp;
    const double shape = (double)g.shape0;
    a.mu0 = g.mu0;
    a.sd0 = g.sd0;
    a.inv_sd0 = 1.0 / g.sd0;
    a.lp_const = r * (-0.5 * std::log(2.0 * M_PI * g.sd0 * g.sd0) + shape * std::log(g.rate0) - std::lgamma(shape)) +
                 std::lgamma((double)r);
    a.shape_m1 = shape - 1.0;
    a.rate = g.rate0;
    a.half_nd_log2pi = 0.5 * (double)c->n_obs * std::log(2.0 * M_PI);
    a.mala_eps = g.mala_step;
    a.mu0_f = (float)a.mu0;
    a.inv_sd0_f = (float)a.inv_sd0;
    a.lp_const_f = (float)a.lp_const;
    a.shape_m1_f = (float)a.shape_m1;
    a.rate_f = (float)a.rate;
    a.mala_eps_f = (float)a.mala_eps;
    a.hnl_f[0] = (float)a.half_nd_log2pi;
    a.hnl_f[1] = (float)(a.half_nd_log2pi - (double)a.hnl_f[0]);
    a.key = key_of(c);
    a.stream = cfg.stream_id;
    a.index0 = (uint32_t)c->shard_off;
    a.shard_out = static_cast<Partial *>(c->shard_out);
    if (c->shard_n) a.log_n = std::log((double)c->shard_n);  // equal weights are 1 / N of the whole sampler
    return a;
}

enum GmmKernel { GMM_INIT, GMM_REWEIGHT, GMM_MCMC };

// a mixture shard's finalisation on every rank's partials (kind: 0 init,
// 1 reweight, 2 mcmc), the sampler's N in place of the shard's
template <typename R, int MOVE>
int gmm_shard_finalize_move(smc_ctx *c, const Partial *parts, int32_t world, int kind) {
    GmmArgs<R> a = gmm_args<R>(c);
    a.n = c->shard_n;
    a.shard_out = nullptr;
    gmm_shard_finalize_kernel<R, MOVE><<<1, kBlock, 0, c->stream>>>(a, parts, world, kind);
    return cuda_check(cudaGetLastError());
}
template <typename R>
int gmm_shard_finalize_r(smc_ctx *c, const Partial *parts, int32_t world, int kind) {
    switch (c->cfg.gmm.move) {
        case SMC_GMM_RW: return gmm_shard_finalize_move<R, kMoveRW>(c, parts, world, kind);
        case SMC_GMM_MALA: return gmm_shard_finalize_move<R, kMoveMALA>(c, parts, world, kind);
        case SMC_GMM_RW_MALA: return gmm_shard_finalize_move<R, kMoveRWMALA>(c, parts, world, kind);
    }
    return SMC_E_ARG;
}

template <typename R, int NC, int MOVE>
int gmm_launch_move(smc_ctx *c, GmmKernel k) {
    constexpr bool G = (MOVE != kMoveRW);
    GmmArgs<R> a = gmm_args<R>(c);
    const size_t smem = (((size_t)a.nd * sizeof(R)) + 15) & ~size_t(15);
    const unsigned gq = (unsigned)((kQuad * a.n + kBlock - 1) / kBlock);
    const unsigned gw = (unsigned)c->L.nbw;
    switch (k) {
        case GMM_INIT:
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(gmm_init_kernel<R, NC, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            gmm_init_kernel<R, NC, G><<<gq, kBlock, smem, c->stream>>>(a);
            break;
        case GMM_REWEIGHT:
            gmm_reweight_kernel<R, NC><<<gw, kBlock, 0, c->stream>>>(a);
            break;
        case GMM_MCMC:
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(gmm_mcmc_kernel<R, NC, MOVE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            gmm_mcmc_kernel<R, NC, MOVE><<<gq, kBlock, smem, c->stream>>>(a);
            break;
    }
    return cuda_check(cudaGetLastError());
}

template <typename R, int NC>
int gmm_launch_nc(smc_ctx *c, GmmKernel k) {
    switch (c->cfg.gmm.move) {
        case SMC_GMM_RW: return gmm_launch_move<R, NC, kMoveRW>(c, k);
        case SMC_GMM_MALA: return gmm_launch_move<R, NC, kMoveMALA>(c, k);
        case SMC_GMM_RW_MALA: return gmm_launch_move<R, NC, kMoveRWMALA>(c, k);
    }
    return SMC_E_ARG;
}

template <typename R>
int gmm_launch(smc_ctx *c, GmmKernel k) {
    switch (c->cfg.gmm.n_comp) {
        case 1: return gmm_launch_nc<R, 1>(c, k);
        case 2: return gmm_launch_nc<R, 2>(c, k);
        case 3: return gmm_launch_nc<R, 3>(c, k);
        case 4: return gmm_launch_nc<R, 4>(c, k);
        case 5: return gmm_launch_nc<R, 5>(c, k);
        case 6: return gmm_launch_nc<R, 6>(c, k);
        case 7: return gmm_launch_nc<R, 7>(c, k);
        case 8: return gmm_launch_nc<R, 8>(c, k);
    }
    return SMC_E_ARG;
}

// tempered log-target and gradient at count given points (rows of pitch count)
template <typename R, int NC>
int gmm_log_target_nc(smc_ctx *c, const void *u, int64_t count, double alpha, void *logt, void *grad) {
    GmmArgs<R> a = gmm_args<R>(c);
    const size_t smem = (((size_t)a.nd * sizeof(R)) + 15) & ~size_t(15);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(gmm_log_target_kernel<R, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned g = (unsigned)((kQuad * count + kBlock - 1) / kBlock);
    gmm_log_target_kernel<R, NC><<<g, kBlock, smem, c->stream>>>(a, static_cast<const R *>(u), count, count, alpha,
                                                                 static_cast<R *>(logt), static_cast<R *>(grad));
    return cuda_check(cudaGetLastError());
}

template <typename R>
int gmm_log_target_r(smc_ctx *c, const void *u, int64_t count, double alpha, void *logt, void *grad) {
    switch (c->cfg.gmm.n_comp) {
        case 1: return gmm_log_target_nc<R, 1>(c, u, count, alpha, logt, grad);
        case 2: return gmm_log_target_nc<R, 2>(c, u, count, alpha, logt, grad);
        case 3: return gmm_log_target_nc<R, 3>(c, u, count, alpha, logt, grad);
        case 4: return gmm_log_target_nc<R, 4>(c, u, count, alpha, logt, grad);
        case 5: return gmm_log_target_nc<R, 5>(c, u, count, alpha, logt, grad);
        case 6: return gmm_log_target_nc<R, 6>(c, u, count, alpha, logt, grad);
        case 7: return gmm_log_target_nc<R, 7>(c, u, count, alpha, logt, grad);
        case 8: return gmm_log_target_nc<R, 8>(c, u, count, alpha, logt, grad);
    }
    return SMC_E_ARG;
}

int gmm_log_target_any(smc_ctx *c, const void *u, int64_t count, double alpha, void *logt, void *grad) {
    return (c->cfg.precision == 32) ? gmm_log_target_r<float>(c, u, count, alpha, logt, grad)
                                    : gmm_log_target_r<double>(c, u, count, alpha, logt, grad);
}

int gmm_launch_any(smc_ctx *c, GmmKernel k) {
    return (c->cfg.precision == 32) ? gmm_launch<float>(c, k) : gmm_launch<double>(c, k);
}

// SMC_ALPHA_ADAPTIVE: alpha_t of the coming iteration (gmm_alpha_kernel),
// written into the schedule array before the reweighting reads it
template <typename R>
int gmm_launch_alpha(smc_ctx *c) {
    static int per_sm[64] = {}, sms[64] = {};
    int slots = 0;
    if (int rc = coop_capacity(reinterpret_cast<const void *>(gmm_alpha_kernel<R>), per_sm, sms, &slots)) return rc;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)slots, c->L.nbw, (int64_t)kMaxCoopGrid}));
    const double log_target = std::log(c->cfg.gmm.ess_target * (double)c->cfg.n_particles);
    const int dep = c->dependent_launch;
    c->dependent_launch = 0;  // the first kernel of the iteration: an ordinary node
    const int rc = launch_coop(c, grid, gmm_alpha_kernel<R>, gmm_args<R>(c), (int32_t)(3 * c->cfg.gmm.n_comp + 1),
                               log_target, c->alpha, reinterpret_cast<AlphaPartial<R> *>(c->ws + c->L.adapt));
    c->dependent_launch = dep;
    return rc;
}

int gmm_shard_launch(smc_ctx *c, int kind, void *d_partial) {
    c->shard_out = d_partial;
    const int rc = gmm_launch_any(c, kind == 0 ? GMM_INIT : kind == 1 ? GMM_REWEIGHT : GMM_MCMC);
    c->shard_out = nullptr;
    return rc;
}

int gmm_shard_finalize_any(smc_ctx *c, const void *d_partials, int32_t world, int kind) {
    const Partial *p = static_cast<const Partial *>(d_partials);
    return (c->cfg.precision == 32) ? gmm_shard_finalize_r<float>(c, p, world, kind)
                                    : gmm_shard_finalize_r<double>(c, p, world, kind);
}

int gmm_launch_reweight(smc_ctx *c) {
    if (c->cfg.gmm.schedule == SMC_ALPHA_ADAPTIVE) {
        const int rc = (c->cfg.precision == 32) ? gmm_launch_alpha<float>(c) : gmm_launch_alpha<double>(c);
        if (rc) return rc;
    }
    return gmm_launch_any(c, GMM_REWEIGHT);
}
int gmm_launch_mcmc(smc_ctx *c) { return gmm_launch_any(c, GMM_MCMC); }

int gmm_initialize(smc_ctx *c) {
    const int rc = gmm_launch_any(c, GMM_INIT);
    if (!rc) c->t_host = 0;
    return rc;
}

int gmm_move(smc_ctx *c) {
    if (c->t_host + 1 > c->cfg.gmm.n_iter) return SMC_E_ARG;
    const int rc = gmm_launch_reweight(c);
    if (!rc) c->t_host += 1;
    return rc;
}

int gmm_mcmc(smc_ctx *c) {
    if (c->t_host < 1) return SMC_OK;  // nothing to move at t = 0 (equal weights, alpha = 0)
    return gmm_launch_any(c, GMM_MCMC);
}

}  // namespace

// ============================================================== batched ==

namespace {

struct BatchPlan {
    int32_t nf = 0, tmax = 0, ntiles = 0, nstiles = 0;
    int64_t ntot = 0;  // concatenated particles (each filter padded to 64)
    std::vector<int32_t> perm;  // internal -> caller index
    std::vector<int64_t> n, off, obs_off, rec_off;
    std::vector<int32_t> T, tfirst, sfirst, tile_filter, stile_filter, act_tiles, act_stiles, frac;
    std::vector<uint32_t> stream_of;
    std::vector<unsigned long long> mrec;  // floor((2^64 - 1) / N) per filter
    std::vector<double> log_n;
    size_t o_fst, o_bs, o_rec, o_part, o_tsum, o_x, o_lw, o_anc, o_obs, o_n, o_off, o_obs_off, o_rec_off, o_T,
        o_tfirst, o_sfirst, o_tf, o_stf, o_act, o_acts, o_stream, o_mrec, o_logn, o_nlogn, o_obs_f, o_frac,
        total = 0;
    size_t rsize = 4;
};

bool batch_valid(const smc_config *cfg, const int64_t *n, const int32_t *T, int32_t nf) {
    if (!cfg || !n || !T || nf < 1 || nf > 65536) return false;
    if (cfg->model != SMC_MODEL_CV && cfg->model != SMC_MODEL_CV_GAUSS) return false;
    if (cfg->precision != 32 && cfg->precision != 64) return false;
    if (cfg->scheme != SMC_SYSTEMATIC && cfg->scheme != SMC_STRATIFIED) return false;
    // per-context options the batched kernels do not implement
    if (cfg->flags & (SMC_FLAG_RECORD | SMC_FLAG_POST_MEAN | SMC_FLAG_INPLACE)) return false;
    if (!(cfg->threshold == cfg->threshold) || !(cfg->cv.obs_scale > 0) || !(cfg->cv.obs_df > 0)) return false;
    for (int32_t b = 0; b < nf; ++b)
        if (n[b] < 1 || n[b] > (int64_t(1) << 30) || T[b] < 1) return false;
    return true;
}

bool batch_plan(const smc_config *cfg, const int64_t *n, const int32_t *T, int32_t nf, BatchPlan &P) {
    if (!batch_valid(cfg, n, T, nf)) return false;
    P.nf = nf;
    P.rsize = (cfg->precision == 32) ? 4 : 8;
    P.perm.resize(nf);
    std::iota(P.perm.begin(), P.perm.end(), 0);
    std::stable_sort(P.perm.begin(), P.perm.end(), [&](int32_t a, int32_t b) { return T[a] > T[b]; });
    P.n.resize(nf);
    P.off.resize(nf);
    P.obs_off.resize(nf);
    P.rec_off.resize(nf);
    P.T.resize(nf);
    P.tfirst.resize(nf + 1);
    P.sfirst.resize(nf + 1);
    P.frac.resize(nf);
    P.stream_of.resize(nf);
    P.mrec.resize(nf);
    P.log_n.resize(nf);
    int64_t o = 0, oo = 0;
    int32_t tf = 0, sf = 0;
    for (int32_t i = 0; i < nf; ++i) {
        const int32_t b = P.perm[i];
        P.n[i] = n[b];
        P.T[i] = T[b];
        P.off[i] = o;
        o += (n[b] + 63) & ~int64_t(63);
        P.obs_off[i] = oo;
        P.rec_off[i] = oo;
        oo += T[b];
        P.tfirst[i] = tf;
        // the move tiles of the plain filter of the same precision
        const int64_t tile_n = (cfg->precision == 64) ? pf64_move_threads(n[b]) : kPfTile;
        tf += (int32_t)((n[b] + tile_n - 1) / tile_n);
        P.sfirst[i] = sf;
        sf += (int32_t)((n[b] + kScanTile - 1) / kScanTile);
        P.frac[i] = 61 - ceil_log2(n[b]);
        P.stream_of[i] = cfg->stream_id + (uint32_t)b;
        P.mrec[i] = ~0ull / (unsigned long long)n[b];
        P.log_n[i] = std::log((double)n[b]);
    }
    P.tfirst[nf] = tf;
    P.sfirst[nf] = sf;
    P.ntot = o;
    P.ntiles = tf;
    P.nstiles = sf;
    P.tmax = P.T[0];
    P.tile_filter.resize(tf);
    P.stile_filter.resize(sf);
    for (int32_t i = 0; i < nf; ++i) {
        for (int32_t k = P.tfirst[i]; k < P.tfirst[i + 1]; ++k) P.tile_filter[k] = i;
        for (int32_t k = P.sfirst[i]; k < P.sfirst[i + 1]; ++k) P.stile_filter[k] = i;
    }
    // filters active at iteration t: those with T > t, a prefix in this order
    P.act_tiles.assign(P.tmax, 0);
    P.act_stiles.assign(P.tmax, 0);
    int32_t a = nf;
    for (int32_t t = 0; t < P.tmax; ++t) {
        while (a > 0 && P.T[a - 1] <= t) --a;
        P.act_tiles[t] = P.tfirst[a];
        P.act_stiles[t] = P.sfirst[a];
    }
    size_t off_b = 0;
    auto take = [&](size_t bytes) {
        const size_t r = off_b;
        off_b += align_up(bytes);
        return r;
    };
    P.o_fst = take(sizeof(DevState) * nf);
    P.o_bs = take(sizeof(BatchState));
    P.o_rec = take(sizeof(smc_record) * (size_t)oo);
    P.o_part = take(sizeof(Partial) * (size_t)tf);
    P.o_tsum = take(8 * (size_t)sf);
    P.o_x = take(2 * 4 * (size_t)P.ntot * P.rsize);
    P.o_lw = take(2 * (size_t)P.ntot * P.rsize);
    P.o_anc = take(4 * (size_t)P.ntot);
    P.o_obs = take(16 * (size_t)oo);
    P.o_obs_f = take(8 * (size_t)oo);  // float copy (FP32 batches)
    P.o_n = take(8 * (size_t)nf);
    P.o_off = take(8 * (size_t)nf);
    P.o_obs_off = take(8 * (size_t)nf);
    P.o_rec_off = take(8 * (size_t)nf);
    P.o_T = take(4 * (size_t)nf);
    P.o_tfirst = take(4 * (size_t)(nf + 1));
    P.o_sfirst = take(4 * (size_t)(nf + 1));
    P.o_tf = take(4 * (size_t)tf);
    P.o_stf = take(4 * (size_t)sf);
    P.o_act = take(4 * (size_t)P.tmax);
    P.o_acts = take(4 * (size_t)P.tmax);
    P.o_stream = take(4 * (size_t)nf);
    P.o_mrec = take(8 * (size_t)nf);
    P.o_logn = take(8 * (size_t)nf);
    P.o_nlogn = take(8 * (size_t)nf);  // -log N in the batch precision
    P.o_frac = take(4 * (size_t)nf);
    P.total = off_b;
    return true;
}

}  // namespace

struct smc_batch {
    smc_config cfg;
    BatchPlan P;
    char *ws;
    cudaStream_t stream;
    int device, nsm;
    int32_t t_host;
    int initialized;
    int grid_per_sm;
    int chunk;  // tiles per work item of the persistent kernels
    cudaGraphExec_t graph;
    int graph_grid, graph_chunk;
    std::vector<int32_t> inv;  // caller -> internal
};

namespace {

template <typename T>
T *at(smc_batch *b, size_t o) {
    return reinterpret_cast<T *>(b->ws + o);
}

template <typename R>
BatchArgs<R> batch_args(smc_batch *bt) {
    const BatchPlan &P = bt->P;
    BatchArgs<R> B;
    PfArgs<R> &a = B.proto;
    std::memset(&a, 0, sizeof(a));
    const smc_config &g = bt->cfg;
    a.threshold = g.threshold;
    set_threshold_df(a, g.threshold);
    a.delta = R(g.cv.delta);
    a.sd_pos = R(g.cv.sd_pos);
    a.sd_vel = R(g.cv.sd_vel);
    a.sd_pos0 = R(g.cv.sd_pos0);
    a.sd_vel0 = R(g.cv.sd_vel0);
    const double s = g.cv.obs_scale, nu = g.cv.obs_df;
    a.inv_scale = R(1.0 / s);
    a.inv_nu = R(1.0 / nu);
    a.half_nu1 = R(0.5 * (nu + 1.0));
    a.gaussian = (g.model == SMC_MODEL_CV_GAUSS) ? 1 : 0;
    double cst;
    if (a.gaussian) cst = -0.5 * std::log(2.0 * M_PI) - std::log(s);
    else cst = std::lgamma(0.5 * (nu + 1.0)) - std::lgamma(0.5 * nu) - 0.5 * std::log(nu * M_PI) - std::log(s);
    a.ll_const = R(2.0 * cst);
    a.key = make_uint2((uint32_t)(g.seed & 0xffffffffu), (uint32_t)(g.seed >> 32));
    for (int k = 0; k < 2; ++k) {
        R *base = at<R>(bt, P.o_x) + (size_t)k * 4 * P.ntot;
        for (int r = 0; r < 4; ++r) B.x[k][r] = base + (size_t)r * P.ntot;
        B.lw[k] = at<R>(bt, P.o_lw) + (size_t)k * P.ntot;
    }
    B.anc = at<int32_t>(bt, P.o_anc);
    B.obs = at<double>(bt, P.o_obs);
    B.rec = at<smc_record>(bt, P.o_rec);
    B.part = at<Partial>(bt, P.o_part);
    B.tsum = at<unsigned long long>(bt, P.o_tsum);
    B.fst = at<DevState>(bt, P.o_fst);
    B.bs = at<BatchState>(bt, P.o_bs);
    B.n = at<int64_t>(bt, P.o_n);
    B.off = at<int64_t>(bt, P.o_off);
    B.tfirst = at<int32_t>(bt, P.o_tfirst);
    B.sfirst = at<int32_t>(bt, P.o_sfirst);
    B.tile_filter = at<int32_t>(bt, P.o_tf);
    B.stile_filter = at<int32_t>(bt, P.o_stf);
    B.act_tiles = at<int32_t>(bt, P.o_act);
    B.act_stiles = at<int32_t>(bt, P.o_acts);
    B.obs_off = at<int64_t>(bt, P.o_obs_off);
    B.rec_off = at<int64_t>(bt, P.o_rec_off);
    B.n_iter = at<int32_t>(bt, P.o_T);
    B.stream_of = at<uint32_t>(bt, P.o_stream);
    B.mrec = at<unsigned long long>(bt, P.o_mrec);
    B.log_n = at<double>(bt, P.o_logn);
    B.neg_log_n = at<R>(bt, P.o_nlogn);
    B.obs_r = (sizeof(R) == 4) ? at<R>(bt, P.o_obs_f) : reinterpret_cast<const R *>(B.obs);
    B.frac = at<int32_t>(bt, P.o_frac);
    B.tmax = P.tmax;
    B.stratified = (g.scheme == SMC_STRATIFIED) ? 1 : 0;
    B.chunk = bt->chunk;
    return B;
}

template <typename R>
int batch_launch_iteration(smc_batch *bt, int grid) {
    const BatchArgs<R> B = batch_args<R>(bt);
    batch_pf_kernel<R><<<grid, kBlock, 0, bt->stream>>>(B);
    batch_reduce_kernel<R><<<grid, kBlock, 0, bt->stream>>>(B);
    if (B.stratified) batch_select_kernel<R, true><<<grid, kBlock, 0, bt->stream>>>(B);
    else batch_select_kernel<R, false><<<grid, kBlock, 0, bt->stream>>>(B);
    return cuda_check(cudaGetLastError());
}

int batch_iteration(smc_batch *bt, int grid) {
    return (bt->cfg.precision == 32) ? batch_launch_iteration<float>(bt, grid)
                                     : batch_launch_iteration<double>(bt, grid);
}

int batch_grid(smc_batch *bt) { return bt->grid_per_sm * bt->nsm; }

int batch_reset_and_init(smc_batch *bt) {
    const int nf = bt->P.nf;
    batch_reset_kernel<<<(nf + 255) / 256, 256, 0, bt->stream>>>(at<DevState>(bt, bt->P.o_fst), nf,
                                                                  at<BatchState>(bt, bt->P.o_bs));
    int rc = cuda_check(cudaGetLastError());
    if (rc) return rc;
    rc = batch_iteration(bt, batch_grid(bt));
    if (rc) return rc;
    bt->t_host = 0;
    bt->initialized = 1;
    return SMC_OK;
}

int batch_graph(smc_batch *bt) {
    const int grid = batch_grid(bt);
    if (bt->graph && bt->graph_grid == grid && bt->graph_chunk == bt->chunk) return SMC_OK;
    if (bt->graph) {
        cudaGraphExecDestroy(bt->graph);
        bt->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SMC_E_CUDA;
    const int rc = batch_iteration(bt, grid);
    const cudaError_t e = cudaStreamEndCapture(bt->stream, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return SMC_E_CUDA;
    }
    const cudaError_t e2 = cudaGraphInstantiate(&bt->graph, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        bt->graph = nullptr;
        return SMC_E_CUDA;
    }
    bt->graph_grid = grid;
    bt->graph_chunk = bt->chunk;
    return SMC_OK;
}

int batch_read_states(smc_batch *bt, std::vector<DevState> &h) {
    h.resize(bt->P.nf);
    int rc = cuda_check(cudaMemcpyAsync(h.data(), at<DevState>(bt, bt->P.o_fst), sizeof(DevState) * bt->P.nf,
                                        cudaMemcpyDeviceToHost, bt->stream));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(bt->stream));
    if (rc) return rc;
    for (const DevState &d : h)
        if (d.error) return d.error;
    return SMC_OK;
}

}  // namespace

extern "C" {

size_t smc_batch_workspace_bytes(const smc_config *cfg, const int64_t *n, const int32_t *T, int32_t nf) {
    BatchPlan P;
    if (!batch_plan(cfg, n, T, nf, P)) return 0;
    return P.total;
}

int smc_batch_create(smc_batch **out, const smc_config *cfg, const int64_t *n, const int32_t *T, int32_t nf,
                     void *d_ws, size_t bytes, void *cuda_stream) {
    if (!out) return SMC_E_ARG;
    *out = nullptr;
    smc_batch *bt = new (std::nothrow) smc_batch();
    if (!bt) return SMC_E_ARG;
    if (!batch_plan(cfg, n, T, nf, bt->P)) {
        delete bt;
        return SMC_E_ARG;
    }
    const BatchPlan &P = bt->P;
    if (!d_ws || bytes < P.total || ((uintptr_t)d_ws & (kAlign - 1))) {
        delete bt;
        return SMC_E_WORKSPACE;
    }
    bt->cfg = *cfg;
    bt->ws = static_cast<char *>(d_ws);
    bt->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&bt->device);
    cudaDeviceGetAttribute(&bt->nsm, cudaDevAttrMultiProcessorCount, bt->device);
    bt->grid_per_sm = 4;
    bt->chunk = 1;
    bt->graph = nullptr;
    bt->graph_grid = 0;
    bt->t_host = -1;
    bt->initialized = 0;
    bt->inv.resize(nf);
    for (int32_t i = 0; i < nf; ++i) bt->inv[P.perm[i]] = i;
    auto up = [&](size_t o, const void *src, size_t nbytes) {
        return cuda_check(cudaMemcpyAsync(bt->ws + o, src, nbytes, cudaMemcpyHostToDevice, bt->stream));
    };
    int rc = cuda_check(cudaMemsetAsync(bt->ws, 0, P.o_x, bt->stream));
    if (!rc) rc = up(P.o_n, P.n.data(), 8 * (size_t)nf);
    if (!rc) rc = up(P.o_off, P.off.data(), 8 * (size_t)nf);
    if (!rc) rc = up(P.o_obs_off, P.obs_off.data(), 8 * (size_t)nf);
    if (!rc) rc = up(P.o_rec_off, P.rec_off.data(), 8 * (size_t)nf);
    if (!rc) rc = up(P.o_T, P.T.data(), 4 * (size_t)nf);
    if (!rc) rc = up(P.o_tfirst, P.tfirst.data(), 4 * (size_t)(nf + 1));
    if (!rc) rc = up(P.o_sfirst, P.sfirst.data(), 4 * (size_t)(nf + 1));
    if (!rc) rc = up(P.o_tf, P.tile_filter.data(), 4 * (size_t)P.ntiles);
    if (!rc) rc = up(P.o_stf, P.stile_filter.data(), 4 * (size_t)P.nstiles);
    if (!rc) rc = up(P.o_act, P.act_tiles.data(), 4 * (size_t)P.tmax);
    if (!rc) rc = up(P.o_acts, P.act_stiles.data(), 4 * (size_t)P.tmax);
    if (!rc) rc = up(P.o_stream, P.stream_of.data(), 4 * (size_t)nf);
    if (!rc) rc = up(P.o_mrec, P.mrec.data(), 8 * (size_t)nf);
    if (!rc) rc = up(P.o_logn, P.log_n.data(), 8 * (size_t)nf);
    std::vector<double> nl64(nf);
    std::vector<float> nl32(nf);
    for (int32_t i = 0; i < nf; ++i) {
        nl64[i] = -P.log_n[i];
        nl32[i] = (float)nl64[i];
    }
    if (!rc) rc = (P.rsize == 4) ? up(P.o_nlogn, nl32.data(), 4 * (size_t)nf) : up(P.o_nlogn, nl64.data(), 8 * (size_t)nf);
    if (!rc) rc = up(P.o_frac, P.frac.data(), 4 * (size_t)nf);
    if (!rc) rc = cuda_check(cudaStreamSynchronize(bt->stream));
    if (rc) {
        delete bt;
        return rc;
    }
    *out = bt;
    return SMC_OK;
}

int smc_batch_destroy(smc_batch *bt) {
    if (!bt) return SMC_E_ARG;
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    delete bt;
    return SMC_OK;
}

int smc_batch_set_streams(smc_batch *bt, const uint32_t *stream_ids) {
    if (!bt || !stream_ids) return SMC_E_ARG;
    for (int32_t f = 0; f < bt->P.nf; ++f) bt->P.stream_of[bt->inv[f]] = stream_ids[f];
    int rc = cuda_check(cudaMemcpyAsync(bt->ws + bt->P.o_stream, bt->P.stream_of.data(), 4 * (size_t)bt->P.nf,
                                        cudaMemcpyHostToDevice, bt->stream));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(bt->stream));  // the host vector may change again
    return rc;
}

int smc_batch_set_data(smc_batch *bt, int32_t filter, const double *obs, int on_device) {
    if (!bt || !obs || filter < 0 || filter >= bt->P.nf) return SMC_E_ARG;
    const int32_t i = bt->inv[filter];
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    double *dst = at<double>(bt, bt->P.o_obs) + 2 * bt->P.obs_off[i];
    int rc = cuda_check(cudaMemcpyAsync(dst, obs, 16 * (size_t)bt->P.T[i], k, bt->stream));
    if (!rc && bt->P.rsize == 4) {
        const int64_t m = 2 * (int64_t)bt->P.T[i];
        to_float_kernel<<<(unsigned)((m + 255) / 256), 256, 0, bt->stream>>>(
            dst, at<float>(bt, bt->P.o_obs_f) + 2 * bt->P.obs_off[i], m);
        rc = cuda_check(cudaGetLastError());
    }
    if (!rc && !on_device) rc = cuda_check(cudaStreamSynchronize(bt->stream));
    return rc;
}

int smc_batch_initialize(smc_batch *bt) {
    if (!bt) return SMC_E_ARG;
    return batch_reset_and_init(bt);
}

int smc_batch_iterate(smc_batch *bt, int32_t n) {
    if (!bt || n < 0) return SMC_E_ARG;
    if (!bt->initialized) return SMC_E_STATE;
    if (bt->t_host + n > bt->P.tmax - 1) return SMC_E_ARG;
    const bool use_graph = bt->stream != nullptr;
    if (use_graph) {
        int rc = batch_graph(bt);
        if (rc) return rc;
        for (int32_t i = 0; i < n; ++i)
            if (cudaGraphLaunch(bt->graph, bt->stream) != cudaSuccess) return SMC_E_CUDA;
    } else {
        for (int32_t i = 0; i < n; ++i) {
            int rc = batch_iteration(bt, batch_grid(bt));
            if (rc) return rc;
        }
    }
    bt->t_host += n;
    return SMC_OK;
}

int smc_batch_run(smc_batch *bt) {
    if (!bt) return SMC_E_ARG;
    int rc = batch_reset_and_init(bt);
    if (rc) return rc;
    return smc_batch_iterate(bt, bt->P.tmax - 1);
}

int smc_batch_tune(smc_batch *bt, int32_t *blocks_per_sm, int32_t *tiles_per_item) {
    if (!bt) return SMC_E_ARG;
    // the launch shape of the persistent kernels: resident blocks per SM and
    // consecutive tiles per work item (the tile itself, the plain move
    // kernel's tile of the same precision, fixes the reduction order that
    // makes every filter bit-identical to its plain run)
    const int cand_g[6] = {1, 2, 3, 4, 6, 8};
    const int cand_c[3] = {1, 2, 4};
    float best = 1e30f;
    int best_g = bt->grid_per_sm, best_c = bt->chunk;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SMC_E_CUDA;
    const int reps = std::min(10, bt->P.tmax - 1);
    for (int c : cand_c) {
        for (int g : cand_g) {
            bt->grid_per_sm = g;
            bt->chunk = c;
            int rc = batch_reset_and_init(bt);
            if (rc) return rc;
            cudaEventRecord(e0, bt->stream);
            for (int r = 0; r < reps; ++r)
                if ((rc = batch_iteration(bt, batch_grid(bt)))) return rc;
            cudaEventRecord(e1, bt->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) return SMC_E_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_g = g;
                best_c = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bt->grid_per_sm = best_g;
    bt->chunk = best_c;
    if (blocks_per_sm) *blocks_per_sm = best_g;
    if (tiles_per_item) *tiles_per_item = best_c;
    return batch_reset_and_init(bt);
}

int smc_batch_log_evidence(smc_batch *bt, double *h_out) {
    if (!bt || !h_out) return SMC_E_ARG;
    std::vector<DevState> h;
    const int rc = batch_read_states(bt, h);
    for (int32_t f = 0; f < bt->P.nf; ++f) h_out[f] = h.empty() ? 0.0 : h[bt->inv[f]].log_evidence;
    return rc;
}

int smc_batch_read_history(smc_batch *bt, int32_t filter, smc_record *hr, int32_t count, int32_t *n_written) {
    if (!bt || !hr || count < 0 || filter < 0 || filter >= bt->P.nf) return SMC_E_ARG;
    std::vector<DevState> h;
    const int rc = batch_read_states(bt, h);
    if (rc && rc != SMC_E_NONFINITE) return rc;
    const int32_t i = bt->inv[filter];
    const int32_t last = h[i].t;
    const int32_t m = std::min(count, last + 1);
    if (m > 0) {
        const int rc2 = cuda_check(cudaMemcpyAsync(hr, at<smc_record>(bt, bt->P.o_rec) + bt->P.rec_off[i] + (last - m + 1),
                                                   sizeof(smc_record) * (size_t)m, cudaMemcpyDeviceToHost, bt->stream));
        if (rc2) return rc2;
        if (cudaStreamSynchronize(bt->stream) != cudaSuccess) return SMC_E_CUDA;
    }
    if (n_written) *n_written = std::max(m, 0);
    return rc;
}

int smc_batch_read_state(smc_batch *bt, int32_t filter, void *dst, int on_device) {
    if (!bt || !dst || filter < 0 || filter >= bt->P.nf) return SMC_E_ARG;
    std::vector<DevState> h;
    const int rc = batch_read_states(bt, h);
    if (rc && rc != SMC_E_NONFINITE) return rc;
    const BatchPlan &P = bt->P;
    const int32_t i = bt->inv[filter];
    const size_t rs = P.rsize;
    const char *base = bt->ws + P.o_x + (size_t)(h[i].cur & 1) * 4 * P.ntot * rs + (size_t)P.off[i] * rs;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    int rc2 = copy_pitched(dst, (size_t)P.n[i] * rs, base, (size_t)P.ntot * rs, (size_t)P.n[i] * rs, 4, k, bt->stream);
    if (!rc2) rc2 = cuda_check(cudaStreamSynchronize(bt->stream));
    return rc2 ? rc2 : rc;
}

}  // extern "C"

// ============================================================ gradient ==

namespace {

// digamma by upward recurrence to x >= 6, then the asymptotic series
// psi(x) ~ ln x - 1/(2x) - sum_k B_2k / (2k x^2k)
double digamma_host(double x) {
    double r = 0.0;
    while (x < 6.0) {
        r -= 1.0 / x;
        x += 1.0;
    }
    const double f = 1.0 / (x * x);
    return r + std::log(x) - 0.5 / x -
           f * (1.0 / 12 - f * (1.0 / 120 - f * (1.0 / 252 - f * (1.0 / 240 - f * (1.0 / 132)))));
}

template <typename R>
void set_slots(PfArgs<R> &a, const char *src, char *dst, int64_t ld) {
    for (int r = 0; r < 4; ++r) {
        a.x[0][r] = reinterpret_cast<R *>(const_cast<char *>(src)) + (size_t)r * ld;
        a.x[1][r] = reinterpret_cast<R *>(dst) + (size_t)r * ld;
    }
    a.lw[0] = reinterpret_cast<R *>(const_cast<char *>(src)) + (size_t)4 * ld;
    a.lw[1] = reinterpret_cast<R *>(dst) + (size_t)4 * ld;
}

// resampling decisions of the recorded run (host copy), T = t_host + 1
int recorded_flags(smc_ctx *c, std::vector<int> &flags) {
    const int32_t T = c->t_host + 1;
    if (T < 1 || T > c->cfg.max_records) return SMC_E_STATE;
    std::vector<smc_record> h(T);
    int32_t nw = 0;
    const int rc = smc_read_history(c, h.data(), T, &nw);
    if (rc) return rc;
    if (nw != T) return SMC_E_STATE;
    flags.resize(T);
    for (int32_t t = 0; t < T; ++t) flags[t] = h[t].resampled;
    return SMC_OK;
}

double *scal(smc_ctx *c) { return reinterpret_cast<double *>(c->ws + c->L.scal); }

template <typename R>
int pf_replay_impl(smc_ctx *c, const double th[4], double *h_out) {
    std::vector<int> flags;
    int rc = recorded_flags(c, flags);
    if (rc) return rc;
    const int32_t T = c->t_host + 1;
    PfArgs<R> a = pf_args<R>(c);
    a.sd_pos = R(th[0]);
    a.sd_vel = R(th[1]);
    set_obs_params(a, th[2], th[3], c->cfg.model == SMC_MODEL_CV_GAUSS);
    a.part = reinterpret_cast<Partial *>(c->ws + c->L.rep_part);
    double *sc = scal(c);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(sc + 16);
    if ((rc = cuda_check(cudaMemsetAsync(sc, 0, 256, c->stream)))) return rc;
    char *rep[2] = {c->ws + c->L.rep, c->ws + c->L.rep + 5 * row_bytes(c)};
    const int32_t *hist = reinterpret_cast<const int32_t *>(c->ws + c->L.hist);
    for (int32_t t = 0; t < T; ++t) {
        set_slots<R>(a, rep[(t + 1) & 1], rep[t & 1], c->L.ld);
        const int gather = (t > 0 && flags[t - 1]) ? 1 : 0;
        a.anc = gather ? hist + (size_t)(t - 1) * c->L.ld : c->anc;
        pf_replay_kernel<R><<<(unsigned)c->L.nbw, kBlock, 0, c->stream>>>(a, t, gather, sc + 2 + ((t + 1) & 1),
                                                                           sc + 2 + (t & 1), sc + 4, ticket);
        if ((rc = cuda_check(cudaGetLastError()))) return rc;
    }
    if ((rc = cuda_check(cudaMemcpyAsync(h_out, sc + 4, 8, cudaMemcpyDeviceToHost, c->stream)))) return rc;
    return cuda_check(cudaStreamSynchronize(c->stream));
}

template <typename R>
int pf_grad_impl(smc_ctx *c, double *grad) {
    std::vector<int> flags;
    int rc = recorded_flags(c, flags);
    if (rc) return rc;
    const int32_t T = c->t_host + 1;
    const int64_t n = c->cfg.n_particles, ld = c->L.ld;
    const int ck = c->L.ck;
    PfArgs<R> a = pf_args<R>(c);
    a.part = reinterpret_cast<Partial *>(c->ws + c->L.rep_part);
    double *sc = scal(c);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(sc + 16);
    if ((rc = cuda_check(cudaMemsetAsync(sc, 0, 256, c->stream)))) return rc;
    const int32_t *hist = reinterpret_cast<const int32_t *>(c->ws + c->L.hist);
    float *gb[2] = {reinterpret_cast<float *>(c->ws + c->L.gbar), reinterpret_cast<float *>(c->ws + c->L.gbar) + ld};
    R *xb = reinterpret_cast<R *>(c->ws + c->L.xbar);
    R *atb = reinterpret_cast<R *>(c->ws + c->L.at);
    auto slot = [&](int64_t s, int k) -> char * {
        return k == 0 ? ckpt_slot(c, s) : c->ws + c->L.seg + (size_t)k * 5 * row_bytes(c);
    };
    AdjArgs<R> g;
    g.n = n;
    g.ld = ld;
    g.obs = c->obs;
    g.rec = c->rec;
    g.rec_cap = c->cfg.max_records;
    g.grad = sc + 8;
    g.part = a.part;
    g.ticket = ticket;
    const double s = c->cfg.cv.obs_scale, nu = c->cfg.cv.obs_df;
    g.delta = R(c->cfg.cv.delta);
    g.inv_scale = R(1.0 / s);
    g.scale = R(s);
    g.nu = R(nu);
    g.inv_nu = R(1.0 / nu);
    g.half_nu1 = R(0.5 * (nu + 1.0));
    g.dnu_const = R(0.5 * (digamma_host(0.5 * (nu + 1.0)) - digamma_host(0.5 * nu)) - 0.5 / nu);
    g.gaussian = (c->cfg.model == SMC_MODEL_CV_GAUSS) ? 1 : 0;
    g.key = key_of(c);
    g.stream = c->cfg.stream_id;
    const int64_t nseg = (T + ck - 1) / ck;
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
        const int32_t t0 = (int32_t)(sg * ck), t1 = std::min<int32_t>(t0 + ck, T);
        // recompute iterations t0 + 1 .. t1 - 1 from the checkpoint at t0
        for (int32_t t = t0 + 1; t < t1; ++t) {
            set_slots<R>(a, slot(sg, t - 1 - t0), slot(sg, t - t0), ld);
            const int gather = flags[t - 1] ? 1 : 0;
            a.anc = gather ? hist + (size_t)(t - 1) * ld : c->anc;
            pf_replay_kernel<R><<<(unsigned)c->L.nbw, kBlock, 0, c->stream>>>(
                a, t, gather, &c->rec[(t - 1) % c->cfg.max_records].log_norm, sc + 20, sc + 21, ticket);
            if ((rc = cuda_check(cudaGetLastError()))) return rc;
        }
        // reverse sweep through the segment
        for (int32_t t = t1 - 1; t >= t0; --t) {
            const char *sl = slot(sg, t - t0);
            g.x = reinterpret_cast<const R *>(sl);
            g.lw = reinterpret_cast<const R *>(sl) + 4 * ld;
            g.gbar_next = gb[(t + 1) & 1];
            g.gbar = gb[t & 1];
            g.xbar_f = (t == T - 1) ? nullptr : xb;
            g.at = atb;
            g.S_next_in = sc + ((t + 1) & 1);
            g.S_out = sc + (t & 1);
            g.t = t;
            g.last = (t == T - 1) ? 1 : 0;
            pf_adjoint_kernel<R><<<(unsigned)c->L.nbw, kBlock, 0, c->stream>>>(g);
            if ((rc = cuda_check(cudaGetLastError()))) return rc;
            if (t > 0) {
                if (flags[t - 1]) {
                    pf_parent_gather_kernel<R><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, c->stream>>>(
                        hist + (size_t)(t - 1) * ld, atb, xb, n, ld);
                    if ((rc = cuda_check(cudaGetLastError()))) return rc;
                } else {
                    std::swap(xb, atb);  // identity ancestry: the parent adjoint is A^T xbar itself
                }
            }
        }
    }
    if ((rc = cuda_check(cudaMemcpyAsync(grad, sc + 8, 32, cudaMemcpyDeviceToHost, c->stream)))) return rc;
    return cuda_check(cudaStreamSynchronize(c->stream));
}

}  // namespace

extern "C" {

int smc_pf_grad(smc_ctx *c, double grad[4]) {
    if (!c || !grad) return SMC_E_ARG;
    if (!recording(c) || !c->initialized) return SMC_E_STATE;
    const int rc = read_state(c);
    if (rc) return rc;
    return (c->cfg.precision == 32) ? pf_grad_impl<float>(c, grad) : pf_grad_impl<double>(c, grad);
}

int smc_pf_replay(smc_ctx *c, const double theta[4], double *h_log_evidence) {
    if (!c || !theta || !h_log_evidence) return SMC_E_ARG;
    if (!recording(c) || !c->initialized) return SMC_E_STATE;
    if (!(theta[2] > 0) || !(theta[3] > 0)) return SMC_E_ARG;
    const int rc = read_state(c);
    if (rc) return rc;
    return (c->cfg.precision == 32) ? pf_replay_impl<float>(c, theta, h_log_evidence)
                                    : pf_replay_impl<double>(c, theta, h_log_evidence);
}

int smc_read_ancestor_history(smc_ctx *c, int32_t t, int32_t *dst, int on_device) {
    if (!c || !dst || t < 0) return SMC_E_ARG;
    if (!recording(c) || t > c->t_host) return SMC_E_STATE;
    const int32_t *src = reinterpret_cast<const int32_t *>(c->ws + c->L.hist) + (size_t)t * c->L.ld;
    return copy_out(c, dst, src, (size_t)c->cfg.n_particles * 4, on_device);
}

}  // extern "C"

// ========================================= resampling without allocation ==
//
// smc_resample_systematic_noalloc: systematic ancestors straight from a
// caller's log-weights, for callers that must not allocate device memory.
// Its scratch (a state block for the kernels, the per-tile sums of the
// fixed-point weights, the running maximum) is one file-scope device array
// of fixed size, so the entry point calls no allocator; the price is a size
// limit and one shared scratch area per device.

namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 22;                    // particles per call
constexpr int kNoAllocMaxTiles = (int)(kNoAllocMaxN / kScanTile);     // 2048 scan tiles
struct NoAllocScratch {
    DevState st;
    unsigned long long tsum[kNoAllocMaxTiles];
    int max_key;
    int nan_seen;  // a NaN log-weight was read (the maximum alone would drop it)
};
// every GPU that loads the library holds this array (about 17 KB) until exit
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// device address of the array, per device: looked up once per device
// (concurrent first calls from several host threads store the same value)
std::atomic<NoAllocScratch *> g_noalloc_ptr[64];

// one-time set-up on the current device: the array's device address (in
// host code its name is only a host-side stand-in)
int noalloc_scratch(NoAllocScratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SMC_E_CUDA;
    NoAllocScratch *p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void *q = nullptr;
        if (cudaGetSymbolAddress(&q, g_noalloc_scratch) != cudaSuccess || !q) return SMC_E_CUDA;
        p = static_cast<NoAllocScratch *>(q);
        g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return SMC_OK;
}

// float keys that order like the floats (for an integer atomicMax)
__device__ __forceinline__ int float_key(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// clear the shared scratch for this call: state block, running maximum and
// the NaN flag
__global__ void noalloc_clear_kernel(NoAllocScratch *s, int32_t t) {
    DevState *st = &s->st;
    const int W = (int)(sizeof(DevState) / 4);
    for (int i = threadIdx.x; i < W; i += blockDim.x) reinterpret_cast<uint32_t *>(st)[i] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        st->t = t;
        st->due = 1;
        s->max_key = float_key(-INFINITY);
        s->nan_seen = 0;
    }
}

__global__ void __launch_bounds__(kBlock) noalloc_max_kernel(const float *lw, int64_t n, NoAllocScratch *s) {
    float m = -INFINITY;
    bool nan = false;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
        const float v = lw[i];
        nan |= (v != v);
        m = fmaxf(m, v);
    }
    m = warp_maxf(m);
    if (__any_sync(0xffffffffu, nan) && (threadIdx.x & 31) == 0) s->nan_seen = 1;
    if ((threadIdx.x & 31) == 0) atomicMax(&s->max_key, float_key(m));
}

// a NaN or a maximum that is not finite: the call fails like the context
// API's weighting step (SMC_E_NONFINITE) and the later kernels write nothing
__global__ void noalloc_set_max_kernel(NoAllocScratch *s) {
    const float m = key_float(s->max_key);
    s->st.max_lw = (double)m;
    s->st.max_lw_f = m;
    if (s->nan_seen || !(m > -INFINITY) || !(m < INFINITY)) s->st.error = SMC_E_NONFINITE;
}

}  // namespace

extern "C" int smc_resample_systematic_noalloc(const float *d_log_weight, int64_t n, uint64_t seed, uint32_t stream_id,
                                               int32_t t, int32_t *d_ancestors, void *cuda_stream) {
    if (!d_log_weight || !d_ancestors || n < 1 || t < 0) return SMC_E_ARG;
    if (n > kNoAllocMaxN) return SMC_E_ARG;  // beyond the fixed scratch
    if (((uintptr_t)d_log_weight & 15) || ((uintptr_t)d_ancestors & 3)) return SMC_E_ARG;
    NoAllocScratch *s = nullptr;
    int rc = noalloc_scratch(&s);
    if (rc) return rc;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    DevState *st = &s->st;
    const unsigned tiles = (unsigned)((n + kScanTile - 1) / kScanTile);
    noalloc_clear_kernel<<<1, kBlock, 0, stream>>>(s, t);
    noalloc_max_kernel<<<std::min<unsigned>(tiles * 4, 1184u), kBlock, 0, stream>>>(d_log_weight, n, s);
    noalloc_set_max_kernel<<<1, 1, 0, stream>>>(s);
    if ((rc = cuda_check(cudaGetLastError()))) return rc;
    QGen<float> qg;
    qg.lw[0] = qg.lw[1] = d_log_weight;
    qg.frac = 61 - ceil_log2(n);
    qg.cur_lw = nullptr;
    qg.m = 0;
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    tile_reduce_kernel<QGen<float>><<<tiles, kBlock, 0, stream>>>(qg, n, s->tsum, nullptr, &st->scan_ticket[SLOT_CDF],
                                                                   st, 1);
    GridTargets<false> tg{};
    tg.n = n;
    tg.key = key;
    tg.stream = stream_id;
    tg.mrec = ~0ull / (unsigned long long)n;
    scan_select_kernel<QGen<float>, GridTargets<false>, AncOut, NoSink><<<tiles, kBlock, 0, stream>>>(
        qg, tg, AncOut{d_ancestors}, NoSink{}, n, s->tsum, nullptr, st, 1,
        0);
    return cuda_check(cudaGetLastError());
}

extern "C" int smc_resample_noalloc_status(void *cuda_stream, int32_t *h_status) {
    if (!h_status) return SMC_E_ARG;
    NoAllocScratch *s = nullptr;
    int rc = noalloc_scratch(&s);
    if (rc) return rc;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    int32_t v = 0;
    if ((rc = cuda_check(cudaMemcpyAsync(&v, &s->st.error, sizeof(v), cudaMemcpyDeviceToHost, stream)))) return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(stream)))) return rc;
    *h_status = v;
    return SMC_OK;
}
