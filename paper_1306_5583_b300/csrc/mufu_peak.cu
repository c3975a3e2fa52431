// Measured issue rate of the special-function (MUFU) pipe on the current
// device, the roofline denominator of the likelihood-bound GMM moves.
//
// Every thread runs kChains independent dependency chains of alternating
// base-2 exponentials and logarithms (ex2.approx / lg2.approx in inline PTX,
// so the compiler can neither fold nor reorder them: x -> 2^x -> log2 2^x
// keeps every value near 0.5).  With enough warps in flight the chains hide
// the pipe latency and the kernel runs at the pipe's throughput.  The rate
// is reported as MUFU operations per second; divided by the SM count and the
// SM clock sampled meanwhile it gives operations per clock per SM.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2a(float x) {
    float y;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// kind 0: alternating ex2 / lg2 (x -> log2 2^x); 1: ex2 alone (x -> 2^(-x/2),
// one FMA-pipe multiply per operation); 2: lg2 alone (x -> log2 x + 2, one
// FMA-pipe add per operation).  Two MUFU operations per chain and round.
template <int kKind>
__global__ void __launch_bounds__(256) mufu_chains_kernel(int32_t iters, float *sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 1e-3f * (float)c + 1e-7f * (float)threadIdx.x;
    for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (kKind == 0) x[c] = lg2a(ex2a(x[c]));
            else if (kKind == 1) x[c] = ex2a(-0.5f * ex2a(-0.5f * x[c]));
            else x[c] = lg2a(lg2a(x[c] + 2.0f) + 2.0f);
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += x[c];
    if (acc == 12345.0f) sink[blockIdx.x] = acc;  // keeps the chains live
}

}  // namespace

extern "C" {

// ops_per_s: MUFU operations per second of one launch of blocks_per_sm x SMs
// blocks of 256 threads, each thread 2 x kChains x iters operations of the
// given kind, timed with CUDA events on a private stream after one warm-up
// launch.  ms: the launch's duration.  Returns 0, or 5 when a CUDA call
// fails.
int smc_mufu_rate(int32_t kind, int32_t blocks_per_sm, int32_t iters, double *ops_per_s, double *ms) {
    if (kind < 0 || kind > 2 || blocks_per_sm < 1 || iters < 1 || !ops_per_s || !ms) return 1;
    void (*kern)(int32_t, float *) =
        kind == 0 ? mufu_chains_kernel<0> : (kind == 1 ? mufu_chains_kernel<1> : mufu_chains_kernel<2>);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 5;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 5;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *sink = nullptr;
    int rc = 0;
    const unsigned grid = (unsigned)(blocks_per_sm * sms);
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&sink, grid * sizeof(float)) != cudaSuccess) {
        rc = 5;
    } else {
        kern<<<grid, 256, 0, s>>>(iters, sink);
        cudaEventRecord(e0, s);
        kern<<<grid, 256, 0, s>>>(iters, sink);
        cudaEventRecord(e1, s);
        float t = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            rc = 5;
        } else {
            const double ops = (double)grid * 256.0 * 2.0 * kChains * (double)iters;
            *ms = t;
            *ops_per_s = ops / (t * 1e-3);
        }
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return rc;
}

}  // extern "C"
