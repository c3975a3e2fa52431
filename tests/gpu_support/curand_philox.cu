// Test-only: evaluates the CUDA toolkit's curand Philox4x32-10 device
// function (public header, called as a library routine) on given counters
// and keys, so GPU tests can cross-check libsmc's own generator.
#include <cstdint>
#include <curand_kernel.h>

__global__ void curand_philox_kernel(const uint4 *ctr, uint2 key, uint4 *out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key);
}

extern "C" int curand_philox4x32_10(const uint32_t *d_ctr, const uint32_t *key, uint32_t *d_out, int64_t n) {
    if (n <= 0) return 0;
    curand_philox_kernel<<<(unsigned)((n + 255) / 256), 256>>>(reinterpret_cast<const uint4 *>(d_ctr),
                                                                make_uint2(key[0], key[1]),
                                                                reinterpret_cast<uint4 *>(d_out), n);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
