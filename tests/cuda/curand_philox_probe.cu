// Test probe: evaluates the CUDA toolkit's own Philox4x32-10 device function
// (curand_Philox4x32_10 from curand_philox4x32_x.h, called, not copied) on
// given counters and keys, so the tests can compare it with the oracle's and
// the library's independently written Philox.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void probe_kernel(const uint4 *ctr, const uint2 *key, uint4 *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int probe_curand_philox(const uint32_t *h_ctr, const uint32_t *h_key, uint32_t *h_out,
                                   int n) {
    uint4 *d_ctr = nullptr, *d_out = nullptr;
    uint2 *d_key = nullptr;
    if (cudaMalloc(&d_ctr, n * sizeof(uint4)) || cudaMalloc(&d_out, n * sizeof(uint4)) ||
        cudaMalloc(&d_key, n * sizeof(uint2)))
        return -1;
    cudaMemcpy(d_ctr, h_ctr, n * sizeof(uint4), cudaMemcpyHostToDevice);
    cudaMemcpy(d_key, h_key, n * sizeof(uint2), cudaMemcpyHostToDevice);
    probe_kernel<<<(n + 127) / 128, 128>>>(d_ctr, d_key, d_out, n);
    cudaError_t e = cudaMemcpy(h_out, d_out, n * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(d_ctr);
    cudaFree(d_out);
    cudaFree(d_key);
    return e == cudaSuccess ? 0 : -2;
}
