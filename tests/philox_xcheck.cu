// Test helper: Philox4x32-10 words from cuRAND's device implementation
// (curand_Philox4x32_10), for comparing the oracle's Philox against a library.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_curand_philox(const uint4* ctr, const uint2* key, uint4* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

// ctr: n x 4 words, key: n x 2 words, out: n x 4 words (host buffers); returns a cudaError_t.
extern "C" int curand_philox_words(const unsigned* ctr, const unsigned* key, unsigned* out, int n) {
    uint4 *dc = nullptr, *dout = nullptr;
    uint2* dk = nullptr;
    cudaError_t e = cudaMalloc(&dc, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(uint2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_curand_philox<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return (int)e;
}
