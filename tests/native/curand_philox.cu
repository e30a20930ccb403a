// Test helper: NVIDIA's own Philox4x32-10 (cuRAND's device function curand_Philox4x32_10),
// evaluated on the GPU for a list of (counter, key) pairs, as an independent implementation
// to check the CPU oracle's Philox against.  Built by tests/test_gpu_curand_philox.py.
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdint>

__global__ void philox_blocks(const uint4 *ctr, const uint2 *key, uint4 *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

// ctr: host uint32 [n][4], key: host uint32 [n][2], out: host uint32 [n][4]; returns 0 on success
extern "C" int curand_philox_blocks(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n)
{
    uint4 *dc = nullptr, *dout = nullptr;
    uint2 *dk = nullptr;
    cudaError_t e = cudaMalloc(&dc, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(uint2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        philox_blocks<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return e == cudaSuccess ? 0 : int(e);
}
