// Test helper: the library's Box-Muller radius (bbe_rng.cuh: bm_radius2, which takes its square
// root with sqrt_f32x2) for every one of the 2^24 first words a Philox block can give it
// (wa >> 8 = m for m = 0 .. 2^24 - 1), and the same radius with the IEEE square root
// (__fsqrt_rn) of the same argument.  Built by tests/test_gpu_radius.py.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../paper_2108_02419_gb300/csrc/bbe_rng.cuh"

__global__ void radii(float *ours, float *ieee, uint32_t n)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;  // even: one pair per thread
    const uint32_t m = 2u * i;
    if (m + 1u >= n + 1u) return;
    const float2 r = bbe::bm_radius2(m << 8, (m + 1u) << 8);
    ours[m] = r.x;
    ours[m + 1u] = r.y;
    const float2 u1 = __fmul2_rn(make_float2(__uint2float_rn(m + 1u), __uint2float_rn(m + 2u)), bbe::splat2(0x1p-24f));
    const float2 m2l = __fmul2_rn(bbe::splat2(-2.0f), bbe::log_f32x2(u1));
    ieee[m] = __fsqrt_rn(m2l.x);
    ieee[m + 1u] = __fsqrt_rn(m2l.y);
}

// ours, ieee: host float[2^24]; returns 0 on success
extern "C" int bm_radii(float *ours, float *ieee)
{
    const uint32_t n = 1u << 24;
    float *d_ours = nullptr, *d_ieee = nullptr;
    cudaError_t e = cudaMalloc(&d_ours, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_ieee, sizeof(float) * n);
    if (e == cudaSuccess) {
        radii<<<(n / 2 + 255) / 256, 256>>>(d_ours, d_ieee, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(ours, d_ours, sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ieee, d_ieee, sizeof(float) * n, cudaMemcpyDeviceToHost);
    cudaFree(d_ours);
    cudaFree(d_ieee);
    return e == cudaSuccess ? 0 : int(e);
}
