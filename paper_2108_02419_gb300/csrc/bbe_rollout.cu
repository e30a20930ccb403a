// bbe_rollout.cu -- the probability finalisers of the rollout counts: win probabilities and
// odds (the dry-run estimate p_c = count_c / R of Section 3, decimal odds 1 / p_c) and place
// probabilities.
// (The rollout kernels themselves, win and place counts, are in bbe_win.cuh.)
//
// Each is one binary32 round-to-nearest division per output, so the results are bit-identical
// to any implementation of the same definition.
#include <cuda_runtime.h>

#include "bbe_internal.h"

namespace bbe {

namespace {

__global__ void win_probs_kernel(DevBatch b, const int32_t *__restrict__ counts, float *__restrict__ probs,
                                 float *__restrict__ odds)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n_total) return;
    const int r = b.comp_race[i];
    const float p = __fdiv_rn(__int2float_rn(counts[i]), __ll2float_rn(b.R[r]));
    probs[i] = p;
    if (odds) odds[i] = __fdiv_rn(1.0f, p);
}

// probs[i] = (sum of place counts of competitor i over places 0 .. top-1) / R of its race
__global__ void place_probs_kernel(DevBatch b, int places, const int32_t *__restrict__ counts, int top,
                                   float *__restrict__ probs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n_total) return;
    int64_t s = 0;
    for (int j = 0; j < top; ++j) s += counts[int64_t(i) * places + j];
    probs[i] = __fdiv_rn(__ll2float_rn(s), __ll2float_rn(b.R[b.comp_race[i]]));
}

}  // namespace

cudaError_t launch_place_probs(const DevBatch &b, int places, const int32_t *counts, int top, float *probs,
                               cudaStream_t stream)
{
    const int threads = 256;
    const int blocks = (b.n_total + threads - 1) / threads;
    if (blocks > 0) place_probs_kernel<<<blocks, threads, 0, stream>>>(b, places, counts, top, probs);
    return cudaGetLastError();
}

cudaError_t launch_win_probs(const DevBatch &b, const int32_t *counts, float *probs, float *odds,
                             cudaStream_t stream)
{
    const int threads = 256;
    const int blocks = (b.n_total + threads - 1) / threads;
    if (blocks > 0) win_probs_kernel<<<blocks, threads, 0, stream>>>(b, counts, probs, odds);
    return cudaGetLastError();
}

}  // namespace bbe
