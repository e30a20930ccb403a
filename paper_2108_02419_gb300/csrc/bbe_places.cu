// bbe_places.cu -- finishing-place counts (include/bbe.h: bbe_place_counts).
//
// Section 3 runs a race until its last competitor crosses the line and lets in-play betting
// stop earlier, for instance when the third-placed competitor crosses; place and each-way
// markets (Section 2) need the places.  Every rollout here runs until K = min(places, n)
// competitors have crossed.  All competitors keep moving under Eq. 1 until the rollout ends
// (finished ones included), and the competitors that cross in the same step are placed by
// their crossing time within the step, tau = (L - d) / S, then by index.  The first place is
// the winner of the win-probability path, on the same random stream.
//
// Layout: one competitor per lane (lane j of a segment holds competitor j for the whole
// rollout; n <= 32), floor(32 / n) segments per warp, each running its own sequence of
// rollouts of the warp's race; the step is bbe_lane.cuh's lane_step.  When the rollout ends
// lane j of the segment adds one to the count of (competitor placed j-th, place j) in a
// per-warp shared-memory table, flushed to global memory once per work item.  The step
// arithmetic is the win kernel's operation for operation (binary32 round-to-nearest
// intrinsics, compiled with --fmad=false).
#include <cuda_runtime.h>

#include <cmath>

#include "bbe_internal.h"
#include "bbe_lane.cuh"

namespace bbe {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct PlaceStage {
    float4 pq[32];  // (mu, sigma, P, theta)
    float kr[32];
    float d0[32], prev0[32];
    int cnt[32 * 32];  // [competitor][place] counts of the current work item
};

template <int DIST>
__global__ void __launch_bounds__(256) place_kernel(RolloutLaunch l)
{
    extern __shared__ PlaceStage place_stage[];
    PlaceStage &st = place_stage[threadIdx.x >> 5];
    const DevBatch &b = l.b;
    const int lane = threadIdx.x & 31;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(l.queue, 1);
        it = __shfl_sync(kFull, it, 0);
        if (it >= l.n_items) break;
        const WorkItem w = l.items[it];
        const int r = w.race;
        const int off = b.race_off[r];
        const int n = b.race_off[r + 1] - off;
        const int K = min(l.places, n);
        const int nseg = 32 / n;
        const int seg = lane / n;
        const int c = lane - seg * n;  // competitor held by this lane
        const bool lane_used = seg < nseg;
        const int segbase = seg * n;

        __syncwarp();
        if (lane < n) {
            const int ci = off + lane;
            const float mu = b.mu[ci], P = b.P[ci];
            st.pq[lane] = make_float4(mu, b.sigma[ci], P, b.theta[ci]);
            st.kr[lane] = __fmul_rn(kKappa, __fsub_rn(__fmul_rn(2.0f, b.rho[ci]), 1.0f));
            st.d0[lane] = b.d0[ci];
            st.prev0[lane] = b.prev0 ? b.prev0[ci] : __fmul_rn(mu, P);
        }
        for (int i = lane; i < n * K; i += 32) st.cnt[i] = 0;
        __syncwarp();

        const float L = b.L[r];
        const float invL = __fdiv_rn(1.0f, L);
        const uint32_t rid = b.race_ids ? uint32_t(b.race_ids[r]) : b.race_id0 + uint32_t(r);
        LaneComp cp{0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (lane_used) {
            const float4 q = st.pq[c];
            cp = LaneComp{q.x, q.y, q.z, q.w, st.kr[c]};
        }
        const int kend = w.k_begin + w.k_count;
        int k = w.k_begin + seg;
        bool active = lane_used && k < kend;
        int t = 0, placed = 0, my_order = 0;
        float d = lane_used ? st.d0[c] : INFINITY;
        float prev = lane_used ? st.prev0[c] : 0.0f;
        bool finished = false;
        float zc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        long long steps = 0;
        bool hit_limit = false;

        while (__any_sync(kFull, active)) {
            const bool running = active;
            const bool aborted = running && t >= l.max_steps;
            const float S = lane_step<DIST>(d, prev, cp, n, segbase, lane_used, running, c, t, uint32_t(k), rid, invL, zc,
                                            l.round_key);
            const float dn = __fadd_rn(d, S);
            bool fin = running && !aborted && !finished && dn >= L;
            // this step's finishers of each segment, earliest crossing first
            const float tau = fin ? __fdiv_rn(__fsub_rn(L, d), S) : INFINITY;
            while (__any_sync(kFull, fin)) {
                float best = INFINITY;
                int bc = -1;
                for (int j = 0; j < n; ++j) {
                    const int src = lane_used ? segbase + j : lane;
                    const float tj = __shfl_sync(kFull, fin ? tau : INFINITY, src);
                    if (tj < best) {
                        best = tj;
                        bc = j;
                    }
                }
                if (bc >= 0) {
                    if (c == placed && placed < K) my_order = bc;
                    ++placed;
                    if (c == bc) {
                        finished = true;
                        fin = false;
                    }
                }
            }
            if (running) {
                if (placed >= K || aborted) {
                    if (!aborted && c < K) atomicAdd(&st.cnt[my_order * K + c], 1);
                    if (c == 0) steps += aborted ? t : t + 1;
                    hit_limit |= aborted;
                    k += nseg;
                    active = k < kend;
                    t = 0;
                    placed = 0;
                    finished = false;
                    d = st.d0[c];
                    prev = st.prev0[c];
                } else {
                    d = dn;
                    prev = S;
                    ++t;
                }
            }
        }
        // one flush per work item
        __syncwarp();
        for (int i = lane; i < n * K; i += 32) {
            const int v = st.cnt[i];
            if (v != 0) atomicAdd(&l.counts[(off + i / K) * l.places + i % K], v);
        }
        unsigned long long stp = (unsigned long long)steps;
        for (int o = 16; o > 0; o >>= 1) stp += __shfl_xor_sync(kFull, stp, o);
        if (lane == 0 && l.steps != nullptr) atomicAdd(&l.steps[r], stp);
        if (__any_sync(kFull, hit_limit) && lane == 0) atomicOr(l.status, kStatusStepLimit);
    }
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

cudaError_t launch_places(RolloutLaunch l, int num_sms, cudaStream_t stream)
{
    const int block = 256;
    const size_t smem = size_t(block / 32) * sizeof(PlaceStage);
    int nb = 1;
    cudaError_t e = cudaSuccess;
    switch (l.b.dist) {
    case BBE_DIST_NORMAL:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, place_kernel<BBE_DIST_NORMAL>, block, smem);
        break;
    case BBE_DIST_UNIFORM:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, place_kernel<BBE_DIST_UNIFORM>, block, smem);
        break;
    default:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, place_kernel<BBE_DIST_TWO_POINT>, block, smem);
        break;
    }
    if (e != cudaSuccess) return e;
    l.block = block;
    l.grid = num_sms * (nb > 0 ? nb : 1);
    switch (l.b.dist) {
    case BBE_DIST_NORMAL: place_kernel<BBE_DIST_NORMAL><<<l.grid, block, smem, stream>>>(l); break;
    case BBE_DIST_UNIFORM: place_kernel<BBE_DIST_UNIFORM><<<l.grid, block, smem, stream>>>(l); break;
    default: place_kernel<BBE_DIST_TWO_POINT><<<l.grid, block, smem, stream>>>(l); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_place_probs(const DevBatch &b, int places, const int32_t *counts, int top, float *probs,
                               cudaStream_t stream)
{
    const int threads = 256;
    const int blocks = (b.n_total + threads - 1) / threads;
    if (blocks > 0) place_probs_kernel<<<blocks, threads, 0, stream>>>(b, places, counts, top, probs);
    return cudaGetLastError();
}

}  // namespace bbe
