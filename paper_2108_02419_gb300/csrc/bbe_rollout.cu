// bbe_rollout.cu -- the Monte Carlo rollout kernel and the win-probability finaliser.
//
// One warp runs the rollouts of one race at a time with competitors in lanes: a race of
// n competitors occupies a segment of n lanes, and a warp packs floor(32 / n) segments,
// each running its own sequence of rollouts of the same race (Section 3 dry-runs).
// Warps pull work items (race, rollout range) from a global queue: one persistent launch
// covers races of any size mix.  Per step every lane evaluates Eq. 1 for its competitor:
// the nearest competitor strictly in front (i+) comes from warp shuffles over the
// segment, finishing is detected with a ballot, and the winner (least within-step
// crossing time, lowest index on ties) by a shuffle reduction.  Win counts stay in
// registers (lane c of a segment counts competitor c) and are reduced once per work item.
//
// The arithmetic is pinned to binary32 round-to-nearest with explicit intrinsics, and this
// file is compiled with --fmad=false, so the counts are bit-identical to any
// implementation that follows the same operation order.
#include <cuda_runtime.h>

#include <cmath>

#include "bbe_internal.h"
#include "bbe_rng.cuh"

namespace bbe {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int DIST>
__global__ void __launch_bounds__(1024) rollout_kernel(RolloutLaunch l)
{
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
        const int nseg = 32 / n;
        const int seg = lane / n;
        const int j = lane - seg * n;  // competitor index within the race
        const bool lane_used = seg < nseg;
        const int segbase = seg * n;
        const unsigned segbits = !lane_used ? 0u : (n == 32 ? kFull : (((1u << n) - 1u) << segbase));

        // stage competitor j's parameters in registers
        const int ci = off + (lane_used ? j : 0);
        const float d0 = b.d0[ci];
        const float mu = b.mu[ci];
        const float sigma = b.sigma[ci];
        const float P = b.P[ci];
        const float theta = b.theta[ci];
        const float kr = __fmul_rn(kKappa, __fsub_rn(__fmul_rn(2.0f, b.rho[ci]), 1.0f));
        const float prev0 = b.prev0 ? b.prev0[ci] : __fmul_rn(mu, P);
        const float L = b.L[r];
        const float invL = __fdiv_rn(1.0f, L);
        const uint32_t rid = b.race_id0 + uint32_t(r);

        const int kend = w.k_begin + w.k_count;
        int k = w.k_begin + seg;
        bool active = lane_used && k < kend;
        float d = d0, prev = prev0;
        int t = 0;
        Words4 wd{0u, 0u, 0u, 0u};
        float z_cos = 0.0f, z_sin = 0.0f;
        int wins = 0;
        long long steps = 0;
        bool hit_limit = false;

        while (__any_sync(kFull, active)) {
            // delta(v_c): z for (race, rollout k, step t, competitor j)
            float z = 0.0f;
            if (active) {
                if ((t & 3) == 0) wd = philox4x32_10(uint32_t(k), uint32_t(t) >> 2, uint32_t(j), rid, b.seed_lo, b.seed_hi);
                if (DIST == BBE_DIST_NORMAL) {
                    if ((t & 1) == 0) {
                        const bool hi = (t & 2) != 0;
                        box_muller(hi ? wd.w2 : wd.w0, hi ? wd.w3 : wd.w1, z_cos, z_sin);
                    }
                    z = (t & 1) ? z_sin : z_cos;
                } else {
                    const int q = t & 3;
                    const uint32_t wsel = q == 0 ? wd.w0 : (q == 1 ? wd.w1 : (q == 2 ? wd.w2 : wd.w3));
                    z = DIST == BBE_DIST_UNIFORM ? uniform_z(wsel) : two_point_z(wsel);
                }
            }
            // responsiveness R_c
            const float Rc = __fmaf_rn(kr, __fmaf_rn(d, invL, -0.5f), 1.0f);
            // i+: nearest competitor strictly in front (lowest index among equals)
            bool has_front = false;
            float front_d = 0.0f, front_prev = 0.0f;
            for (int i = 0; i < n; ++i) {
                const float di = __shfl_sync(kFull, d, segbase + i);
                const float pi = __shfl_sync(kFull, prev, segbase + i);
                if (di > d && (!has_front || di < front_d)) {
                    has_front = true;
                    front_d = di;
                    front_prev = pi;
                }
            }
            const bool blocked = has_front && !(__fsub_rn(front_d, d) > theta);
            float S;
            if (blocked) {
                S = __fmul_rn(Rc, prev < front_prev ? prev : front_prev);
            } else {
                S = __fmul_rn(__fmul_rn(Rc, P), __fmaf_rn(sigma, z, mu));
            }
            S = S < kStepFloor ? kStepFloor : S;
            const float dn = __fadd_rn(d, S);

            const bool aborted = active && t >= l.max_steps;
            const bool fin = active && !aborted && dn >= L;
            const unsigned fin_mask = __ballot_sync(kFull, fin);
            const unsigned abort_mask = __ballot_sync(kFull, aborted);
            const bool seg_fin = (fin_mask & segbits) != 0u;
            const bool seg_abort = (abort_mask & segbits) != 0u;
            int winner = -1;
            if (fin_mask != 0u) {
                const float tau = fin ? __fdiv_rn(__fsub_rn(L, d), S) : INFINITY;
                float best = INFINITY;
                for (int i = 0; i < n; ++i) {
                    const float ti = __shfl_sync(kFull, tau, segbase + i);
                    if (ti < best) {
                        best = ti;
                        winner = i;
                    }
                }
            }
            if (active) {
                if (seg_fin && j == winner) ++wins;
                if (seg_fin || seg_abort) {
                    steps += seg_fin ? (t + 1) : t;
                    hit_limit |= seg_abort;
                    k += nseg;
                    active = k < kend;
                    d = d0;
                    prev = prev0;
                    t = 0;
                } else {
                    d = dn;
                    prev = S;
                    ++t;
                }
            }
        }
        // one reduction per work item: wins of competitor j summed over the segments
        int total = 0;
        for (int s = 0; s < nseg; ++s) total += __shfl_sync(kFull, wins, s * n + j);
        if (seg == 0 && total != 0) atomicAdd(&l.counts[off + j], total);
        unsigned long long st = (lane_used && j == 0) ? (unsigned long long)steps : 0ull;
        for (int o = 16; o > 0; o >>= 1) st += __shfl_xor_sync(kFull, st, o);
        if (lane == 0 && l.steps != nullptr) atomicAdd(&l.steps[r], st);
        if (__any_sync(kFull, hit_limit) && lane == 0) atomicOr(l.status, kStatusStepLimit);
    }
}

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

}  // namespace

cudaError_t launch_rollout(const RolloutLaunch &l, cudaStream_t stream)
{
    switch (l.b.dist) {
    case BBE_DIST_NORMAL: rollout_kernel<BBE_DIST_NORMAL><<<l.grid, l.block, 0, stream>>>(l); break;
    case BBE_DIST_UNIFORM: rollout_kernel<BBE_DIST_UNIFORM><<<l.grid, l.block, 0, stream>>>(l); break;
    default: rollout_kernel<BBE_DIST_TWO_POINT><<<l.grid, l.block, 0, stream>>>(l); break;
    }
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
