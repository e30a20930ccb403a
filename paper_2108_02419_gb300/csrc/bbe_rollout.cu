// bbe_rollout.cu -- the Monte Carlo rollout kernel and the win-probability finaliser.
//
// One warp runs the rollouts of one race at a time with competitors in lanes: a race of
// n competitors occupies a segment of n lanes, and a warp packs floor(32 / n) segments,
// each running its own sequence of rollouts of the same race (Section 3 dry-runs).
// Warps pull work items (race, rollout range) from a global queue: one persistent launch
// covers races of any size mix.  The race's parameters are staged in shared memory per
// warp.  Per step every lane evaluates Eq. 1 for the competitor it holds; lanes keep the
// competitors in rank order, so the nearest competitor in front (i+) is one shuffle away;
// finishing is detected with a ballot and the winner (least within-step crossing time,
// lowest index on ties) found from the ballot mask, or by a shuffle reduction when
// several cross in the same step.  Each lane counts the wins of the competitor that starts
// every rollout in it; the counts are reduced once per work item.
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

// Per-warp staging of the current race: competitor parameters by competitor index, and the
// competitor holding each rank (ascending position, then index) at the start of a rollout.
struct WarpStage {
    float mu[32], sigma[32], P[32], theta[32], kr[32], d0[32], prev0[32];
    int init_c[32];
};

struct Params {
    float mu, sigma, P, theta, kr;
};

__device__ __forceinline__ Params load_params(const WarpStage &st, int c)
{
    return Params{st.mu[c], st.sigma[c], st.P[c], st.theta[c], st.kr[c]};
}

// Lanes of a segment hold the race's competitors in rank order: lane p holds the competitor
// with the p-th smallest (position, index).  The nearest competitor strictly in front of the
// one in lane p is then the one in lane p+1 (or, when positions are equal, the first later
// lane with a larger position), found with one shuffle.  After each step the order is
// restored by odd-even transposition (each competitor's state moves with it); overtakes are
// rare, so this costs a ballot per step and a few shuffles per overtake.
template <int DIST>
__global__ void __launch_bounds__(512) rollout_kernel(RolloutLaunch l)
{
    extern __shared__ WarpStage stage_all[];
    WarpStage &st = stage_all[threadIdx.x >> 5];
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
        const int p = lane - seg * n;  // rank slot within the segment
        const bool lane_used = seg < nseg;
        const int segbase = seg * n;
        const unsigned segmask = !lane_used ? 0u : (n == 32 ? kFull : (((1u << n) - 1u) << segbase));
        const bool has_next = lane_used && p + 1 < n;

        // stage the race: lane j < n loads competitor j (coalesced) and ranks it
        __syncwarp();
        float my_d0 = INFINITY;
        if (lane < n) {
            const int ci = off + lane;
            const float mu = b.mu[ci], P = b.P[ci];
            my_d0 = b.d0[ci];
            st.mu[lane] = mu;
            st.sigma[lane] = b.sigma[ci];
            st.P[lane] = P;
            st.theta[lane] = b.theta[ci];
            st.kr[lane] = __fmul_rn(kKappa, __fsub_rn(__fmul_rn(2.0f, b.rho[ci]), 1.0f));
            st.d0[lane] = my_d0;
            st.prev0[lane] = b.prev0 ? b.prev0[ci] : __fmul_rn(mu, P);
        }
        int rank = 0;
        for (int i = 0; i < n; ++i) {
            const float di = __shfl_sync(kFull, my_d0, i);
            rank += (di < my_d0 || (di == my_d0 && i < lane)) ? 1 : 0;
        }
        if (lane < n) st.init_c[rank] = lane;
        __syncwarp();

        const float L = b.L[r];
        const float invL = __fdiv_rn(1.0f, L);
        const uint32_t rid = b.race_id0 + uint32_t(r);
        const int home = lane_used ? st.init_c[p] : 0;  // this lane counts wins of `home`
        const int kend = w.k_begin + w.k_count;
        int k = w.k_begin + seg;
        bool active = lane_used && k < kend;
        int t = 0;
        unsigned gstep = 0;
        int c = home;
        float d = st.d0[c], prev = st.prev0[c];
        Params q = load_params(st, c);
        uint32_t w1 = 0u, w2 = 0u, w3 = 0u;  // Philox words of the current 4-step block
        float zs = 0.0f;                    // sine half of the current Box-Muller pair
        int wins = 0;
        long long steps = 0;
        bool hit_limit = false;

        while (__any_sync(kFull, active)) {
            const bool running = active && t >= 0;
            // delta(v_c): z for (race, rollout k, step t, competitor c)
            float z = 0.0f;
            if (running) {
                if (DIST == BBE_DIST_NORMAL) {
                    if ((t & 1) == 0) {
                        uint32_t wa = w2, wb = w3;
                        if ((t & 3) == 0) {
                            const Words4 wd = philox4x32_10(uint32_t(k), uint32_t(t) >> 2, uint32_t(c), rid,
                                                            b.seed_lo, b.seed_hi);
                            wa = wd.w0;
                            wb = wd.w1;
                            w2 = wd.w2;
                            w3 = wd.w3;
                        }
                        box_muller(wa, wb, z, zs);
                    } else {
                        z = zs;
                    }
                } else {
                    uint32_t wsel;
                    if ((t & 3) == 0) {
                        const Words4 wd = philox4x32_10(uint32_t(k), uint32_t(t) >> 2, uint32_t(c), rid,
                                                        b.seed_lo, b.seed_hi);
                        wsel = wd.w0;
                        w1 = wd.w1;
                        w2 = wd.w2;
                        w3 = wd.w3;
                    } else {
                        const int qq = t & 3;
                        wsel = qq == 1 ? w1 : (qq == 2 ? w2 : w3);
                    }
                    z = DIST == BBE_DIST_UNIFORM ? uniform_z(wsel) : two_point_z(wsel);
                }
            }
            // responsiveness R_c
            const float Rc = __fmaf_rn(q.kr, __fmaf_rn(d, invL, -0.5f), 1.0f);
            // i+: the next rank; with equal positions, the first later rank strictly in front
            float fd = __shfl_down_sync(kFull, d, 1);
            float fp = __shfl_down_sync(kFull, prev, 1);
            bool has_front = has_next;
            if (__any_sync(kFull, running && has_next && fd == d)) {
                has_front = false;
                for (int i = 1; i < n; ++i) {
                    const bool ok = lane_used && p + i < n;
                    const int src = ok ? segbase + p + i : lane;
                    const float di = __shfl_sync(kFull, d, src);
                    const float pi = __shfl_sync(kFull, prev, src);
                    if (ok && !has_front && di > d) {
                        has_front = true;
                        fd = di;
                        fp = pi;
                    }
                }
            }
            // Eq. 1
            const bool blocked = has_front && !(__fsub_rn(fd, d) > q.theta);
            float S = blocked ? __fmul_rn(Rc, fminf(prev, fp))
                              : __fmul_rn(__fmul_rn(Rc, q.P), __fmaf_rn(q.sigma, z, q.mu));
            S = fmaxf(S, kStepFloor);
            const float dn = __fadd_rn(d, S);

            // finish: least within-step crossing time, ties to the lowest competitor index
            const bool aborted = running && t >= l.max_steps;
            const bool fin = running && !aborted && dn >= L;
            const unsigned fmask = __ballot_sync(kFull, fin);
            const unsigned amask = __ballot_sync(kFull, aborted);
            const unsigned my_f = fmask & segmask;
            const bool seg_done = ((fmask | amask) & segmask) != 0u;
            if (fmask != 0u) {
                int wl = my_f ? (__ffs(my_f) - 1) : lane;
                if (__any_sync(kFull, __popc(my_f) > 1)) {
                    const float tau = fin ? __fdiv_rn(__fsub_rn(L, d), S) : INFINITY;
                    float best = INFINITY;
                    int bestc = 1 << 30, bl = wl;
                    for (int i = 0; i < n; ++i) {
                        const int src = lane_used ? segbase + i : lane;
                        const float ti = __shfl_sync(kFull, tau, src);
                        const int ci = __shfl_sync(kFull, c, src);
                        if (ti < best || (ti == best && ti < INFINITY && ci < bestc)) {
                            best = ti;
                            bestc = ci;
                            bl = src;
                        }
                    }
                    if (my_f) wl = bl;
                }
                const int cw = __shfl_sync(kFull, c, wl);
                if (my_f != 0u && home == cw) ++wins;
            }

            // advance, or start the segment's next rollout
            if (active) {
                if (running) {
                    if (seg_done) {
                        steps += my_f ? (t + 1) : t;
                        hit_limit |= (my_f == 0u);
                        k += nseg;
                        active = k < kend;
                        // packed segments start rollouts on a common 4-step phase so
                        // the warp draws Philox blocks together
                        t = nseg > 1 ? -int((4u - ((gstep + 1u) & 3u)) & 3u) : 0;
                        c = home;
                        d = st.d0[c];
                        prev = st.prev0[c];
                        q = load_params(st, c);
                    } else {
                        d = dn;
                        prev = S;
                        ++t;
                    }
                } else {
                    ++t;
                }
            }
            ++gstep;

            // restore rank order (odd-even transposition), moving each competitor's state
            {
                const float nd = __shfl_down_sync(kFull, d, 1);
                const int nc = __shfl_down_sync(kFull, c, 1);
                bool ooo = has_next && (nd < d || (nd == d && nc < c));
                while (__any_sync(kFull, ooo)) {
#pragma unroll
                    for (int ph = 0; ph < 2; ++ph) {
                        const bool lower = ((p - ph) & 1) == 0;
                        const int pp = lower ? p + 1 : p - 1;
                        const bool valid = lane_used && pp >= 0 && pp < n;
                        const int pl = valid ? segbase + pp : lane;
                        const float od = __shfl_sync(kFull, d, pl);
                        const int oc = __shfl_sync(kFull, c, pl);
                        const bool mine_greater = d > od || (d == od && c > oc);
                        const bool swap = valid && (lower ? mine_greater : !mine_greater);
                        const int src = swap ? pl : lane;
                        c = __shfl_sync(kFull, c, src);
                        d = __shfl_sync(kFull, d, src);
                        prev = __shfl_sync(kFull, prev, src);
                        w1 = __shfl_sync(kFull, w1, src);
                        w2 = __shfl_sync(kFull, w2, src);
                        w3 = __shfl_sync(kFull, w3, src);
                        zs = __shfl_sync(kFull, zs, src);
                        if (swap) q = load_params(st, c);
                    }
                    const float nd2 = __shfl_down_sync(kFull, d, 1);
                    const int nc2 = __shfl_down_sync(kFull, c, 1);
                    ooo = has_next && (nd2 < d || (nd2 == d && nc2 < c));
                }
            }
        }
        // one reduction per work item: wins of each home competitor summed over segments
        int total = 0;
        for (int s2 = 0; s2 < nseg; ++s2) total += __shfl_sync(kFull, wins, s2 * n + (lane_used ? p : 0));
        if (seg == 0 && total != 0) atomicAdd(&l.counts[off + home], total);
        unsigned long long stp = (lane_used && p == 0) ? (unsigned long long)steps : 0ull;
        for (int o = 16; o > 0; o >>= 1) stp += __shfl_xor_sync(kFull, stp, o);
        if (lane == 0 && l.steps != nullptr) atomicAdd(&l.steps[r], stp);
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
    const size_t smem = size_t(l.block / 32) * sizeof(WarpStage);
    switch (l.b.dist) {
    case BBE_DIST_NORMAL: rollout_kernel<BBE_DIST_NORMAL><<<l.grid, l.block, smem, stream>>>(l); break;
    case BBE_DIST_UNIFORM: rollout_kernel<BBE_DIST_UNIFORM><<<l.grid, l.block, smem, stream>>>(l); break;
    default: rollout_kernel<BBE_DIST_TWO_POINT><<<l.grid, l.block, smem, stream>>>(l); break;
    }
    return cudaGetLastError();
}

int rollout_resident_blocks(int dist, int block)
{
    const size_t smem = size_t(block / 32) * sizeof(WarpStage);
    int nb = 0;
    cudaError_t e;
    switch (dist) {
    case BBE_DIST_NORMAL: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rollout_kernel<BBE_DIST_NORMAL>, block, smem); break;
    case BBE_DIST_UNIFORM: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rollout_kernel<BBE_DIST_UNIFORM>, block, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rollout_kernel<BBE_DIST_TWO_POINT>, block, smem); break;
    }
    return e == cudaSuccess ? nb : 1;
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
