// bbe_rollout.cu -- the place-count rollout kernel and the probability finalisers.
//
// The place-count kernel (include/bbe.h: bbe_place_counts, bbe_order_counts) runs every rollout
// of Section 3's dry-runs to the K-th finisher.  One warp runs the rollouts of one race at a
// time: a race of n competitors occupies a segment of ceil(n / V) lanes, each lane holding V
// consecutive ranks (V = 1, 2 or 4), and a warp packs floor(32 / lanes) segments, each running
// its own sequence of rollouts of the same race.  Warps pull work items (race, rollout range)
// from a global queue; the race's parameters are staged in shared memory per warp.
//
// Per step every slot evaluates Eq. 1 for the competitor it holds.  Slots keep the competitors
// in rank order (ascending position, then index), so the nearest competitor strictly in front
// (i+) is the next slot: a register (same lane) or one shuffle (next lane).  Finishing is
// detected with a ballot; finished competitors keep moving in their rank slots, the finishers
// of a step are placed by repeated argmin of (crossing time, index), the lane of place j
// records its competitor, and completed rollouts are tallied in a per-warp [competitor][place]
// table in shared memory that reaches the global counts once per work item.  (Win counts,
// K = 1, come from the dedicated kernel in bbe_win.cuh.)
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

// Per-warp staging of the current race, indexed by competitor: parameters, start state,
// the competitor holding each rank at the start of a rollout, and the normals of the
// current 4-step Philox block that are still to be used (by segment and competitor, so
// that they stay with the competitor when ranks change).
struct WarpStage {
    float4 pq[32];  // (mu, sigma, P, theta)
    float kr[32];
    float d0[32], prev0[32];
    int init_c[32];
    float zc[3][128];
};

// One count for `key` in a hash table of `cap` entries (a power of two, at least twice the keys
// it will hold, so a free entry is always found): MurmurHash3's 64-bit finaliser (Appleby)
// picks the first entry, linear probing the next ones; an entry is claimed by compare-and-swap
// from empty.  Where a key lands depends on the order of insertion; the set of (key, count)
// pairs does not.  The probe loop is bounded by the table size.
__device__ __forceinline__ void hist_insert(unsigned long long *keys, int32_t *counts, int64_t cap,
                                            unsigned long long key, int32_t *status)
{
    unsigned long long h = key;
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    const unsigned long long mask = (unsigned long long)(cap - 1);
    unsigned long long i = h & mask;
    for (int64_t probe = 0; probe < cap; ++probe) {
        const unsigned long long prev = atomicCAS(keys + i, kEmptyOrderKey, key);
        if (prev == kEmptyOrderKey || prev == key) {
            atomicAdd(counts + i, 1);
            return;
        }
        i = (i + 1) & mask;
    }
    atomicOr(status, kStatusTableFull);
}

// (da, ca) comes after (db, cb) in rank order
__device__ __forceinline__ bool key_gt(float da, int ca, float db, int cb)
{
    return da > db || (da == db && ca > cb);
}

// The state of one competitor that moves with it when ranks change.
struct Slot {
    int c;
    float d, prev;
};

__device__ __forceinline__ Slot shfl_slot(const Slot &s, int src)
{
    return Slot{__shfl_sync(kFull, s.c, src), __shfl_sync(kFull, s.d, src), __shfl_sync(kFull, s.prev, src)};
}

// z for step t of competitor c in rollout k (Eq. 1's delta(v_c) = mu + sigma z): a
// Philox block serves steps t .. t+3 (t a multiple of 4); its first z is returned and the
// other three are cached in shared memory for the following steps.
template <int DIST>
__device__ __forceinline__ float draw_z(WarpStage &st, int zi, int c, int t, uint32_t k, uint32_t rid,
                                        const uint32_t (&rk)[20])
{
    const Words4 wd = philox4x32_10(k, uint32_t(t) >> 2, uint32_t(c), rid, rk);
    float z0, z1, z2, z3;
    if (DIST == BBE_DIST_NORMAL) {
        box_muller2(wd, z0, z1, z2, z3);
    } else if (DIST == BBE_DIST_UNIFORM) {
        z0 = uniform_z(wd.w0);
        z1 = uniform_z(wd.w1);
        z2 = uniform_z(wd.w2);
        z3 = uniform_z(wd.w3);
    } else {
        z0 = two_point_z(wd.w0);
        z1 = two_point_z(wd.w1);
        z2 = two_point_z(wd.w2);
        z3 = two_point_z(wd.w3);
    }
    st.zc[0][zi] = z1;
    st.zc[1][zi] = z2;
    st.zc[2][zi] = z3;
    return z0;
}

// Place counts: the rollout ends when K = min(places, n) competitors have crossed;
// competitors past the line keep moving and keep their rank slots (a competitor has finished
// exactly when its position is at least L, since positions only grow).
//
// Launch bounds: the finishing order lives in registers, so the kernel may use up to 128 rather
// than spill (measured faster on GB300).
template <int DIST, int V>
__global__ void __launch_bounds__(512, 1) rollout_kernel(RolloutLaunch l)
{
    extern __shared__ WarpStage stage_all[];
    WarpStage &st = stage_all[threadIdx.x >> 5];
    // a [competitor][place] count table per warp after the stages
    int *cnt = reinterpret_cast<int *>(stage_all + (blockDim.x >> 5)) + (threadIdx.x >> 5) * 1024;
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
        const int nl = (n + V - 1) / V;  // lanes per segment
        const int nseg = 32 / nl;
        const int seg = lane / nl;
        const int ql = lane - seg * nl;  // lane within the segment
        const bool lane_used = seg < nseg;
        const int segbase = seg * nl;
        const int zbase = lane_used ? seg * n : 0;  // this segment's row of the z cache
        const unsigned segmask = !lane_used ? 0u : (nl == 32 ? kFull : (((1u << nl) - 1u) << segbase));
        const bool has_next_lane = lane_used && ql + 1 < nl;
        const int rank0 = ql * V;
        bool valid[V];
#pragma unroll
        for (int v = 0; v < V; ++v) valid[v] = lane_used && rank0 + v < n;

        // stage the race: lane j < n loads competitor j (coalesced) and ranks it
        __syncwarp();
        float my_d0 = INFINITY;
        if (lane < n) {
            const int ci = off + lane;
            const float mu = b.mu[ci], P = b.P[ci];
            my_d0 = b.d0[ci];
            st.pq[lane] = make_float4(mu, b.sigma[ci], P, b.theta[ci]);
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
        const int K = min(l.places, n);
        for (int i = lane; i < n * K; i += 32) cnt[i] = 0;
        __syncwarp();

        const float L = b.L[r];
        const float invL = __fdiv_rn(1.0f, L);
        const uint32_t rid = b.race_ids ? uint32_t(b.race_ids[r]) : b.race_id0 + uint32_t(r);
        // unsigned: k + nseg stays below 2^32 for any k_end <= 2^31 - 1
        const unsigned kend = unsigned(w.k_begin) + unsigned(w.k_count);
        unsigned k = unsigned(w.k_begin) + unsigned(seg);
        bool active = lane_used && k < kend;
        int t = 0;
        unsigned gstep = 0;
        int home[V];  // the competitor that starts every rollout in each slot
        Slot s[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            home[v] = valid[v] ? st.init_c[rank0 + v] : 0;
            s[v].c = home[v];
            s[v].d = valid[v] ? st.d0[home[v]] : INFINITY;
            s[v].prev = st.prev0[home[v]];
        }
        long long steps = 0;
        bool hit_limit = false;
        int placed = 0;      // competitors placed in the segment's current rollout
        int my_ord[V];       // competitor in place ql + m * nl
#pragma unroll
        for (int m = 0; m < V; ++m) my_ord[m] = 0;

        // every work item starts with an active segment, and segments change state only at a
        // finish or a step-limit abort, so the warp checks for remaining work only after such a
        // step (measured faster)
        for (;;) {
            bool fired = false;  // a segment finished or was cut off in this step
            __syncwarp();  // z-cache writes of earlier steps are visible to every lane
            const bool running = active && t >= 0;
            // i+: the next rank (same lane, or slot 0 of the next lane).  The same shuffles
            // verify the rank order: every slot's next rank must be strictly in front.
            float fd[V], fp[V];
            bool hf[V];
            auto set_next = [&](float nd, float np) {
#pragma unroll
                for (int v = 0; v < V - 1; ++v) {
                    fd[v] = s[v + 1].d;
                    fp[v] = s[v + 1].prev;
                    hf[v] = valid[v + 1];
                }
                fd[V - 1] = nd;
                fp[V - 1] = np;
                hf[V - 1] = valid[V - 1] && has_next_lane;
            };
            auto next_ranks = [&]() {
                const float nd = __shfl_down_sync(kFull, s[0].d, 1);
                set_next(nd, __shfl_down_sync(kFull, s[0].prev, 1));
            };
            next_ranks();
            bool bad = false;
#pragma unroll
            for (int v = 0; v < V; ++v) bad |= hf[v] && !(fd[v] > s[v].d);
            if (__any_sync(kFull, bad)) {
                // an overtake in the last step (or equal positions): restore rank order by
                // odd-even transposition, then handle ties by a search over the segment.
                // after(by_key, a, b): a belongs behind b, by position then competitor index,
                // or by position alone
                auto after = [](bool by_key, const Slot &a, const Slot &b) {
                    return by_key ? key_gt(a.d, a.c, b.d, b.c) : a.d > b.d;
                };
                // some pair of neighbouring ranks is out of order by key
                auto key_ooo = [&]() {
                    bool o = false;
#pragma unroll
                    for (int v = 0; v + 1 < V; ++v) o |= valid[v + 1] && after(true, s[v], s[v + 1]);
                    const float nd = __shfl_down_sync(kFull, s[0].d, 1);
                    const int nc = __shfl_down_sync(kFull, s[0].c, 1);
                    return o || (has_next_lane && key_gt(s[V - 1].d, s[V - 1].c, nd, nc));
                };
                // odd-even transposition passes while any lane has a pair out of order; returns
                // the position of the next lane's first rank after the last pass
                auto transpose = [&](bool by_key, bool ooo) {
                    float nd = 0.0f;
                    while (__any_sync(kFull, ooo)) {
                        ooo = false;
                        if (V == 1) {
#pragma unroll
                            for (int ph = 0; ph < 2; ++ph) {
                                const bool lower = ((ql - ph) & 1) == 0;
                                const int pq = lower ? ql + 1 : ql - 1;
                                const bool ok = lane_used && pq >= 0 && pq < nl;
                                const int pl = ok ? segbase + pq : lane;
                                const Slot o = shfl_slot(s[0], pl);
                                const bool sw = lower ? after(by_key, s[0], o) : after(by_key, o, s[0]);
                                if (ok && sw) s[0] = o;
                            }
                        } else {
                            // ranks q*V + v: even pairs (2i, 2i+1) lie inside a lane; odd pairs
                            // are the inner ones (1,2), (3,4).. of a lane and (V-1 of lane q, 0 of
                            // lane q+1)
#pragma unroll
                            for (int v = 0; v + 1 < V; v += 2) {
                                if (valid[v + 1] && after(by_key, s[v], s[v + 1])) {
                                    const Slot tmp = s[v];
                                    s[v] = s[v + 1];
                                    s[v + 1] = tmp;
                                }
                            }
#pragma unroll
                            for (int v = 1; v + 1 < V; v += 2) {
                                if (valid[v + 1] && after(by_key, s[v], s[v + 1])) {
                                    const Slot tmp = s[v];
                                    s[v] = s[v + 1];
                                    s[v + 1] = tmp;
                                }
                            }
                            const Slot from_next = shfl_slot(s[0], has_next_lane ? lane + 1 : lane);
                            const Slot from_prev = shfl_slot(s[V - 1], (lane_used && ql > 0) ? lane - 1 : lane);
                            const bool swap_hi = has_next_lane && after(by_key, s[V - 1], from_next);
                            const bool swap_lo = lane_used && ql > 0 && after(by_key, from_prev, s[0]);
                            if (swap_hi) s[V - 1] = from_next;
                            if (swap_lo) s[0] = from_prev;
#pragma unroll
                            for (int v = 0; v + 1 < V; ++v) ooo |= valid[v + 1] && after(by_key, s[v], s[v + 1]);
                        }
                        nd = __shfl_down_sync(kFull, s[0].d, 1);
                        const int nc = by_key ? __shfl_down_sync(kFull, s[0].c, 1) : 0;
                        ooo |= has_next_lane && after(by_key, s[V - 1], Slot{nc, nd, 0.0f});
                    }
                    return nd;
                };
                // order by position first, entered on the check above (equal positions cost
                // one pass that swaps nothing); competitors at equal positions are put in index
                // order below, only when there are any.  The last pass's shuffle gives the next
                // lane's first position.
                const float nd_sorted = transpose(false, bad);
                set_next(nd_sorted, __shfl_down_sync(kFull, s[0].prev, 1));
                bool tie = false;
#pragma unroll
                for (int v = 0; v < V; ++v) tie |= hf[v] && fd[v] == s[v].d;
                if (__any_sync(kFull, tie)) {
                    // equal positions: index order among them, then for each slot the first
                    // later rank with a larger position
                    transpose(true, key_ooo());
#pragma unroll
                    for (int v = 0; v < V; ++v) hf[v] = false;
                    for (int j = 0; j < nl; ++j) {
                        const int src = lane_used ? segbase + j : lane;
#pragma unroll
                        for (int u = 0; u < V; ++u) {
                            const float dj = __shfl_sync(kFull, s[u].d, src);
                            const float pj = __shfl_sync(kFull, s[u].prev, src);
                            const int rj = j * V + u;
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                if (valid[v] && rj > rank0 + v && rj < n && !hf[v] && dj > s[v].d) {
                                    hf[v] = true;
                                    fd[v] = dj;
                                    fp[v] = pj;
                                }
                            }
                        }
                    }
                }
            }
            // delta(v_c): z for (race, rollout k, step t, competitor c)
            float z[V];
#pragma unroll
            for (int v = 0; v < V; ++v) z[v] = 0.0f;
            // one branch per lane for all its slots: a Philox block at the first step of four,
            // else the cached normals (an invalid slot reads a harmless entry of its segment)
            if (running) {
                if ((t & 3) == 0) {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (valid[v]) z[v] = draw_z<DIST>(st, zbase + s[v].c, s[v].c, t, uint32_t(k), rid, l.round_key);
                } else {
                    const float *zrow = st.zc[(t & 3) - 1] + zbase;
#pragma unroll
                    for (int v = 0; v < V; ++v) z[v] = zrow[s[v].c];
                }
            }
            // Eq. 1, then advance
            const bool aborted = running && t >= l.max_steps;
            float S[V], dn[V];
            bool fin[V], any_fin = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float4 q = st.pq[s[v].c];  // (mu, sigma, P, theta)
                const float kr = st.kr[s[v].c];
                const float Rc = __fmaf_rn(kr, __fmaf_rn(s[v].d, invL, -0.5f), 1.0f);
                const bool blocked = hf[v] && !(__fsub_rn(fd[v], s[v].d) > q.w);
                float Sv = blocked ? __fmul_rn(Rc, fminf(s[v].prev, fp[v]))
                                   : __fmul_rn(__fmul_rn(Rc, q.z), __fmaf_rn(q.y, z[v], q.x));
                Sv = fmaxf(Sv, kStepFloor);
                S[v] = Sv;
                dn[v] = __fadd_rn(s[v].d, Sv);
                fin[v] = running && valid[v] && !aborted && dn[v] >= L && s[v].d < L;
                any_fin |= fin[v];
            }
            // finish: least within-step crossing time, ties to the lowest competitor index
            bool seg_fin = false, seg_done = false;
            // place this step's new finishers of each segment, earliest crossing first
            if (__ballot_sync(kFull, any_fin || aborted) != 0u) {
                fired = true;
                const unsigned amask = __ballot_sync(kFull, aborted);
                for (;;) {
                    unsigned fm[V];
                    int nfin = 0;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        fm[v] = __ballot_sync(kFull, fin[v]) & segmask;
                        nfin += __popc(fm[v]);
                    }
                    if (!__any_sync(kFull, nfin > 0)) break;
                    int wl = lane, wv = 0;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        if (fm[v] != 0u) {
                            wl = __ffs(fm[v]) - 1;
                            wv = v;
                        }
                    }
                    if (__any_sync(kFull, nfin > 1)) {
                        float best = INFINITY;
                        int bestc = 1 << 30, bl = wl, bv = wv;
                        for (int j = 0; j < nl; ++j) {
                            const int src = lane_used ? segbase + j : lane;
#pragma unroll
                            for (int u = 0; u < V; ++u) {
                                const float tau = fin[u] ? __fdiv_rn(__fsub_rn(L, s[u].d), S[u]) : INFINITY;
                                const float tj = __shfl_sync(kFull, tau, src);
                                const int cj = __shfl_sync(kFull, s[u].c, src);
                                if (tj < best || (tj == best && tj < INFINITY && cj < bestc)) {
                                    best = tj;
                                    bestc = cj;
                                    bl = src;
                                    bv = u;
                                }
                            }
                        }
                        if (nfin > 1) {
                            wl = bl;
                            wv = bv;
                        }
                    }
                    int cw = 0;
#pragma unroll
                    for (int u = 0; u < V; ++u) {
                        const int cu = __shfl_sync(kFull, s[u].c, wl);
                        cw = wv == u ? cu : cw;
                    }
                    if (nfin > 0) {
#pragma unroll
                        for (int m = 0; m < V; ++m)
                            if (placed == ql + m * nl) my_ord[m] = cw;
                        ++placed;
                        if (lane == wl) {
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                if (v == wv) fin[v] = false;
                        }
                    }
                }
                seg_fin = placed >= K;
                seg_done = seg_fin || (amask & segmask) != 0u;
            }

            // advance, or start the segment's next rollout
            if (active) {
                if (running) {
                    if (seg_done) {
                        // one count per place of a completed rollout (a cut-off one counts for nobody)
#pragma unroll
                        for (int m = 0; m < V; ++m) {
                            const int j = ql + m * nl;
                            if (seg_fin && j < K) atomicAdd(&cnt[my_ord[m] * K + j], 1);
                        }
                        if ((l.orders != nullptr || l.hist_keys != nullptr) && seg_fin) {
                            // the ordered top K, gathered from the lanes holding places 0 .. K-1:
                            // as one base-n number (the dense tables, K <= 3) and as the order
                            // key, the mixed-radix number whose digit j (radix n - j) is the
                            // place-j finisher's index among the competitors not yet placed
                            unsigned code = 0u, taken = 0u;
                            unsigned long long key = 0ull;
                            for (int j = 0; j < K; ++j) {
                                const int mj = j / nl;
                                int mine = my_ord[0];
#pragma unroll
                                for (int m = 1; m < V; ++m)
                                    if (m == mj) mine = my_ord[m];
                                const int cj = __shfl_sync(segmask, mine, segbase + (j - mj * nl));
                                code = code * unsigned(n) + unsigned(cj);
                                key = key * unsigned(n - j) + unsigned(__popc(((1u << cj) - 1u) & ~taken));
                                taken |= 1u << cj;
                            }
                            if (ql == 0) {
                                if (l.orders != nullptr) atomicAdd(&l.orders[l.order_off[r] + code], 1);
                                if (l.hist_keys != nullptr) {
                                    const int64_t h0 = l.hist_off[r];
                                    hist_insert(l.hist_keys + h0, l.hist_counts + h0, l.hist_off[r + 1] - h0, key,
                                                l.status);
                                }
                            }
                        }
                        placed = 0;
                        steps += seg_fin ? (t + 1) : t;
                        hit_limit |= !seg_fin;
                        k += nseg;
                        active = k < kend;
                        // packed segments start rollouts on a common 4-step phase so the
                        // warp draws its Philox blocks together
                        t = nseg > 1 ? -int((4u - ((gstep + 1u) & 3u)) & 3u) : 0;
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const int hc = home[v];
                            s[v].c = hc;
                            s[v].d = valid[v] ? st.d0[hc] : INFINITY;
                            s[v].prev = st.prev0[hc];
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            if (valid[v]) {
                                s[v].d = dn[v];
                                s[v].prev = S[v];
                            }
                        }
                        ++t;
                    }
                } else {
                    ++t;
                }
            }
            ++gstep;
            if (fired && !__any_sync(kFull, active)) break;
        }
        // one flush of the place table per work item
        __syncwarp();
        for (int i = lane; i < n * K && l.counts != nullptr; i += 32) {
            const int c = cnt[i];
            if (c != 0) atomicAdd(&l.counts[(off + i / K) * l.places + i % K], c);
        }
        unsigned long long stp = (lane_used && ql == 0) ? (unsigned long long)steps : 0ull;
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

// per warp: its stage and its [competitor][place] count table
size_t stage_bytes(int block) { return size_t(block / 32) * (sizeof(WarpStage) + 1024 * sizeof(int)); }

template <int V>
cudaError_t launch_v(const RolloutLaunch &l, cudaStream_t stream)
{
    const size_t smem = stage_bytes(l.block);
    switch (l.b.dist) {
    case BBE_DIST_NORMAL: rollout_kernel<BBE_DIST_NORMAL, V><<<l.grid, l.block, smem, stream>>>(l); break;
    case BBE_DIST_UNIFORM: rollout_kernel<BBE_DIST_UNIFORM, V><<<l.grid, l.block, smem, stream>>>(l); break;
    default: rollout_kernel<BBE_DIST_TWO_POINT, V><<<l.grid, l.block, smem, stream>>>(l); break;
    }
    return cudaGetLastError();
}

template <int V>
int resident_v(int dist, int block)
{
    const size_t smem = stage_bytes(block);
    int nb = 0;
    cudaError_t e;
    switch (dist) {
    case BBE_DIST_NORMAL:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rollout_kernel<BBE_DIST_NORMAL, V>, block, smem);
        break;
    case BBE_DIST_UNIFORM:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rollout_kernel<BBE_DIST_UNIFORM, V>, block, smem);
        break;
    default:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rollout_kernel<BBE_DIST_TWO_POINT, V>, block, smem);
        break;
    }
    return e == cudaSuccess ? nb : 1;
}

}  // namespace

cudaError_t launch_place_rollout(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream)
{
    switch (slots_per_lane) {
    case 4: return launch_v<4>(l, stream);
    case 3:
    case 2: return launch_v<2>(l, stream);
    default: return launch_v<1>(l, stream);
    }
}

int place_resident_blocks(int dist, int slots_per_lane, int block)
{
    switch (slots_per_lane) {
    case 4: return resident_v<4>(dist, block);
    case 3:
    case 2: return resident_v<2>(dist, block);
    default: return resident_v<1>(dist, block);
    }
}

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
