// bbe_win.cuh -- the rollout kernel: the Section 3 dry-runs under Eq. 1, each rollout run to its
// first finisher (win counts) or, in place mode, to its K-th (place counts, ordered tallies and
// the finishing-order histogram).
//
// Layout.  A warp holds 32 V slots (V = 1..4 per lane; slot i = 32 v + lane, so the lanes of
// one register hold consecutive slots).  A race of n competitors takes floor(32 V / n)
// segments of n consecutive slots: slot s n + c holds competitor c for the whole work item, and
// each segment runs its own rollouts of the race.  A competitor never changes slot, so the four
// normals of its current Philox block live in registers, and so do its parameters (or, in the
// register-lean variant for three and four slots per lane, a shared-memory address of them).
//
// The nearest competitor strictly in front (i+).  Each step every slot publishes (d, previous
// step) in shared memory and reads the entry of its rank successor (rank order: ascending
// position, then index), whose address it keeps in a register.  In a segment where every
// successor is strictly in front, the successor is i+.  The same read detects an overtake or
// an equal position (successor not strictly in front); on that rare step the segment is
// re-sorted by odd-even transposition over a rank table in shared memory, and a slot whose
// successor stands level with it takes the first later rank strictly in front.
//
// The step loop is unrolled over the four steps of a Philox block: a block draws one
// Philox4x32-10 output per slot and both of its Box-Muller pairs, then runs four steps whose
// normals are registers chosen at compile time.  Every rollout starts on a block boundary (a
// segment that finishes waits for the next one; the counter of step t is t >> 2 in any case).
// A finished segment takes its next rollout index from a per-warp counter, so the segments of
// a work item stay busy until its rollouts run out.
//
// Finishing.  A ballot finds the steps with finishers; each finisher offers the key
// (within-step crossing time tau = (L - d) / S, slot) to its segment's minimum in shared
// memory, which gives the least tau and, on equal tau, the lowest competitor index.  Wins are
// tallied per competitor in shared memory and reach the global counts once per work item.
// Place mode records each crossing with its key (sub-step, tau, slot) and places a block's
// crossings at the block's end; a segment whose K-th place is filled ends its rollout, and its
// places and order are tallied when it restarts.
//
// Loop bookkeeping.  After a block without a finish or a step-limit cut-off nothing can have
// changed which slots run, so the warp's reduction of restart and liveness flags runs only after
// blocks with one; a warp-uniform count-down rules out the step limit until a block could reach it.
//
// The arithmetic is the pinned binary32 round-to-nearest sequence of include/bbe.h (explicit
// intrinsics, file compiled with --fmad=false), so the counts are bit-identical to any
// implementation that follows it, whatever the layout.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "bbe_internal.h"
#include "bbe_rng.cuh"

namespace bbe {

namespace win {

constexpr unsigned kAll = 0xffffffffu;
constexpr unsigned long long kNoKey = ~0ull;

template <int V>
struct WinStage {
    static constexpr int NS = 32 * V;   // slots per warp
    static constexpr int ROW = NS + 2;  // entries per position row: slots, the sentinel, padding to 16 bytes
    float2 pos[2][ROW];                 // (d, previous step) per slot, one row per step parity
    float4 pq[32];                      // per competitor: (mu, sigma, P, theta)
    float kr[32];                       // per competitor: kappa (2 rho - 1)
    float d0[32], prev0[32];            // per competitor: start state of every rollout
    int rank0[32], byrank0[32];         // start rank of competitor c; competitor at start rank r
    int wins[32];                       // wins per competitor in the current work item
    int order[NS];                      // order[segment base + r]: slot holding rank r
    int rnk[NS];                        // rank of each slot
    int flag[NS];                       // by segment base + rank: the slot there swaps with its successor
    unsigned segk[NS];                  // by segment base: rollout index handed to a restart
    unsigned long long key[NS];         // by segment base: least crossing key of the block (win mode)
    unsigned long long fkey[NS];        // place mode: each slot's crossing (sub-step, slot) of the block, or none
    float2 fcross[NS];                  // place mode: (d, S) of that crossing step
    unsigned next_k;                    // next rollout index of the work item
};

template <int DIST>
__device__ __forceinline__ void draw_block(uint32_t k, uint32_t blk, uint32_t c, uint32_t rid,
                                           const uint32_t (&rkey)[20], float (&z)[4])
{
    const Words4 wd = philox4x32_10(k, blk, c, rid, rkey);
    if (DIST == BBE_DIST_NORMAL) {
        box_muller2(wd, z[0], z[1], z[2], z[3]);
    } else if (DIST == BBE_DIST_UNIFORM) {
        z[0] = uniform_z(wd.w0);
        z[1] = uniform_z(wd.w1);
        z[2] = uniform_z(wd.w2);
        z[3] = uniform_z(wd.w3);
    } else {
        z[0] = two_point_z(wd.w0);
        z[1] = two_point_z(wd.w1);
        z[2] = two_point_z(wd.w2);
        z[3] = two_point_z(wd.w3);
    }
}

// Registers per thread: enough for one or two slots per lane to run without spilling at 7 or 8
// resident 4-warp blocks per SM (measured faster than the compiler's unbounded choice), and
// for the register-lean three- and four-slot variants.
template <int V, int MODE>
struct WinRegs {
    static constexpr int value = MODE == 0 ? (V == 1 ? 48 : (V == 2 ? 72 : 80)) : (V == 1 ? 48 : (V == 2 ? 72 : 80));
};
// Parameters read from shared memory each step instead of held in registers.
template <int V>
struct WinLean {
    static constexpr bool value = V >= 3;
};

// MODE 0: win counts, each rollout run to its first finisher.  MODE 1: place counts (and the
// ordered tallies), each rollout run until K = min(l.places, n) competitors have crossed; the
// finished ones keep moving and blocking, a competitor has crossed exactly when its position is
// at least L (positions only grow), and the finishers of a step are placed in (tau, slot) order.
template <int DIST, int V, int LAW, int MODE>
__global__ void __maxnreg__((WinRegs<V, MODE>::value)) win_rollout_kernel(RolloutLaunch l)
{
    constexpr bool PS = WinLean<V>::value;
    using Stage = WinStage<V>;
    constexpr int NS = Stage::NS;
    constexpr int ROWB = Stage::ROW * int(sizeof(float2));
    constexpr int kSent = NS * int(sizeof(float2));  // byte offset of the sentinel (+inf: no one in front)
    extern __shared__ __align__(16) unsigned char win_smem[];
    Stage &st = reinterpret_cast<Stage *>(win_smem)[threadIdx.x >> 5];
    char *const posb = reinterpret_cast<char *>(&st.pos[0][0]);
    // place mode, per warp after all the stages: the finisher of each place (by segment base +
    // place), the places filled and the sub-step of the K-th place (by segment base), then the
    // work item's [competitor][place] table
    int *pl_ord = nullptr, *pl_n = nullptr, *pl_kj = nullptr, *pl_cnt = nullptr;
    if constexpr (MODE == 1) {
        pl_ord = reinterpret_cast<int *>(win_smem + (blockDim.x >> 5) * sizeof(Stage)) +
                 (threadIdx.x >> 5) * (3 * NS + l.place_cells);
        pl_n = pl_ord + NS;
        pl_kj = pl_ord + 2 * NS;
        pl_cnt = pl_ord + 3 * NS;
    }
    const DevBatch &b = l.b;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        st.pos[0][NS] = make_float2(INFINITY, INFINITY);
        st.pos[1][NS] = make_float2(INFINITY, INFINITY);
    }
    bool hit_limit = false;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(l.queue, 1);
        it = __shfl_sync(kAll, it, 0);
        if (it >= l.n_items) break;
        const WorkItem w = l.items[it];
        const int r = BBE_INDEX(w.race, b.n_races, l.status);
        const int off = b.race_off[r];
        const int n = BBE_INDEX(b.race_off[r + 1] - off - 1, 32, l.status) + 1;  // 1..32
        (void)BBE_INDEX(off + n - 1, b.n_total, l.status);
        const int nseg = l.seg_cap > 0 ? min(NS / n, l.seg_cap) : NS / n;  // segments of this warp

        // stage the race: lane j < n loads competitor j (coalesced) and ranks it by (d0, j)
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
            st.wins[lane] = 0;
        }
        int rank = 0;
        for (int i = 0; i < n; ++i) {
            const float di = __shfl_sync(kAll, my_d0, i);
            rank += (di < my_d0 || (di == my_d0 && i < lane)) ? 1 : 0;
        }
        if (lane < n) {
            st.rank0[lane] = rank;
            st.byrank0[BBE_INDEX(rank, 32, l.status)] = lane;
        }
        for (int i = lane; i < NS; i += 32) {
            st.key[i] = kNoKey;
            st.flag[i] = 0;
        }
        const int K = MODE == 1 ? min(l.places, n) : 1;  // places run per rollout
        if constexpr (MODE == 1) {
            for (int i = lane; i < NS; i += 32) {
                pl_n[i] = 0;
                st.fkey[i] = kNoKey;
            }
            for (int i = lane; i < n * K; i += 32) pl_cnt[i] = 0;
        }
        if (lane == 0) st.next_k = unsigned(w.k_begin) + unsigned(nseg);
        __syncwarp();

        const float L = b.L[r];
        const float invL = __fdiv_rn(1.0f, L);
        const float t0r = LAW == BBE_LAW_TIME ? b.t0[r] : 0.0f;     // time law: elapsed steps
        const float invTr = LAW == BBE_LAW_TIME ? b.invT[r] : 0.0f;  // time law: 1 / expected duration
        const uint32_t rid = b.race_ids ? uint32_t(b.race_ids[r]) : b.race_id0 + uint32_t(r);
        // unsigned: rollout indices stay below 2^31 + 2^7
        const unsigned kend = unsigned(w.k_begin) + unsigned(w.k_count);

        // per slot: segment base, competitor parameters, state, front address, rollout, block
        int sb[V], fo[V];
        unsigned kk[V], blk[V];
        float mu[V], sg[V], P[V], th[V], kr[V], d[V], pv[V];
        const float4 *pqa[V];  // register-lean variant: this slot's (mu, sigma, P, theta)
        const float *kra[V];   // register-lean variant: this slot's kappa (2 rho - 1)
        bool alive[V], pend[V], cut[V];  // running; rollout ended, to restart; stopped at max_steps
        unsigned long long steps = 0;
        bool blk_fin = false;  // warp-uniform: some slot crossed the line in this block (a finish)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int slot = 32 * v + lane;
            const int seg = slot / n;
            const bool used = seg < nseg;
            sb[v] = used ? seg * n : slot;
            const int c = used ? slot - seg * n : 0;
            kk[v] = unsigned(w.k_begin) + unsigned(seg);
            alive[v] = used && kk[v] < kend;
            pend[v] = false;
            cut[v] = false;
            blk[v] = 0;
            if constexpr (PS) {
                pqa[v] = &st.pq[c];
                kra[v] = &st.kr[c];
            } else {
                const float4 q = st.pq[c];
                mu[v] = q.x;
                sg[v] = q.y;
                P[v] = q.z;
                th[v] = q.w;
                kr[v] = st.kr[c];
            }
            d[v] = st.d0[c];
            pv[v] = st.prev0[c];
            const int r0 = st.rank0[c];
            fo[v] = (used && r0 + 1 < n) ? BBE_INDEX(sb[v] + st.byrank0[r0 + 1], NS, l.status) * int(sizeof(float2)) : kSent;
            if (alive[v]) {
                st.order[BBE_INDEX(sb[v] + r0, NS, l.status)] = slot;
                st.rnk[slot] = r0;
            }
        }
        __syncwarp();

        // A segment whose rank order broke (an overtake, or equal positions): odd-even
        // transposition by (position, slot) over the segment's rank table, then each slot's
        // successor, and i+ for a slot level with its successor.  pb is the step's row.
        auto full_sort = [&](const char *pb, float (&fd)[V], float (&fp)[V]) {
            const float2 *row = reinterpret_cast<const float2 *>(pb);
            int rk[V];
#pragma unroll
            for (int v = 0; v < V; ++v) rk[v] = alive[v] ? st.rnk[32 * v + lane] : 0;
            // a sort of n keys ends within n phases; 32 passes bound the loop for any input
            for (int pass = 0; pass < 32; ++pass) {
                bool swapped = false;
#pragma unroll
                for (int ph = 0; ph < 2; ++ph) {
                    int nr[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        nr[v] = rk[v];
                        const int slot = 32 * v + lane;
                        const bool lower = ((rk[v] ^ ph) & 1) == 0;
                        const int pr = lower ? rk[v] + 1 : rk[v] - 1;
                        if (alive[v] && pr >= 0 && pr < n) {
                            const int ps = BBE_INDEX(st.order[BBE_INDEX(sb[v] + pr, NS, l.status)], NS, l.status);
                            const float pd = row[ps].x;
                            const bool inv = lower ? (d[v] > pd || (d[v] == pd && slot > ps))
                                                   : (pd > d[v] || (pd == d[v] && ps > slot));
                            if (inv) {
                                nr[v] = pr;
                                swapped = true;
                            }
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        rk[v] = nr[v];
                        if (alive[v]) st.order[BBE_INDEX(sb[v] + nr[v], NS, l.status)] = 32 * v + lane;
                    }
                    __syncwarp();
                }
                if (!__any_sync(kAll, swapped)) break;
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (!alive[v]) continue;
                st.rnk[32 * v + lane] = rk[v];
                fo[v] = rk[v] + 1 < n ? BBE_INDEX(st.order[BBE_INDEX(sb[v] + rk[v] + 1, NS, l.status)], NS, l.status) *
                                            int(sizeof(float2))
                                      : kSent;
                float2 f = *reinterpret_cast<const float2 *>(pb + fo[v]);
                if (!(f.x > d[v])) {
                    // level with the successor: the first later rank strictly in front, if any
                    f = make_float2(INFINITY, INFINITY);
                    for (int q = rk[v] + 2; q < n; ++q) {
                        const float2 g = row[BBE_INDEX(st.order[BBE_INDEX(sb[v] + q, NS, l.status)], NS, l.status)];
                        if (g.x > d[v]) {
                            f = g;
                            break;
                        }
                    }
                }
                fd[v] = f.x;
                fp[v] = f.y;
            }
            __syncwarp();
        };

        // The common case first: isolated overtakes.  A slot whose successor is now strictly
        // behind it swaps ranks with that successor, unless a neighbouring pair swaps too (a
        // chain); then every slot re-reads its successor, and what is still out of order or
        // level goes to the full sort.
        auto repair = [&](const char *pb, float (&fd)[V], float (&fp)[V]) {
            int rk[V];
            bool init[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                rk[v] = alive[v] ? st.rnk[32 * v + lane] : 0;
                init[v] = alive[v] && fd[v] < d[v];
                if (init[v]) st.flag[BBE_INDEX(sb[v] + rk[v], NS, l.status)] = 1;
            }
            __syncwarp();
            bool ok[V];
#pragma unroll
            for (int v = 0; v < V; ++v)
                ok[v] = init[v] && !(rk[v] > 0 && st.flag[sb[v] + rk[v] - 1]) && !(rk[v] + 2 < n && st.flag[sb[v] + rk[v] + 1]);
            __syncwarp();
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (!init[v]) continue;
                st.flag[sb[v] + rk[v]] = 0;
                if (ok[v]) {
                    const int slot = 32 * v + lane;
                    const int f = BBE_INDEX(st.order[BBE_INDEX(sb[v] + rk[v] + 1, NS, l.status)], NS, l.status);
                    st.order[sb[v] + rk[v]] = f;
                    st.order[sb[v] + rk[v] + 1] = slot;
                    st.rnk[f] = rk[v];
                    st.rnk[slot] = rk[v] + 1;
                }
            }
            __syncwarp();
            bool again = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (!alive[v]) continue;
                const int r1 = st.rnk[32 * v + lane] + 1;
                fo[v] = r1 < n ? BBE_INDEX(st.order[BBE_INDEX(sb[v] + r1, NS, l.status)], NS, l.status) * int(sizeof(float2))
                               : kSent;
                const float2 f = *reinterpret_cast<const float2 *>(pb + fo[v]);
                fd[v] = f.x;
                fp[v] = f.y;
                again |= !(f.x > d[v]);
            }
            if (__any_sync(kAll, again)) full_sort(pb, fd, fp);
        };

        // Place mode, the end of a Philox block in which some slot crossed the line or may have
        // reached max_steps: the block's crossings of each segment take the next places one at
        // a time in key order (sub-step, tau, slot), and a segment whose K-th place is filled
        // ends its rollout (its places and order are tallied when it restarts); a rollout
        // stopped at max_steps that did not end earlier counts for nobody.  Ending at the
        // block's end costs nothing: a segment whose rollout ended waits for the next block in
        // any case, and its slots record no further crossings (d < L fails past the line).
        // (Measured slower for win counts, which end their rollouts within the step.)
        auto block_end = [&]() {
            __syncwarp();
            {
                unsigned long long fk[V];
                bool more = false;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int slot = 32 * v + lane;
                    fk[v] = st.fkey[slot];
                    if (fk[v] != kNoKey) {
                        const float2 c = st.fcross[slot];
                        const float tau = __fdiv_rn(__fsub_rn(L, c.x), c.y);
                        fk[v] |= static_cast<unsigned long long>(__float_as_uint(tau)) << 8;
                        st.fkey[slot] = kNoKey;
                        more = true;
                    }
                }
                // one crossing per segment per round; a segment has at most n of them
                for (int round = 0; round < NS && __any_sync(kAll, more); ++round) {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (fk[v] != kNoKey) atomicMin(&st.key[sb[v]], fk[v]);
                    __syncwarp();
                    bool won[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        won[v] = fk[v] != kNoKey && st.key[sb[v]] == fk[v];
                        if (won[v]) {
                            const int p = BBE_INDEX(pl_n[sb[v]], n, l.status);
                            pl_ord[sb[v] + p] = 32 * v + lane - sb[v];
                            pl_n[sb[v]] = p + 1;
                            if (p == K - 1) pl_kj[sb[v]] = int(fk[v] >> 40);
                        }
                    }
                    __syncwarp();
                    more = false;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        if (fk[v] != kNoKey) st.key[sb[v]] = kNoKey;
                        if (won[v]) fk[v] = kNoKey;
                        more |= fk[v] != kNoKey;
                    }
                    __syncwarp();
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (!alive[v] && !cut[v]) continue;
                const int slot = 32 * v + lane;
                const int jend = pl_n[sb[v]] >= K ? pl_kj[sb[v]] : -1;  // sub-step of the K-th place
                if (jend >= 0) {
                    if (slot == sb[v]) steps += (unsigned long long)(blk[v] * 4u + unsigned(jend) + 1u);
                    pend[v] = true;
                } else if (cut[v]) {
                    if (slot == sb[v]) steps += (unsigned long long)l.max_steps;
                    hit_limit = true;
                    pend[v] = true;
                }
                alive[v] = alive[v] && !pend[v];
                cut[v] = false;
            }
            __syncwarp();
        };

        // Place mode, at a block boundary: the segments that completed a rollout (K places filled;
        // a rollout cut off at max_steps fills fewer and counts for nobody) add one count per
        // place and, for the ordered tallies, their order: as one base-n number (the dense
        // tables, K <= 3) and as the order key, the mixed-radix number whose digit j (radix
        // n - j) is the place-j finisher's index among the competitors not yet placed.
        auto tally_completed = [&]() {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (!pend[v] || pl_n[sb[v]] < K) continue;
                const int c = 32 * v + lane - sb[v];  // this slot's competitor
                if (c < K) atomicAdd(&pl_cnt[BBE_INDEX(pl_ord[sb[v] + c] * K + c, n * K, l.status)], 1);
                if (c == 0 && (l.orders != nullptr || l.hist_keys != nullptr)) {
                    unsigned code = 0u, taken = 0u;
                    unsigned long long key = 0ull;
                    for (int j = 0; j < K; ++j) {
                        const int cj = pl_ord[sb[v] + j];
                        code = code * unsigned(n) + unsigned(cj);
                        key = key * unsigned(n - j) + unsigned(__popc(((1u << cj) - 1u) & ~taken));
                        taken |= 1u << cj;
                    }
                    if (l.orders != nullptr) {
#if defined(BBE_CHECKED) && BBE_CHECKED
                        unsigned cells = 1u;  // n^K entries in the race's dense table
                        for (int j = 0; j < K; ++j) cells *= unsigned(n);
#endif
                        atomicAdd(&l.orders[l.order_off[r] + BBE_INDEX(code, cells, l.status)], 1);
                    }
                    if (l.hist_keys != nullptr) {
                        const int64_t h0 = l.hist_off[r];
                        hist_insert(l.hist_keys + h0, l.hist_counts + h0, l.hist_off[r + 1] - h0, key, l.status);
                    }
                }
            }
            __syncwarp();
        };

        // One step of every slot: sub-step J of the Philox block (its normal is z[v][J]); CHK
        // when some segment may reach max_steps within the block.
        auto step = [&](auto Jc, auto CHKc, const float (&z)[V][4]) {
            constexpr int J = decltype(Jc)::value;
            constexpr bool CHK = decltype(CHKc)::value;
            constexpr int BO = (J & 1) * ROWB;
            if constexpr (CHK) {
                // a rollout reaching step max_steps stops there and counts for nobody (in place
                // mode unless it ended earlier in the block, decided at the block's end)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (alive[v] && int(blk[v]) * 4 + J >= l.max_steps) {
                        alive[v] = false;
                        if constexpr (MODE == 0) {
                            pend[v] = true;
                            hit_limit = true;
                            if (32 * v + lane == sb[v]) steps += (unsigned long long)l.max_steps;
                        } else {
                            cut[v] = true;
                        }
                    }
                }
            }
            // publish this step's (d, previous step) of every slot
#pragma unroll
            for (int v = 0; v < V; ++v)
                *reinterpret_cast<float2 *>(posb + BO + (32 * v + lane) * 8) = make_float2(d[v], pv[v]);
            __syncwarp();
            float fd[V], fp[V];
            bool bad = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 f = *reinterpret_cast<const float2 *>(posb + BO + BBE_INDEX(fo[v], kSent + 1, l.status));
                fd[v] = f.x;
                fp[v] = f.y;
                bad |= alive[v] && !(f.x > d[v]);
            }
            if (__any_sync(kAll, bad)) repair(posb + BO, fd, fp);
            // Eq. 1 (a successor at +inf is never within theta: the free branch)
            float S[V], dn[V];
            bool fv[V], fin = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float kv, thv, Pv, sgv, muv;
                if constexpr (PS) {
                    const float4 q = *pqa[v];
                    muv = q.x;
                    sgv = q.y;
                    Pv = q.z;
                    thv = q.w;
                    kv = *kra[v];
                } else {
                    muv = mu[v];
                    sgv = sg[v];
                    Pv = P[v];
                    thv = th[v];
                    kv = kr[v];
                }
                const float Rc = responsiveness<LAW>(kv, d[v], invL, t0r, int(blk[v]) * 4 + J, invTr);
                const bool blocked = !(__fsub_rn(fd[v], d[v]) > thv);
                float Sv = blocked ? __fmul_rn(Rc, fminf(pv[v], fp[v]))
                                   : __fmul_rn(__fmul_rn(Rc, Pv), __fmaf_rn(sgv, z[v][J], muv));
                Sv = fmaxf(Sv, kStepFloor);
                S[v] = Sv;
                dn[v] = __fadd_rn(d[v], Sv);
                fv[v] = alive[v] && dn[v] >= L && (MODE == 0 || d[v] < L);
                fin |= fv[v];
            }
            if constexpr (MODE == 1) {
                // place mode: a crossing is recorded with its key (sub-step, within-step crossing
                // time tau, slot) and placed at the block's end; tau > 0, so its bit pattern orders
                // like its value, and key order is the order of finish with ties to the lower
                // competitor index (the slot order within a segment)
                if (__any_sync(kAll, fin)) {
                    blk_fin = true;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        if (fv[v]) {
                            // tau joins the key at the block's end (one division there, none here)
                            st.fkey[32 * v + lane] = (static_cast<unsigned long long>(J) << 40) | unsigned(32 * v + lane);
                            st.fcross[32 * v + lane] = make_float2(d[v], S[v]);
                        }
                    }
                }
            } else if (__any_sync(kAll, fin)) {
                // win mode: least (tau, slot) per segment, at once; tau > 0, so its bit pattern
                // orders like its value
                blk_fin = true;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (fv[v]) {
                        const float tau = __fdiv_rn(__fsub_rn(L, d[v]), S[v]);
                        atomicMin(&st.key[sb[v]], (static_cast<unsigned long long>(__float_as_uint(tau)) << 32) |
                                                      unsigned(32 * v + lane));
                    }
                }
                __syncwarp();
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (alive[v]) {
                        const unsigned long long kw = st.key[sb[v]];
                        if (kw != kNoKey) {
                            const int slot = 32 * v + lane;
                            if (int(unsigned(kw)) == slot) atomicAdd(&st.wins[BBE_INDEX(slot - sb[v], 32, l.status)], 1);
                            alive[v] = false;
                            pend[v] = true;
                            if (slot == sb[v]) steps += (unsigned long long)(blk[v] * 4u + unsigned(J) + 1u);
                        }
                    }
                }
                __syncwarp();
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (fv[v]) st.key[sb[v]] = kNoKey;
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                d[v] = dn[v];
                pv[v] = S[v];
            }
        };

        // blocks before one in which a rollout could reach max_steps (the check starts there)
        unsigned left = l.max_steps >= 4 ? unsigned(l.max_steps - 4) / 4u + 1u : 0u;
        // warp-uniform: the last block may have changed which slots run (a finish, a cut-off);
        // after a block without either the reduction below would find nothing to do
        bool blk_event = true;
        for (;;) {
            if (blk_event) {
            blk_event = false;
            // segments that finished in the last block start their next rollout; one reduction
            // says whether any did and whether anything still runs
            bool pany = false, aany = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                pany |= pend[v];
                aany |= alive[v];
            }
            const unsigned state = __reduce_or_sync(kAll, (pany ? 1u : 0u) | (aany ? 2u : 0u));
            if (state & 1u) {
                if constexpr (MODE == 1) tally_completed();
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (pend[v] && 32 * v + lane == sb[v]) {
                        st.segk[sb[v]] = atomicAdd(&st.next_k, 1u);
                        if constexpr (MODE == 1) pl_n[sb[v]] = 0;
                    }
                __syncwarp();
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (!pend[v]) continue;
                    pend[v] = false;
                    const unsigned knew = st.segk[sb[v]];
                    if (knew < kend) {
                        const int slot = 32 * v + lane;
                        const int c = slot - sb[v];
                        kk[v] = knew;
                        alive[v] = true;
                        blk[v] = 0;
                        d[v] = st.d0[c];
                        pv[v] = st.prev0[c];
                        const int r0 = st.rank0[c];
                        fo[v] = r0 + 1 < n ? (sb[v] + st.byrank0[r0 + 1]) * int(sizeof(float2)) : kSent;
                        st.order[sb[v] + r0] = slot;
                        st.rnk[slot] = r0;
                    }
                }
                __syncwarp();
                bool any_alive = false;
#pragma unroll
                for (int v = 0; v < V; ++v) any_alive |= alive[v];
                if (!__any_sync(kAll, any_alive)) break;
            } else if (!(state & 2u)) {
                break;
            }
            }

            // the block's normals: one Philox4x32-10 output per slot, counter (k, t >> 2, c, race)
            float z[V][4];
#pragma unroll
            for (int v = 0; v < V; ++v)
                draw_block<DIST>(kk[v], blk[v], uint32_t(32 * v + lane - sb[v]), rid, l.round_key, z[v]);
            // no slot is further into its rollout than the blocks the work item has run, so a
            // warp-uniform count-down rules out the step limit in all but the longest items
            bool near_limit = false;
            if (left == 0u) {
#pragma unroll
                for (int v = 0; v < V; ++v) near_limit |= alive[v] && int(blk[v]) * 4 + 4 > l.max_steps;
            } else {
                --left;
            }
            blk_fin = false;
            if (left == 0u && __any_sync(kAll, near_limit)) {
                blk_event = true;
                step(std::integral_constant<int, 0>{}, std::true_type{}, z);
                step(std::integral_constant<int, 1>{}, std::true_type{}, z);
                step(std::integral_constant<int, 2>{}, std::true_type{}, z);
                step(std::integral_constant<int, 3>{}, std::true_type{}, z);
                if constexpr (MODE == 1) block_end();
            } else {
                step(std::integral_constant<int, 0>{}, std::false_type{}, z);
                step(std::integral_constant<int, 1>{}, std::false_type{}, z);
                step(std::integral_constant<int, 2>{}, std::false_type{}, z);
                step(std::integral_constant<int, 3>{}, std::false_type{}, z);
                if constexpr (MODE == 1) {
                    if (blk_fin) block_end();
                }
                blk_event = blk_event || blk_fin;
            }
#pragma unroll
            for (int v = 0; v < V; ++v) ++blk[v];
        }

        // one global atomic per competitor with wins (per competitor and place in place mode), one
        // per work item for the step total
        __syncwarp();
        if constexpr (MODE == 1) {
            for (int i = lane; i < n * K && l.counts != nullptr; i += 32) {
                const int cc = pl_cnt[i];
                if (cc != 0) atomicAdd(&l.counts[(off + i / K) * l.places + i % K], cc);
            }
        } else {
            if (lane < n && st.wins[lane] != 0) atomicAdd(&l.counts[off + lane], st.wins[lane]);
        }
        for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(kAll, steps, o);
        if (lane == 0 && l.steps != nullptr) atomicAdd(l.steps + r, steps);
    }
    if (__any_sync(kAll, hit_limit) && lane == 0) atomicOr(l.status, kStatusStepLimit);
}

// Dynamic shared memory of a block: the warps' stages, then in place mode each warp's place
// lists (3 x 32 V ints) and [competitor][place] table (place_cells ints).
template <int V, int MODE>
size_t win_stage_bytes(int block, int place_cells)
{
    const size_t warps = size_t(block / 32);
    return warps * sizeof(WinStage<V>) + (MODE == 1 ? warps * (3 * 32 * V + size_t(place_cells)) * sizeof(int) : 0);
}

// The largest place table a launch may ask for (32 competitors x 32 places).
constexpr int kMaxPlaceCells = 32 * 32;

template <int V, int LAW, int MODE>
cudaError_t launch_win_vl(const RolloutLaunch &l, cudaStream_t stream)
{
    const size_t smem = win_stage_bytes<V, MODE>(l.block, l.place_cells);
    switch (l.b.dist) {
    case BBE_DIST_NORMAL: win_rollout_kernel<BBE_DIST_NORMAL, V, LAW, MODE><<<l.grid, l.block, smem, stream>>>(l); break;
    case BBE_DIST_UNIFORM: win_rollout_kernel<BBE_DIST_UNIFORM, V, LAW, MODE><<<l.grid, l.block, smem, stream>>>(l); break;
    default: win_rollout_kernel<BBE_DIST_TWO_POINT, V, LAW, MODE><<<l.grid, l.block, smem, stream>>>(l); break;
    }
    return cudaGetLastError();
}

// Blocks resident per SM.  Also lets the kernels take the dynamic shared memory of the largest
// block (16 warps may need more than the default 48 KB); every launch path asks this first.
template <int DIST, int V, int LAW, int MODE>
int win_resident_dvl(int block, int place_cells)
{
    const void *fn = reinterpret_cast<const void *>(win_rollout_kernel<DIST, V, LAW, MODE>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(win_stage_bytes<V, MODE>(512, MODE == 1 ? kMaxPlaceCells : 0))) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int nb = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, win_rollout_kernel<DIST, V, LAW, MODE>,
                                                                        block, win_stage_bytes<V, MODE>(block, place_cells));
    return e == cudaSuccess ? nb : 1;
}

// The launch and the residency query of the kernels of one responsiveness law and mode (each
// law's kernels are compiled in a translation unit of their own).
template <int LAW, int MODE>
cudaError_t launch_law(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream)
{
    switch (slots_per_lane) {
    case 4: return launch_win_vl<4, LAW, MODE>(l, stream);
    case 3: return launch_win_vl<3, LAW, MODE>(l, stream);
    case 2: return launch_win_vl<2, LAW, MODE>(l, stream);
    default: return launch_win_vl<1, LAW, MODE>(l, stream);
    }
}

template <int LAW, int MODE>
int resident_law(int dist, int slots_per_lane, int block, int place_cells)
{
    auto one = [&](auto Vc) {
        constexpr int V = decltype(Vc)::value;
        switch (dist) {
        case BBE_DIST_NORMAL: return win_resident_dvl<BBE_DIST_NORMAL, V, LAW, MODE>(block, place_cells);
        case BBE_DIST_UNIFORM: return win_resident_dvl<BBE_DIST_UNIFORM, V, LAW, MODE>(block, place_cells);
        default: return win_resident_dvl<BBE_DIST_TWO_POINT, V, LAW, MODE>(block, place_cells);
        }
    };
    switch (slots_per_lane) {
    case 4: return one(std::integral_constant<int, 4>{});
    case 3: return one(std::integral_constant<int, 3>{});
    case 2: return one(std::integral_constant<int, 2>{});
    default: return one(std::integral_constant<int, 1>{});
    }
}

cudaError_t launch_position_law(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream);
int resident_position_law(int dist, int slots_per_lane, int block);
cudaError_t launch_time_law(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream);
int resident_time_law(int dist, int slots_per_lane, int block);

}  // namespace win

}  // namespace bbe
