// bbe_internal.h -- types shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "bbe.h"

namespace bbe {

// Device view of a staged batch.  Per-competitor arrays are CSR over race_off.
struct DevBatch {
    const int32_t *race_off;  // [n_races + 1]
    const float *L;           // [n_races]
    const int64_t *R;         // [n_races]
    const int32_t *comp_race; // [n_total]: race of each competitor
    const float *d0, *mu, *sigma, *rho, *P, *theta, *prev0;  // [n_total]
    const int32_t *race_ids;  // [n_races] stream id of each race, or null: race_id0 + r
    int32_t n_races;
    int32_t n_total;
    uint32_t race_id0;
    uint32_t seed_lo, seed_hi;
    int32_t dist;
    int32_t law;              // responsiveness law: BBE_LAW_POSITION or BBE_LAW_TIME
    const float *t0;          // time law: [n_races] steps elapsed before the state
    const float *invT;        // time law: [n_races] 1 / expected duration in steps
};

// Responsiveness R_c of Eq. 1 at the start of step t of a dry-run (binary32, the oracle's
// operation order): the position law from the fraction of the track covered, the time law
// from the fraction of the expected duration elapsed, held at 1 once it is over.
template <int LAW>
__device__ __forceinline__ float responsiveness(float kr, float d, float invL, float t0, int t, float invT)
{
    if constexpr (LAW == BBE_LAW_TIME) {
        const float u = fminf(__fmul_rn(__fadd_rn(t0, __int2float_rn(t)), invT), 1.0f);
        return __fmaf_rn(kr, __fadd_rn(u, -0.5f), 1.0f);
    } else {
        return __fmaf_rn(kr, __fmaf_rn(d, invL, -0.5f), 1.0f);
    }
}

// A unit of the persistent kernel's work queue: rollouts k_begin .. k_begin+k_count-1
// of one race.
struct WorkItem {
    int32_t race;
    int32_t k_begin;
    int32_t k_count;
    int32_t pad;
};

struct RolloutLaunch {
    DevBatch b;
    const WorkItem *items;
    int32_t n_items;
    int32_t *queue;           // work-queue head, zeroed before each launch
    int32_t *counts;          // [n_total]
    unsigned long long *steps;  // [n_races] or null
    int32_t *status;          // device status bits
    int32_t max_steps;
    int32_t grid, block;
    uint32_t round_key[20];  // Philox round keys (k0, k1) of rounds 0..9, from the seed
    int32_t places;          // place-count kernel: places per competitor in `counts` (null: no place table)
    int32_t place_cells;     // place-count kernel: ints of each warp's [competitor][place] table (>= n K)
    int32_t seg_cap;         // most segments (concurrent rollouts) per warp, or 0: as many as fit
    int32_t *orders;         // place-count kernel, or null: ordered top-`places` tallies, n^places per race
    const int64_t *order_off;  // [n_races]: first entry of each race's tally table in `orders`
    unsigned long long *hist_keys;  // place-count kernel, or null: finishing-order hash tables (keys)
    int32_t *hist_counts;           // the count beside each key
    const int64_t *hist_off;        // [n_races + 1]: each race's table (a power of two of entries)
};

// An empty entry of a finishing-order hash table (no order key reaches it: keys < 2^64 - 1).
constexpr unsigned long long kEmptyOrderKey = ~0ull;

// Philox4x32-10 key schedule: round i uses (seed_lo + i * 0x9E3779B9, seed_hi + i * 0xBB67AE85).
inline void fill_round_keys(RolloutLaunch &l)
{
    for (int i = 0; i < 10; ++i) {
        l.round_key[2 * i] = l.b.seed_lo + uint32_t(i) * 0x9E3779B9u;
        l.round_key[2 * i + 1] = l.b.seed_hi + uint32_t(i) * 0xBB67AE85u;
    }
}

// Device status bits written by the kernels.
constexpr int32_t kStatusStepLimit = 1;
constexpr int32_t kStatusTableFull = 2;  // a finishing-order hash table had no free entry
constexpr int32_t kStatusBadIndex = 4;   // checked build: a device index check failed

// BBE_INDEX(i, n, status): the index i of an array of n entries.  The checked build (BBE_CHECKED
// defined; build.build(checked=True)) tests 0 <= i < n, and on failure records kStatusBadIndex in
// the status word and uses index 0 instead, so no access leaves its array; other builds use i
// as it is, with no code added.
#if defined(BBE_CHECKED) && BBE_CHECKED
#define BBE_INDEX(i, n, status) ::bbe::checked_index((i), (n), (status))
#else
#define BBE_INDEX(i, n, status) (i)
#endif

#ifdef __CUDACC__
template <typename I, typename N>
__device__ __forceinline__ I checked_index(I i, N n, int32_t *status)
{
    bool bad = int64_t(i) >= int64_t(n);
    if constexpr (std::is_signed<I>::value) bad = bad || i < I(0);
    if (bad) {
        atomicOr(status, kStatusBadIndex);
        return I(0);
    }
    return i;
}

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
#endif

// slots_per_lane: competitors held per lane (1 to 4; the place-count kernel takes 1, 2 or 4).
cudaError_t launch_rollout(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream);
// Blocks of `block` threads of the rollout kernel that fit on one SM at once.
int rollout_resident_blocks(int dist, int slots_per_lane, int block);
cudaError_t launch_win_probs(const DevBatch &b, const int32_t *counts, float *probs, float *odds,
                             cudaStream_t stream);
// The rollout kernel in place mode: counts [n_total][l.places], rollouts to the K-th finisher.
cudaError_t launch_place_rollout(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream);
int place_resident_blocks(int dist, int slots_per_lane, int block, int place_cells);
cudaError_t launch_place_probs(const DevBatch &b, int places, const int32_t *counts, int top, float *probs,
                               cudaStream_t stream);

void set_error(const std::string &msg);

}  // namespace bbe

// A staged batch of race states (opaque to the ABI, shared by the library's units).
struct bbe_batch {
    using DevBatch = bbe::DevBatch;
    using WorkItem = bbe::WorkItem;
    uint64_t serial = 0;  // unique per staged batch (cache key for plans built from it)
    int device = 0;
    int num_sms = 0;
    int32_t n_races = 0;
    int32_t n_total = 0;
    int32_t max_n = 0;
    uint64_t seed = 0;
    int32_t dist = 0;
    uint32_t race_id0 = 0;

    // host copies (scheduling, cost estimates, range checks and sub-batches)
    std::vector<int32_t> h_off;
    std::vector<float> h_L;
    std::vector<int64_t> h_R;
    std::vector<float> h_d0, h_mu, h_sigma, h_rho, h_P, h_theta;
    std::vector<float> h_prev;      // empty when the default previous step is used
    std::vector<int32_t> h_race_ids;  // empty when race r has stream id race_id0 + r
    std::vector<int64_t> h_k0;        // first rollout index of each race; empty when all are 0
    std::vector<float> h_t0, h_T;     // time law: elapsed steps and expected duration per race (empty: position law)
    void *law_mem = nullptr;          // time law: device t0[n_races], invT[n_races]

    // library-owned device memory
    void *arena = nullptr;
    DevBatch dev{};
    WorkItem *d_items = nullptr;  // items grouped by slots per lane (1, 2, 3, 4)
    int32_t n_items_v[4] = {0, 0, 0, 0};  // item counts per group
    int32_t *d_queue = nullptr;        // one queue head per group
    int32_t *d_status = nullptr;

    bbe_launch_cfg cfg{};
    int8_t slots_by_n[BBE_MAX_COMPETITORS + 1] = {};  // layout per competitor count (0: the default)
    int8_t default_slots = 2;  // the automatic layout: two per lane, one for a batch too small to fill the GPU
    int32_t seg_cap = 0;       // segments per warp at most (0: as many as fit); set for very small batches
    int32_t resident[4] = {1, 1, 1, 1};  // rollout-kernel blocks resident per SM, per group
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // graph cache (captured on the second pass with the same output buffers)
    int32_t *last_counts = nullptr;
    int64_t *last_steps = nullptr;

    // finishing-order tally layout (bbe_order_counts): first entry of each race's table
    int32_t order_places = 0;
    std::vector<int64_t> h_order_off;  // [n_races + 1]
    int64_t *d_order_off = nullptr;
    // finishing-order histogram layout (bbe_order_histogram): each race's hash table
    int32_t hist_places = 0;
    std::vector<int64_t> h_hist_off;  // [n_races + 1]
    int64_t *d_hist_off = nullptr;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int32_t *g_counts = nullptr;
    int64_t *g_steps = nullptr;

    // Streams that carried work reading this batch, each with an event recorded after its
    // latest use.  The batch's device memory comes from the library's stream-ordered pool and is
    // freed on the library's release stream behind those events, so replacing a buffer or
    // destroying the batch waits for this batch's own work only, never for the whole device.
    mutable std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
    cudaStream_t free_stream = nullptr;  // uploads of a rebuilt work list (made on first need)
};


namespace bbe {
// bbe_race_init with an optional explicit stream id per race (host array, may be null).
bbe_status stage_batch(bbe_batch **out, int32_t n_races, const int32_t *race_off, const float *track_len,
                       const int64_t *rollouts, const float *pos, const float *mu, const float *sigma,
                       const float *resp, const float *pref, const float *theta, const float *prev_step,
                       uint64_t seed, bbe_dist dist, uint32_t race_id0, const int32_t *race_ids,
                       cudaStream_t stream);
// Run rollouts k0[r] .. k0[r] + R[r] - 1 of race r instead of 0 .. R[r] - 1 (host array;
// k0[r] + R[r] <= 2^31 - 1).  The counts of such a batch added to those of rollouts
// 0 .. k0[r] - 1 equal the counts of one batch of k0[r] + R[r] rollouts.
bbe_status set_first_rollouts(bbe_batch *b, const int64_t *k0);
// Record that work just enqueued on `s` reads the batch (see bbe_batch::uses).
cudaError_t note_use(const bbe_batch *b, cudaStream_t s);
}  // namespace bbe

