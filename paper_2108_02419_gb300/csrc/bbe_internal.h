// bbe_internal.h -- types shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
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
    int32_t n_races;
    int32_t n_total;
    uint32_t race_id0;
    uint32_t seed_lo, seed_hi;
    int32_t dist;
};

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
};

// Device status bits written by the kernels.
constexpr int32_t kStatusStepLimit = 1;

// slots_per_lane: competitors held per lane (1 or 2).
cudaError_t launch_rollout(const RolloutLaunch &l, int slots_per_lane, cudaStream_t stream);
// Blocks of `block` threads of the rollout kernel that fit on one SM at once.
int rollout_resident_blocks(int dist, int slots_per_lane, int block);
cudaError_t launch_win_probs(const DevBatch &b, const int32_t *counts, float *probs, float *odds,
                             cudaStream_t stream);

void set_error(const std::string &msg);

}  // namespace bbe
