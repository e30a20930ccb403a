// bbe_noalloc.cu -- bbe_rollout_noalloc: the rollout pass without any memory allocation.
//
// Some callers cannot allocate GPU memory at the point where they need win counts: code
// running inside a memory pool they do not own, a real-time loop that must not call
// cudaMalloc (it can synchronise the device and stall other streams), or a host process
// whose allocator is locked by another framework.  bbe_race_init allocates a staged copy of
// the batch and a work list; this entry point instead reads the caller's device arrays
// directly and keeps its work list, queue heads and status word in one fixed, file-scope
// device array (g_noalloc_scratch below), which every GPU that loads the library holds
// until the process exits.  It runs the same rollout kernel as bbe_rollout_batch, so the
// counts are identical.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "bbe_internal.h"

namespace {

constexpr int kMaxRaces = BBE_NOALLOC_MAX_RACES;
constexpr int kMaxItems = BBE_NOALLOC_MAX_ITEMS;
constexpr int kPlanThreads = 1024;
constexpr int kMaxDevices = 64;
constexpr int kSlots = 2;              // competitors per lane: the library's automatic layout
constexpr int kRolloutsPerLane = 32;   // the library's default work-item size

struct NoallocHeader {
    int32_t queue;       // work-queue head of the rollout kernel
    int32_t status;      // device status bits written by the rollout kernel
    int32_t plan_error;  // bbe_status of the lowest-numbered invalid race, 0 if none
    int32_t plan_race;   // that race
    int32_t n_items;     // work items in the list
    int32_t pad[3];
};

struct NoallocScratch {
    NoallocHeader h;
    int32_t race_items[kMaxRaces];   // per-race item counts, then offsets
    bbe::WorkItem items[kMaxItems];  // the work list, race by race
};

// The only memory this entry point uses besides the caller's arrays.  Host code must not
// pass its name to a kernel (in host code it is a stand-in, not a device address); the
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

struct PlanArgs {
    int32_t n_races;
    int32_t n_competitors;
    const int32_t *race_off;
    const float *L;
    const int64_t *R;
    const float *d0, *mu, *sigma, *rho, *P, *theta, *prev0;
};

// Rollouts per work item: the library's (kRolloutsPerLane per segment of the warp, the warp
// holding floor(64 / n) segments), raised so that a race has at most `cap` items.
__device__ int64_t chunk_for(int n, int64_t R, int cap)
{
    const int64_t base = int64_t(kRolloutsPerLane) * (32 * kSlots / n);
    const int64_t need = (R + cap - 1) / cap;
    return base > need ? base : need;
}

// One block validates the batch, counts the work items of every race and writes the work
// list into the scratch array.  Every read of the caller's per-competitor arrays is
// bounded by n_competitors after the offsets have been checked.  An invalid batch writes no
// items and reports its lowest-numbered invalid race (as bbe_race_init does).
__global__ void __launch_bounds__(kPlanThreads) plan_kernel(PlanArgs a)
{
    NoallocScratch &sc = g_noalloc_scratch;
    __shared__ int s_err;  // least (race * 8 + |status|) over invalid races
    __shared__ int s_part[kPlanThreads];
    __shared__ int s_total;
    const int tid = threadIdx.x;
    if (tid == 0) s_err = INT_MAX;
    __syncthreads();
    const int cap = kMaxItems / a.n_races;
    for (int r = tid; r < a.n_races; r += kPlanThreads) {
        int err = 0;
        const int o0 = a.race_off[r], o1 = a.race_off[r + 1];
        if (r == 0 && o0 != 0) err = BBE_ERR_ARG;
        if (o0 < 0 || o1 > a.n_competitors || o1 < o0) err = BBE_ERR_ARG;
        const int n = o1 - o0;
        if (!err && (n < 1 || n > BBE_MAX_COMPETITORS)) err = BBE_ERR_UNSUPPORTED;
        const float L = a.L[r];
        const int64_t R = a.R[r];
        if (!err && (!isfinite(L) || !(L > 0.0f) || R < 1 || R > 0x7FFFFFFFLL)) err = BBE_ERR_ARG;
        for (int i = o0; !err && i < o1; ++i) {
            const float d = a.d0[i];
            if (!isfinite(d) || d < 0.0f) err = BBE_ERR_ARG;
            else if (d >= L) err = BBE_ERR_FINISHED;
            else if (!isfinite(a.mu[i]) || !(a.mu[i] > 0.0f) || !isfinite(a.sigma[i]) || !(a.sigma[i] >= 0.0f))
                err = BBE_ERR_ARG;
            else if (!(a.rho[i] >= 0.0f && a.rho[i] <= 1.0f) || !(a.P[i] > 0.0f && a.P[i] <= 1.0f))
                err = BBE_ERR_ARG;
            else if (!isfinite(a.theta[i]) || !(a.theta[i] >= 0.0f))
                err = BBE_ERR_ARG;
            else if (a.prev0 && (!isfinite(a.prev0[i]) || !(a.prev0[i] > 0.0f)))
                err = BBE_ERR_ARG;
        }
        int items = 0;
        if (err) atomicMin(&s_err, r * 8 - err);
        else items = int((R + chunk_for(n, R, cap) - 1) / chunk_for(n, R, cap));
        sc.race_items[r] = items;
    }
    __syncthreads();
    // exclusive scan of the per-race item counts (contiguous chunks of races per thread)
    const int per = (a.n_races + kPlanThreads - 1) / kPlanThreads;
    const int r0 = tid * per;
    const int r1 = min(a.n_races, r0 + per);
    int sum = 0;
    for (int r = r0; r < r1; ++r) sum += sc.race_items[r];
    s_part[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int i = 0; i < kPlanThreads; ++i) {
            const int x = s_part[i];
            s_part[i] = run;
            run += x;
        }
        s_total = run;
        // at most cap items per race keeps the list within the array; checked all the same
        if (run > kMaxItems && s_err == INT_MAX) s_err = 8 * a.n_races - BBE_ERR_RANGE;
    }
    __syncthreads();
    int run = s_part[tid];
    for (int r = r0; r < r1; ++r) {
        const int x = sc.race_items[r];
        sc.race_items[r] = run;
        run += x;
    }
    __syncthreads();
    const bool ok = s_err == INT_MAX;
    if (ok) {
        for (int r = tid; r < a.n_races; r += kPlanThreads) {
            const int n = a.race_off[r + 1] - a.race_off[r];
            const int64_t R = a.R[r];
            const int64_t chunk = chunk_for(n, R, cap);
            int pos = sc.race_items[r];
            for (int64_t k = 0; k < R; k += chunk, ++pos) {
                const int64_t cnt = R - k < chunk ? R - k : chunk;
                sc.items[pos] = bbe::WorkItem{r, int32_t(k), int32_t(cnt), 0};
            }
        }
    }
    if (tid == 0) {
        sc.h.queue = 0;
        sc.h.status = 0;
        sc.h.plan_error = ok ? 0 : -(s_err & 7);
        sc.h.plan_race = ok ? -1 : s_err >> 3;
        sc.h.n_items = ok ? s_total : 0;
    }
}

std::mutex g_mu;
NoallocScratch *g_scratch_addr[kMaxDevices] = {};

bbe_status scratch_for_current_device(NoallocScratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        bbe::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return BBE_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            bbe::set_error(std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
            return BBE_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_scratch_addr[dev];
    return BBE_OK;
}

// p is device memory of device `dev` (or managed memory, which any device may read)
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}

}  // namespace

#define NA_TRY(expr)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            bbe::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));            \
            return BBE_ERR_CUDA;                                                            \
        }                                                                                   \
    } while (0)

extern "C" BBE_API bbe_status bbe_rollout_noalloc(int32_t n_races, int32_t n_competitors, const int32_t *race_off,
                                                  const float *track_len, const int64_t *rollouts, const float *pos,
                                                  const float *mu, const float *sigma, const float *resp,
                                                  const float *pref, const float *theta, const float *prev_step,
                                                  uint64_t seed, bbe_dist dist, uint32_t race_id0,
                                                  int32_t *win_counts, int64_t *steps_total, void *cuda_stream)
{
    if (n_races < 1 || n_races > kMaxRaces) {
        bbe::set_error("bbe_rollout_noalloc: n_races must be 1.." + std::to_string(kMaxRaces) + ", got " +
                       std::to_string(n_races));
        return BBE_ERR_RANGE;
    }
    if (n_competitors < 1 || n_competitors > kMaxRaces * BBE_MAX_COMPETITORS) {
        bbe::set_error("bbe_rollout_noalloc: n_competitors out of range");
        return BBE_ERR_RANGE;
    }
    if (int(dist) < 0 || int(dist) > 2) {
        bbe::set_error("bbe_rollout_noalloc: unknown distribution");
        return BBE_ERR_ARG;
    }
    int dev = 0, sms = 0;
    NA_TRY(cudaGetDevice(&dev));
    const void *required[] = {race_off, track_len, rollouts, pos, mu, sigma, resp, pref, theta, win_counts};
    for (const void *p : required) {
        if (!p || !on_device(p, dev)) {
            bbe::set_error("bbe_rollout_noalloc: every array must be non-null memory of the current device "
                           "(pref and theta included; only prev_step and steps_total may be NULL)");
            return BBE_ERR_ARG;
        }
    }
    if ((prev_step && !on_device(prev_step, dev)) || (steps_total && !on_device(steps_total, dev))) {
        bbe::set_error("bbe_rollout_noalloc: prev_step / steps_total must be memory of the current device");
        return BBE_ERR_ARG;
    }
    NoallocScratch *sc = nullptr;
    bbe_status st = scratch_for_current_device(&sc);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);

    plan_kernel<<<1, kPlanThreads, 0, s>>>(
        PlanArgs{n_races, n_competitors, race_off, track_len, rollouts, pos, mu, sigma, resp, pref, theta, prev_step});
    NA_TRY(cudaGetLastError());
    NoallocHeader h;
    NA_TRY(cudaMemcpyAsync(&h, &sc->h, sizeof(h), cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
    if (h.plan_error != 0) {
        bbe::set_error("bbe_rollout_noalloc: race " + std::to_string(h.plan_race) +
                       " is invalid (offsets, sizes 1..32, L > 0, R in 1..2^31-1, 0 <= d < L, mu > 0, "
                       "sigma >= 0, rho in [0,1], P in (0,1], theta >= 0, prev > 0)");
        return static_cast<bbe_status>(h.plan_error);
    }

    NA_TRY(cudaMemsetAsync(win_counts, 0, size_t(n_competitors) * sizeof(int32_t), s));
    if (steps_total) NA_TRY(cudaMemsetAsync(steps_total, 0, size_t(n_races) * sizeof(int64_t), s));
    NA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int block = 128;
    bbe::DevBatch b{race_off, track_len, rollouts, nullptr, pos, mu, sigma, resp, pref, theta, prev_step,
                    nullptr, n_races, n_competitors, race_id0, uint32_t(seed), uint32_t(seed >> 32), int32_t(dist)};
    if (h.n_items > 0) {
        bbe::RolloutLaunch l{};
        l.b = b;
        l.items = sc->items;
        l.n_items = h.n_items;
        l.queue = &sc->h.queue;
        l.counts = win_counts;
        l.steps = reinterpret_cast<unsigned long long *>(steps_total);
        l.status = &sc->h.status;
        l.max_steps = BBE_MAX_STEPS_DEFAULT;
        l.block = block;
        l.grid = sms * std::max(1, std::min(16, bbe::rollout_resident_blocks(int(dist), kSlots, block)));
        l.grid = std::max(1, std::min(l.grid, (l.n_items + block / 32 - 1) / (block / 32)));  // no idle warps
        bbe::fill_round_keys(l);
        NA_TRY(bbe::launch_rollout(l, kSlots, s));
    }
    int32_t status = 0;
    NA_TRY(cudaMemcpyAsync(&status, &sc->h.status, sizeof(status), cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
    if (status & bbe::kStatusBadIndex) {
        bbe::set_error("bbe_rollout_noalloc: a device index check failed (checked build)");
        return BBE_ERR_RANGE;
    }
    if (status & bbe::kStatusStepLimit) {
        bbe::set_error("bbe_rollout_noalloc: a rollout reached max_steps without a finisher");
        return BBE_ERR_STEP_LIMIT;
    }
    return BBE_OK;
}
