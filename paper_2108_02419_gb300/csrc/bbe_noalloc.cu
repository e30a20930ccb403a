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

struct NoallocHeader {
    int32_t queue[2];    // work-queue heads of the two rollout kernels
    int32_t status;      // device status bits written by the rollout kernels
    int32_t plan_error;  // bbe_status of the first invalid input found, 0 if none
    int32_t n_items[2];  // items per slots-per-lane value (1, 2)
    int32_t pad[2];
};

struct NoallocScratch {
    NoallocHeader h;
    int32_t race_items[2][kMaxRaces];  // per-race item counts, then offsets
    bbe::WorkItem items[kMaxItems];    // one-slot items first, then two-slot items
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

__device__ int slots_for_n(int n)
{
    if (n < 2) return 1;
    const int used1 = n * (32 / n);
    const int used2 = n * (32 / ((n + 1) / 2));
    return 2 * used1 < used2 ? 2 : 1;
}

__device__ int64_t chunk_for(int n, int64_t R, int cap)
{
    const int v = slots_for_n(n);
    const int nseg = 32 / ((n + v - 1) / v);
    const int64_t base = 32 * int64_t(nseg);
    const int64_t need = (R + cap - 1) / cap;  // keeps a race to at most `cap` items
    return base > need ? base : need;
}

__device__ void note_error(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// One block validates the batch, counts the work items of every race and writes the work
// list into the scratch array.  Every read of the caller's per-competitor arrays is
// bounded by n_competitors after the offsets have been checked.
__global__ void __launch_bounds__(kPlanThreads) plan_kernel(PlanArgs a)
{
    NoallocScratch &sc = g_noalloc_scratch;
    __shared__ int s_err;
    __shared__ int s_part[2][kPlanThreads];
    __shared__ int s_total[2];
    const int tid = threadIdx.x;
    if (tid == 0) s_err = 0;
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
        int items = 0, v = 1;
        if (err) {
            note_error(&s_err, err);
        } else {
            v = slots_for_n(n);
            const int64_t chunk = chunk_for(n, R, cap);
            items = int((R + chunk - 1) / chunk);
        }
        sc.race_items[v - 1][r] = items;
        sc.race_items[2 - v][r] = 0;
    }
    __syncthreads();
    // exclusive scan of the per-race item counts (contiguous chunks of races per thread)
    const int per = (a.n_races + kPlanThreads - 1) / kPlanThreads;
    const int r0 = tid * per;
    const int r1 = min(a.n_races, r0 + per);
    for (int v = 0; v < 2; ++v) {
        int sum = 0;
        for (int r = r0; r < r1; ++r) sum += sc.race_items[v][r];
        s_part[v][tid] = sum;
    }
    __syncthreads();
    if (tid < 2) {
        int run = 0;
        for (int i = 0; i < kPlanThreads; ++i) {
            const int x = s_part[tid][i];
            s_part[tid][i] = run;
            run += x;
        }
        s_total[tid] = run;
    }
    __syncthreads();
    for (int v = 0; v < 2; ++v) {
        int run = s_part[v][tid];
        for (int r = r0; r < r1; ++r) {
            const int x = sc.race_items[v][r];
            sc.race_items[v][r] = run;
            run += x;
        }
    }
    __syncthreads();
    const bool ok = s_err == 0;
    if (ok) {
        for (int r = tid; r < a.n_races; r += kPlanThreads) {
            const int n = a.race_off[r + 1] - a.race_off[r];
            const int v = slots_for_n(n);
            const int64_t R = a.R[r];
            const int64_t chunk = chunk_for(n, R, cap);
            int pos = (v == 2 ? s_total[0] : 0) + sc.race_items[v - 1][r];
            for (int64_t k = 0; k < R; k += chunk, ++pos) {
                const int64_t cnt = R - k < chunk ? R - k : chunk;
                sc.items[pos] = bbe::WorkItem{r, int32_t(k), int32_t(cnt), 0};
            }
        }
    }
    if (tid == 0) {
        sc.h.queue[0] = 0;
        sc.h.queue[1] = 0;
        sc.h.status = 0;
        sc.h.plan_error = s_err;
        sc.h.n_items[0] = ok ? s_total[0] : 0;
        sc.h.n_items[1] = ok ? s_total[1] : 0;
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

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
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
    const void *required[] = {race_off, track_len, rollouts, pos, mu, sigma, resp, pref, theta, win_counts};
    for (const void *p : required) {
        if (!p || !on_device(p)) {
            bbe::set_error("bbe_rollout_noalloc: every array must be non-null device memory "
                           "(pref and theta included; only prev_step and steps_total may be NULL)");
            return BBE_ERR_ARG;
        }
    }
    if ((prev_step && !on_device(prev_step)) || (steps_total && !on_device(steps_total))) {
        bbe::set_error("bbe_rollout_noalloc: prev_step / steps_total must be device memory");
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
        bbe::set_error("bbe_rollout_noalloc: invalid race batch (offsets, sizes 1..32, L > 0, R in 1..2^31-1, "
                       "0 <= d < L, mu > 0, sigma >= 0, rho in [0,1], P in (0,1], theta >= 0, prev > 0)");
        return static_cast<bbe_status>(h.plan_error);
    }

    NA_TRY(cudaMemsetAsync(win_counts, 0, size_t(n_competitors) * sizeof(int32_t), s));
    if (steps_total) NA_TRY(cudaMemsetAsync(steps_total, 0, size_t(n_races) * sizeof(int64_t), s));
    int dev = 0, sms = 0;
    NA_TRY(cudaGetDevice(&dev));
    NA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int block = 128;
    bbe::DevBatch b{race_off, track_len, rollouts, nullptr, pos, mu, sigma, resp, pref, theta, prev_step,
                    nullptr, n_races, n_competitors, race_id0, uint32_t(seed), uint32_t(seed >> 32), int32_t(dist)};
    for (int v = 2; v >= 1; --v) {
        if (h.n_items[v - 1] == 0) continue;
        bbe::RolloutLaunch l{};
        l.b = b;
        l.items = sc->items + (v == 2 ? h.n_items[0] : 0);
        l.n_items = h.n_items[v - 1];
        l.queue = &sc->h.queue[v - 1];
        l.counts = win_counts;
        l.steps = reinterpret_cast<unsigned long long *>(steps_total);
        l.status = &sc->h.status;
        l.max_steps = BBE_MAX_STEPS_DEFAULT;
        l.block = block;
        l.grid = sms * std::max(1, std::min(16, bbe::rollout_resident_blocks(int(dist), v, block)));
        bbe::fill_round_keys(l);
        NA_TRY(bbe::launch_rollout(l, v, s));
    }
    int32_t status = 0;
    NA_TRY(cudaMemcpyAsync(&status, &sc->h.status, sizeof(status), cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
    if (status & bbe::kStatusStepLimit) {
        bbe::set_error("bbe_rollout_noalloc: a rollout reached max_steps without a finisher");
        return BBE_ERR_STEP_LIMIT;
    }
    return BBE_OK;
}
