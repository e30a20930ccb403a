// bbe_capi.cu -- the C ABI declared in include/bbe.h: validation and staging of race
// batches, the persistent launch (replayed from an instantiated CUDA graph), the launch
// autotuner and the win-probability finaliser.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "bbe_internal.h"

namespace bbe {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

}  // namespace bbe

using bbe::set_error;

namespace {

#define BBE_CUDA_TRY(expr)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));                 \
            return BBE_ERR_CUDA;                                                            \
        }                                                                                   \
    } while (0)

constexpr int32_t kDefaultWarpsPerBlock = 4;
constexpr int32_t kDefaultBlocksPerSm = 16;
constexpr int32_t kDefaultRolloutsPerLane = 32;
constexpr int64_t kMaxItemsPerRace = 256;
constexpr int64_t kMaxItems = int64_t(1) << 21;

bool finite(float x) { return std::isfinite(x); }

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

bool is_host_memory(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeUnregistered || at.type == cudaMemoryTypeHost;
}

// copy caller memory (host or device) into a host vector: memcpy for host memory, an
// asynchronous device-to-host copy otherwise (the caller synchronises the stream)
bbe_status copy_in(void *dst, const void *src, size_t bytes, cudaStream_t s, const char *what)
{
    if (bytes == 0) return BBE_OK;
    if (is_host_memory(src)) {
        std::memcpy(dst, src, bytes);
        return BBE_OK;
    }
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    if (e != cudaSuccess) {
        set_error(std::string("copy of ") + what + ": " + cudaGetErrorString(e));
        return BBE_ERR_CUDA;
    }
    return BBE_OK;
}

// Device memory of staged batches comes from one stream-ordered pool per device owned by the
// library, which keeps up to kPoolKeep bytes of freed memory for the next batch (the default
// pool hands freed memory back at once, and mapping it again costs ~90 us per batch); it is
// never the process's default pool, whose settings other libraries may rely on.
constexpr uint64_t kPoolKeep = uint64_t(256) << 20;
// Arenas up to this size are uploaded in one copy from a host image of the arena.
constexpr size_t kOneCopyBytes = size_t(4) << 20;

cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t s)
{
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = pools.find(dev);
        if (it == pools.end()) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
            uint64_t keep = kPoolKeep;
            if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
            pools[dev] = pool;
        } else {
            pool = it->second;
        }
    }
    return cudaMallocFromPoolAsync(ptr, bytes, pool, s);
}

void free_graph(bbe_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);  // an executable graph still running is freed when it ends
    b->gexec = nullptr;
    b->g_counts = nullptr;
    b->g_steps = nullptr;
}

cudaError_t ensure_free_stream(bbe_batch *b)
{
    return b->free_stream ? cudaSuccess : cudaStreamCreateWithFlags(&b->free_stream, cudaStreamNonBlocking);
}

// One stream per device on which the library releases batch memory (made once): each release
// waits there for the events of its own batch's uses, so the host and the callers' streams never
// wait, and no stream is made per batch.
cudaError_t release_stream(cudaStream_t *out)
{
    static std::mutex mu;
    static std::map<int, cudaStream_t> streams;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    auto it = streams.find(dev);
    if (it == streams.end()) {
        cudaStream_t st = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
        it = streams.emplace(dev, st).first;
    }
    *out = it->second;
    return cudaSuccess;
}

// Free `p` (stream-ordered allocation) once every recorded use of the batch has completed; the
// host does not wait.
cudaError_t free_behind_uses(bbe_batch *b, void *p)
{
    if (!p) return cudaSuccess;
    cudaStream_t rs = nullptr;
    cudaError_t e = release_stream(&rs);
    for (auto &u : b->uses)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(rs, u.second, 0);
    if (e == cudaSuccess) e = cudaFreeAsync(p, rs);
    return e;
}

// Expected steps of one rollout: the leader's remaining distance over the largest mean
// step (used only to order the work queue, longest items first).
double est_steps(const bbe_batch *b, int r)
{
    const int a = b->h_off[r], e = b->h_off[r + 1];
    float lead = 0.0f, vmax = 0.0f;
    for (int i = a; i < e; ++i) {
        lead = std::max(lead, b->h_d0[i]);
        vmax = std::max(vmax, b->h_mu[i]);
    }
    return 1.0 + double(b->h_L[r] - lead) / double(std::max(vmax, 1e-3f));
}

// Slots-per-lane groups: group g holds races run with kSlots[g] competitors per lane.
constexpr int kGroups = 4;
constexpr int kSlots[kGroups] = {1, 2, 3, 4};

int group_of(int v) { return v - 1; }

// Competitors per lane for a race of n.  Automatic choice (`dflt`): two, the layout measured
// fastest on GB300 for the uneven mix of 2..24 competitors (3.13e11 competitor-steps/s against
// 1.72e11 with one per lane up to 5 and four for 21..24, whose four-slot kernel runs short of
// registers); one for a batch too small to fill the GPU's warps (build_items), where the
// latency of a warp's step decides (a 5-competitor race of 10^3 rollouts: 0.061 ms a pass
// against 0.091).  `mode` forces a layout, `by_n` gives one per competitor count.
int slots_for(int n, int mode, const int8_t *by_n = nullptr, int dflt = 2)
{
    const int v = mode != 0 ? mode : (by_n && by_n[n] ? by_n[n] : dflt);  // forced, the per-count table, or automatic
    return n >= v ? v : std::min(n, 2);  // a layout wider than the race falls back
}

// A run of work items of one race, each of `chunk` rollouts, the first from rollout k0 on;
// `first` is the run's first index in the list (the run ends where the next one starts).
struct ItemRun {
    int32_t race, k0, chunk, first;
};

// items[i] for every list index i: the run holding i (the last whose first index is at most i,
// by binary search over the runs in list order), then its item i - first.
__global__ void expand_items(const ItemRun *__restrict__ runs, int32_t n_runs, int32_t total,
                             bbe::WorkItem *__restrict__ items)
{
    const int32_t i = int32_t(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= total) return;
    int32_t lo = 0, hi = n_runs - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (runs[mid].first <= i) lo = mid;
        else hi = mid - 1;
    }
    const ItemRun r = runs[lo];
    items[i] = bbe::WorkItem{r.race, r.k0 + (i - r.first) * r.chunk, r.chunk, 0};
}

bbe_status build_items(bbe_batch *b, cudaStream_t upload = nullptr)
{
    // Per race: full chunks of `chunk` rollouts (all of one cost) and a remainder.  The list puts
    // longer work first: full chunks race by race in descending cost per chunk, then the
    // remainders in descending cost.  Sorting races rather than items keeps the host work
    // proportional to the number of races.
    struct RacePlan {
        int32_t race;
        int64_t chunk, full, rem, k0;
        double cost_full, cost_rem;
    };
    std::vector<RacePlan> plans[kGroups];
    // keep the whole list near kMaxItems items: very large batches get larger items
    int64_t total_rollouts = 0;
    for (int r = 0; r < b->n_races; ++r) total_rollouts += b->h_R[r];
    const int64_t min_chunk = (total_rollouts + kMaxItems - 1) / kMaxItems;
    int64_t race_items = kMaxItemsPerRace;  // items per race at most (lifted for very small batches)
    auto chunk_of = [&](int r, int64_t per_lane, int nseg) {
        // at least per_lane rollouts per segment, at most race_items items per race
        return std::max<int64_t>(std::max<int64_t>(per_lane * nseg, (b->h_R[r] + race_items - 1) / race_items), min_chunk);
    };
    auto nseg_of = [&](int r) {  // segments of a warp: floor(32 V / n) slots of n
        const int n = b->h_off[r + 1] - b->h_off[r];
        const int fit = 32 * slots_for(n, b->cfg.slots_per_lane, b->slots_by_n, b->default_slots) / n;
        return b->seg_cap > 0 ? std::min(fit, b->seg_cap) : fit;
    };
    // A batch too small to give every warp the GPU can hold (64 per SM) a work item runs fewer
    // rollouts per lane, down to one: the chunking decides which warp runs a rollout, never its
    // result.  (An item holds at most 32 x per_lane rollouts, so large batches skip the count.)
    int64_t per_lane = b->cfg.rollouts_per_lane;
    const int64_t warp_slots = int64_t(std::max(1, b->num_sms)) * 64;
    auto items_at = [&](int64_t pl) {  // items of the list at pl rollouts per lane, counted up to warp_slots
        int64_t items = 0;
        for (int r = 0; r < b->n_races && items < warp_slots; ++r) {
            const int64_t chunk = chunk_of(r, pl, nseg_of(r));
            items += (b->h_R[r] + chunk - 1) / chunk;
        }
        return items;
    };
    b->default_slots = 2;
    b->seg_cap = 0;
    while (per_lane > 1 && total_rollouts < warp_slots * per_lane * 32) {
        if (items_at(per_lane) >= warp_slots) break;
        per_lane = std::max<int64_t>(1, per_lane / 2);
    }
    // still short of work for every warp at one rollout per lane: one competitor per lane, and
    // as few concurrent rollouts per warp as keep the list within the warp slots (a warp's step
    // then waits on fewer segments' rank repairs; a race may then take up to one item per warp
    // slot, so that each segment runs one rollout)
    if (per_lane == 1 && total_rollouts < warp_slots * 32 && items_at(1) < warp_slots) {
        b->default_slots = 1;
        race_items = warp_slots;
        for (int32_t cap = 1; cap < 32; cap *= 2) {
            b->seg_cap = cap;
            if (items_at(1) < warp_slots) break;
            b->seg_cap = 0;
        }
        if (b->seg_cap == 0) race_items = kMaxItemsPerRace;
    }
    size_t total = 0;
    for (int r = 0; r < b->n_races; ++r) {
        const int n = b->h_off[r + 1] - b->h_off[r];
        const int v = slots_for(n, b->cfg.slots_per_lane, b->slots_by_n, b->default_slots);
        const int nseg = nseg_of(r);
        const int64_t chunk = chunk_of(r, per_lane, nseg);
        const double st = est_steps(b, r);
        RacePlan pl{r, chunk, b->h_R[r] / chunk, b->h_R[r] % chunk, b->h_k0.empty() ? 0 : b->h_k0[r], 0.0, 0.0};
        pl.cost_full = double((chunk + nseg - 1) / nseg) * st;
        pl.cost_rem = double((pl.rem + nseg - 1) / nseg) * st;
        total += size_t(pl.full) + (pl.rem > 0 ? 1 : 0);
        plans[group_of(v)].push_back(pl);
    }
    if (total > size_t(INT32_MAX)) {
        set_error("work list too long; raise rollouts_per_lane");
        return BBE_ERR_RANGE;
    }
    // the list as runs of equal items (a race's full chunks, then its remainder), expanded into
    // items on the device: 16 bytes per run cross the bus instead of 16 per item
    std::vector<ItemRun> runs;
    runs.reserve(size_t(2) * size_t(b->n_races));
    int32_t listed = 0;
    for (int g = 0; g < kGroups; ++g) {
        std::vector<RacePlan> &pg = plans[g];
        const int32_t before = listed;
        std::stable_sort(pg.begin(), pg.end(), [](const RacePlan &x, const RacePlan &y) { return x.cost_full > y.cost_full; });
        for (const RacePlan &pl : pg) {
            if (pl.full == 0) continue;
            runs.push_back(ItemRun{pl.race, int32_t(pl.k0), int32_t(pl.chunk), listed});
            listed += int32_t(pl.full);
        }
        std::stable_sort(pg.begin(), pg.end(), [](const RacePlan &x, const RacePlan &y) { return x.cost_rem > y.cost_rem; });
        for (const RacePlan &pl : pg) {
            if (pl.rem == 0) continue;
            runs.push_back(ItemRun{pl.race, int32_t(pl.k0 + pl.full * pl.chunk), int32_t(pl.rem), listed});
            listed += 1;
        }
        b->n_items_v[g] = listed - before;
    }

    // the new list is in place before the call returns (made on `upload`, the staging call's
    // stream, else on the batch's free stream); the old one is freed behind this batch's work
    // that may still read it
    bbe::WorkItem *fresh = nullptr;
    ItemRun *d_runs = nullptr;
    if (!upload) {
        BBE_CUDA_TRY(ensure_free_stream(b));
        upload = b->free_stream;
    }
    BBE_CUDA_TRY(pool_alloc(reinterpret_cast<void **>(&fresh), std::max<size_t>(1, size_t(listed)) * sizeof(bbe::WorkItem), upload));
    if (!runs.empty()) {
        BBE_CUDA_TRY(pool_alloc(reinterpret_cast<void **>(&d_runs), runs.size() * sizeof(ItemRun), upload));
        BBE_CUDA_TRY(cudaMemcpyAsync(d_runs, runs.data(), runs.size() * sizeof(ItemRun), cudaMemcpyHostToDevice, upload));
        expand_items<<<unsigned((listed + 255) / 256), 256, 0, upload>>>(d_runs, int32_t(runs.size()), listed, fresh);
        BBE_CUDA_TRY(cudaGetLastError());
        BBE_CUDA_TRY(cudaFreeAsync(d_runs, upload));
    }
    BBE_CUDA_TRY(cudaStreamSynchronize(upload));
    free_graph(b);
    BBE_CUDA_TRY(free_behind_uses(b, b->d_items));
    b->d_items = fresh;
    return BBE_OK;
}

bbe_status check_cfg(const bbe_launch_cfg &c)
{
    if (c.warps_per_block < 1 || c.warps_per_block > 16 || c.blocks_per_sm < 1 || c.blocks_per_sm > 32 ||
        c.rollouts_per_lane < 1 || c.rollouts_per_lane > 65536 || c.max_steps < 1 || c.max_steps > (1 << 30) ||
        c.slots_per_lane < 0 || c.slots_per_lane > 4) {
        set_error("launch configuration out of range");
        return BBE_ERR_ARG;
    }
    return BBE_OK;
}

bbe::RolloutLaunch make_launch(const bbe_batch *b, int32_t *counts, int64_t *steps, int g)
{
    bbe::RolloutLaunch l{};
    l.b = b->dev;
    int first = 0;
    for (int h = 0; h < g; ++h) first += b->n_items_v[h];
    l.items = b->d_items + first;
    l.n_items = b->n_items_v[g];
    l.queue = b->d_queue + g;
    l.counts = counts;
    l.steps = reinterpret_cast<unsigned long long *>(steps);
    l.status = b->d_status;
    l.max_steps = b->cfg.max_steps;
    l.seg_cap = b->seg_cap;
    l.block = 32 * b->cfg.warps_per_block;
    // persistent grid: never more blocks than can be resident at once, nor more warps than work
    // items (a warp runs one item at a time; a small batch then launches and drains faster)
    l.grid = std::max(1, b->num_sms * std::min(b->cfg.blocks_per_sm, std::max(1, b->resident[g])));
    l.grid = std::max(1, std::min(l.grid, (l.n_items + b->cfg.warps_per_block - 1) / b->cfg.warps_per_block));
    bbe::fill_round_keys(l);
    return l;
}

// The launch sequence of one rollout pass: reset queues, status and outputs, then one
// persistent kernel per non-empty slots-per-lane group, the group with most slots first.
// With a side stream the first kernel runs on `s` and the others on `side`, so that they
// fill SMs as the first kernel's blocks retire.
cudaError_t enqueue_pass(const bbe_batch *b, int32_t *counts, int64_t *steps, cudaStream_t s, cudaStream_t side)
{
    cudaError_t e = cudaMemsetAsync(b->d_queue, 0, kGroups * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, size_t(b->n_total) * sizeof(int32_t), s);
    if (e == cudaSuccess && steps) e = cudaMemsetAsync(steps, 0, size_t(b->n_races) * sizeof(int64_t), s);
    int groups[kGroups], ng = 0;
    for (int g = kGroups - 1; g >= 0; --g)
        if (b->n_items_v[g] > 0) groups[ng++] = g;
    if (e != cudaSuccess || ng == 0) return e;
    if (ng > 1 && side) {
        e = cudaEventRecord(b->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, b->ev_fork, 0);
        if (e == cudaSuccess) e = bbe::launch_rollout(make_launch(b, counts, steps, groups[0]), kSlots[groups[0]], s);
        for (int i = 1; i < ng && e == cudaSuccess; ++i)
            e = bbe::launch_rollout(make_launch(b, counts, steps, groups[i]), kSlots[groups[i]], side);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join, side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join, 0);
        return e;
    }
    for (int i = 0; i < ng && e == cudaSuccess; ++i)
        e = bbe::launch_rollout(make_launch(b, counts, steps, groups[i]), kSlots[groups[i]], s);
    return e;
}

// The streams and events a pass needs, made on first need: the side stream and fork/join events
// only for a pass of more than one layout group, the capture stream only for a captured graph.
bbe_status ensure_aux(bbe_batch *b, bool capture = false)
{
    int groups = 0;
    for (int g = 0; g < kGroups; ++g) groups += b->n_items_v[g] > 0 ? 1 : 0;
    if (capture && !b->capture_stream)
        BBE_CUDA_TRY(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    if (groups > 1) {
        if (!b->side_stream) BBE_CUDA_TRY(cudaStreamCreateWithFlags(&b->side_stream, cudaStreamNonBlocking));
        if (!b->ev_fork) BBE_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
        if (!b->ev_join) BBE_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
    }
    return BBE_OK;
}

bbe_status ensure_graph(bbe_batch *b, int32_t *counts, int64_t *steps)
{
    if (b->gexec && b->g_counts == counts && b->g_steps == steps) return BBE_OK;
    free_graph(b);
    bbe_status st = ensure_aux(b, true);
    if (st) return st;
    BBE_CUDA_TRY(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_pass(b, counts, steps, b->capture_stream, b->side_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        set_error(std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return BBE_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->gexec = nullptr;
        set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
        return BBE_ERR_CUDA;
    }
    b->g_counts = counts;
    b->g_steps = steps;
    return BBE_OK;
}

template <typename T>
T *carve(char *&p, size_t count)
{
    T *out = reinterpret_cast<T *>(p);
    p += (count * sizeof(T) + 255) / 256 * 256;
    return out;
}

}  // namespace

bbe_status bbe::stage_batch(bbe_batch **out, int32_t n_races, const int32_t *race_off, const float *track_len,
                            const int64_t *rollouts, const float *pos, const float *mu, const float *sigma,
                            const float *resp, const float *pref, const float *theta, const float *prev_step,
                            uint64_t seed, bbe_dist dist, uint32_t race_id0, const int32_t *race_ids,
                            cudaStream_t s)
{
    if (!out) {
        set_error("out is NULL");
        return BBE_ERR_ARG;
    }
    *out = nullptr;
    if (n_races < 1 || !race_off || !track_len || !rollouts || !pos || !mu || !sigma || !resp) {
        set_error("n_races < 1 or a required array is NULL");
        return BBE_ERR_ARG;
    }
    if (int(dist) < 0 || int(dist) > 2) {
        set_error("unknown distribution");
        return BBE_ERR_ARG;
    }
    std::vector<int32_t> off(size_t(n_races) + 1);
    bbe_status st = copy_in(off.data(), race_off, off.size() * sizeof(int32_t), s, "race_off");
    if (st) return st;
    BBE_CUDA_TRY(cudaStreamSynchronize(s));
    if (off[0] != 0) {
        set_error("race_off[0] != 0");
        return BBE_ERR_ARG;
    }
    int32_t max_n = 0;
    for (int r = 0; r < n_races; ++r) {
        const int64_t n = int64_t(off[r + 1]) - off[r];
        if (n < 0) {
            set_error("race_off is not monotone at race " + std::to_string(r));
            return BBE_ERR_ARG;
        }
        if (n < 1 || n > BBE_MAX_COMPETITORS) {
            set_error("race " + std::to_string(r) + " has " + std::to_string(n) + " competitors (supported: 1..32)");
            return BBE_ERR_UNSUPPORTED;
        }
        max_n = std::max<int32_t>(max_n, int32_t(n));
    }
    const int32_t nt = off[n_races];

    auto b = new bbe_batch();
    static std::atomic<uint64_t> next_serial{1};
    b->serial = next_serial.fetch_add(1);
    b->n_races = n_races;
    b->n_total = nt;
    b->max_n = max_n;
    b->seed = seed;
    b->dist = int32_t(dist);
    b->race_id0 = race_id0;
    b->h_off = off;
    b->h_L.resize(n_races);
    b->h_R.resize(n_races);
    b->h_d0.resize(nt);
    b->h_mu.resize(nt);
    b->h_sigma.resize(nt);
    b->h_rho.resize(nt);
    b->h_P.assign(nt, 1.0f);
    b->h_theta.assign(nt, BBE_THETA_DEFAULT);
    if (race_ids) b->h_race_ids.assign(race_ids, race_ids + n_races);
    std::vector<float> &h_sigma = b->h_sigma, &h_rho = b->h_rho, &h_P = b->h_P, &h_theta = b->h_theta,
                       &h_prev = b->h_prev;
    auto fail = [&](bbe_status code) {
        bbe_destroy_batch(b);  // frees whatever was allocated so far
        return code;
    };
    if ((st = copy_in(b->h_L.data(), track_len, n_races * sizeof(float), s, "track_len")) ||
        (st = copy_in(b->h_R.data(), rollouts, n_races * sizeof(int64_t), s, "rollouts")) ||
        (st = copy_in(b->h_d0.data(), pos, nt * sizeof(float), s, "pos")) ||
        (st = copy_in(b->h_mu.data(), mu, nt * sizeof(float), s, "mu")) ||
        (st = copy_in(h_sigma.data(), sigma, nt * sizeof(float), s, "sigma")) ||
        (st = copy_in(h_rho.data(), resp, nt * sizeof(float), s, "resp")) ||
        (pref && (st = copy_in(h_P.data(), pref, nt * sizeof(float), s, "pref"))) ||
        (theta && (st = copy_in(h_theta.data(), theta, nt * sizeof(float), s, "theta"))))
        return fail(st);
    if (prev_step) {
        h_prev.resize(nt);
        if ((st = copy_in(h_prev.data(), prev_step, nt * sizeof(float), s, "prev_step"))) return fail(st);
    }
    {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error(std::string("staging copies: ") + cudaGetErrorString(e));
            return fail(BBE_ERR_CUDA);
        }
    }
    // validation (Section 3: S > 0, P in [0,1], positions on the track)
    for (int r = 0; r < n_races; ++r) {
        const float L = b->h_L[r];
        if (!finite(L) || !(L > 0.0f)) {
            set_error("track_len of race " + std::to_string(r) + " is not a positive finite number");
            return fail(BBE_ERR_ARG);
        }
        if (b->h_R[r] < 1 || b->h_R[r] > INT32_MAX) {
            set_error("rollouts of race " + std::to_string(r) + " outside 1..2^31-1");
            return fail(BBE_ERR_ARG);
        }
        for (int i = off[r]; i < off[r + 1]; ++i) {
            const float d = b->h_d0[i];
            auto where = [&]() { return " (race " + std::to_string(r) + ", competitor " + std::to_string(i - off[r]) + ")"; };
            if (!finite(d) || d < 0.0f) {
                set_error("position must be finite and >= 0" + where());
                return fail(BBE_ERR_ARG);
            }
            if (d >= L) {
                set_error("competitor already finished (d >= L)" + where());
                return fail(BBE_ERR_FINISHED);
            }
            if (!finite(b->h_mu[i]) || !(b->h_mu[i] > 0.0f) || !finite(h_sigma[i]) || !(h_sigma[i] >= 0.0f)) {
                set_error("need finite mu > 0 and sigma >= 0" + where());
                return fail(BBE_ERR_ARG);
            }
            if (!(h_rho[i] >= 0.0f && h_rho[i] <= 1.0f)) {
                set_error("responsiveness rho outside [0, 1]" + where());
                return fail(BBE_ERR_ARG);
            }
            if (!(h_P[i] > 0.0f && h_P[i] <= 1.0f)) {
                set_error("preference P outside (0, 1]" + where());
                return fail(BBE_ERR_ARG);
            }
            if (!finite(h_theta[i]) || !(h_theta[i] >= 0.0f)) {
                set_error("theta must be finite and >= 0" + where());
                return fail(BBE_ERR_ARG);
            }
            if (prev_step && (!finite(h_prev[i]) || !(h_prev[i] > 0.0f))) {
                set_error("prev_step must be finite and > 0" + where());
                return fail(BBE_ERR_ARG);
            }
        }
    }
    std::vector<int32_t> comp_race(nt);
    for (int r = 0; r < n_races; ++r)
        for (int i = off[r]; i < off[r + 1]; ++i) comp_race[i] = r;

    // one device arena for the staged batch
    size_t bytes = 0;
    auto add = [&](size_t n) { bytes += (n + 255) / 256 * 256; };
    add((n_races + 1) * 4); add(n_races * 4); add(n_races * 8); add(size_t(nt) * 4); add(n_races * 4);
    for (int i = 0; i < 7; ++i) add(size_t(nt) * 4);
    add(4 * kGroups); add(4);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = pool_alloc(&b->arena, bytes, s);
    if (e != cudaSuccess) {
        set_error(std::string("device allocation: ") + cudaGetErrorString(e));
        return fail(BBE_ERR_CUDA);
    }
    char *p = static_cast<char *>(b->arena);
    int32_t *d_off = carve<int32_t>(p, n_races + 1);
    float *d_L = carve<float>(p, n_races);
    int64_t *d_R = carve<int64_t>(p, n_races);
    int32_t *d_cr = carve<int32_t>(p, nt);
    int32_t *d_ids = carve<int32_t>(p, n_races);
    float *d_d0 = carve<float>(p, nt), *d_mu = carve<float>(p, nt), *d_sigma = carve<float>(p, nt);
    float *d_rho = carve<float>(p, nt), *d_P = carve<float>(p, nt), *d_theta = carve<float>(p, nt);
    float *d_prev = carve<float>(p, nt);
    b->d_queue = carve<int32_t>(p, kGroups);
    b->d_status = carve<int32_t>(p, 1);
    // A small batch's arena is assembled on the host in its own layout and goes up in one copy
    // (one transfer's overhead instead of one per array); a large one goes up array by array,
    // with no extra host pass over it.  The queue heads and status are reset before use.
    struct Up {
        void *dst;
        const void *src;
        size_t n;
    };
    std::vector<Up> ups = {{d_off, off.data(), off.size() * 4},       {d_L, b->h_L.data(), size_t(n_races) * 4},
                           {d_R, b->h_R.data(), size_t(n_races) * 8}, {d_cr, comp_race.data(), size_t(nt) * 4},
                           {d_d0, b->h_d0.data(), size_t(nt) * 4},   {d_mu, b->h_mu.data(), size_t(nt) * 4},
                           {d_sigma, h_sigma.data(), size_t(nt) * 4}, {d_rho, h_rho.data(), size_t(nt) * 4},
                           {d_P, h_P.data(), size_t(nt) * 4},         {d_theta, h_theta.data(), size_t(nt) * 4}};
    if (prev_step) ups.push_back({d_prev, h_prev.data(), size_t(nt) * 4});
    if (race_ids) ups.push_back({d_ids, b->h_race_ids.data(), size_t(n_races) * 4});
    std::vector<char> img;
    if (bytes <= kOneCopyBytes) {
        img.assign(bytes, 0);
        for (const Up &u : ups)
            std::memcpy(img.data() + (static_cast<const char *>(u.dst) - static_cast<const char *>(b->arena)), u.src, u.n);
        ups.assign(1, Up{b->arena, img.data(), bytes});
    }
    for (const Up &u : ups) {
        e = cudaMemcpyAsync(u.dst, u.src, u.n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            set_error(std::string("staging upload: ") + cudaGetErrorString(e));
            return fail(BBE_ERR_CUDA);
        }
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error(std::string("staging upload: ") + cudaGetErrorString(e));
        return fail(BBE_ERR_CUDA);
    }
    b->dev = bbe::DevBatch{d_off,   d_L,      d_R,   d_cr, d_d0, d_mu, d_sigma, d_rho, d_P, d_theta,
                           prev_step ? d_prev : nullptr, race_ids ? d_ids : nullptr, n_races, nt, race_id0,
                           uint32_t(seed), uint32_t(seed >> 32), int32_t(dist)};
    b->cfg = bbe_launch_cfg{kDefaultWarpsPerBlock, kDefaultBlocksPerSm, kDefaultRolloutsPerLane, BBE_MAX_STEPS_DEFAULT, 0};
    for (int g = 0; g < kGroups; ++g)
        b->resident[g] = bbe::rollout_resident_blocks(b->dist, kSlots[g], 32 * kDefaultWarpsPerBlock);
    if ((st = build_items(b, s))) return fail(st);
    *out = b;
    return BBE_OK;
}

bbe_status bbe::set_first_rollouts(bbe_batch *b, const int64_t *k0)
{
    if (!b || !k0) {
        set_error("batch or k0 is NULL");
        return BBE_ERR_ARG;
    }
    for (int r = 0; r < b->n_races; ++r) {
        if (k0[r] < 0 || k0[r] + b->h_R[r] > INT32_MAX) {
            set_error("first rollout index out of range");
            return BBE_ERR_RANGE;
        }
    }
    b->h_k0.assign(k0, k0 + b->n_races);
    return build_items(b);
}

cudaError_t bbe::note_use(const bbe_batch *b, cudaStream_t s)
{
    // work captured into a caller's graph runs when that graph does: its lifetime is the caller's
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;
    for (auto &u : b->uses)
        if (u.first == s) return cudaEventRecord(u.second, s);
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    b->uses.emplace_back(s, ev);
    return cudaEventRecord(ev, s);
}

extern "C" {

const char *bbe_last_error(void) { return bbe::g_last_error.c_str(); }

bbe_status bbe_race_init(bbe_batch **out, int32_t n_races, const int32_t *race_off, const float *track_len,
                         const int64_t *rollouts, const float *pos, const float *mu, const float *sigma,
                         const float *resp, const float *pref, const float *theta, const float *prev_step,
                         uint64_t seed, bbe_dist dist, uint32_t race_id0, void *cuda_stream)
{
    return bbe::stage_batch(out, n_races, race_off, track_len, rollouts, pos, mu, sigma, resp, pref, theta,
                            prev_step, seed, dist, race_id0, nullptr, as_stream(cuda_stream));
}

bbe_status bbe_rollout_batch(bbe_batch *b, int32_t *win_counts, int64_t *steps_total, void *cuda_stream)
{
    if (!b || !win_counts) {
        set_error("batch or win_counts is NULL");
        return BBE_ERR_ARG;
    }
    const bool cached = b->gexec && b->g_counts == win_counts && b->g_steps == steps_total;
    if (!cached && !(b->last_counts == win_counts && b->last_steps == steps_total)) {
        // first pass with these buffers: launch directly; a graph is captured if they come again
        b->last_counts = win_counts;
        b->last_steps = steps_total;
        bbe_status st = ensure_aux(b);
        if (st) return st;
        BBE_CUDA_TRY(enqueue_pass(b, win_counts, steps_total, as_stream(cuda_stream), b->side_stream));
        BBE_CUDA_TRY(bbe::note_use(b, as_stream(cuda_stream)));
        return BBE_OK;
    }
    bbe_status st = ensure_graph(b, win_counts, steps_total);
    if (st) return st;
    BBE_CUDA_TRY(cudaGraphLaunch(b->gexec, as_stream(cuda_stream)));
    BBE_CUDA_TRY(bbe::note_use(b, as_stream(cuda_stream)));
    return BBE_OK;
}

bbe_status bbe_win_probs(const bbe_batch *b, const int32_t *win_counts, float *probs, float *odds, void *cuda_stream)
{
    if (!b || !win_counts || !probs) {
        set_error("batch, win_counts or probs is NULL");
        return BBE_ERR_ARG;
    }
    BBE_CUDA_TRY(bbe::launch_win_probs(b->dev, win_counts, probs, odds, as_stream(cuda_stream)));
    BBE_CUDA_TRY(bbe::note_use(b, as_stream(cuda_stream)));
    return BBE_OK;
}

namespace {
// The rollout kernel in place mode over the whole batch: place table (nullable) and, with
// `orders`, the ordered top-`places` tallies at b->d_order_off.
bbe_status run_place_mode(bbe_batch *b, int32_t places, int32_t *place_counts, int32_t *orders,
                          int64_t *steps_total, cudaStream_t s, unsigned long long *hist_keys = nullptr,
                          int32_t *hist_counts = nullptr)
{
    if (place_counts)
        BBE_CUDA_TRY(cudaMemsetAsync(place_counts, 0, size_t(b->n_total) * size_t(places) * sizeof(int32_t), s));
    if (steps_total) BBE_CUDA_TRY(cudaMemsetAsync(steps_total, 0, size_t(b->n_races) * sizeof(int64_t), s));
    BBE_CUDA_TRY(cudaMemsetAsync(b->d_queue, 0, kGroups * sizeof(int32_t), s));
    BBE_CUDA_TRY(cudaMemsetAsync(b->d_status, 0, sizeof(int32_t), s));
    for (int g = kGroups - 1; g >= 0; --g) {
        if (b->n_items_v[g] == 0) continue;
        bbe::RolloutLaunch l = make_launch(b, place_counts, steps_total, g);
        l.places = places;
        l.orders = orders;
        l.order_off = orders ? b->d_order_off : nullptr;
        l.hist_keys = hist_keys;
        l.hist_counts = hist_counts;
        l.hist_off = hist_keys ? b->d_hist_off : nullptr;
        l.place_cells = b->max_n * std::min(places, b->max_n);
        const int res = bbe::place_resident_blocks(b->dev.dist, kSlots[g], l.block, l.place_cells);
        l.grid = std::max(1, b->num_sms * std::min(b->cfg.blocks_per_sm, std::max(1, res)));
        l.grid = std::max(1, std::min(l.grid, (l.n_items + b->cfg.warps_per_block - 1) / b->cfg.warps_per_block));
        BBE_CUDA_TRY(bbe::launch_place_rollout(l, kSlots[g], s));
    }
    BBE_CUDA_TRY(bbe::note_use(b, s));
    return BBE_OK;
}

// per-race first entries of the order tally tables for `places` (n_r ^ min(places, n_r) entries)
void order_layout(const bbe_batch *b, int32_t places, std::vector<int64_t> &off)
{
    off.assign(size_t(b->n_races) + 1, 0);
    for (int r = 0; r < b->n_races; ++r) {
        const int n = b->h_off[r + 1] - b->h_off[r];
        int64_t cells = 1;
        for (int j = 0; j < std::min(places, n); ++j) cells *= n;
        off[size_t(r) + 1] = off[size_t(r)] + cells;
    }
}
// Number of ordered tuples of K distinct competitors out of n, n! / (n - K)!, or 0 when it
// exceeds 2^64 - 1 (the order keys would not fit in 64 bits beside the empty marker).
uint64_t ordered_tuples(int n, int K)
{
    uint64_t f = 1;
    for (int j = 0; j < K; ++j) {
        const uint64_t m = uint64_t(n - j);
        if (f > (~0ull) / m) return 0;
        f *= m;
    }
    return f;
}

// per-race hash tables of the finishing-order histogram for `places`: the least power of two
// at least twice the most distinct orders the race can show, min(R_r, n_r! / (n_r - K_r)!), and
// at least 2; false (with the error set) for a race whose order keys do not fit in 64 bits
bool hist_layout(const bbe_batch *b, int32_t places, std::vector<int64_t> &off)
{
    off.assign(size_t(b->n_races) + 1, 0);
    for (int r = 0; r < b->n_races; ++r) {
        const int n = b->h_off[r + 1] - b->h_off[r];
        const uint64_t f = ordered_tuples(n, std::min(places, n));
        if (f == 0) {
            set_error("race " + std::to_string(r) + ": the orders of its first " + std::to_string(std::min(places, n)) +
                      " of " + std::to_string(n) + " competitors exceed 2^64 - 1 keys; ask for fewer places");
            return false;
        }
        const uint64_t most = std::min<uint64_t>(f, uint64_t(b->h_R[r]));
        int64_t cap = 2;
        while (uint64_t(cap) < 2 * most) cap *= 2;
        off[size_t(r) + 1] = off[size_t(r)] + cap;
    }
    return true;
}
}  // namespace

bbe_status bbe_place_counts(bbe_batch *b, int32_t places, int32_t *place_counts, int64_t *steps_total,
                            void *cuda_stream)
{
    if (!b || !place_counts) {
        set_error("batch or place_counts is NULL");
        return BBE_ERR_ARG;
    }
    if (places < 1 || places > BBE_MAX_COMPETITORS) {
        set_error("places outside 1..BBE_MAX_COMPETITORS");
        return BBE_ERR_ARG;
    }
    return run_place_mode(b, places, place_counts, nullptr, steps_total, as_stream(cuda_stream));
}

bbe_status bbe_order_table_size(const bbe_batch *b, int32_t places, int64_t *entries)
{
    if (!b || !entries || places < 1 || places > BBE_MAX_ORDER_PLACES) {
        set_error("bbe_order_table_size: batch or entries is NULL, or places outside 1..BBE_MAX_ORDER_PLACES");
        return BBE_ERR_ARG;
    }
    std::vector<int64_t> off;
    order_layout(b, places, off);
    *entries = off.back();
    return BBE_OK;
}

bbe_status bbe_order_counts(bbe_batch *b, int32_t places, int32_t *order_counts, int32_t *place_counts,
                            int64_t *steps_total, void *cuda_stream)
{
    if (!b || !order_counts || places < 1 || places > BBE_MAX_ORDER_PLACES) {
        set_error("bbe_order_counts: batch or order_counts is NULL, or places outside 1..BBE_MAX_ORDER_PLACES");
        return BBE_ERR_ARG;
    }
    cudaStream_t s = as_stream(cuda_stream);
    if (b->order_places != places || !b->d_order_off) {
        order_layout(b, places, b->h_order_off);
        BBE_CUDA_TRY(free_behind_uses(b, b->d_order_off));
        b->d_order_off = nullptr;
        b->order_places = 0;
        BBE_CUDA_TRY(pool_alloc(reinterpret_cast<void **>(&b->d_order_off), b->h_order_off.size() * sizeof(int64_t), s));
        BBE_CUDA_TRY(cudaMemcpyAsync(b->d_order_off, b->h_order_off.data(), b->h_order_off.size() * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, s));  // the host copy lives with the batch
        b->order_places = places;
    }
    BBE_CUDA_TRY(cudaMemsetAsync(order_counts, 0, size_t(b->h_order_off.back()) * sizeof(int32_t), s));
    return run_place_mode(b, places, place_counts, order_counts, steps_total, s);
}

bbe_status bbe_order_histogram_layout(const bbe_batch *b, int32_t places, int64_t *table_off, int64_t *entries)
{
    if (!b || places < 1 || places > BBE_MAX_COMPETITORS) {
        set_error("bbe_order_histogram_layout: batch is NULL, or places outside 1..BBE_MAX_COMPETITORS");
        return BBE_ERR_ARG;
    }
    std::vector<int64_t> off;
    if (!hist_layout(b, places, off)) return BBE_ERR_RANGE;
    if (table_off) std::copy(off.begin(), off.end(), table_off);
    if (entries) *entries = off.back();
    return BBE_OK;
}

bbe_status bbe_order_histogram(bbe_batch *b, int32_t places, uint64_t *keys, int32_t *counts, int32_t *place_counts,
                               int64_t *steps_total, void *cuda_stream)
{
    cudaStream_t s = as_stream(cuda_stream);
    if (!b || !keys || !counts || places < 1 || places > BBE_MAX_COMPETITORS) {
        set_error("bbe_order_histogram: batch, keys or counts is NULL, or places outside 1..BBE_MAX_COMPETITORS");
        return BBE_ERR_ARG;
    }
    if (b->hist_places != places || !b->d_hist_off) {
        std::vector<int64_t> off;
        if (!hist_layout(b, places, off)) return BBE_ERR_RANGE;
        BBE_CUDA_TRY(free_behind_uses(b, b->d_hist_off));
        b->d_hist_off = nullptr;
        b->hist_places = 0;
        BBE_CUDA_TRY(pool_alloc(reinterpret_cast<void **>(&b->d_hist_off), off.size() * sizeof(int64_t), s));
        BBE_CUDA_TRY(cudaMemcpyAsync(b->d_hist_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        BBE_CUDA_TRY(cudaStreamSynchronize(s));  // `off` is pageable and goes out of scope
        b->h_hist_off = std::move(off);
        b->hist_places = places;
    }
    const size_t entries = size_t(b->h_hist_off.back());
    BBE_CUDA_TRY(cudaMemsetAsync(keys, 0xFF, entries * sizeof(uint64_t), s));
    BBE_CUDA_TRY(cudaMemsetAsync(counts, 0, entries * sizeof(int32_t), s));
    return run_place_mode(b, places, place_counts, nullptr, steps_total, s,
                          reinterpret_cast<unsigned long long *>(keys), counts);
}

bbe_status bbe_order_key_encode(int32_t n, int32_t places, const int32_t *order, uint64_t *key)
{
    const int K = std::min(places, n);
    if (!order || !key || n < 1 || n > BBE_MAX_COMPETITORS || places < 1 || ordered_tuples(n, K) == 0) {
        set_error("bbe_order_key_encode: order or key is NULL, n outside 1..BBE_MAX_COMPETITORS, places < 1, or the "
                  "orders exceed 2^64 - 1 keys");
        return BBE_ERR_ARG;
    }
    uint32_t taken = 0;
    uint64_t k = 0;
    for (int j = 0; j < K; ++j) {
        const int c = order[j];
        if (c < 0 || c >= n || (taken >> c) & 1u) {
            set_error("bbe_order_key_encode: order holds a competitor outside 0..n-1 or the same competitor twice");
            return BBE_ERR_ARG;
        }
        int below = 0;  // competitors with a lower index not yet placed
        for (int i = 0; i < c; ++i) below += ((taken >> i) & 1u) ? 0 : 1;
        k = k * uint64_t(n - j) + uint64_t(below);
        taken |= 1u << c;
    }
    *key = k;
    return BBE_OK;
}

bbe_status bbe_order_key_decode(int32_t n, int32_t places, uint64_t key, int32_t *order)
{
    const int K = std::min(places, n);
    const uint64_t f = (n >= 1 && n <= BBE_MAX_COMPETITORS && places >= 1) ? ordered_tuples(n, K) : 0;
    if (!order || f == 0 || key >= f) {
        set_error("bbe_order_key_decode: order is NULL, n outside 1..BBE_MAX_COMPETITORS, places < 1, or key outside "
                  "0 .. n!/(n-K)! - 1");
        return BBE_ERR_ARG;
    }
    // the digits from the last (radix n - K + 1) to the first (radix n)
    int digit[BBE_MAX_COMPETITORS];
    for (int j = K - 1; j >= 0; --j) {
        const uint64_t radix = uint64_t(n - j);
        digit[j] = int(key % radix);
        key /= radix;
    }
    uint32_t taken = 0;
    for (int j = 0; j < K; ++j) {
        int c = 0, seen = 0;  // the digit[j]-th (from 0) competitor not yet placed
        for (;; ++c) {
            if ((taken >> c) & 1u) continue;
            if (seen == digit[j]) break;
            ++seen;
        }
        order[j] = c;
        taken |= 1u << c;
    }
    return BBE_OK;
}

namespace {
// P_c = prod_i (1 - w_i min(1, |f_r,i - p_c,i|)), one thread per competitor; its race by binary
// search of race_off
__global__ void preference_kernel(int n_races, const int32_t *__restrict__ race_off, int F,
                                  const float *__restrict__ factors, const float *__restrict__ prefs,
                                  const float *__restrict__ weights, float *__restrict__ P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= race_off[n_races]) return;
    int lo = 0, hi = n_races;  // race_off[lo] <= i < race_off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (race_off[mid] <= i) lo = mid;
        else hi = mid;
    }
    float p = 1.0f;
    for (int k = 0; k < F; ++k) {
        const float m = fminf(fabsf(__fsub_rn(factors[size_t(lo) * F + k], prefs[size_t(i) * F + k])), 1.0f);
        p = __fmul_rn(p, __fsub_rn(1.0f, __fmul_rn(weights[k], m)));
    }
    P[i] = p;
}
}  // namespace

bbe_status bbe_preference_coefficients(int32_t n_races, const int32_t *race_off, int32_t n_competitors,
                                       int32_t n_factors, const float *factors, const float *preferences,
                                       const float *weights, float *P, void *cuda_stream)
{
    if (n_races < 1 || n_competitors < 0 || n_factors < 1 || !race_off || !factors || !preferences || !weights || !P) {
        set_error("bbe_preference_coefficients: bad arguments");
        return BBE_ERR_ARG;
    }
    if (n_competitors == 0) return BBE_OK;
    const int threads = 256;
    preference_kernel<<<unsigned((n_competitors + threads - 1) / threads), threads, 0, as_stream(cuda_stream)>>>(
        n_races, race_off, n_factors, factors, preferences, weights, P);
    BBE_CUDA_TRY(cudaGetLastError());
    return BBE_OK;
}

bbe_status bbe_place_probs(const bbe_batch *b, int32_t places, const int32_t *place_counts, int32_t top,
                           float *probs, void *cuda_stream)
{
    if (!b || !place_counts || !probs) {
        set_error("batch, place_counts or probs is NULL");
        return BBE_ERR_ARG;
    }
    if (places < 1 || places > BBE_MAX_COMPETITORS || top < 1 || top > places) {
        set_error("places outside 1..BBE_MAX_COMPETITORS or top outside 1..places");
        return BBE_ERR_ARG;
    }
    BBE_CUDA_TRY(bbe::launch_place_probs(b->dev, places, place_counts, top, probs, as_stream(cuda_stream)));
    BBE_CUDA_TRY(bbe::note_use(b, as_stream(cuda_stream)));
    return BBE_OK;
}

bbe_status bbe_batch_set_law(bbe_batch *b, bbe_law law, const float *elapsed, const float *horizon,
                             void *cuda_stream)
{
    if (!b || (law != BBE_LAW_POSITION && law != BBE_LAW_TIME) || (law == BBE_LAW_TIME && !horizon)) {
        set_error("bbe_batch_set_law: batch is NULL, the law is unknown, or the time law has no horizon");
        return BBE_ERR_ARG;
    }
    cudaStream_t s = as_stream(cuda_stream);
    if (law == BBE_LAW_POSITION) {
        b->dev.law = BBE_LAW_POSITION;
        b->h_t0.clear();
        b->h_T.clear();
        free_graph(b);
        return BBE_OK;
    }
    const size_t nr = size_t(b->n_races);
    std::vector<float> t0(nr, 0.0f), T(nr);
    bbe_status st;
    if ((elapsed && (st = copy_in(t0.data(), elapsed, nr * sizeof(float), s, "elapsed"))) ||
        (st = copy_in(T.data(), horizon, nr * sizeof(float), s, "horizon")))
        return st;
    BBE_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<float> inv(nr);
    for (size_t r = 0; r < nr; ++r) {
        if (!finite(t0[r]) || !(t0[r] >= 0.0f) || !finite(T[r]) || !(T[r] > 0.0f)) {
            set_error("bbe_batch_set_law: race " + std::to_string(r) + " needs a finite elapsed >= 0 and horizon > 0");
            return BBE_ERR_ARG;
        }
        inv[r] = 1.0f / T[r];  // binary32 division, round to nearest
    }
    void *mem = nullptr;
    BBE_CUDA_TRY(pool_alloc(&mem, 2 * nr * sizeof(float), s));
    float *d_t0 = static_cast<float *>(mem), *d_inv = d_t0 + nr;
    BBE_CUDA_TRY(cudaMemcpyAsync(d_t0, t0.data(), nr * sizeof(float), cudaMemcpyHostToDevice, s));
    BBE_CUDA_TRY(cudaMemcpyAsync(d_inv, inv.data(), nr * sizeof(float), cudaMemcpyHostToDevice, s));
    BBE_CUDA_TRY(cudaStreamSynchronize(s));
    BBE_CUDA_TRY(free_behind_uses(b, b->law_mem));
    b->law_mem = mem;
    b->h_t0 = std::move(t0);
    b->h_T = std::move(T);
    b->dev.law = BBE_LAW_TIME;
    b->dev.t0 = d_t0;
    b->dev.invT = d_inv;
    free_graph(b);  // the captured launch parameters change
    return BBE_OK;
}

bbe_status bbe_batch_status(bbe_batch *b, void *cuda_stream)
{
    if (!b) {
        set_error("batch is NULL");
        return BBE_ERR_ARG;
    }
    cudaStream_t s = as_stream(cuda_stream);
    int32_t flags = 0;
    BBE_CUDA_TRY(cudaMemcpyAsync(&flags, b->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BBE_CUDA_TRY(cudaStreamSynchronize(s));
    if (flags & bbe::kStatusBadIndex) {
        set_error("a device index check failed (checked build)");
        return BBE_ERR_RANGE;
    }
    if (flags & bbe::kStatusTableFull) {
        set_error("a finishing-order hash table had no free entry");
        return BBE_ERR_RANGE;
    }
    if (flags & bbe::kStatusStepLimit) {
        set_error("a rollout reached max_steps without a finisher");
        return BBE_ERR_STEP_LIMIT;
    }
    return BBE_OK;
}

bbe_status bbe_batch_set_cfg(bbe_batch *b, const bbe_launch_cfg *cfg)
{
    if (!b || !cfg) {
        set_error("batch or cfg is NULL");
        return BBE_ERR_ARG;
    }
    bbe_launch_cfg c = *cfg;
    if (c.warps_per_block == 0) c.warps_per_block = kDefaultWarpsPerBlock;
    if (c.blocks_per_sm == 0) c.blocks_per_sm = kDefaultBlocksPerSm;
    if (c.rollouts_per_lane == 0) c.rollouts_per_lane = kDefaultRolloutsPerLane;
    if (c.max_steps == 0) c.max_steps = BBE_MAX_STEPS_DEFAULT;
    bbe_status st = check_cfg(c);
    if (st) return st;
    const bool rebuild = c.rollouts_per_lane != b->cfg.rollouts_per_lane || c.slots_per_lane != b->cfg.slots_per_lane;
    b->cfg = c;
    for (int g = 0; g < kGroups; ++g)
        b->resident[g] = bbe::rollout_resident_blocks(b->dist, kSlots[g], 32 * c.warps_per_block);
    free_graph(b);
    return rebuild ? build_items(b) : BBE_OK;
}

bbe_status bbe_batch_get_cfg(const bbe_batch *b, bbe_launch_cfg *cfg)
{
    if (!b || !cfg) {
        set_error("batch or cfg is NULL");
        return BBE_ERR_ARG;
    }
    *cfg = b->cfg;
    return BBE_OK;
}

bbe_status bbe_batch_layout(const bbe_batch *b, int32_t *slots_by_n)
{
    if (!b || !slots_by_n) {
        set_error("batch or slots_by_n is NULL");
        return BBE_ERR_ARG;
    }
    slots_by_n[0] = 0;
    for (int n = 1; n <= BBE_MAX_COMPETITORS; ++n)
        slots_by_n[n] = slots_for(n, b->cfg.slots_per_lane, b->slots_by_n, b->default_slots);
    return BBE_OK;
}

bbe_status bbe_batch_set_layout(bbe_batch *b, const int32_t *slots_by_n)
{
    if (!b) {
        set_error("batch is NULL");
        return BBE_ERR_ARG;
    }
    int8_t tab[BBE_MAX_COMPETITORS + 1] = {};
    for (int n = 1; slots_by_n && n <= BBE_MAX_COMPETITORS; ++n) {
        if (slots_by_n[n] < 0 || slots_by_n[n] > 4) {
            set_error("slots_by_n entries must be 0..4");
            return BBE_ERR_ARG;
        }
        tab[n] = int8_t(slots_by_n[n]);
    }
    std::memcpy(b->slots_by_n, tab, sizeof(tab));
    return build_items(b);
}

bbe_status bbe_batch_autotune(bbe_batch *b, int32_t *win_counts, double budget_ms, void *cuda_stream)
{
    if (!b || !win_counts || !(budget_ms > 0.0)) {
        set_error("batch or win_counts is NULL, or budget_ms <= 0");
        return BBE_ERR_ARG;
    }
    cudaStream_t s = as_stream(cuda_stream);
    const bbe_launch_cfg start = b->cfg;
    int8_t start_tab[BBE_MAX_COMPETITORS + 1];
    std::memcpy(start_tab, b->slots_by_n, sizeof(start_tab));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BBE_CUDA_TRY(cudaEventCreate(&e0));
    BBE_CUDA_TRY(cudaEventCreate(&e1));
    double spent = 0.0;
    bbe_status st = BBE_OK;
    // one pass of batch x into counts, timed on the device (the launch path of a first pass)
    auto time_pass = [&](bbe_batch *x, int32_t *counts, float &ms) -> bbe_status {
        bbe_status e = ensure_aux(x);
        if (e) return e;
        if (cudaEventRecord(e0, s) != cudaSuccess || enqueue_pass(x, counts, nullptr, s, x->side_stream) != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || bbe::note_use(x, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            set_error("autotune: a timed pass failed");
            return BBE_ERR_CUDA;
        }
        spent += ms;
        return BBE_OK;
    };
    float ms = 0.0f;
    int8_t tab[BBE_MAX_COMPETITORS + 1] = {};
    bbe_launch_cfg best = start;
    best.slots_per_lane = 0;
    float best_ms = INFINITY;  // of `best`, the best of three whole-batch passes
    {
        // 1. competitors per lane, for each competitor count of the batch: a sample of up to 64 of
        // its races (spread over the batch), one pass per layout; another layout replaces the
        // default of two only when at least 5 % faster
        std::vector<std::vector<int32_t>> by_n(BBE_MAX_COMPETITORS + 1);
        for (int r = 0; r < b->n_races; ++r) by_n[size_t(b->h_off[r + 1] - b->h_off[r])].push_back(r);
        for (int n = 1; n <= BBE_MAX_COMPETITORS && st == BBE_OK && spent < budget_ms; ++n) {
            const std::vector<int32_t> &all = by_n[size_t(n)];
            if (all.empty()) continue;
            std::vector<int32_t> pick;
            const size_t stride = std::max<size_t>(1, all.size() / 64);
            for (size_t i = 0; i < all.size() && pick.size() < 64; i += stride) pick.push_back(all[i]);
            std::vector<int32_t> off(1, 0);
            std::vector<float> L, d0, mu, sg, rho, P, th;
            std::vector<int64_t> R;
            for (int32_t r : pick) {
                L.push_back(b->h_L[size_t(r)]);
                R.push_back(b->h_R[size_t(r)]);
                for (int i = b->h_off[size_t(r)]; i < b->h_off[size_t(r) + 1]; ++i) {
                    d0.push_back(b->h_d0[size_t(i)]);
                    mu.push_back(b->h_mu[size_t(i)]);
                    sg.push_back(b->h_sigma[size_t(i)]);
                    rho.push_back(b->h_rho[size_t(i)]);
                    P.push_back(b->h_P[size_t(i)]);
                    th.push_back(b->h_theta[size_t(i)]);
                }
                off.push_back(int32_t(d0.size()));
            }
            bbe_batch *sub = nullptr;
            st = bbe::stage_batch(&sub, int32_t(pick.size()), off.data(), L.data(), R.data(), d0.data(), mu.data(),
                                  sg.data(), rho.data(), P.data(), th.data(), nullptr, b->seed, bbe_dist(b->dist),
                                  0u, nullptr, s);
            if (st == BBE_OK && b->dev.law == BBE_LAW_TIME) {
                std::vector<float> el, hz;
                for (int32_t r : pick) {
                    el.push_back(b->h_t0[size_t(r)]);
                    hz.push_back(b->h_T[size_t(r)]);
                }
                st = bbe_batch_set_law(sub, BBE_LAW_TIME, el.data(), hz.data(), s);
                if (st) bbe_destroy_batch(sub);
            }
            if (st) break;
            int32_t *sc = nullptr;
            if (pool_alloc(reinterpret_cast<void **>(&sc), d0.size() * sizeof(int32_t), s) != cudaSuccess) {
                set_error("autotune: scratch allocation failed");
                st = BBE_ERR_CUDA;
                bbe_destroy_batch(sub);
                break;
            }
            float t_v[5] = {INFINITY, INFINITY, INFINITY, INFINITY, INFINITY};
            for (int v = 1; v <= 4 && st == BBE_OK; ++v) {
                if (v > n && v > 2) continue;  // a forced layout wider than the race falls back to two
                bbe_launch_cfg c = start;
                c.slots_per_lane = v;
                if ((st = bbe_batch_set_cfg(sub, &c))) break;
                if ((st = time_pass(sub, sc, ms))) break;  // first launch of the layout on this sample
                if ((st = time_pass(sub, sc, ms))) break;
                t_v[v] = ms;
            }
            // another layout replaces the default of two only when clearly faster on the sample
            int vbest = 2;
            for (int v = 1; v <= 4; ++v)
                if (t_v[v] < t_v[vbest] * (vbest == 2 ? 0.95f : 1.0f)) vbest = v;
            tab[n] = int8_t(vbest);
            cudaFreeAsync(sc, s);
            bbe_destroy_batch(sub);
        }
    }
    // the best of three whole-batch passes with the batch's current layout and shape
    auto best_of_three = [&](float &t) -> bbe_status {
        t = INFINITY;
        for (int rep = 0; rep < 3; ++rep) {
            const bbe_status e = time_pass(b, win_counts, ms);
            if (e) return e;
            t = std::min(t, ms);
        }
        return BBE_OK;
    };
    bbe_launch_cfg first = start;
    first.slots_per_lane = 0;
    float first_ms = INFINITY;
    if (st == BBE_OK) {
        // 2. the per-count layout against the starting one on the whole batch: each layout group
        // is a launch of its own with its own tail, which the per-count samples do not see, so
        // the new table stays only if the whole batch runs at least 2 % faster with it
        st = bbe_batch_set_cfg(b, &first);
        if (st == BBE_OK) st = build_items(b);
        if (st == BBE_OK) st = best_of_three(first_ms);
        if (st == BBE_OK && std::memcmp(tab, start_tab, sizeof(tab)) != 0) {
            std::memcpy(b->slots_by_n, tab, sizeof(tab));
            float t_tab = INFINITY;
            if ((st = build_items(b)) == BBE_OK && (st = best_of_three(t_tab)) == BBE_OK) {
                if (t_tab < 0.98f * first_ms) {
                    first_ms = t_tab;
                } else {
                    std::memcpy(b->slots_by_n, start_tab, sizeof(start_tab));
                    st = build_items(b);
                }
            }
        }
    }
    if (st == BBE_OK) {
        // 3. block shape and work-item size with that layout, each timed on the whole batch (the
        // best of three passes); the starting shape stays unless another is at least 2 % faster
        best_ms = first_ms;
        const bbe_launch_cfg cands[] = {{4, 16, 32, start.max_steps, 0}, {8, 8, 32, start.max_steps, 0},
                                        {2, 32, 32, start.max_steps, 0}, {4, 16, 16, start.max_steps, 0},
                                        {4, 16, 64, start.max_steps, 0}, {8, 8, 16, start.max_steps, 0}};
        for (size_t i = 0; i < sizeof(cands) / sizeof(cands[0]) && st == BBE_OK && spent < budget_ms; ++i) {
            if (std::memcmp(&cands[i], &first, sizeof(first)) == 0) continue;
            if ((st = bbe_batch_set_cfg(b, &cands[i]))) break;
            float t = INFINITY;
            if ((st = best_of_three(t))) break;
            if (t < best_ms && t < 0.98f * first_ms) {
                best_ms = t;
                best = cands[i];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) {
        std::memcpy(b->slots_by_n, start_tab, sizeof(start_tab));
        bbe_batch_set_cfg(b, &start);
        build_items(b);
        return st;
    }
    return bbe_batch_set_cfg(b, &best);
}

bbe_status bbe_batch_info(const bbe_batch *b, int32_t *n_races, int64_t *n_competitors, int64_t *total_rollouts,
                          int32_t *max_competitors)
{
    if (!b) {
        set_error("batch is NULL");
        return BBE_ERR_ARG;
    }
    if (n_races) *n_races = b->n_races;
    if (n_competitors) *n_competitors = b->n_total;
    if (total_rollouts) *total_rollouts = std::accumulate(b->h_R.begin(), b->h_R.end(), int64_t(0));
    if (max_competitors) *max_competitors = b->max_n;
    return BBE_OK;
}

bbe_status bbe_batch_launches(const bbe_batch *b, int32_t *kernels_per_pass)
{
    if (!b || !kernels_per_pass) {
        set_error("batch or kernels_per_pass is NULL");
        return BBE_ERR_ARG;
    }
    int32_t k = 0;
    for (int g = 0; g < kGroups; ++g) k += b->n_items_v[g] > 0 ? 1 : 0;
    *kernels_per_pass = k;
    return BBE_OK;
}

void bbe_destroy_batch(bbe_batch *b)
{
    if (!b) return;
    int cur = -1;
    const bool switched = cudaGetDevice(&cur) == cudaSuccess && cur != b->device && cudaSetDevice(b->device) == cudaSuccess;
    // The memory is freed in stream order behind the batch's own recorded work: the host waits
    // for nothing and no other stream is held up.  Streams and events still in use are released
    // by CUDA when their work completes.
    free_graph(b);
    for (void *p : {static_cast<void *>(b->d_items), static_cast<void *>(b->d_order_off), static_cast<void *>(b->d_hist_off), b->arena,
                    b->law_mem}) {
        if (p && free_behind_uses(b, p) != cudaSuccess) {
            // no free stream could be made: wait for this batch's uses on the host instead
            cudaGetLastError();
            for (auto &u : b->uses) cudaEventSynchronize(u.second);
            cudaFree(p);
        }
    }
    for (auto &u : b->uses) cudaEventDestroy(u.second);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->side_stream) cudaStreamDestroy(b->side_stream);
    if (b->free_stream) cudaStreamDestroy(b->free_stream);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
    if (switched) cudaSetDevice(cur);
}

}  // extern "C"
