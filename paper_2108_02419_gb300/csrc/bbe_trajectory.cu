// bbe_trajectory.cu -- the actual race and its bettors (include/bbe.h: bbe_race_trajectory,
// bbe_snapshot_batch, bbe_bettor_predictions).
//
// Section 6 describes the workload the simulator exists for: one simulation of the race
// itself, and from every snapshot of it (say once per second) each of B rational bettors runs
// d dry-runs (RP(d), Section 3) to re-estimate the outcome; Section 4 lists simpler bettors
// that predict the winner from the race so far (LinEx, LW, UD, ZI).
//   trajectory_kernel   one warp per race, one competitor per lane: a full run (until the last
//                       competitor crosses) of rollout k of the race's stream, writing the
//                       positions and step sizes of every step (the space-time series that
//                       Section 6 plots).
//   bbe_snapshot_batch  (host) a batch with one race per (snapshot, bettor): the snapshot's
//                       state, the bettor's own stream id and d rollouts, to be run by
//                       bbe_rollout_batch like any batch.
//   predictors_kernel   one thread per snapshot: the rule-based bettors' predictions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "bbe_internal.h"
#include "bbe_lane.cuh"

namespace bbe {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct TrajLaunch {
    DevBatch b;
    uint32_t k;
    int32_t cap, max_steps;
    float *pos, *stp;
    int32_t *nsteps, *status;
    uint32_t round_key[20];
};

template <int DIST>
__global__ void __launch_bounds__(128) trajectory_kernel(TrajLaunch l)
{
    const int lane = threadIdx.x & 31;
    const int r = int((blockIdx.x * size_t(blockDim.x) + threadIdx.x) >> 5);
    const DevBatch &b = l.b;
    if (r >= b.n_races) return;
    const int off = b.race_off[r];
    const int n = b.race_off[r + 1] - off;
    const bool used = lane < n;
    LaneComp cp{0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float d = INFINITY, prev = 0.0f;
    if (used) {
        const int ci = off + lane;
        const float mu = b.mu[ci], P = b.P[ci];
        cp = LaneComp{mu, b.sigma[ci], P, b.theta[ci], __fmul_rn(kKappa, __fsub_rn(__fmul_rn(2.0f, b.rho[ci]), 1.0f))};
        d = b.d0[ci];
        prev = b.prev0 ? b.prev0[ci] : __fmul_rn(mu, P);
    }
    const float L = b.L[r];
    const float invL = __fdiv_rn(1.0f, L);
    const uint32_t rid = b.race_ids ? uint32_t(b.race_ids[r]) : b.race_id0 + uint32_t(r);
    float zc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float *pos = l.pos + size_t(off) * size_t(l.cap);
    float *stp = l.stp ? l.stp + size_t(off) * size_t(l.cap) : nullptr;
    int t = 0;
    for (;;) {
        if (t >= l.max_steps) {
            if (lane == 0) atomicOr(l.status, kStatusStepLimit);
            break;
        }
        const float S = lane_step<DIST>(d, prev, cp, n, 0, used, used, lane, t, l.k, rid, invL, zc, l.round_key, b.law,
                                        b.law == BBE_LAW_TIME ? b.t0[r] : 0.0f, b.law == BBE_LAW_TIME ? b.invT[r] : 0.0f);
        const float dn = __fadd_rn(d, S);
        if (used && t < l.cap) {
            pos[size_t(t) * n + lane] = dn;
            if (stp) stp[size_t(t) * n + lane] = S;
        }
        prev = S;
        d = dn;
        ++t;
        if (__all_sync(kFull, !used || dn >= L)) break;
    }
    if (lane == 0) l.nsteps[r] = t;
}

struct PredArgs {
    DevBatch b;
    int32_t race, cap, every, n_snap, window;
    float ud_gap;
    uint32_t zi_stream;
    const float *pos, *stp;
    const int32_t *nsteps;
    int32_t *pred;
    uint32_t round_key[20];
};

// One thread per snapshot s at time t_s = s * every (the race's state after t_s steps).
//   LW    the leader (largest position; equal positions: lower index)
//   UD    the second-placed competitor while its distance to the leader is below ud_gap, else
//         the leader
//   LinEx each competitor's mean step over the last min(window, t_s) steps (its previous step
//         input at t_s = 0) taken as its speed for the rest of the race; the least time to the
//         line (L - d) / v wins, equal times: lower index
//   ZI    a competitor drawn uniformly: (w0 * n) >> 32 for the first word w0 of Philox
//         counter (s, 0, 0, zi_stream)
// Snapshots past the recorded trajectory get -1.
__global__ void predictors_kernel(PredArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_snap) return;
    const DevBatch &b = a.b;
    const int off = b.race_off[a.race];
    const int n = b.race_off[a.race + 1] - off;
    const int ts = s * a.every;
    const int T = min(a.nsteps[a.race], a.cap);
    int32_t *out = a.pred + size_t(s) * 4;
    if (ts > T) {
        out[0] = out[1] = out[2] = out[3] = -1;
        return;
    }
    const float *pos = a.pos + size_t(off) * size_t(a.cap);
    const float *stp = a.stp + size_t(off) * size_t(a.cap);
    const float L = b.L[a.race];
    auto d_at = [&](int c) { return ts == 0 ? b.d0[off + c] : pos[size_t(ts - 1) * n + c]; };
    int p1 = 0;
    for (int c = 1; c < n; ++c)
        if (d_at(c) > d_at(p1)) p1 = c;
    int p2 = -1;
    for (int c = 0; c < n; ++c)
        if (c != p1 && (p2 < 0 || d_at(c) > d_at(p2))) p2 = c;
    const int ud = (p2 >= 0 && __fsub_rn(d_at(p1), d_at(p2)) < a.ud_gap) ? p2 : p1;
    const int w = min(a.window, ts);
    int lx = 0;
    float best = INFINITY;
    for (int c = 0; c < n; ++c) {
        float v;
        if (w == 0) {
            v = b.prev0 ? b.prev0[off + c] : __fmul_rn(b.mu[off + c], b.P[off + c]);
        } else {
            float sum = 0.0f;
            for (int m = ts - w; m < ts; ++m) sum = __fadd_rn(sum, stp[size_t(m) * n + c]);
            v = __fdiv_rn(sum, __int2float_rn(w));
        }
        const float tc = __fdiv_rn(__fsub_rn(L, d_at(c)), v);
        if (c == 0 || tc < best) {
            best = tc;
            lx = c;
        }
    }
    const Words4 wd = philox4x32_10(uint32_t(s), 0u, 0u, a.zi_stream, a.round_key);
    const int zi = int((uint64_t(wd.w0) * uint64_t(n)) >> 32);
    out[0] = p1;
    out[1] = ud;
    out[2] = lx;
    out[3] = zi;
}

void fill_keys(uint32_t (&rk)[20], uint32_t lo, uint32_t hi)
{
    for (int i = 0; i < 10; ++i) {
        rk[2 * i] = lo + uint32_t(i) * 0x9E3779B9u;
        rk[2 * i + 1] = hi + uint32_t(i) * 0xBB67AE85u;
    }
}

}  // namespace

}  // namespace bbe

namespace {

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

#define TRAJ_TRY(expr)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            bbe::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));        \
            return BBE_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

}  // namespace

extern "C" {

bbe_status bbe_race_trajectory(bbe_batch *b, uint32_t k, int32_t cap, float *positions, float *step_sizes,
                               int32_t *n_steps, void *cuda_stream)
{
    if (!b || !positions || !n_steps || cap < 1) {
        bbe::set_error("batch, positions or n_steps is NULL, or cap < 1");
        return BBE_ERR_ARG;
    }
    cudaStream_t s = as_stream(cuda_stream);
    TRAJ_TRY(cudaMemsetAsync(b->d_status, 0, sizeof(int32_t), s));
    bbe::TrajLaunch l{};
    l.b = b->dev;
    l.k = k;
    l.cap = cap;
    l.max_steps = b->cfg.max_steps;
    l.pos = positions;
    l.stp = step_sizes;
    l.nsteps = n_steps;
    l.status = b->d_status;
    bbe::fill_keys(l.round_key, l.b.seed_lo, l.b.seed_hi);
    const int warps = 4;
    const unsigned grid = unsigned((b->n_races + warps - 1) / warps);
    switch (l.b.dist) {
    case BBE_DIST_NORMAL: bbe::trajectory_kernel<BBE_DIST_NORMAL><<<grid, 32 * warps, 0, s>>>(l); break;
    case BBE_DIST_UNIFORM: bbe::trajectory_kernel<BBE_DIST_UNIFORM><<<grid, 32 * warps, 0, s>>>(l); break;
    default: bbe::trajectory_kernel<BBE_DIST_TWO_POINT><<<grid, 32 * warps, 0, s>>>(l); break;
    }
    TRAJ_TRY(cudaGetLastError());
    TRAJ_TRY(bbe::note_use(b, s));
    return BBE_OK;
}

bbe_status bbe_snapshot_batch(bbe_batch **out, const bbe_batch *src, int32_t race, const float *positions,
                              const float *step_sizes, const int32_t *n_steps, int32_t cap, int32_t every,
                              int32_t bettors, int64_t dry_runs, uint32_t race_id0, int32_t *n_snapshots,
                              void *cuda_stream)
{
    if (!out || !src || !positions || !step_sizes || !n_steps || !n_snapshots || race < 0 || race >= src->n_races ||
        cap < 1 || every < 1 || bettors < 1 || dry_runs < 1 || dry_runs > INT32_MAX) {
        bbe::set_error("bbe_snapshot_batch: bad arguments");
        return BBE_ERR_ARG;
    }
    *out = nullptr;
    cudaStream_t s = as_stream(cuda_stream);
    const int off = src->h_off[race];
    const int n = src->h_off[race + 1] - off;
    int32_t steps = 0;
    TRAJ_TRY(cudaMemcpyAsync(&steps, n_steps + race, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TRAJ_TRY(cudaStreamSynchronize(s));
    const int T = std::min(steps, cap);
    std::vector<float> pos(size_t(T) * n), stp(size_t(T) * n);
    if (T > 0) {
        TRAJ_TRY(cudaMemcpyAsync(pos.data(), positions + size_t(off) * cap, pos.size() * sizeof(float),
                                 cudaMemcpyDeviceToHost, s));
        TRAJ_TRY(cudaMemcpyAsync(stp.data(), step_sizes + size_t(off) * cap, stp.size() * sizeof(float),
                                 cudaMemcpyDeviceToHost, s));
        TRAJ_TRY(cudaStreamSynchronize(s));
    }
    const float L = src->h_L[race];
    // snapshots t_s = 0, every, 2 every, ... while the state is recorded and nobody has crossed
    std::vector<int> times;
    for (int ts = 0; ts <= T; ts += every) {
        bool open = true;
        for (int c = 0; c < n; ++c) {
            const float d = ts == 0 ? src->h_d0[off + c] : pos[size_t(ts - 1) * n + c];
            open = open && d < L;
        }
        if (!open) break;
        times.push_back(ts);
    }
    const int64_t n_races = int64_t(times.size()) * bettors;
    if (n_races < 1 || n_races * n > INT32_MAX) {
        bbe::set_error("bbe_snapshot_batch: no open snapshot, or too many races");
        return BBE_ERR_RANGE;
    }
    const size_t nr = size_t(n_races);
    std::vector<int32_t> roff(nr + 1, 0);
    std::vector<int32_t> ids(nr, 0);
    std::vector<float> Ls(nr, L);
    std::vector<int64_t> R(nr, dry_runs);
    const size_t nt = size_t(n_races) * n;
    std::vector<float> d0(nt), mu(nt), sg(nt), rho(nt), P(nt), th(nt), pv(nt);
    size_t i = 0;
    for (size_t si = 0; si < times.size(); ++si) {
        const int ts = times[si];
        for (int bt = 0; bt < bettors; ++bt) {
            const size_t rr = si * size_t(bettors) + size_t(bt);
            roff[rr + 1] = roff[rr] + n;
            ids[rr] = int32_t(race_id0 + uint32_t(rr));
            for (int c = 0; c < n; ++c, ++i) {
                const int ci = off + c;
                d0[i] = ts == 0 ? src->h_d0[ci] : pos[size_t(ts - 1) * n + c];
                mu[i] = src->h_mu[ci];
                sg[i] = src->h_sigma[ci];
                rho[i] = src->h_rho[ci];
                P[i] = src->h_P[ci];
                th[i] = src->h_theta[ci];
                pv[i] = ts > 0 ? stp[size_t(ts - 1) * n + c]
                               : (src->h_prev.empty() ? src->h_mu[ci] * src->h_P[ci] : src->h_prev[ci]);
            }
        }
    }
    bbe_status e = bbe::stage_batch(out, int32_t(n_races), roff.data(), Ls.data(), R.data(), d0.data(), mu.data(),
                                    sg.data(), rho.data(), P.data(), th.data(), pv.data(), src->seed,
                                    bbe_dist(src->dist), race_id0, ids.data(), s);
    if (e) return e;
    if (src->dev.law == BBE_LAW_TIME) {
        // a snapshot taken ts steps into the actual race has run t0 + ts steps; same horizon
        std::vector<float> el(nr), hz(nr, src->h_T[size_t(race)]);
        for (size_t si = 0; si < times.size(); ++si)
            for (int bt = 0; bt < bettors; ++bt)
                el[si * size_t(bettors) + size_t(bt)] = src->h_t0[size_t(race)] + float(times[si]);
        if ((e = bbe_batch_set_law(*out, BBE_LAW_TIME, el.data(), hz.data(), s))) {
            bbe_destroy_batch(*out);
            *out = nullptr;
            return e;
        }
    }
    *n_snapshots = int32_t(times.size());
    return BBE_OK;
}

bbe_status bbe_bettor_predictions(const bbe_batch *src, int32_t race, const float *positions, const float *step_sizes,
                                  const int32_t *n_steps, int32_t cap, int32_t every, int32_t n_snapshots,
                                  int32_t linex_window, float ud_gap, uint32_t zi_stream, int32_t *predictions,
                                  void *cuda_stream)
{
    if (!src || !positions || !step_sizes || !n_steps || !predictions || race < 0 || race >= src->n_races || cap < 1 ||
        every < 1 || n_snapshots < 0 || linex_window < 1 || !(ud_gap >= 0.0f)) {
        bbe::set_error("bbe_bettor_predictions: bad arguments");
        return BBE_ERR_ARG;
    }
    if (n_snapshots == 0) return BBE_OK;
    bbe::PredArgs a{};
    a.b = src->dev;
    a.race = race;
    a.cap = cap;
    a.every = every;
    a.n_snap = n_snapshots;
    a.window = linex_window;
    a.ud_gap = ud_gap;
    a.zi_stream = zi_stream;
    a.pos = positions;
    a.stp = step_sizes;
    a.nsteps = n_steps;
    a.pred = predictions;
    bbe::fill_keys(a.round_key, a.b.seed_lo, a.b.seed_hi);
    bbe::predictors_kernel<<<unsigned((n_snapshots + 127) / 128), 128, 0, as_stream(cuda_stream)>>>(a);
    TRAJ_TRY(cudaGetLastError());
    TRAJ_TRY(bbe::note_use(src, as_stream(cuda_stream)));
    return BBE_OK;
}

}  // extern "C"
