/*
 * bbe.h -- C ABI of the GB300 (sm_103a) Monte Carlo race-rollout library.
 *
 * The library estimates, for many race states at once, each competitor's probability of
 * winning the race and the matching decimal odds, by re-running the race from its current
 * state many times: these are the dry-runs of the paper's rational-predictor bettors
 * (Section 3), whose outcomes are counted into frequencies, and the repeated seeded runs
 * that estimate the outcome distribution (Section 6).  One step of a race follows Eq. 1:
 *
 *   d_c(t+1) = d_c(t) + S_c(t),
 *   S_c = R_c * P_c * delta(v_c)          if Delta_c > theta_c (no one close in front)
 *       = R_c * min(S_c(t-1), S_i+(t-1))  otherwise (blocked by the nearest i+ in front)
 *
 * with these readings where the paper leaves the law open:
 *   delta(v_c) = mu_c + sigma_c * z, z ~ N(0,1) (or uniform / two-point, see bbe_dist);
 *   R_c        = 1 + 0.2 (2 rho_c - 1) (d_c / L - 1/2), rho_c in [0,1];
 *   S_c        >= 1e-3 (Section 3: S_c > 0 at all times);
 *   a rollout ends at the first step in which some competitor reaches d >= L; the
 *   winner is the finisher that crossed earliest within that step, i.e. the least
 *   (L - d_c) / S_c, ties to the lowest competitor index.
 * All arithmetic is IEEE binary32 with round-to-nearest-even in a fixed operation order,
 * and the random numbers come from a counter-based Philox4x32-10 stream keyed by
 * (seed) and (rollout k, step t / 4, competitor c, race id r), so the integer win counts
 * are a deterministic function of (state, seed, rollout budget): any partition of the
 * races or rollouts gives the same counts.
 *
 * Conventions for every entry point:
 *   - Return value: BBE_OK or a negative bbe_status; on error nothing was launched and
 *     bbe_last_error() returns a thread-local message.
 *   - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).  Calls that
 *     launch work are asynchronous on that stream unless stated otherwise.
 *   - Buffers passed in are owned by the caller and must stay valid until the work that
 *     uses them has completed; handles (bbe_batch) are owned by the library and freed
 *     with their destroy call.
 *   - Faults found on the device (a rollout that reaches the step limit) are recorded in
 *     a per-batch status word and returned by bbe_batch_status().
 */
#ifndef BBE_H
#define BBE_H

#include <stdint.h>

#if defined(__GNUC__)
#define BBE_API __attribute__((visibility("default")))
#else
#define BBE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BBE_OK = 0,
    BBE_ERR_ARG = -1,         /* null pointer, bad size, non-monotone offsets, NaN/Inf, out-of-range parameter */
    BBE_ERR_UNSUPPORTED = -2, /* a race with fewer than 1 or more than BBE_MAX_COMPETITORS competitors */
    BBE_ERR_FINISHED = -3,    /* a competitor already at or past the finish line (d >= L) */
    BBE_ERR_CUDA = -4,        /* a CUDA runtime call failed (message in bbe_last_error) */
    BBE_ERR_STEP_LIMIT = -5,  /* some rollout reached max_steps without a finisher; it counts for nobody */
    BBE_ERR_TIMEOUT = -6,     /* a bounded device wait gave up (surrogate kernels, bbe_surrogate_status) */
    BBE_ERR_RANGE = -7        /* a value outside the range the call supports */
} bbe_status;

/* Distribution of z in delta(v_c) = mu_c + sigma_c * z.  Section 3 leaves the step
 * generator open (its example is uniform); NORMAL is the default reading. */
typedef enum {
    BBE_DIST_NORMAL = 0,   /* z ~ N(0, 1) by the Box-Muller transform */
    BBE_DIST_UNIFORM = 1,  /* z ~ U(-sqrt 3, sqrt 3): mean 0, variance 1 */
    BBE_DIST_TWO_POINT = 2 /* z = -1 or +1 with probability 1/2 each */
} bbe_dist;

/* Law of the responsiveness R_c(t, d) of Eq. 1.  Section 3 gives only its purpose (a
 * competitor that starts fast and fades, or starts slowly and finishes strongly), written as
 * a function of time and distance; each law below is one reading of it, linear and centred on
 * the middle of the race:
 *   POSITION: R_c = 1 + 0.2 (2 rho_c - 1) (d_c / L - 1/2)  (the fraction of the track covered);
 *   TIME:     R_c = 1 + 0.2 (2 rho_c - 1) (u - 1/2), u = min(1, (t0 + t) / T), the fraction of
 *             the race's expected duration T elapsed, t0 the steps run before the state (a
 *             mid-race snapshot) and t the dry-run's step; in binary32,
 *             u = min(1, (t0 + (float)t) * (1 / T)), R = fma(0.2 (2 rho - 1), u - 0.5, 1). */
typedef enum {
    BBE_LAW_POSITION = 0,
    BBE_LAW_TIME = 1
} bbe_law;

#define BBE_MAX_COMPETITORS 32
#define BBE_MAX_ORDER_PLACES 3 /* ordered places tallied by bbe_order_counts (n^3 <= 32768 per race) */
#define BBE_THETA_DEFAULT 1.0f
#define BBE_MAX_STEPS_DEFAULT (1 << 20)

typedef struct bbe_batch bbe_batch; /* opaque, library-owned */

/* Launch shape of the rollout kernel.  Zero fields mean "library default". */
typedef struct {
    int32_t warps_per_block;    /* 1..16 */
    int32_t blocks_per_sm;      /* 1..32; grid = SMs x blocks_per_sm (persistent) */
    int32_t rollouts_per_lane;  /* rollouts each warp segment runs per work item, 1..65536 (halved, down
                                   to 1, for a batch too small to give every warp slot an item) */
    int32_t max_steps;          /* step limit per rollout, 1..2^30 */
    int32_t slots_per_lane;     /* competitors per lane, 0..4: 0 = automatic (two; one for a batch too
                                   small to give every warp slot an item even at one rollout per
                                   lane), 1..4 = that layout for every race of at least that many
                                   competitors (smaller races take two, or one for a lone
                                   competitor) */
} bbe_launch_cfg;

/* bbe_race_init -- validate a batch of race states and stage it on the current device.
 *
 * Section 3 defines a race r by its track length L_r and, per competitor c, its position
 * d_c, its step distribution v_c (here mu_c, sigma_c), its responsiveness R_c (here the
 * parameter rho_c), its preference coefficient P_c in [0,1] and its blocking threshold
 * theta_c; S_c(t-1) is the competitor's previous step.
 *
 *   out         receives the new handle (set to NULL on error).
 *   n_races     number of races, >= 1.
 *   race_off    int32[n_races + 1], CSR offsets over competitors: race r owns competitors
 *               race_off[r] .. race_off[r+1]-1; race_off[0] = 0; 1 <= size <= 32.
 *   track_len   float[n_races], L_r > 0.
 *   rollouts    int64[n_races], rollout budget R_r, 1 .. 2^31-1.
 *   pos         float[sum n], d_c, 0 <= d_c < L_r.
 *   mu, sigma   float[sum n], mean step mu_c > 0 and spread sigma_c >= 0.
 *   resp        float[sum n], responsiveness parameter rho_c in [0, 1].
 *   pref        float[sum n] or NULL (all 1): P_c in (0, 1].
 *   theta       float[sum n] or NULL (all BBE_THETA_DEFAULT): theta_c >= 0.
 *   prev_step   float[sum n] or NULL (mu_c * P_c): S_c(t-1) > 0 for the first step.
 *   seed        64-bit Philox key.
 *   dist        the distribution of z.
 *   race_id0    id of race 0 in the random stream; race r uses id race_id0 + r, so a batch
 *               split into pieces reproduces the counts of the whole.
 *   cuda_stream stream for the staging copies; the call synchronises it before returning.
 * Every array may live in host or device memory (copied with cudaMemcpyDefault); the
 * library keeps its own device copy, so the caller may free them after the call.
 * Errors: BBE_ERR_ARG, BBE_ERR_UNSUPPORTED, BBE_ERR_FINISHED, BBE_ERR_CUDA. */
BBE_API bbe_status bbe_race_init(bbe_batch **out, int32_t n_races, const int32_t *race_off, const float *track_len,
                         const int64_t *rollouts, const float *pos, const float *mu, const float *sigma,
                         const float *resp, const float *pref, const float *theta, const float *prev_step,
                         uint64_t seed, bbe_dist dist, uint32_t race_id0, void *cuda_stream);

/* bbe_rollout_batch -- run every race's R_r rollouts and count the winners (Section 3
 * dry-runs; Section 6 repeated runs).  One persistent kernel launch (replayed from a CUDA
 * graph) processes all races.
 *   win_counts  device int32[sum n], overwritten: win_counts[race_off[r] + c] = number of
 *               rollouts of race r that competitor c won.  Sum over a race = R_r unless a
 *               rollout hit the step limit.
 *   steps_total device int64[n_races] or NULL, overwritten: total steps over race r's
 *               rollouts (the finishing step included); competitor-steps = n_r x this.
 * Asynchronous on cuda_stream.  Errors: BBE_ERR_ARG, BBE_ERR_CUDA; device faults via
 * bbe_batch_status. */
BBE_API bbe_status bbe_rollout_batch(bbe_batch *batch, int32_t *win_counts, int64_t *steps_total, void *cuda_stream);

/* bbe_win_probs -- frequentist win probabilities p_c = count_c / R_r and decimal odds
 * 1 / p_c (decimal odds are the total returned per unit stake; +Inf when p_c = 0).
 *   win_counts device int32[sum n] from bbe_rollout_batch.
 *   probs      device float[sum n]; odds device float[sum n] or NULL.
 * Asynchronous on cuda_stream.  Errors: BBE_ERR_ARG, BBE_ERR_CUDA. */
BBE_API bbe_status bbe_win_probs(const bbe_batch *batch, const int32_t *win_counts, float *probs, float *odds,
                         void *cuda_stream);

/* bbe_place_counts -- finishing places of every competitor (Section 3: a race runs until its
 * last competitor crosses the line, and in-play betting may stop earlier, for instance when the
 * third-placed competitor crosses; place and each-way markets, Section 2, need the places).
 * Every rollout of race r runs until K = min(places, n_r) competitors have crossed.  Readings:
 * all competitors keep moving under Eq. 1 until the rollout ends, finished ones included (they
 * can still block); competitors crossing in the same step are placed by their crossing time
 * within the step, tau = (L - d) / S, then by lower index.  Same random stream as
 * bbe_rollout_batch, so place 0 is exactly its win count.
 *   places        1 .. BBE_MAX_COMPETITORS.
 *   place_counts  device int32[sum n * places], overwritten: [i * places + j] = rollouts in
 *                 which competitor i finished in place j (0 = first); zero for j >= n_r.
 *   steps_total   nullable device int64[n_races]: steps summed over the race's rollouts.
 * Asynchronous on cuda_stream.  A rollout that reaches max_steps first counts for nobody and
 * sets BBE_ERR_STEP_LIMIT in the batch status.  Errors: BBE_ERR_ARG, BBE_ERR_CUDA. */
BBE_API bbe_status bbe_place_counts(bbe_batch *batch, int32_t places, int32_t *place_counts, int64_t *steps_total,
                                    void *cuda_stream);

/* bbe_order_counts -- finishing-order tallies: how often each ordered tuple of the first K
 * finishers occurs (Section 3: the dry-runs estimate the distribution of outcomes, the order of
 * finish included; a forecast or exacta market pays on the ordered first two, a tricast on the
 * first three).  The rollouts are bbe_place_counts's (same stream, same readings), run to the
 * K-th finisher with K_r = min(places, n_r); each completed rollout adds one to the entry of its
 * ordered tuple (o_1, .., o_K_r), the base-n_r number ((o_1 n_r + o_2) n_r + ..) + o_K_r.
 *   places        1 .. BBE_MAX_ORDER_PLACES (1: the win counts).
 *   order_counts  device int32[bbe_order_table_size entries], overwritten: race r's table of
 *                 n_r ^ K_r entries starts at sum over r' < r of n_r' ^ K_r'.
 *   place_counts  nullable device int32[sum n * places]: bbe_place_counts's table, same pass.
 *   steps_total   nullable device int64[n_races].
 * Every marginal of a race's table is a column of its place counts.  Asynchronous on
 * cuda_stream (the first call with a new `places` uploads the table layout).  Cut-off rollouts
 * count for nobody and set BBE_ERR_STEP_LIMIT.  Errors: BBE_ERR_ARG, BBE_ERR_CUDA. */
BBE_API bbe_status bbe_order_counts(bbe_batch *batch, int32_t places, int32_t *order_counts, int32_t *place_counts,
                                    int64_t *steps_total, void *cuda_stream);

/* bbe_order_table_size -- entries of the order tally buffer for `places` (host; no GPU work).
 * Errors: BBE_ERR_ARG. */
BBE_API bbe_status bbe_order_table_size(const bbe_batch *batch, int32_t places, int64_t *entries);

/* bbe_order_histogram -- the distribution of finishing orders as a histogram (Section 3: the
 * dry-runs estimate the distribution of outcomes; a race's full outcome is the order of all n_r
 * finishers, one of n_r! permutations, so no dense table holds it).  The rollouts are
 * bbe_place_counts's (same stream, same readings), run to the K_r-th finisher with
 * K_r = min(places, n_r) (places >= n_r: the full order); each completed rollout adds one to
 * the count of its order key in race r's hash table.
 * Order key of the ordered tuple (o_0, .., o_{K-1}) of a race of n: the mixed-radix number
 * with digits a_0 .. a_{K-1}, a_j in 0 .. n-j-1 (radix n - j) and a_0 the most significant,
 * where a_j counts the competitors of lower index than o_j that are not among o_0 .. o_{j-1};
 * keys run over 0 .. n!/(n-K)! - 1 (bbe_order_key_encode / _decode convert).  Every race needs
 * n_r!/(n_r-K_r)! <= 2^64 - 1: the full order for n_r <= 20, the first 16 places of 24, the
 * first 13 of 32.
 *   places       1 .. BBE_MAX_COMPETITORS.
 *   keys         device uint64[entries of bbe_order_histogram_layout], overwritten: race r's
 *                table is entries table_off[r] .. table_off[r+1]-1; an unused entry holds
 *                2^64 - 1 (UINT64_MAX) and count 0.
 *   counts       device int32[entries], overwritten: the rollouts that ended in that order.
 *   place_counts nullable device int32[sum n * places]: bbe_place_counts's table, same pass.
 *   steps_total  nullable device int64[n_races].
 * Which entry holds a key depends on the timing of the rollouts; the set of (key, count) pairs
 * of each race does not, and is bit-identical to the tally of the oracle's dry-runs.  A race's
 * table holds a power of two of entries, at least twice min(R_r, n_r!/(n_r-K_r)!), so a free
 * entry is always found (were none found, the batch status would report BBE_ERR_RANGE).
 * Asynchronous on cuda_stream (a call with a new `places` uploads the layout first).  Cut-off
 * rollouts count for nobody and set BBE_ERR_STEP_LIMIT.  Either law of responsiveness.
 * Errors: BBE_ERR_ARG, BBE_ERR_RANGE (a race whose keys exceed 64 bits, named in
 * bbe_last_error), BBE_ERR_CUDA. */
BBE_API bbe_status bbe_order_histogram(bbe_batch *batch, int32_t places, uint64_t *keys, int32_t *counts,
                                       int32_t *place_counts, int64_t *steps_total, void *cuda_stream);

/* bbe_order_histogram_layout -- the hash-table layout bbe_order_histogram uses for `places`
 * (host; no GPU work): table_off (nullable host int64[n_races + 1]) gets each race's first entry
 * and the total, entries (nullable) the total.  Errors: BBE_ERR_ARG, BBE_ERR_RANGE (as above). */
BBE_API bbe_status bbe_order_histogram_layout(const bbe_batch *batch, int32_t places, int64_t *table_off,
                                              int64_t *entries);

/* bbe_order_key_encode / bbe_order_key_decode -- between an ordered tuple order[0 .. K-1]
 * (K = min(places, n), distinct competitors in 0 .. n-1; host int32) and its order key (see
 * bbe_order_histogram).  Host only.  Errors: BBE_ERR_ARG (a repeated or out-of-range
 * competitor, a key >= n!/(n-K)!, or n!/(n-K)! > 2^64 - 1). */
BBE_API bbe_status bbe_order_key_encode(int32_t n, int32_t places, const int32_t *order, uint64_t *key);
BBE_API bbe_status bbe_order_key_decode(int32_t n, int32_t places, uint64_t key, int32_t *order);

/* bbe_place_probs -- probability of finishing in the first `top` places (a place market
 * paying on the first `top` places; top = 1 is the win probability):
 *   probs[i] = (sum over j < top of place_counts[i * places + j]) / R_r.
 * place_counts as written by bbe_place_counts with the same `places`; 1 <= top <= places.
 * Asynchronous.  Errors: BBE_ERR_ARG, BBE_ERR_CUDA. */
BBE_API bbe_status bbe_place_probs(const bbe_batch *batch, int32_t places, const int32_t *place_counts, int32_t top,
                                   float *probs, void *cuda_stream);

/* bbe_preference_coefficients -- the preference coefficients P_c of Eq. 1 from vectors
 * (Section 3: P_c(f_r, p_c) in [0, 1] reduces c's stochastic step by an amount that depends on
 * the mismatch between the race's factors f_r, such as wet or dry going, and the competitor's
 * preferred values p_c; the paper gives no formula).  This library's law:
 *   P_c = prod over factors k in order of (1 - w_k * min(1, |f_r,k - p_c,k|)),
 * binary32 round-to-nearest, each product and difference rounded once.  With weights in [0, 1]
 * the result lies in [0, 1]: 1 for a perfect match, 0 for a full mismatch on a factor of weight 1.
 * Pass the result as bbe_race_init's pref argument.
 *   race_off     device int32[n_races + 1], CSR over competitors (n_competitors = race_off[n_races]).
 *   factors      device float[n_races * n_factors], row-major.
 *   preferences  device float[n_competitors * n_factors], row-major.
 *   weights      device float[n_factors].
 *   P            device float[n_competitors], overwritten.
 * Asynchronous.  Errors: BBE_ERR_ARG (a NULL pointer, n_races < 1, n_factors < 1), BBE_ERR_CUDA. */
BBE_API bbe_status bbe_preference_coefficients(int32_t n_races, const int32_t *race_off, int32_t n_competitors,
                                               int32_t n_factors, const float *factors, const float *preferences,
                                               const float *weights, float *P, void *cuda_stream);

/* bbe_race_trajectory -- one full run of every race of the batch: rollout k of the race's
 * stream (the same stream as bbe_rollout_batch, so use a k outside the dry-runs' 0 .. R-1 for
 * an independent "actual race"), every competitor moving under Eq. 1 until the last one has
 * crossed the line (Section 3) or max_steps pass.  This is the race the bettors of Section 6
 * watch and the space-time series its figure plots.
 *   cap         rows recorded per race, >= 1.
 *   positions   device float[sum n * cap]: race r's rows at race_off[r] * cap; row t
 *               (t < min(n_steps[r], cap)) holds the n positions after step t.
 *   step_sizes  nullable device float[sum n * cap], same layout: S_c(t) of step t.
 *   n_steps     device int32[n_races]: steps until the last competitor crossed.
 * Asynchronous; max_steps sets BBE_ERR_STEP_LIMIT in the batch status.  Errors: BBE_ERR_ARG,
 * BBE_ERR_CUDA. */
BBE_API bbe_status bbe_race_trajectory(bbe_batch *batch, uint32_t k, int32_t cap, float *positions, float *step_sizes,
                                       int32_t *n_steps, void *cuda_stream);

/* bbe_snapshot_batch -- the rational bettors' dry-runs along a trajectory (Section 6: B bettors,
 * each re-estimating the outcome with d dry-runs, RP(d) of Section 3, at every snapshot).
 * Snapshot s is the state of race `race` of src after t_s = s * every steps (t_s = 0: src's
 * own state; else the positions of row t_s - 1 and the step sizes of that row as previous
 * steps), for every t_s whose state is recorded and has nobody across the line.  The new batch
 * holds one race per (snapshot s, bettor b), in that order, with src's competitor parameters,
 * seed and distribution, dry_runs rollouts and stream id race_id0 + s * bettors + b (choose
 * race_id0 so that these ids differ from the ids src uses).  Run it with bbe_rollout_batch.
 *   positions, step_sizes, n_steps, cap: as written by bbe_race_trajectory on src.
 *   n_snapshots (host) receives the number of snapshots.
 * Synchronous on cuda_stream (the trajectory rows are read back).  Errors: BBE_ERR_ARG,
 * BBE_ERR_RANGE (no open snapshot, or more than 2^31 - 1 competitors), BBE_ERR_CUDA. */
BBE_API bbe_status bbe_snapshot_batch(bbe_batch **out, const bbe_batch *src, int32_t race, const float *positions,
                                      const float *step_sizes, const int32_t *n_steps, int32_t cap, int32_t every,
                                      int32_t bettors, int64_t dry_runs, uint32_t race_id0, int32_t *n_snapshots,
                                      void *cuda_stream);

/* bbe_bettor_predictions -- the rule-based bettors of Section 4 at the snapshots of
 * bbe_snapshot_batch (t_s = s * every, s < n_snapshots), predicting the winner from the race so
 * far.  predictions: device int32[n_snapshots * 4], per snapshot:
 *   [0] LW     the leader (largest position; equal positions: lower index);
 *   [1] UD     the second-placed competitor while its distance to the leader is below ud_gap,
 *              else the leader;
 *   [2] LinEx  each competitor's mean step over the last min(linex_window, t_s) steps (its
 *              previous-step input at t_s = 0) taken as its speed for the rest of the race; the
 *              least (L - d) / v, equal values: lower index;
 *   [3] ZI     a uniformly drawn competitor: (w0 * n) >> 32, w0 the first Philox word of
 *              counter (s, 0, 0, zi_stream) under src's seed.
 * Binary32 round-to-nearest arithmetic in the written order; -1 for a snapshot past the
 * recorded trajectory.  Asynchronous.  Errors: BBE_ERR_ARG, BBE_ERR_CUDA. */
BBE_API bbe_status bbe_bettor_predictions(const bbe_batch *src, int32_t race, const float *positions,
                                          const float *step_sizes, const int32_t *n_steps, int32_t cap, int32_t every,
                                          int32_t n_snapshots, int32_t linex_window, float ud_gap, uint32_t zi_stream,
                                          int32_t *predictions, void *cuda_stream);

/* bbe_batch_set_law -- choose the responsiveness law of a staged batch (bbe_law above; a
 * batch starts with BBE_LAW_POSITION).
 *   law         BBE_LAW_POSITION (elapsed and horizon are ignored) or BBE_LAW_TIME.
 *   elapsed     float[n_races], t0 >= 0 per race (finite), or NULL (all 0); host or device.
 *   horizon     float[n_races], T > 0 per race (finite); required for BBE_LAW_TIME; host or
 *               device.  The library keeps its own copy.
 *   cuda_stream stream for the copies; the call synchronises it before returning.
 * bbe_rollout_batch, bbe_race_trajectory and bbe_snapshot_batch (whose snapshots carry
 * elapsed = t0 + the snapshot's step and the same horizon) follow the law.  Place and order
 * tallies and the order histogram follow it too; the surrogate takes position-law batches only
 * (BBE_ERR_UNSUPPORTED otherwise).  Errors: BBE_ERR_ARG (bad law, missing or invalid values),
 * BBE_ERR_CUDA. */
BBE_API bbe_status bbe_batch_set_law(bbe_batch *batch, bbe_law law, const float *elapsed, const float *horizon,
                                     void *cuda_stream);

/* bbe_batch_status -- synchronise cuda_stream and return the batch's device status from
 * the last bbe_rollout_batch, bbe_place_counts, bbe_order_counts or bbe_order_histogram:
 * BBE_OK, BBE_ERR_STEP_LIMIT, BBE_ERR_RANGE (an order hash table without a free entry, which
 * its sizing rules out, or, in the checked build, a failed device index check), or
 * BBE_ERR_CUDA if the stream reported an error. */
BBE_API bbe_status bbe_batch_status(bbe_batch *batch, void *cuda_stream);

/* bbe_batch_set_cfg / bbe_batch_get_cfg -- launch shape used by bbe_rollout_batch.
 * Setting rebuilds the work list.  Errors: BBE_ERR_ARG for out-of-range fields. */
BBE_API bbe_status bbe_batch_set_cfg(bbe_batch *batch, const bbe_launch_cfg *cfg);
BBE_API bbe_status bbe_batch_get_cfg(const bbe_batch *batch, bbe_launch_cfg *cfg);

/* bbe_batch_autotune -- pick this batch's launch by timing it (the batching workload asks for
 * block shapes and rollouts per warp chosen by measurement).  First, for each competitor count
 * present, a sample of up to 64 of its races is run once per layout (1 to 4 competitors per
 * lane) and another layout becomes that count's candidate only when at least 5 % faster on the
 * sample.  Second, the whole batch is timed (the best of three passes) with the candidate
 * per-count layout and with the starting one; every distinct layout is a launch of its own, so
 * the candidate is kept only if the whole batch runs at least 2 % faster with it.  Third, block
 * shapes (warps per block x blocks per SM, capped by occupancy: 4 x 16, 8 x 8, 2 x 32) and
 * work-item sizes (16, 32, 64 rollouts per lane) are each timed the same way; the starting shape
 * stays unless another is at least 2 % faster.
 * win_counts (device int32[sum n]) is scratch.
 * Once `budget_ms` of GPU time is spent the per-count samples not reached keep the default and
 * no further shape is tried (the whole-batch layout check always runs).  Counts do not depend
 * on the launch.  Synchronous; allocates (sample batches).  Errors: BBE_ERR_ARG, BBE_ERR_CUDA
 * (the batch keeps its previous launch). */
BBE_API bbe_status bbe_batch_autotune(bbe_batch *batch, int32_t *win_counts, double budget_ms, void *cuda_stream);

/* bbe_batch_layout -- competitors per lane used for a race of n competitors, n = 1..32, into
 * slots_by_n[n] (int32[BBE_MAX_COMPETITORS + 1]; entry 0 is set to 0).
 * bbe_batch_set_layout -- set that table (entries 0..4; 0 = the default of two; NULL clears
 * it).  It applies while the launch configuration's slots_per_lane is 0, and rebuilds the
 * work list.  Errors: BBE_ERR_ARG. */
BBE_API bbe_status bbe_batch_layout(const bbe_batch *batch, int32_t *slots_by_n);
BBE_API bbe_status bbe_batch_set_layout(bbe_batch *batch, const int32_t *slots_by_n);

/* bbe_batch_launches -- rollout-kernel launches of one bbe_rollout_batch or bbe_place_counts
 * call on this batch (one persistent launch per group of races with the same competitors per
 * lane, 1 to 4, forked from one stream inside the captured graph).  Errors: BBE_ERR_ARG. */
BBE_API bbe_status bbe_batch_launches(const bbe_batch *batch, int32_t *kernels_per_pass);

/* bbe_batch_info -- sizes of a staged batch (any output pointer may be NULL). */
BBE_API bbe_status bbe_batch_info(const bbe_batch *batch, int32_t *n_races, int64_t *n_competitors,
                          int64_t *total_rollouts, int32_t *max_competitors);

/* bbe_destroy_batch -- free a handle (NULL is ignored).  Does not block: the batch's device
 * memory is freed in stream order after the last work that the library enqueued on it (on
 * every stream it was given); work the caller captured into a graph of its own must not run
 * after the batch is destroyed. */
BBE_API void bbe_destroy_batch(bbe_batch *batch);

/* bbe_rollout_noalloc -- the rollout pass of bbe_race_init + bbe_rollout_batch for callers
 * that cannot allocate GPU memory.  The paper has no counterpart: it exists for code that
 * may not call cudaMalloc where it needs win counts (inside a memory pool it does not own,
 * in a latency-bound loop where an allocation could synchronise the device, or under an
 * allocator that another framework holds).
 *
 * It allocates nothing: no cudaMalloc, cudaFree or allocating library call.  Its work list,
 * queue head and status word live in one file-scope device array of 1,114,144 bytes (a
 * 32-byte header, BBE_NOALLOC_MAX_RACES int32 per-race item counts and BBE_NOALLOC_MAX_ITEMS
 * 16-byte work items) that every GPU which loads the library holds until the process exits.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress)
 * with the device current; make that first call before any stream capture on the device.
 *
 * Arguments are those of bbe_race_init plus the outputs of bbe_rollout_batch, with these
 * differences: every array must be memory of the current device (or managed memory; host
 * pointers and other devices' memory are rejected), pref and theta are required,
 * n_competitors = race_off[n_races] is the length of the per-competitor arrays, and the
 * launch shape is fixed: two competitors per lane (the library's automatic layout for a
 * batch that fills the GPU), 4-warp blocks, 32 rollouts per lane and work item.  Counts and step totals are identical to
 * bbe_rollout_batch's for the same inputs.
 *
 * Synchronous: the call synchronises cuda_stream after validating the batch on the device
 * and again after the rollouts, and returns their status.  All calls share the array: calls
 * that overlap on the GPU (from several host threads or streams) race and must be
 * serialised by the caller; each call resets what it reads before use.
 * Errors: BBE_ERR_RANGE (n_races outside 1..BBE_NOALLOC_MAX_RACES), BBE_ERR_ARG,
 * BBE_ERR_UNSUPPORTED, BBE_ERR_FINISHED (as bbe_race_init: the code of the lowest-numbered
 * invalid race, named in bbe_last_error), BBE_ERR_STEP_LIMIT, BBE_ERR_CUDA. */
#define BBE_NOALLOC_MAX_RACES 16384
#define BBE_NOALLOC_MAX_ITEMS 65536
BBE_API bbe_status bbe_rollout_noalloc(int32_t n_races, int32_t n_competitors, const int32_t *race_off,
                                       const float *track_len, const int64_t *rollouts, const float *pos,
                                       const float *mu, const float *sigma, const float *resp, const float *pref,
                                       const float *theta, const float *prev_step, uint64_t seed, bbe_dist dist,
                                       uint32_t race_id0, int32_t *win_counts, int64_t *steps_total,
                                       void *cuda_stream);

/* bbe_last_error -- thread-local message of the last failed call on this thread. */
BBE_API const char *bbe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BBE_H */
