/*
 * bbe_surrogate.h -- learned surrogate of the Monte Carlo win probabilities.
 *
 * The paper's rational bettors estimate win probabilities by simulating the race d times
 * (Section 3); the race simulator is the expensive part of the model (Section 6 moves it to
 * a GPU because millions of dry-runs are needed).  This surrogate is trained on
 * (race state, Monte Carlo win probabilities) pairs that bbe_rollout_batch produces and
 * then answers the same question with one network evaluation per race.  The paper has no
 * learned model; the network below is this library's design:
 *
 *   per competitor c, 16 input columns: x_c[0..4] = [d_c / L, (L - d_c) / 5000, mu_c - 16,
 *            sigma_c - 1, 2 rho_c - 1]; x_c[5..13] derived per race from those: with
 *            v = mu (1 + 0.1 (2 rho - 1) d / L), T = (L - d) / v and s = sigma sqrt(T) / v,
 *            T / 100, the lag behind the race's least T (capped at 100, / 10), s, that lag over
 *            sqrt(s^2 + s_min^2 + 0.01) (capped at 20, / 5), the gap to the nearest competitor
 *            ahead and behind (capped at 100, / 10), 1 / n, and whether c catches the one ahead
 *            (and the one behind catches c) before the line, as a capped share of the remaining
 *            race; x_c[14..15] = 0
 *   encoder  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3)  (width 128)
 *   context  g = mean over the race's competitors of h3
 *   head     u = relu(W4 [h3; g] + b4) (256 -> 128), logit = w5 . u + b5
 *   output   softmax of the logits over the race's competitors (so relabelling the
 *            competitors relabels the output: permutation equivariance)
 *   loss     cross-entropy against the Monte Carlo probabilities, mean over races.
 * Matrix products take bfloat16 operands with float32 accumulation; the master weights and
 * the Adam state are float32.  The forward kernel waits on the tensor cores with a bounded
 * wait (2 s); a wait that gives up is reported by bbe_surrogate_status.  Parameters are one float vector of bbe_surrogate_num_params()
 * values: W1 [128][16] (input columns 14 and 15 are zero), b1 [128], W2 [128][128], b2, W3 [128][128], b3,
 * W4 [128][256], b4, w5 [128], b5 [1] (row-major [out][in]).
 *
 * Conventions are those of bbe.h (status codes, thread-local bbe_last_error, caller-owned
 * buffers, library-owned handles, stream arguments).
 */
#ifndef BBE_SURROGATE_H
#define BBE_SURROGATE_H

#include "bbe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bbe_surrogate bbe_surrogate; /* opaque, library-owned */

typedef struct {
    float lr;             /* Adam step size */
    float beta1, beta2;   /* Adam moment decay rates */
    float eps;            /* Adam denominator guard */
    float weight_decay;   /* decoupled weight decay per step (AdamW); 0 = none */
    int32_t batch_states; /* races per optimizer step, >= 1 */
    int32_t steps;        /* optimizer steps to run in this call, >= 1 */
    uint64_t shuffle_seed;/* seed of the per-epoch shuffle of the races */
} bbe_train_cfg;

/* Number of floats in the parameter vector. */
BBE_API int64_t bbe_surrogate_num_params(void);

/* bbe_surrogate_create -- new network with He-uniform weights drawn from init_seed and zero
 * biases, on the current device.  Errors: BBE_ERR_ARG, BBE_ERR_CUDA. */
BBE_API bbe_status bbe_surrogate_create(bbe_surrogate **out, uint64_t init_seed);

/* bbe_surrogate_set_params / get_params -- copy the float32 parameter vector from / to host
 * memory (num_params floats).  Setting resets the Adam state.  Synchronous. */
BBE_API bbe_status bbe_surrogate_set_params(bbe_surrogate *s, const float *params);
BBE_API bbe_status bbe_surrogate_get_params(const bbe_surrogate *s, float *params);

/* bbe_surrogate_train -- cfg->steps Adam steps on the races of `states` with targets
 * `target_probs` (device float[sum n], e.g. from bbe_win_probs; each race's targets should
 * sum to 1).  Each epoch visits the races in a fresh shuffled order; the epoch position is
 * kept between calls.  The first call on a handle records the ranges of the training
 * states (competitor counts, track lengths, the five input features, P, theta) that
 * bbe_surrogate_infer treats as in range.
 *   loss_log  device float[cfg->steps] or NULL: mean cross-entropy of each step's batch.
 * Asynchronous on cuda_stream after the host-side planning.  Errors: BBE_ERR_ARG,
 * BBE_ERR_CUDA. */
BBE_API bbe_status bbe_surrogate_train(bbe_surrogate *s, const bbe_batch *states, const float *target_probs,
                                       const bbe_train_cfg *cfg, float *loss_log, void *cuda_stream);

/* bbe_surrogate_grad -- gradient of the mean cross-entropy over all races of `states`
 * (device float[num_params], overwritten) and, if loss is not NULL, the loss (device float[1]),
 * without changing the parameters.  Asynchronous.  Errors: BBE_ERR_ARG, BBE_ERR_CUDA. */
BBE_API bbe_status bbe_surrogate_grad(bbe_surrogate *s, const bbe_batch *states, const float *target_probs,
                                      float *grad, float *loss, void *cuda_stream);

/* bbe_surrogate_forward -- network output for every race of `states`: probs device
 * float[sum n] (each race's values sum to 1).  No range check.  Asynchronous. */
BBE_API bbe_status bbe_surrogate_forward(bbe_surrogate *s, const bbe_batch *states, float *probs,
                                         void *cuda_stream);

/* bbe_surrogate_infer -- win probabilities for every race of `states`: races inside the
 * training ranges get the network's output unless the confidence gate (bbe_surrogate_set_gate)
 * rejects it; every other race is simulated with plain Monte Carlo on its own stream id
 * (bbe_rollout_batch), so its probabilities are exactly those of the Monte Carlo path: with
 * the race's own rollout budget by default, or with the budget that the two-stage rule of
 * bbe_surrogate_set_fallback picks (at most the race's own).
 *   probs   device float[sum n], overwritten.
 *   used_mc device uint8[n_races] or NULL: 0 network, 1 Monte Carlo (outside the training
 *           ranges), 2 Monte Carlo (rejected by the confidence gate).
 * Synchronises cuda_stream when the gate is enabled or some race falls back.  Errors:
 * BBE_ERR_ARG, BBE_ERR_CUDA, BBE_ERR_RANGE (no training ranges recorded yet). */
BBE_API bbe_status bbe_surrogate_infer(bbe_surrogate *s, const bbe_batch *states, float *probs, uint8_t *used_mc,
                                       void *cuda_stream);

/* bbe_surrogate_set_inputs -- which input columns the network sees: BBE_SURROGATE_INPUTS_DERIVED
 * (14, the default: the five raw quantities and the nine values derived from them per race) or
 * BBE_SURROGATE_INPUTS_RAW (5: position, remaining distance and the three parameters mu, sigma,
 * rho, with the derived columns zero, i.e. the encoder of the surrogate workload's stated
 * configuration).  Set it before training; it is saved with the checkpoint.  Errors:
 * BBE_ERR_ARG. */
#define BBE_SURROGATE_INPUTS_RAW 5
#define BBE_SURROGATE_INPUTS_DERIVED 14
BBE_API bbe_status bbe_surrogate_set_inputs(bbe_surrogate *s, int32_t inputs);

/* bbe_surrogate_set_gate -- confidence gate of bbe_surrogate_infer: a race whose network output
 * has a second-largest probability above runner_up_max (a contest the network does not call
 * with near-certainty) is simulated with plain Monte Carlo instead.  runner_up_max in [0, 1];
 * values of 0.5 or more disable the gate (the default is 1).  Not stored in checkpoints.
 * Errors: BBE_ERR_ARG. */
BBE_API bbe_status bbe_surrogate_set_gate(bbe_surrogate *s, float runner_up_max);

/* bbe_surrogate_set_fallback -- two-stage Monte Carlo fallback of bbe_surrogate_infer.  With
 * pilot_rollouts = 0 (the default) a fallback race runs its own rollout budget R.  Otherwise it
 * first runs R1 = min(pilot_rollouts, R) rollouts; bbe_surrogate_fallback_budget turns their
 * counts into a total budget R' in [R1, R] that gives each of the race's probabilities a
 * standard deviation of about max_sd at most, and rollouts R1 .. R'-1 of the same stream are
 * added, so the answer is plain Monte Carlo with R' rollouts (k = 0 .. R'-1).  A max-abs error
 * target e over m probabilities calls for max_sd near e / sqrt(2 ln m).  pilot_rollouts in
 * 0 .. 2^31-1, max_sd in (0, 0.5] when pilot_rollouts > 0.  Not stored in checkpoints.
 * Errors: BBE_ERR_ARG. */
BBE_API bbe_status bbe_surrogate_set_fallback(bbe_surrogate *s, int64_t pilot_rollouts, double max_sd);

/* bbe_surrogate_fallback_budget -- the budget rule of the two-stage fallback, on the host.
 *   counts  host int32[n]: wins of each competitor of one race in `pilot` rollouts.
 *   budget  out: with p_c = counts_c / pilot, h_c = 3 sqrt(max(p_c (1 - p_c), 1 / pilot) / pilot)
 *           (three standard errors, floored at one count's worth), q_c the point of
 *           [p_c - h_c, p_c + h_c] nearest 1/2 and v = max_c q_c (1 - q_c) (so v bounds every
 *           p (1 - p) within three standard errors of the pilot's estimate):
 *           budget = min(cap, max(pilot, ceil(v / max_sd^2))), computed in double precision;
 *           a race of one competitor (whose probability is 1) keeps the pilot.
 * Errors: BBE_ERR_ARG (n < 1, NULL pointer, pilot < 1, cap < pilot, max_sd outside (0, 0.5]). */
BBE_API bbe_status bbe_surrogate_fallback_budget(int32_t n, const int32_t *counts, int64_t pilot, int64_t cap,
                                                 double max_sd, int64_t *budget);

/* bbe_surrogate_fallback_stats -- races sent to Monte Carlo by the last bbe_surrogate_infer
 * call on this handle and the rollouts their answers rest on (the sum of their total budgets;
 * 0 when the call failed).  Either pointer may be NULL.  Errors: BBE_ERR_ARG. */
BBE_API bbe_status bbe_surrogate_fallback_stats(const bbe_surrogate *s, int64_t *races, int64_t *rollouts);

/* bbe_surrogate_fallback_times -- host wall time of the last bbe_surrogate_infer's Monte Carlo
 * fallback, by phase, into seconds[5]: staging the fallback races, the pilot (or the whole
 * budget without one: its rollouts and their read-back), the budget rule, staging the top-up,
 * and the top-up with the final probabilities.  Errors: BBE_ERR_ARG. */
BBE_API bbe_status bbe_surrogate_fallback_times(const bbe_surrogate *s, double *seconds);

/* bbe_surrogate_status -- synchronise cuda_stream and report whether a kernel launched on
 * this handle gave up a bounded device wait since the last call (the flag is then cleared;
 * the outputs of the affected calls are undefined).  Errors: BBE_ERR_TIMEOUT, BBE_ERR_ARG,
 * BBE_ERR_CUDA. */
BBE_API bbe_status bbe_surrogate_status(bbe_surrogate *s, void *cuda_stream);

/* bbe_surrogate_wait_probe -- exercise the bounded-wait path without a fault: one warp waits, with
 * the same bounded wait the surrogate kernels use for the tensor cores and bulk copies, on an
 * mbarrier that nothing arrives at; after limit_ns (0 .. 2e9) it gives up and sets the handle's
 * status word, which the next bbe_surrogate_status reports as BBE_ERR_TIMEOUT.  Nothing is left
 * in flight and the context stays usable.  Asynchronous.  Errors: BBE_ERR_ARG, BBE_ERR_CUDA. */
BBE_API bbe_status bbe_surrogate_wait_probe(bbe_surrogate *s, int64_t limit_ns, void *cuda_stream);

/* bbe_surrogate_save / load -- checkpoint: parameters, Adam state, step count, epoch and the
 * position in it, input mode and training ranges, in a little-endian binary file.  load
 * creates a handle on the current device; its first bbe_surrogate_train call continues the
 * saved epoch (the epoch's race order is regenerated from the configuration's shuffle seed), so
 * saving, loading and training on gives the parameters of an uninterrupted run with the same
 * configuration and batch.  Errors: BBE_ERR_ARG (bad file), BBE_ERR_CUDA. */
BBE_API bbe_status bbe_surrogate_save(const bbe_surrogate *s, const char *path);
BBE_API bbe_status bbe_surrogate_load(bbe_surrogate **out, const char *path);

/* bbe_surrogate_destroy -- free a handle (NULL is ignored). */
BBE_API void bbe_surrogate_destroy(bbe_surrogate *s);

#ifdef __cplusplus
}
#endif

#endif /* BBE_SURROGATE_H */
