/*
 * bbe_oracle.c -- plain, slow CPU oracle of the BBE race simulator's Monte Carlo
 * win-probability estimate (Cliff, Hawkins, Keen & Lau-Soto, "Implementing the BBE
 * Agent-Based Model of a Sports-Betting Exchange", 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  The CUDA library never calls it, and it
 * shares no code, header, table or constant generator with the CUDA sources.
 *
 * What it computes (paper sections cited per function):
 *   - Section 3, the discrete-time race: d_c(t+1) = d_c(t) + S_c(t), with S_c from
 *     Eq. 1 (responsiveness R_c, preference P_c, stochastic step delta(v_c), blocking
 *     by the nearest competitor i+ in front when Delta_c <= theta_c, delta_min).
 *   - Section 3, the RP(d) "dry-run" estimator: the race is re-simulated R times from
 *     the current state and the winners are counted (elementary frequentist statistics).
 *
 * Arithmetic: IEEE binary32, round-to-nearest-even, one rounding per written operation.
 * Build with -ffp-contract=off and without fast-math so the compiler fuses nothing; the
 * fused multiply-adds the contract asks for are written as fmaf(), which C99 defines as
 * a single rounding.  The contract (readings of the paper where it is silent) is:
 *
 *   kappa = 0.2f, S_floor = 1e-3f, theta default = 1.0f, max_steps default = 2^20.
 *   invL    = 1 / L
 *   kr_c    = kappa * ((2 * rho_c) - 1)
 *   R_c     = fmaf(kr_c, fmaf(d_c, invL, -0.5f), 1.0f)              responsiveness (position law)
 *   or, with the time law and invT = 1 / T,
 *   u       = min(1, (t0 + (float)t) * invT),  R_c = fmaf(kr_c, u - 0.5f, 1.0f)
 *   i+      = argmin_{i != c, d_i > d_c} d_i   (equal d_i: lowest i)  nearest in front
 *   blocked = i+ exists and not (d_{i+} - d_c > theta_c)             Eq. 1 "otherwise"
 *   S_c     = blocked ? R_c * min(prev_c, prev_{i+})                  Eq. 1, delta_min
 *                     : (R_c * P_c) * fmaf(sigma_c, z, mu_c)           Eq. 1, first case
 *   S_c     = max(S_c, S_floor)                                       Section 3: S > 0
 *   all d_c advance together (synchronous update); prev_c <- S_c
 *   the rollout ends at the first step where some d_c + S_c >= L; the winner is the
 *   finisher with the least tau_c = (L - d_c) / S_c, equal tau: lowest c.
 *
 * Random draws z: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) with key
 * (seed_lo, seed_hi) and counter (k, t >> 2, c, r) for race r, rollout k, step t,
 * competitor c.  NORMAL: Box-Muller (Box & Muller, 1958) on word pair (t >> 1) & 1,
 * cosine branch for even t, sine branch for odd t.  UNIFORM: sqrt(3) * (2u - 1).
 * TWO_POINT: +-1 from the top bit.  log and sin/cos(2 pi u) are evaluated with the
 * fixed operation sequences below (a fitted polynomial for log after an exact range reduction,
 * Taylor series for sin and cos after an exact quadrant reduction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "bbe_oracle.h"

/* ---------------------------------------------------------------- Philox4x32-10 */

/* Philox4x32-10 of Salmon et al. (SC'11): ten rounds; each round multiplies words 0
 * and 2 by the two round multipliers, swaps and xors the high halves with the other
 * words and the key; the key is bumped by the Weyl constants between rounds. */
void bbe_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------ elementary functions */

static float f32_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_from_f32(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* Natural log of a positive normal binary32 x.
 * x = 2^e * m with m in (sqrt(1/2), sqrt(2)];  f = m - 1 is exact (Sterbenz);
 * log m = f * g(f) with g(f) ~ log(1 + f) / f a degree-9 polynomial on [sqrt(1/2) - 1, sqrt(2) - 1]
 * (coefficients from oracle/fit_log.py: Lawson's minimax iteration of least squares on 512
 * Chebyshev nodes, relative error 4.1e-9 before rounding to binary32), evaluated by Horner's rule with fused
 * multiply-adds; log x = e ln2 + log m with ln2 split into a 16-bit head and a tail
 * (Cody & Waite). */
float bbe_oracle_log(float x)
{
    static const float G[10] = {
        0x1.000000p+0f, -0x1.fffff8p-2f, 0x1.555550p-2f, -0x1.000428p-2f, 0x1.99a402p-3f,
        -0x1.542748p-3f, 0x1.227092p-3f, -0x1.0f3768p-3f, 0x1.084e42p-3f, -0x1.383dfep-4f,
    };
    const float LN2_HI = 0x1.62e4p-1f;
    const float LN2_LO = 0x1.7f7d1cp-20f;
    uint32_t b = bits_from_f32(x);
    int e = (int)(b >> 23) - 127;
    uint32_t mb = (b & 0x007FFFFFu) | 0x3F800000u;     /* m in [1, 2) */
    if (mb > 0x3FB504F3u) {                             /* m > sqrt(2): halve m */
        mb -= 0x00800000u;
        e += 1;
    }
    float m = f32_from_bits(mb);
    float f = m - 1.0f;
    float g = G[9];
    for (int k = 8; k >= 0; --k) g = fmaf(f, g, G[k]);
    float logm = f * g;
    float ef = (float)e;
    return fmaf(ef, LN2_HI, fmaf(ef, LN2_LO, logm));
}

/* sin(2 pi u) and cos(2 pi u) for u = m24 * 2^-24, m24 in [0, 2^24).
 * Quadrant q = nearest integer to 4u (exact integer arithmetic); the remainder
 * f = u - q/4 in [-1/8, 1/8) is exact.  With theta = 2 pi f (|theta| <= pi/4) the Taylor
 * series of sin to theta^9 and of cos to theta^10 are evaluated in f by Horner's rule. */
void bbe_oracle_sincos2pi(uint32_t m24, float *sin_out, float *cos_out)
{
    const float S1 = 0x1.921fb6p+2f;   /*  (2pi)^1 / 1!  */
    const float S3 = -0x1.4abbcep+5f;  /* -(2pi)^3 / 3!  */
    const float S5 = 0x1.466bc6p+6f;   /*  (2pi)^5 / 5!  */
    const float S7 = -0x1.32d2ccp+6f;  /* -(2pi)^7 / 7!  */
    const float S9 = 0x1.507834p+5f;   /*  (2pi)^9 / 9!  */
    const float C2 = -0x1.3bd3ccp+4f;  /* -(2pi)^2 / 2!  */
    const float C4 = 0x1.03c1f0p+6f;   /*  (2pi)^4 / 4!  */
    const float C6 = -0x1.55d3c8p+6f;  /* -(2pi)^6 / 6!  */
    const float C8 = 0x1.e1f506p+5f;   /*  (2pi)^8 / 8!  */
    const float C10 = -0x1.a6d1f2p+4f; /* -(2pi)^10 / 10! */
    uint32_t q = (m24 + 0x200000u) >> 22;               /* 0..4 */
    int32_t fm = (int32_t)m24 - (int32_t)(q << 22);     /* [-2^21, 2^21) */
    float f = (float)fm * 0x1p-24f;
    float y = f * f;
    float ps = fmaf(y, S9, S7);
    ps = fmaf(y, ps, S5);
    ps = fmaf(y, ps, S3);
    ps = fmaf(y, ps, S1);
    float sv = f * ps;
    float pc = fmaf(y, C10, C8);
    pc = fmaf(y, pc, C6);
    pc = fmaf(y, pc, C4);
    pc = fmaf(y, pc, C2);
    float cv = fmaf(y, pc, 1.0f);
    switch (q & 3u) {
    case 0: *sin_out = sv;  *cos_out = cv;  break;
    case 1: *sin_out = cv;  *cos_out = -sv; break;
    case 2: *sin_out = -sv; *cos_out = -cv; break;
    default: *sin_out = -cv; *cos_out = sv; break;
    }
}

/* ------------------------------------------------------------- the step generator */

/* delta(v_c) of Eq. 1 is mu_c + sigma_c * z; this returns z for (race r, rollout k,
 * step t, competitor c) under distribution `dist` (Section 3 names the step generator
 * only as "a stochastic function"; the distributions are this library's readings). */
float bbe_oracle_z(int dist, uint64_t seed, uint32_t r, uint32_t k, uint32_t t, uint32_t c)
{
    uint32_t ctr[4] = { k, t >> 2, c, r };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t w[4];
    bbe_oracle_philox4x32_10(ctr, key, w);
    if (dist == BBE_ORACLE_DIST_TWO_POINT) {
        return (w[t & 3u] >> 31) ? 1.0f : -1.0f;
    }
    if (dist == BBE_ORACLE_DIST_UNIFORM) {
        float u = (float)(w[t & 3u] >> 8) * 0x1p-24f;
        return 0x1.bb67aep+0f * ((2.0f * u) - 1.0f);
    }
    /* NORMAL: Box-Muller on the pair selected by bit 1 of t */
    uint32_t wa = ((t >> 1) & 1u) ? w[2] : w[0];
    uint32_t wb = ((t >> 1) & 1u) ? w[3] : w[1];
    float u1 = (float)((wa >> 8) + 1u) * 0x1p-24f;       /* (0, 1] */
    float radius = sqrtf(-2.0f * bbe_oracle_log(u1));
    float sv, cv;
    bbe_oracle_sincos2pi(wb >> 8, &sv, &cv);
    return (t & 1u) ? radius * sv : radius * cv;
}

/* -------------------------------------------------------------- race simulation */

/* Responsiveness R_c(t, d) of Eq. 1.  Section 3 gives only its purpose (fast start and
 * fade, or slow start and fast finish) and writes it as a function of time and distance.
 * Two readings, each linear and centred on the middle of the race:
 *   position law: R = 1 + kappa (2 rho - 1) (d / L - 1/2), the fraction of the track covered;
 *   time law:     R = 1 + kappa (2 rho - 1) (u - 1/2), u = min(1, (t0 + t) / T), the fraction
 *                 of the race's expected duration T elapsed (t0 steps before the state, t in
 *                 the dry-run), held at its end value once T has passed. */
static float responsiveness(float kr, float d, float invL)
{
    return fmaf(kr, fmaf(d, invL, -0.5f), 1.0f);
}

static float responsiveness_time(float kr, float t0, uint32_t t, float invT)
{
    float u = (t0 + (float)t) * invT;
    if (u > 1.0f) u = 1.0f;
    return fmaf(kr, u - 0.5f, 1.0f);
}

/* One step of Section 3 for every competitor, reading only the time-t state
 * (synchronous update).  Returns the step sizes S in S_out. */
static void race_step(const bbe_oracle_race *race, const float *kr, float invL,
                      const float *d, const float *prev, uint64_t seed, uint32_t r,
                      uint32_t k, uint32_t t, float *S_out)
{
    int n = race->n;
    float invT = race->law == BBE_ORACLE_LAW_TIME ? 1.0f / race->T : 0.0f;
    for (int c = 0; c < n; ++c) {
        float R_c = race->law == BBE_ORACLE_LAW_TIME ? responsiveness_time(kr[c], race->t0, t, invT)
                                                     : responsiveness(kr[c], d[c], invL);
        /* i+ : nearest competitor strictly in front of c; equal distance -> lowest i */
        int i_plus = -1;
        for (int i = 0; i < n; ++i) {
            if (i == c || !(d[i] > d[c])) continue;
            if (i_plus < 0 || d[i] < d[i_plus]) i_plus = i;
        }
        float S_c;
        int blocked = 0;
        if (i_plus >= 0) {
            float Delta_c = d[i_plus] - d[c];
            blocked = !(Delta_c > race->theta[c]);
        }
        if (blocked) {
            float delta_min = prev[c] < prev[i_plus] ? prev[c] : prev[i_plus];
            S_c = R_c * delta_min;
        } else {
            float z = bbe_oracle_z(race->dist, seed, r, k, t, (uint32_t)c);
            float delta = fmaf(race->sigma[c], z, race->mu[c]);
            S_c = (R_c * race->P[c]) * delta;
        }
        if (S_c < BBE_ORACLE_S_FLOOR) S_c = BBE_ORACLE_S_FLOOR;
        S_out[c] = S_c;
    }
}

static void race_constants(const bbe_oracle_race *race, float *kr, float *prev0, float *invL)
{
    *invL = 1.0f / race->L;
    for (int c = 0; c < race->n; ++c) {
        kr[c] = BBE_ORACLE_KAPPA * ((2.0f * race->rho[c]) - 1.0f);
        prev0[c] = race->prev0 ? race->prev0[c] : race->mu[c] * race->P[c];
    }
}

/* One rollout (dry-run) k of race r from its current state.  Returns the winner's index,
 * or -1 if max_steps steps pass without a finisher.  *steps receives the number of steps
 * taken (the finishing step included).  If traj is non-null it receives the positions
 * after each step, row-major [steps][n], up to traj_cap rows. */
int bbe_oracle_rollout(const bbe_oracle_race *race, uint64_t seed, uint32_t r, uint32_t k,
                       int64_t max_steps, int64_t *steps, float *traj, int64_t traj_cap)
{
    int n = race->n;
    float *buf = (float *)malloc(sizeof(float) * (size_t)n * 6);
    float *kr = buf, *prev = buf + n, *d = buf + 2 * n, *S = buf + 3 * n, *dn = buf + 4 * n;
    float invL;
    race_constants(race, kr, prev, &invL);
    for (int c = 0; c < n; ++c) d[c] = race->d0[c];
    int winner = -1;
    int64_t t = 0;
    for (;;) {
        if (t == max_steps) break;
        race_step(race, kr, invL, d, prev, seed, r, k, (uint32_t)t, S);
        int any_finished = 0;
        for (int c = 0; c < n; ++c) {
            dn[c] = d[c] + S[c];
            if (dn[c] >= race->L) any_finished = 1;
        }
        if (traj && t < traj_cap) memcpy(traj + t * n, dn, sizeof(float) * (size_t)n);
        if (any_finished) {
            /* the finisher that crossed earliest within the step: least (L - d)/S */
            float best_tau = 0.0f;
            for (int c = 0; c < n; ++c) {
                if (!(dn[c] >= race->L)) continue;
                float tau = (race->L - d[c]) / S[c];
                if (winner < 0 || tau < best_tau) {
                    winner = c;
                    best_tau = tau;
                }
            }
            ++t;
            break;
        }
        for (int c = 0; c < n; ++c) {
            prev[c] = S[c];
            d[c] = dn[c];
        }
        ++t;
    }
    *steps = t;
    free(buf);
    return winner;
}

/* The RP(d) dry-run estimator of Section 3 for one race: R rollouts k = k_begin ..
 * k_begin + R - 1, winners counted in counts[0..n).  Returns 0, or BBE_ORACLE_STEP_LIMIT
 * if some rollout hit max_steps (that rollout then counts for nobody). */
int bbe_oracle_race_counts(const bbe_oracle_race *race, uint64_t seed, uint32_t r,
                           int64_t k_begin, int64_t R, int64_t max_steps,
                           int32_t *counts, int64_t *steps_total)
{
    int status = 0;
    int64_t total = 0;
    for (int c = 0; c < race->n; ++c) counts[c] = 0;
    for (int64_t k = k_begin; k < k_begin + R; ++k) {
        int64_t steps = 0;
        int w = bbe_oracle_rollout(race, seed, r, (uint32_t)k, max_steps, &steps, NULL, 0);
        total += steps;
        if (w < 0) status = BBE_ORACLE_STEP_LIMIT;
        else counts[w] += 1;
    }
    if (steps_total) *steps_total = total;
    return status;
}

/* One rollout k of race r run until `places` competitors have crossed the line.  Section 3
 * runs a race until its last competitor crosses and lets in-play betting stop earlier, for
 * instance when the third-placed competitor crosses; place and each-way markets (Section 2)
 * need the places.  Readings: every competitor keeps moving under Eq. 1 until the rollout
 * ends, finished ones included (the rule names no exception); the competitors that cross in
 * the same step are placed in order of their crossing time within the step,
 * tau = (L - d) / S, equal tau: lower index first.  order[j] receives the competitor in place
 * j for j < places (places <= n).  Returns 0, or BBE_ORACLE_STEP_LIMIT if max_steps steps pass
 * first.  *steps receives the number of steps taken. */
int bbe_oracle_rollout_order(const bbe_oracle_race *race, uint64_t seed, uint32_t r, uint32_t k,
                             int places, int64_t max_steps, int64_t *steps, int32_t *order)
{
    int n = race->n;
    float *buf = (float *)malloc(sizeof(float) * (size_t)n * 5);
    int *finished = (int *)calloc((size_t)n, sizeof(int));
    float *kr = buf, *prev = buf + n, *d = buf + 2 * n, *S = buf + 3 * n, *dn = buf + 4 * n;
    float invL;
    race_constants(race, kr, prev, &invL);
    for (int c = 0; c < n; ++c) d[c] = race->d0[c];
    int placed = 0, status = 0;
    int64_t t = 0;
    for (;;) {
        if (t == max_steps) {
            status = BBE_ORACLE_STEP_LIMIT;
            break;
        }
        race_step(race, kr, invL, d, prev, seed, r, k, (uint32_t)t, S);
        for (int c = 0; c < n; ++c) dn[c] = d[c] + S[c];
        /* this step's new finishers, earliest crossing first */
        for (;;) {
            int best = -1;
            float best_tau = 0.0f;
            for (int c = 0; c < n; ++c) {
                if (finished[c] || !(dn[c] >= race->L)) continue;
                float tau = (race->L - d[c]) / S[c];
                if (best < 0 || tau < best_tau) {
                    best = c;
                    best_tau = tau;
                }
            }
            if (best < 0) break;
            finished[best] = 1;
            if (placed < places) order[placed] = best;
            ++placed;
        }
        ++t;
        if (placed >= places) break;
        for (int c = 0; c < n; ++c) {
            prev[c] = S[c];
            d[c] = dn[c];
        }
    }
    *steps = t;
    free(finished);
    free(buf);
    return status;
}

/* Place counts of one race: R rollouts k = k_begin .. k_begin + R - 1, each run until
 * min(places, n) competitors have crossed; counts[c * places + j] = rollouts in which c
 * finished in place j (j = 0: the winner).  Returns 0, or BBE_ORACLE_STEP_LIMIT if some
 * rollout hit max_steps (that rollout then counts for nobody). */
int bbe_oracle_race_places(const bbe_oracle_race *race, uint64_t seed, uint32_t r,
                           int64_t k_begin, int64_t R, int places, int64_t max_steps,
                           int32_t *counts, int64_t *steps_total)
{
    int n = race->n;
    int kk = places < n ? places : n;
    int status = 0;
    int64_t total = 0;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int i = 0; i < n * places; ++i) counts[i] = 0;
    for (int64_t k = k_begin; k < k_begin + R; ++k) {
        int64_t steps = 0;
        int st = bbe_oracle_rollout_order(race, seed, r, (uint32_t)k, kk, max_steps, &steps, order);
        total += steps;
        if (st != 0) {
            status = st;
            continue;
        }
        for (int j = 0; j < kk; ++j) counts[order[j] * places + j] += 1;
    }
    if (steps_total) *steps_total = total;
    free(order);
    return status;
}

/* Finishing-order tallies (Section 3: the rollouts estimate the distribution of outcomes; the
 * ordered top places are the outcome a forecast or exacta-style market is about).  Rollouts
 * k_begin .. k_begin+R-1 run to the kk-th finisher, kk = min(places, n); each completed rollout adds
 * one to the entry of its ordered top-kk tuple (o_1, .., o_kk), entry index
 * (..((o_1) n + o_2) n + ..) + o_kk of the n^kk counts.  A rollout cut off by max_steps counts for
 * nobody.  Returns 0 or BBE_ORACLE_STEP_LIMIT; *steps_total sums the steps of every rollout. */
int bbe_oracle_race_orders(const bbe_oracle_race *race, uint64_t seed, uint32_t r,
                           int64_t k_begin, int64_t R, int places, int64_t max_steps,
                           int32_t *counts, int64_t *steps_total)
{
    int n = race->n;
    int kk = places < n ? places : n;
    int64_t cells = 1;
    for (int j = 0; j < kk; ++j) cells *= n;
    int status = 0;
    int64_t total = 0;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < cells; ++i) counts[i] = 0;
    for (int64_t k = k_begin; k < k_begin + R; ++k) {
        int64_t steps = 0;
        int st = bbe_oracle_rollout_order(race, seed, r, (uint32_t)k, kk, max_steps, &steps, order);
        total += steps;
        if (st != 0) {
            status = st;
            continue;
        }
        int64_t code = 0;
        for (int j = 0; j < kk; ++j) code = code * n + order[j];
        counts[code] += 1;
    }
    if (steps_total) *steps_total = total;
    free(order);
    return status;
}

/* The finishing order of each of rollouts k_begin .. k_begin + R - 1 of race r, run to the
 * kk-th finisher, kk = min(places, n) (Section 3: the dry-runs give the distribution of
 * outcomes): orders[i * kk + j] = the competitor in place j of rollout k_begin + i, or -1 in
 * the whole row of a rollout cut off at max_steps.  The histogram of the rows is the order
 * distribution.  Returns 0, or BBE_ORACLE_STEP_LIMIT if some rollout was cut off. */
int bbe_oracle_race_order_list(const bbe_oracle_race *race, uint64_t seed, uint32_t r, int64_t k_begin, int64_t R,
                               int places, int64_t max_steps, int32_t *orders, int64_t *steps_total)
{
    int n = race->n;
    int kk = places < n ? places : n;
    int status = 0;
    int64_t total = 0;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < R; ++i) {
        int64_t steps = 0;
        int st = bbe_oracle_rollout_order(race, seed, r, (uint32_t)(k_begin + i), kk, max_steps, &steps, order);
        total += steps;
        if (st != 0) status = st;
        for (int j = 0; j < kk; ++j) orders[i * kk + j] = st != 0 ? -1 : order[j];
    }
    if (steps_total) *steps_total = total;
    free(order);
    return status;
}

/* One full run of race r (rollout k of its stream): every competitor moves under Eq. 1 until
 * the last one has crossed the line (Section 3) or max_steps steps pass; the space-time series
 * of the race (Section 6 plots one).  For t < min(steps, cap): d_traj[t * n + c] = d_c after
 * step t and s_traj[t * n + c] = S_c(t) (either may be NULL).  Returns 0, or
 * BBE_ORACLE_STEP_LIMIT; *steps = steps taken. */
int bbe_oracle_trajectory(const bbe_oracle_race *race, uint64_t seed, uint32_t r, uint32_t k, int64_t max_steps,
                          int64_t *steps, float *d_traj, float *s_traj, int64_t cap)
{
    int n = race->n;
    float *buf = (float *)malloc(sizeof(float) * (size_t)n * 5);
    float *kr = buf, *prev = buf + n, *d = buf + 2 * n, *S = buf + 3 * n, *dn = buf + 4 * n;
    float invL;
    race_constants(race, kr, prev, &invL);
    for (int c = 0; c < n; ++c) d[c] = race->d0[c];
    int status = 0;
    int64_t t = 0;
    for (;;) {
        if (t == max_steps) {
            status = BBE_ORACLE_STEP_LIMIT;
            break;
        }
        race_step(race, kr, invL, d, prev, seed, r, k, (uint32_t)t, S);
        int all_in = 1;
        for (int c = 0; c < n; ++c) {
            dn[c] = d[c] + S[c];
            if (!(dn[c] >= race->L)) all_in = 0;
        }
        if (t < cap) {
            if (d_traj) memcpy(d_traj + t * n, dn, sizeof(float) * (size_t)n);
            if (s_traj) memcpy(s_traj + t * n, S, sizeof(float) * (size_t)n);
        }
        for (int c = 0; c < n; ++c) {
            prev[c] = S[c];
            d[c] = dn[c];
        }
        ++t;
        if (all_in) break;
    }
    *steps = t;
    free(buf);
    return status;
}

/* Preference coefficients P_c(f_r, p_c) of Eq. 1 from factor and preference vectors
 * (Section 3: a coefficient in [0, 1] that reduces the step by an amount depending on the
 * mismatch between the race's factors f_r and the competitor's preferences p_c; the paper gives
 * no formula).  Reading: P_c = prod_i (1 - w_i * min(1, |f_r,i - p_c,i|)), i = 0 .. F-1 in order,
 * binary32, with weights w_i in [0, 1], so a perfect match gives 1 and a full mismatch on a
 * factor of weight 1 gives 0.  factors [n_races][F], prefs [sum n][F], P [sum n]. */
void bbe_oracle_preference(int n_races, const int32_t *race_off, int F, const float *factors, const float *prefs,
                           const float *weights, float *P)
{
    for (int r = 0; r < n_races; ++r) {
        for (int c = race_off[r]; c < race_off[r + 1]; ++c) {
            float p = 1.0f;
            for (int i = 0; i < F; ++i) {
                float m = fabsf(factors[r * F + i] - prefs[c * F + i]);
                if (m > 1.0f) m = 1.0f;
                p = p * (1.0f - weights[i] * m);
            }
            P[c] = p;
        }
    }
}

/* Frequentist win probabilities and decimal odds (Section 2: decimal odds are the
 * total returned per unit stake, so odds = 1/p): p_c = count_c / R. */
void bbe_oracle_win_probs(int n, const int32_t *counts, int64_t R, float *probs, float *odds)
{
    float Rf = (float)R;
    for (int c = 0; c < n; ++c) {
        float p = (float)counts[c] / Rf;
        probs[c] = p;
        if (odds) odds[c] = 1.0f / p;
    }
}

/* ------------------------------------------------------ batch helpers for the tests */

void bbe_oracle_log_batch(const float *x, float *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = bbe_oracle_log(x[i]);
}

void bbe_oracle_sincos2pi_batch(const uint32_t *m24, float *s, float *c, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) bbe_oracle_sincos2pi(m24[i], &s[i], &c[i]);
}

void bbe_oracle_z_batch(int dist, uint64_t seed, uint32_t r, uint32_t k0, int64_t nk,
                        uint32_t nt, uint32_t c, float *z)
{
    for (int64_t kk = 0; kk < nk; ++kk)
        for (uint32_t t = 0; t < nt; ++t)
            z[kk * nt + t] = bbe_oracle_z(dist, seed, r, k0 + (uint32_t)kk, t, c);
}
