/*
 * bbe_oracle.h -- declarations of the CPU oracle (test infrastructure only; see
 * bbe_oracle.c).  Independent of the CUDA library's header.
 */
#ifndef BBE_ORACLE_H
#define BBE_ORACLE_H

#include <stdint.h>

#define BBE_ORACLE_DIST_NORMAL 0
#define BBE_ORACLE_DIST_UNIFORM 1
#define BBE_ORACLE_DIST_TWO_POINT 2

#define BBE_ORACLE_KAPPA 0x1.99999ap-3f   /* 0.2f */
#define BBE_ORACLE_S_FLOOR 0x1.0624dep-10f /* 1e-3f */
#define BBE_ORACLE_STEP_LIMIT (-5)
#define BBE_ORACLE_LAW_POSITION 0
#define BBE_ORACLE_LAW_TIME 1

/* One race of Section 3: n competitors on a track of length L; per competitor the
 * position d0, the step distribution's mean mu and spread sigma, responsiveness rho,
 * preference coefficient P, blocking threshold theta and (nullable) previous step. */
typedef struct {
    int n;
    float L;
    const float *d0;
    const float *mu;
    const float *sigma;
    const float *rho;
    const float *P;
    const float *theta;
    const float *prev0; /* nullable: mu * P */
    int dist;
    int law;            /* responsiveness law: BBE_ORACLE_LAW_POSITION or BBE_ORACLE_LAW_TIME */
    float t0;           /* time law: steps elapsed before the state (a mid-race snapshot) */
    float T;            /* time law: the race's expected duration in steps, > 0 */
} bbe_oracle_race;

void bbe_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
float bbe_oracle_log(float x);
void bbe_oracle_sincos2pi(uint32_t m24, float *sin_out, float *cos_out);
float bbe_oracle_z(int dist, uint64_t seed, uint32_t r, uint32_t k, uint32_t t, uint32_t c);
int bbe_oracle_rollout(const bbe_oracle_race *race, uint64_t seed, uint32_t r, uint32_t k,
                       int64_t max_steps, int64_t *steps, float *traj, int64_t traj_cap);
int bbe_oracle_race_counts(const bbe_oracle_race *race, uint64_t seed, uint32_t r,
                           int64_t k_begin, int64_t R, int64_t max_steps,
                           int32_t *counts, int64_t *steps_total);
int bbe_oracle_rollout_order(const bbe_oracle_race *race, uint64_t seed, uint32_t r, uint32_t k,
                             int places, int64_t max_steps, int64_t *steps, int32_t *order);
int bbe_oracle_race_places(const bbe_oracle_race *race, uint64_t seed, uint32_t r,
                           int64_t k_begin, int64_t R, int places, int64_t max_steps,
                           int32_t *counts, int64_t *steps_total);
int bbe_oracle_race_orders(const bbe_oracle_race *race, uint64_t seed, uint32_t r,
                           int64_t k_begin, int64_t R, int places, int64_t max_steps,
                           int32_t *counts, int64_t *steps_total);
int bbe_oracle_race_order_list(const bbe_oracle_race *race, uint64_t seed, uint32_t r, int64_t k_begin, int64_t R,
                               int places, int64_t max_steps, int32_t *orders, int64_t *steps_total);
int bbe_oracle_trajectory(const bbe_oracle_race *race, uint64_t seed, uint32_t r, uint32_t k, int64_t max_steps,
                          int64_t *steps, float *d_traj, float *s_traj, int64_t cap);
void bbe_oracle_preference(int n_races, const int32_t *race_off, int F, const float *factors, const float *prefs,
                           const float *weights, float *P);
void bbe_oracle_win_probs(int n, const int32_t *counts, int64_t R, float *probs, float *odds);
void bbe_oracle_log_batch(const float *x, float *y, int64_t n);
void bbe_oracle_sincos2pi_batch(const uint32_t *m24, float *s, float *c, int64_t n);
void bbe_oracle_z_batch(int dist, uint64_t seed, uint32_t r, uint32_t k0, int64_t nk,
                        uint32_t nt, uint32_t c, float *z);

#endif
