// bbe_lane.cuh -- one step of Eq. 1 in the one-competitor-per-lane layout (the trajectory
// kernel: one rollout per race, so the rollout kernel's rank tables and packed segments do not
// pay).
//
// A race of n competitors occupies a segment of n lanes (lane segbase + c holds competitor c
// for the whole rollout).  i+ (the nearest competitor strictly in front, lowest index among
// equal positions) is found by a scan of the segment; the four normals of the current Philox
// block (counter (k, t >> 2, c, race id)) are kept in the lane's registers.  The arithmetic
// is the rollout kernel's, operation for operation: binary32 round-to-nearest intrinsics, and
// the including translation unit is compiled with --fmad=false.
#pragma once

#include "bbe_internal.h"
#include "bbe_rng.cuh"

namespace bbe {

// per-lane constants of a competitor
struct LaneComp {
    float mu, sigma, P, theta, kr;
};

template <int DIST>
__device__ __forceinline__ void lane_draw_block(float (&zc)[4], int c, int t, uint32_t k, uint32_t rid,
                                                const uint32_t (&rk)[20])
{
    const Words4 wd = philox4x32_10(k, uint32_t(t) >> 2, uint32_t(c), rid, rk);
    if (DIST == BBE_DIST_NORMAL) {
        box_muller2(wd, zc[0], zc[1], zc[2], zc[3]);
    } else if (DIST == BBE_DIST_UNIFORM) {
        zc[0] = uniform_z(wd.w0);
        zc[1] = uniform_z(wd.w1);
        zc[2] = uniform_z(wd.w2);
        zc[3] = uniform_z(wd.w3);
    } else {
        zc[0] = two_point_z(wd.w0);
        zc[1] = two_point_z(wd.w1);
        zc[2] = two_point_z(wd.w2);
        zc[3] = two_point_z(wd.w3);
    }
}

// S_c(t) of Eq. 1 (with the floor) for the competitor of this lane at position d with previous
// step prev.  Called by all 32 lanes of the warp; lanes outside a segment pass lane_used false.
template <int DIST>
__device__ __forceinline__ float lane_step(float d, float prev, const LaneComp &cp, int n, int segbase,
                                           bool lane_used, bool running, int c, int t, uint32_t k, uint32_t rid,
                                           float invL, float (&zc)[4], const uint32_t (&rk)[20], int law = BBE_LAW_POSITION,
                                           float t0 = 0.0f, float invT = 0.0f)
{
    const int lane = threadIdx.x & 31;
    float fd = INFINITY, fp = 0.0f;
    bool hf = false;
    for (int j = 0; j < n; ++j) {
        const int src = lane_used ? segbase + j : lane;
        const float dj = __shfl_sync(0xffffffffu, d, src);
        const float pj = __shfl_sync(0xffffffffu, prev, src);
        if (dj > d && dj < fd) {
            fd = dj;
            fp = pj;
            hf = true;
        }
    }
    if (running && (t & 3) == 0) lane_draw_block<DIST>(zc, c, t, k, rid, rk);
    const int ph = t & 3;
    const float z = ph == 0 ? zc[0] : (ph == 1 ? zc[1] : (ph == 2 ? zc[2] : zc[3]));
    const float Rc = law == BBE_LAW_TIME ? responsiveness<BBE_LAW_TIME>(cp.kr, d, invL, t0, t, invT)
                                         : responsiveness<BBE_LAW_POSITION>(cp.kr, d, invL, t0, t, invT);
    const bool blocked = hf && !(__fsub_rn(fd, d) > cp.theta);
    const float S = blocked ? __fmul_rn(Rc, fminf(prev, fp)) : __fmul_rn(__fmul_rn(Rc, cp.P), __fmaf_rn(cp.sigma, z, cp.mu));
    return fmaxf(S, kStepFloor);
}

}  // namespace bbe
