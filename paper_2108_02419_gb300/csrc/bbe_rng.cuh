// bbe_rng.cuh -- device-side random step generator delta(v_c) of Eq. 1.
//
// Counter-based Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) keyed by the 64-bit
// seed, counter (k, t >> 2, c, r); four 32-bit words serve four consecutive steps of
// one competitor in one rollout.  The normal variate uses the Box-Muller transform
// (Box & Muller, 1958) on the word pair (t >> 1) & 1; its log and sin/cos(2 pi u) are
// evaluated with fixed, fully specified binary32 operation sequences (every add, multiply,
// fused multiply-add, divide and square root is an explicit round-to-nearest intrinsic),
// so the results do not depend on compiler contraction or on the CUDA math library:
//
//   log x:  x = 2^e m, m in (sqrt(1/2), sqrt(2)], f = m - 1 (exact),
//           log m = f g(f), g a degree-9 fit of log(1 + f) / f on [sqrt(1/2) - 1, sqrt(2) - 1]
//           (Lawson's minimax iteration of least squares on 512 Chebyshev nodes, 50 rounds,
//           constant term 1, coefficients rounded to binary32) [Horner, fma],
//           log x = e ln2_hi + (e ln2_lo + log m).
//   sqrt:   correctly rounded (see sqrt_f32x2).
//   sincos: u = m24 2^-24, q = round(4u) by integer arithmetic, f = u - q/4 exactly,
//           Taylor series of sin(2 pi f) to degree 9 and cos(2 pi f) to degree 10 in f
//           [Horner, fma], then the quadrant rotation by q mod 4.
#pragma once
#include <cstdint>

namespace bbe {

constexpr float kKappa = 0x1.99999ap-3f;   // 0.2f: responsiveness amplitude
constexpr float kStepFloor = 0x1.0624dep-10f;  // 1e-3f: S_c > 0 at all times

struct Words4 {
    uint32_t w0, w1, w2, w3;
};

// Philox4x32-10 with the round keys given: rk[2i], rk[2i+1] are the key words of round i.
// With rk in the kernel's parameter block every round is the high and low halves of two
// 32x32-bit products (taken as two separate multiplies each, which issue faster on sm_103a than
// one 64-bit product) and two three-input XORs with constant-bank operands.
__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                const uint32_t (&rk)[20])
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        c0 = hi1 ^ c1 ^ rk[2 * i];
        c2 = hi0 ^ c3 ^ rk[2 * i + 1];
        c1 = lo1;
        c3 = lo0;
    }
    return Words4{c0, c1, c2, c3};
}

// The float arithmetic below works on two values at once (__ffma2_rn, __fadd2_rn, __fmul2_rn:
// one instruction for both, each component rounded exactly as __fmaf_rn, __fadd_rn and
// __fmul_rn round it), because a Philox block always feeds two Box-Muller pairs.
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

// Natural log of two positive normal floats (the Box-Muller radius only needs (0, 1]).
__device__ __forceinline__ float2 log_f32x2(float2 x)
{
    uint32_t ba = __float_as_uint(x.x), bb = __float_as_uint(x.y);
    int ea = int(ba >> 23) - 127, eb = int(bb >> 23) - 127;
    uint32_t ma = (ba & 0x007FFFFFu) | 0x3F800000u, mb = (bb & 0x007FFFFFu) | 0x3F800000u;
    const bool ha = ma > 0x3FB504F3u, hb = mb > 0x3FB504F3u;
    ma = ha ? ma - 0x00800000u : ma;
    mb = hb ? mb - 0x00800000u : mb;
    ea = ha ? ea + 1 : ea;
    eb = hb ? eb + 1 : eb;
    const float2 f = __fadd2_rn(make_float2(__uint_as_float(ma), __uint_as_float(mb)), splat2(-1.0f));
    float2 g = __ffma2_rn(f, splat2(-0x1.383dfep-4f), splat2(0x1.084e42p-3f));
    g = __ffma2_rn(f, g, splat2(-0x1.0f3768p-3f));
    g = __ffma2_rn(f, g, splat2(0x1.227092p-3f));
    g = __ffma2_rn(f, g, splat2(-0x1.542748p-3f));
    g = __ffma2_rn(f, g, splat2(0x1.99a402p-3f));
    g = __ffma2_rn(f, g, splat2(-0x1.000428p-2f));
    g = __ffma2_rn(f, g, splat2(0x1.555550p-2f));
    g = __ffma2_rn(f, g, splat2(-0x1.fffff8p-2f));
    g = __ffma2_rn(f, g, splat2(1.0f));
    const float2 logm = __fmul2_rn(f, g);
    const float2 ef = make_float2(__int2float_rn(ea), __int2float_rn(eb));
    return __ffma2_rn(ef, splat2(0x1.62e4p-1f), __ffma2_rn(ef, splat2(0x1.7f7d1cp-20f), logm));
}

// sin and cos of 2 pi m / 2^24 for m = wa >> 8 and m = wb >> 8.  With q = round(m / 2^22)
// (halves up) the remainder m - q 2^22 in [-2^21, 2^21) is the low 22 bits of m sign-extended,
// (int)(w << 2) >> 10, and q mod 4 is the top two bits of u = w + 2^29: bit 30 says whether
// sin and cos trade places, bit 31 whether sin changes sign, and bit 31 of u + 2^30 whether
// cos does (the sign flips are XORs of the sign bit, exactly the negations).
__device__ __forceinline__ void sincos2pi_words(uint32_t wa, uint32_t wb, float2 &s_out, float2 &c_out)
{
    const int32_t fa = int32_t(wa << 2) >> 10, fb = int32_t(wb << 2) >> 10;
    const float2 f = __fmul2_rn(make_float2(__int2float_rn(fa), __int2float_rn(fb)), splat2(0x1p-24f));
    const float2 y = __fmul2_rn(f, f);
    float2 ps = __ffma2_rn(y, splat2(0x1.507834p+5f), splat2(-0x1.32d2ccp+6f));
    ps = __ffma2_rn(y, ps, splat2(0x1.466bc6p+6f));
    ps = __ffma2_rn(y, ps, splat2(-0x1.4abbcep+5f));
    ps = __ffma2_rn(y, ps, splat2(0x1.921fb6p+2f));
    const float2 sv = __fmul2_rn(f, ps);
    float2 pc = __ffma2_rn(y, splat2(-0x1.a6d1f2p+4f), splat2(0x1.e1f506p+5f));
    pc = __ffma2_rn(y, pc, splat2(-0x1.55d3c8p+6f));
    pc = __ffma2_rn(y, pc, splat2(0x1.03c1f0p+6f));
    pc = __ffma2_rn(y, pc, splat2(-0x1.3bd3ccp+4f));
    const float2 cv = __ffma2_rn(y, pc, splat2(1.0f));
    // rotate (sin, cos) of the remainder by q quarter turns
    const uint32_t ua = wa + 0x20000000u, ub = wb + 0x20000000u;
    const bool oa = (ua & 0x40000000u) != 0u, ob = (ub & 0x40000000u) != 0u;
    const float aa = oa ? cv.x : sv.x, ab = ob ? cv.y : sv.y;
    const float ca = oa ? sv.x : cv.x, cb = ob ? sv.y : cv.y;
    s_out = make_float2(__uint_as_float(__float_as_uint(aa) ^ (ua & 0x80000000u)),
                        __uint_as_float(__float_as_uint(ab) ^ (ub & 0x80000000u)));
    c_out = make_float2(__uint_as_float(__float_as_uint(ca) ^ ((ua + 0x40000000u) & 0x80000000u)),
                        __uint_as_float(__float_as_uint(cb) ^ ((ub + 0x40000000u) & 0x80000000u)));
}

// Correctly rounded square roots of x.x and x.y, each -0 or a positive normal float (the
// Box-Muller radius: -2 log u1 is -0 for u1 = 1, else in [1.19e-7, 33.3]).  Markstein's
// sequence (P. Markstein, "IA-64 and Elementary Functions", 2000): from the hardware estimate
// y ~ 1/sqrt(x) (rsqrtf), g = x y and h = y / 2; one coupled Newton step with the residual
// e = 1/2 - g h refines both (g' = g + g e ~ sqrt x, h' = h + h e ~ 1 / (2 sqrt x), relative
// errors of order 2^-44); the exact residual d = x - g'^2 (an FMA) then gives g' + d h',
// rounded once, which is the correctly rounded square root.  A GPU test compares all 2^24
// radii the generator can produce with the IEEE square root and with the CPU oracle's.
__device__ __forceinline__ float2 sqrt_f32x2(float2 x)
{
    // x = -0: the estimate of the least normal keeps g = -0 * 2^63 = -0, and sqrt(-0) = -0
    const float2 y = make_float2(rsqrtf(fmaxf(x.x, 0x1p-126f)), rsqrtf(fmaxf(x.y, 0x1p-126f)));
    const float2 g = __fmul2_rn(x, y);
    const float2 h = __fmul2_rn(y, splat2(0.5f));
    const float2 e = __ffma2_rn(make_float2(-g.x, -g.y), h, splat2(0.5f));
    const float2 g1 = __ffma2_rn(g, e, g);
    const float2 h1 = __ffma2_rn(h, e, h);
    const float2 d = __ffma2_rn(make_float2(-g1.x, -g1.y), g1, x);
    return __ffma2_rn(d, h1, g1);
}

// The Box-Muller radii sqrt(-2 log u1) of the two pairs of a Philox block, u1 = ((wa >> 8) + 1)
// 2^-24 in (0, 1] for wa = w0 and w2.
// (w & ~0xff) has at most 24 significant bits, so its conversion is exact, and
// (w & ~0xff) 2^-32 + 2^-24 = ((w >> 8) + 1) 2^-24 is exact in one FMA.
__device__ __forceinline__ float2 bm_radius2(uint32_t wa, uint32_t wb)
{
    const float2 u1 = __ffma2_rn(make_float2(__uint2float_rn(wa & 0xFFFFFF00u), __uint2float_rn(wb & 0xFFFFFF00u)),
                                 splat2(0x1p-32f), splat2(0x1p-24f));
    return sqrt_f32x2(__fmul2_rn(splat2(-2.0f), log_f32x2(u1)));
}

// The two Box-Muller pairs of one Philox block: (z0, z1) = r (cos, sin) of (w0, w1) and
// (z2, z3) of (w2, w3), with r = sqrt(-2 log u1), u1 = ((wa >> 8) + 1) 2^-24 in (0, 1] and
// angle 2 pi (wb >> 8) 2^-24.
__device__ __forceinline__ void box_muller2(const Words4 &wd, float &z0, float &z1, float &z2, float &z3)
{
    const float2 radius = bm_radius2(wd.w0, wd.w2);
    float2 sv, cv;
    sincos2pi_words(wd.w1, wd.w3, sv, cv);
    const float2 zc = __fmul2_rn(radius, cv);
    const float2 zs = __fmul2_rn(radius, sv);
    z0 = zc.x;
    z1 = zs.x;
    z2 = zc.y;
    z3 = zs.y;
}

__device__ __forceinline__ float uniform_z(uint32_t w)
{
    const float u = __fmul_rn(__uint2float_rn(w >> 8), 0x1p-24f);
    return __fmul_rn(0x1.bb67aep+0f, __fsub_rn(__fmul_rn(2.0f, u), 1.0f));
}

__device__ __forceinline__ float two_point_z(uint32_t w) { return (w >> 31) ? 1.0f : -1.0f; }

}  // namespace bbe
