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
//           (least squares on Chebyshev nodes reweighted towards the minimax relative
//           error) [Horner, fma], log x = e ln2_hi + (e ln2_lo + log m).
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
// With rk in the kernel's parameter block every round is two 32x32->64 multiplies and two
// three-input XORs with constant-bank operands.
__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                const uint32_t (&rk)[20])
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint64_t p0 = uint64_t(0xD2511F53u) * c0;
        const uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
        const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
        const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
        c0 = hi1 ^ c1 ^ rk[2 * i];
        c2 = hi0 ^ c3 ^ rk[2 * i + 1];
        c1 = lo1;
        c3 = lo0;
    }
    return Words4{c0, c1, c2, c3};
}

// Natural log of a positive normal float (the Box-Muller radius only needs (0, 1]).
__device__ __forceinline__ float log_f32(float x)
{
    uint32_t b = __float_as_uint(x);
    int e = int(b >> 23) - 127;
    uint32_t mb = (b & 0x007FFFFFu) | 0x3F800000u;
    const bool halve = mb > 0x3FB504F3u;
    mb = halve ? mb - 0x00800000u : mb;
    e = halve ? e + 1 : e;
    const float f = __fsub_rn(__uint_as_float(mb), 1.0f);
    float g = __fmaf_rn(f, -0x1.36ee94p-4f, 0x1.07eecap-3f);
    g = __fmaf_rn(f, g, -0x1.0f4ebcp-3f);
    g = __fmaf_rn(f, g, 0x1.228226p-3f);
    g = __fmaf_rn(f, g, -0x1.542678p-3f);
    g = __fmaf_rn(f, g, 0x1.99a2f8p-3f);
    g = __fmaf_rn(f, g, -0x1.000428p-2f);
    g = __fmaf_rn(f, g, 0x1.555552p-2f);
    g = __fmaf_rn(f, g, -0x1.fffff8p-2f);
    g = __fmaf_rn(f, g, 1.0f);
    const float logm = __fmul_rn(f, g);
    const float ef = __int2float_rn(e);
    return __fmaf_rn(ef, 0x1.62e4p-1f, __fmaf_rn(ef, 0x1.7f7d1cp-20f, logm));
}

// sin and cos of 2 pi m24 / 2^24.
__device__ __forceinline__ void sincos2pi_f32(uint32_t m24, float &s_out, float &c_out)
{
    const uint32_t q = (m24 + 0x200000u) >> 22;
    const int32_t fm = int32_t(m24) - int32_t(q << 22);
    const float f = __fmul_rn(__int2float_rn(fm), 0x1p-24f);
    const float y = __fmul_rn(f, f);
    float ps = __fmaf_rn(y, 0x1.507834p+5f, -0x1.32d2ccp+6f);
    ps = __fmaf_rn(y, ps, 0x1.466bc6p+6f);
    ps = __fmaf_rn(y, ps, -0x1.4abbcep+5f);
    ps = __fmaf_rn(y, ps, 0x1.921fb6p+2f);
    const float sv = __fmul_rn(f, ps);
    float pc = __fmaf_rn(y, -0x1.a6d1f2p+4f, 0x1.e1f506p+5f);
    pc = __fmaf_rn(y, pc, -0x1.55d3c8p+6f);
    pc = __fmaf_rn(y, pc, 0x1.03c1f0p+6f);
    pc = __fmaf_rn(y, pc, -0x1.3bd3ccp+4f);
    const float cv = __fmaf_rn(y, pc, 1.0f);
    const uint32_t quad = q & 3u;
    // rotate (sin, cos) of the remainder by q quarter turns
    const float a = (quad & 1u) ? cv : sv;   // |sin| of the result
    const float b = (quad & 1u) ? sv : cv;   // |cos| of the result
    s_out = (quad >= 2u) ? -a : a;
    c_out = (quad == 1u || quad == 2u) ? -b : b;
}

// Box-Muller pair from two Philox words: (r cos, r sin) with r = sqrt(-2 log u1),
// u1 = ((wa >> 8) + 1) 2^-24 in (0, 1], angle 2 pi (wb >> 8) 2^-24.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float &z_cos, float &z_sin)
{
    const float u1 = __fmul_rn(__uint2float_rn((wa >> 8) + 1u), 0x1p-24f);
    const float radius = __fsqrt_rn(__fmul_rn(-2.0f, log_f32(u1)));
    float sv, cv;
    sincos2pi_f32(wb >> 8, sv, cv);
    z_cos = __fmul_rn(radius, cv);
    z_sin = __fmul_rn(radius, sv);
}

__device__ __forceinline__ float uniform_z(uint32_t w)
{
    const float u = __fmul_rn(__uint2float_rn(w >> 8), 0x1p-24f);
    return __fmul_rn(0x1.bb67aep+0f, __fsub_rn(__fmul_rn(2.0f, u), 1.0f));
}

__device__ __forceinline__ float two_point_z(uint32_t w) { return (w >> 31) ? 1.0f : -1.0f; }

}  // namespace bbe
