// Correctly rounded FP64 reciprocal, quotient and square root computed on the
// integer pipes.
//
// On this GPU the FP64 pipe retires 2 fused multiply-adds per clock per SM
// (measured), a sixty-fourth of the FP32 rate, while the integer pipes sit
// mostly idle in the kernels that need these operations (the weight build's
// pivots, back substitution and r^3 assembly).  The library's FP64 reciprocal,
// divide and square root run their refinement steps on the FP64 pipe; the
// routines here produce the same correctly rounded results from integer
// arithmetic on the 53-bit significands instead, leaving the FP64 pipe to the
// elimination's multiply-adds.
//
// Method (fixed-point Newton-Raphson with an exact remainder test; see e.g.
// J.-M. Muller et al., Handbook of Floating-Point Arithmetic, ch. on division
// and square root, and T. Granlund, P. Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994, for the reciprocal-based
// quotient): a 64-bit fixed-point estimate of 1/m (or 1/sqrt(m)) is seeded by
// the FP32 approximation unit and refined by two Newton steps in 64 x 64-bit
// integer products to within a few units of 2^-64 relative; it gives a
// candidate integer quotient (root) within one of the truncated exact value;
// the exact remainder, computed modulo 2^64 (it is known to be far below
// 2^63 in magnitude), corrects the candidate to the truncated value and
// decides the rounding to nearest.  A quotient of two 53-bit significands, or
// the square root of a 105/106-bit integer, is never exactly halfway between
// two representable values, so no tie-breaking is needed.
//
// Inputs outside the fast paths (zeros where noted, subnormals, infinities,
// NaN, results that would leave the normal range) go to the library routine,
// so every result equals the library's correctly rounded one (tested bit for
// bit on seeded operands, tests/test_gpu_intfp64.py).
#pragma once

#include <stdint.h>

namespace rbffd {

static constexpr uint64_t IF_SIGN = 0x8000000000000000ull;
static constexpr uint64_t IF_FRAC = 0x000fffffffffffffull;
static constexpr uint64_t IF_HIDDEN = 0x0010000000000000ull;   // 2^52

__device__ __forceinline__ uint64_t if_bits(double x) {
    return (uint64_t)__double_as_longlong(x);
}
__device__ __forceinline__ double if_double(uint64_t b) {
    return __longlong_as_double((long long)b);
}

// Y ~ 2^116 / m for a significand 2^52 < m < 2^53 (so 2^63 < Y < 2^64),
// within a few units.  Seed: the FP32 approximate reciprocal of the top 23
// fraction bits (relative error below 2^-21); each Newton step
// Y <- Y + Y (2^127 - X Y) / 2^127, X = m 2^11, squares the error.
__device__ __forceinline__ uint64_t if_rcp_fix(uint64_t m) {
    const float xf = __uint_as_float(0x3f800000u | (uint32_t)((m >> 29) & 0x7fffffu));
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(xf));
    const uint32_t rb = __float_as_uint(r);
    uint64_t Y = rb >= 0x3f800000u ? ~0ull : (uint64_t)((rb & 0x7fffffu) | 0x800000u) << 40;
    const uint64_t X = m << 11;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const uint64_t ph = __umul64hi(X, Y), pl = X * Y;
        // floor((2^127 - X Y) / 2^64), a small signed number
        const int64_t dh = (int64_t)((1ull << 63) - ph) - (int64_t)(pl != 0);
        if (dh >= 0) Y += __umul64hi(Y, (uint64_t)dh) << 1;
        else Y -= __umul64hi(Y, (uint64_t)(-dh)) << 1;
    }
    return Y;
}

// RN(1/p).  Also returns the fixed-point reciprocal Yp of p's significand for
// if_div (0 when the significand is a power of two, whose quotients are exact
// exponent shifts).  The library reciprocal for zero, subnormal, huge,
// infinite or NaN p.
__device__ __forceinline__ double if_rcp(double p, uint64_t* Yp) {
    const uint64_t b = if_bits(p);
    const int ep = (int)((b >> 52) & 0x7ff);
    const uint64_t frac = b & IF_FRAC;
    *Yp = 0;
    if (ep == 0 || ep >= 2045) {
        const double r = __drcp_rn(p);
        if (ep != 0 && ep < 2047 && frac != 0) *Yp = if_rcp_fix(frac | IF_HIDDEN);
        return r;
    }
    const uint64_t sign = b & IF_SIGN;
    if (frac == 0) return if_double(sign | (uint64_t)(2046 - ep) << 52);
    const uint64_t m = frac | IF_HIDDEN;
    const uint64_t Y = if_rcp_fix(m);
    *Yp = Y;
    // q = RN(2^105 / m), 2^52 < q < 2^53; remainder 2^105 - q m modulo 2^64
    uint64_t q = Y >> 11;
    int64_t R = (int64_t)(0ull - q * m);
    if (R < 0) { --q; R += (int64_t)m; }
    if (R < 0) { --q; R += (int64_t)m; }
    if (R >= (int64_t)m) { ++q; R -= (int64_t)m; }
    if (R >= (int64_t)m) { ++q; R -= (int64_t)m; }
    q += (uint64_t)(2 * R > (int64_t)m);
    return if_double(sign | (uint64_t)(2045 - ep) << 52 | (q - IF_HIDDEN));
}

// RN(b / p) given Yp from if_rcp(p).  The library quotient for subnormal,
// infinite or NaN operands and for results outside the normal range.
__device__ __forceinline__ double if_div(double bv, double p, uint64_t Yp) {
    const uint64_t bb = if_bits(bv), pb = if_bits(p);
    const int eb = (int)((bb >> 52) & 0x7ff), ep = (int)((pb >> 52) & 0x7ff);
    const uint64_t sign = (bb ^ pb) & IF_SIGN;
    if (ep == 0 || ep == 2047 || eb == 2047) return __ddiv_rn(bv, p);
    if (eb == 0) {
        if ((bb & ~IF_SIGN) == 0) return if_double(sign);   // +-0 / p
        return __ddiv_rn(bv, p);
    }
    const uint64_t mb = (bb & IF_FRAC) | IF_HIDDEN;
    const uint64_t pf = pb & IF_FRAC;
    if (pf == 0) {   // p a power of two: an exact exponent shift
        const int E = eb - ep + 1023;
        if (E < 1 || E > 2046) return __ddiv_rn(bv, p);
        return if_double(sign | (uint64_t)E << 52 | (mb - IF_HIDDEN));
    }
    if (Yp == 0) return __ddiv_rn(bv, p);
    const uint64_t mp = pf | IF_HIDDEN;
    // q = RN(mb 2^t / mp) with t = 52 (mb >= mp) or 53, so 2^52 <= q < 2^53
    const int t = mb >= mp ? 52 : 53;
    int E = eb - ep + 1023 - (t - 52);
    if (E < 1 || E > 2046) return __ddiv_rn(bv, p);
    const uint64_t H = __umul64hi(mb << 11, Yp);   // ~ (mb / mp) 2^63
    uint64_t q = H >> (63 - t);
    int64_t R = (int64_t)((mb << t) - q * mp);     // exact: |R| < 2^56
    if (R < 0) { --q; R += (int64_t)mp; }
    if (R < 0) { --q; R += (int64_t)mp; }
    if (R >= (int64_t)mp) { ++q; R -= (int64_t)mp; }
    if (R >= (int64_t)mp) { ++q; R -= (int64_t)mp; }
    q += (uint64_t)(2 * R > (int64_t)mp);
    if (q == (IF_HIDDEN << 1)) {   // rounded up to 2^53
        q = IF_HIDDEN;
        if (++E > 2046) return __ddiv_rn(bv, p);
    }
    return if_double(sign | (uint64_t)E << 52 | (q - IF_HIDDEN));
}

// RN(sqrt(x)).  The library square root for negative, subnormal, infinite or
// NaN x; +-0 returns itself.
__device__ __forceinline__ double if_sqrt(double x) {
    const uint64_t b = if_bits(x);
    if ((b & ~IF_SIGN) == 0) return x;
    const int e = (int)((b >> 52) & 0x7ff);
    if ((b & IF_SIGN) || e == 0 || e == 2047) return __dsqrt_rn(x);
    const uint64_t frac = b & IF_FRAC;
    const int k = e - 1075;              // x = m 2^k
    const int odd = k & 1;
    const uint64_t E = (uint64_t)((k >> 1) + 1049);
    if (frac == 0 && !odd) return if_double(E << 52);   // an even power of two
    // M = m 2^(52 + odd) (105 or 106 bits), sqrt(M) in [2^52, 2^53)
    const uint64_t m = frac | IF_HIDDEN;
    const uint64_t Z = m << (10 + odd);  // M / 2^42: z = Z / 2^62 in [1, 4)
    float r;
    const float zf = __ull2float_rz(Z) * 2.168404344971009e-19f;   // x 2^-62
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(zf));
    const uint32_t rb = __float_as_uint(r);
    // Y ~ 2^64 / sqrt(z), refined by Y <- Y + Y (2^62 - z Y^2 2^-66) / 2^63
    uint64_t Y = rb >= 0x3f800000u ? ~0ull : (uint64_t)((rb & 0x7fffffu) | 0x800000u) << 40;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const uint64_t T = __umul64hi(Y, Y);   // ~ 2^64 / z
        const uint64_t U = __umul64hi(T, Z);   // ~ 2^62
        const int64_t d = (int64_t)((1ull << 62) - U);
        if (d >= 0) Y += __umul64hi(Y, (uint64_t)d) << 1;
        else Y -= __umul64hi(Y, (uint64_t)(-d)) << 1;
    }
    uint64_t q = __umul64hi(Z, Y) >> 10;        // ~ sqrt(M)
    const uint64_t Mlo = m << (52 + odd);       // M modulo 2^64
    int64_t R = (int64_t)(Mlo - q * q);         // exact: |R| < 2^56
    if (R < 0) { R += (int64_t)(2 * q - 1); --q; }
    if (R < 0) { R += (int64_t)(2 * q - 1); --q; }
    if (R >= (int64_t)(2 * q + 1)) { R -= (int64_t)(2 * q + 1); ++q; }
    if (R >= (int64_t)(2 * q + 1)) { R -= (int64_t)(2 * q + 1); ++q; }
    q += (uint64_t)(R > (int64_t)q);            // sqrt(M) > q + 1/2
    return if_double(E << 52 | (q - IF_HIDDEN));
}

}  // namespace rbffd
