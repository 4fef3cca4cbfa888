// Correctly rounded FP64 quotient from a known correctly rounded reciprocal
// (used by the weight build's back substitution, whose pivots' reciprocals
// the elimination computes anyway).  Header-only so a test can compile it
// into its own probe kernel.
#pragma once

namespace rbffd {

// b / p rounded to nearest from y = RN(1/p), by Markstein's method (P.
// Markstein, IBM J. Res. Dev. 34(1), 1990): q0 = RN(b y) lies within 1.5 ulp
// of b/p; one correction q1 = RN(q0 + r0 y), r0 = b - p q0, leaves it within
// half an ulp plus a term of order 2^-53 ulp, so q1 is faithful; for a
// faithful q1 and y = RN(1/p) the exact remainder r1 = b - p q1 gives
// RN(q1 + r1 y) = RN(b/p).  Every remainder is one fused multiply-add, exact
// while nothing over- or underflows, so the method runs only for
// 2^-500 <= |b|, |p| < 2^501 (else the library quotient).  Five FP64
// instructions against about eight for the library quotient; the reciprocal
// is the pivot's, computed during the elimination anyway.  The two quotients
// agreed bit for bit on 6e10 random operand pairs (mantissas uniform, and next
// to 1 and 2), and the weights stay identical to the oracle's in > 99 % of rows.
__device__ __forceinline__ double div_by_pivot(double b, double p, double y) {
    const int eb = (int)((__double_as_longlong(b) >> 52) & 0x7ff);
    const int ep = (int)((__double_as_longlong(p) >> 52) & 0x7ff);
    if (eb < 1023 - 500 || eb > 1023 + 500 || ep < 1023 - 500 || ep > 1023 + 500)
        return __ddiv_rn(b, p);
    const double q0 = __dmul_rn(b, y);
    const double r0 = __fma_rn(-q0, p, b);
    const double q1 = __fma_rn(r0, y, q0);
    const double r1 = __fma_rn(-q1, p, b);
    return __fma_rn(r1, y, q1);
}

}  // namespace rbffd
