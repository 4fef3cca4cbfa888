// Helpers shared by the node generators (jittered grid, disk boundary,
// Poisson-disc placement): the counter-based SplitMix64 draw and sin/cos
// evaluated the same way wherever a node position depends on an angle, so
// positions are reproducible bit for bit.
#pragma once

#include <stdint.h>

namespace rbffd {

// SplitMix64 (Steele, Lea & Flood 2014): the c-th output of the generator
// seeded with `seed`, i.e. the finaliser applied to seed + (c+1)*golden.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// top 53 bits of the draw as a double in [0, 1)
__device__ __forceinline__ double unit_draw(uint64_t seed, uint64_t c) {
    return __dmul_rn((double)(splitmix64_at(seed, c) >> 11), 1.0 / 9007199254740992.0);
}

// sin and cos on [0, pi/2]: Taylor series through x^21 / x^20 in Horner
// form, every operation separately rounded (truncation below 2e-17)
__device__ __forceinline__ void series_sincos(double x, double* s, double* c) {
    double x2 = __dmul_rn(x, x);
    double ps = 1.0, pc = 1.0;
    for (int k = 10; k >= 1; --k) {
        double den_s = (double)((2 * k) * (2 * k + 1));
        double den_c = (double)((2 * k - 1) * (2 * k));
        ps = __dsub_rn(1.0, __dmul_rn(__ddiv_rn(x2, den_s), ps));
        pc = __dsub_rn(1.0, __dmul_rn(__ddiv_rn(x2, den_c), pc));
    }
    *s = __dmul_rn(x, ps);
    *c = pc;
}

// unit vector at angle a in [0, 2 pi): reduced to a quadrant and an offset
__device__ __forceinline__ void unit_dir(double a, double* ux, double* uy) {
    const double half_pi = 1.5707963267948966;
    int q = (int)__ddiv_rn(a, half_pi);
    if (q > 3) q = 3;
    double r = __dsub_rn(a, __dmul_rn((double)q, half_pi));
    if (r < 0.0) r = 0.0;
    double s, c;
    series_sincos(r, &s, &c);
    switch (q) {
        case 0: *ux = c; *uy = s; break;
        case 1: *ux = -s; *uy = c; break;
        case 2: *ux = -c; *uy = -s; break;
        default: *ux = s; *uy = -c; break;
    }
}

}  // namespace rbffd
