// Probe for the integer-pipe FP64 routines of the weight build
// (csrc/intfp64.cuh): if_rcp, if_div and if_sqrt against the library's
// correctly rounded reciprocal, quotient and square root, bit for bit, on
// seeded operands.  Operand families: 0 uniform significands, exponents in
// [-60, 60]; 1 significands next to 1 and 2 (the hard cases for rounding);
// 2 exponents in [-1020, 1020] (fallbacks at the ends of the range); 3 powers
// of two, zeros, subnormals and exact squares.  Prints one line per routine
// and family: "<routine> family F operands P mismatches K".
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "intfp64.cuh"

__device__ __forceinline__ uint64_t mix64(uint64_t x) {   // SplitMix64 finaliser
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ double operand(uint64_t r, uint64_t r2, int fam, bool positive) {
    uint64_t mant = r & 0xfffffffffffffull;
    int span = 121;
    if (fam == 1) mant = (r & 1) ? 0xfffffffffffffull - ((r >> 1) & 0xff) : ((r >> 1) & 0xff);
    if (fam == 2) span = 2041;
    int e = (int)((r2 >> 3) % span) - span / 2;
    const uint64_t sign = positive ? 0 : (r2 >> 63) << 63;
    if (fam == 3) {
        switch (r2 & 7) {
            case 0: mant = 0; break;                                           // power of two
            case 1: return __longlong_as_double((long long)sign);              // zero
            case 2: return __longlong_as_double((long long)(sign | (r & 0xfffffffffffffull)));  // subnormal
            case 3: {                                                          // exact square
                const uint64_t q = (1ull << 25) + (r % ((1ull << 26) + (1ull << 25)));
                return (double)(q * q) * (positive ? 1.0 : ((r2 >> 63) ? -1.0 : 1.0));
            }
            default: break;
        }
    }
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 1023) << 52) | mant));
}

__global__ void probe(int which, int fam, int iters, unsigned long long* bad) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nb = 0;
    for (int i = 0; i < iters; ++i) {
        const uint64_t id = ((uint64_t)which << 56) | ((uint64_t)fam << 48) | (t * (uint64_t)iters + i);
        const uint64_t a = mix64(4 * id), a2 = mix64(4 * id + 1);
        const uint64_t c = mix64(4 * id + 2), c2 = mix64(4 * id + 3);
        double got, want;
        if (which == 0) {
            const double p = operand(a, a2, fam, false);
            uint64_t Y;
            got = rbffd::if_rcp(p, &Y);
            want = __drcp_rn(p);
        } else if (which == 1) {
            const double b = operand(c, c2, fam == 1 ? 0 : fam, false);
            const double p = operand(a, a2, fam, false);
            uint64_t Y;
            rbffd::if_rcp(p, &Y);
            got = rbffd::if_div(b, p, Y);
            want = __ddiv_rn(b, p);
        } else {
            const double x = operand(a, a2, fam, true);
            got = rbffd::if_sqrt(x);
            want = __dsqrt_rn(x);
        }
        // NaN results compare as NaN (any payload)
        const bool both_nan = got != got && want != want;
        if (!both_nan && __double_as_longlong(got) != __double_as_longlong(want)) ++nb;
    }
    if (nb) atomicAdd(bad, nb);
}

int main() {
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return 2;
    const int blocks = 152 * 8, threads = 256, iters = 128;
    const char* names[3] = {"rcp", "div", "sqrt"};
    for (int which = 0; which < 3; ++which)
        for (int fam = 0; fam < 4; ++fam) {
            unsigned long long h = 0;
            cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice);
            probe<<<blocks, threads>>>(which, fam, iters, d);
            if (cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
            printf("%s family %d operands %llu mismatches %llu\n", names[which], fam,
                   (unsigned long long)blocks * threads * iters, h);
        }
    cudaFree(d);
    return 0;
}
