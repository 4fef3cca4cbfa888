// Probe for the weight build's quotient (csrc/fp64div.cuh): div_by_pivot(b, p,
// RN(1/p)) against the library's correctly rounded b / p, bit for bit, on
// seeded operand pairs.  Modes: 0 uniform mantissas, 1 mantissas next to 1
// and 2 (the hard cases for rounding), 2 exponents beyond the fast path's
// range (the library fallback).  Prints one line per mode: "mode M pairs P
// mismatches K".
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "fp64div.cuh"

__device__ __forceinline__ uint64_t mix64(uint64_t x) {   // SplitMix64 finaliser
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ double operand(uint64_t r, int mode) {
    uint64_t mant = r & 0xfffffffffffffull;
    if (mode == 1) mant = (r & 1) ? 0xfffffffffffffull - ((r >> 1) & 0xff) : ((r >> 1) & 0xff);
    const int span = mode == 2 ? 1401 : 121;            // exponents in [-700, 700] or [-60, 60]
    const int e = (int)((r >> 52) % span) - span / 2;
    const uint64_t sign = (r >> 63) << 63;
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 1023) << 52) | mant));
}

__global__ void probe(int mode, int iters, unsigned long long* bad) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nb = 0;
    for (int i = 0; i < iters; ++i) {
        const uint64_t id = (uint64_t)mode << 48 | (t * (uint64_t)iters + i);
        const double b = operand(mix64(2 * id), mode == 1 ? 0 : mode);
        const double p = operand(mix64(2 * id + 1), mode);
        const double q = rbffd::div_by_pivot(b, p, __drcp_rn(p));
        if (__double_as_longlong(q) != __double_as_longlong(__ddiv_rn(b, p))) ++nb;
    }
    if (nb) atomicAdd(bad, nb);
}

int main() {
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return 2;
    const int blocks = 152 * 8, threads = 256, iters = 256;
    for (int mode = 0; mode < 3; ++mode) {
        unsigned long long h = 0;
        cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice);
        probe<<<blocks, threads>>>(mode, iters, d);
        if (cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
        printf("mode %d pairs %llu mismatches %llu\n", mode,
               (unsigned long long)blocks * threads * iters, h);
    }
    cudaFree(d);
    return 0;
}
