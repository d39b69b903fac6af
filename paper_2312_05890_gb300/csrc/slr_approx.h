// The approximate counter's generator and sampling kernel (internal to the library).
//
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the n-th output of the
// generator seeded with s is mix(s + (n + 1) g) with g = 0x9E3779B97F4A7C15
// and mix the generator's output function; used as a counter-based generator,
// so that the host, the device and any other implementation draw the same
// numbers for the same (seed, index).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "slr_device.cuh"

namespace slr {

constexpr unsigned long long kSplitMixGamma = 0x9E3779B97F4A7C15ull;
// point index reserved for the coin of a split
constexpr int kApproxCoinPoint = (1 << 24) - 1;
constexpr int kApproxMaxTrials = 64;

__host__ __device__ inline unsigned long long splitmix64(unsigned long long seed, unsigned long long n) {
    unsigned long long z = seed + (n + 1ull) * kSplitMixGamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// draw index of coordinate i of point k of split j in trial t
__host__ __device__ inline unsigned long long approx_draw_index(int t, int j, int k, int i) {
    return ((unsigned long long)t << 40) | ((unsigned long long)j << 34) | ((unsigned long long)k << 10) |
           (unsigned long long)i;
}

// uniform double in [0, 1): the top 53 bits
__host__ __device__ inline double splitmix_uniform(unsigned long long seed, unsigned long long n) {
    return (double)(splitmix64(seed, n) >> 11) * 0x1p-53;
}

int approx_width(const NetParams<double> &net);
size_t approx_sample_smem(const NetParams<double> &net);
// Samples n points of the box [lo, hi] (float64, device) and appends the
// coordinate `dim` of each unsafe point to coord (device, room for n); count
// (device) receives how many.
cudaError_t launch_approx_sample(const NetParams<double> &net, const double *lo, const double *hi, int dim,
                                 unsigned long long seed, int trial, int split, int n, double *coord,
                                 unsigned long long *count, int sms, cudaStream_t s);

}  // namespace slr
