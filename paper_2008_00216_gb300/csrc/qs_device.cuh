// Device-side helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qsgb {

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

// Insert a zero bit at position p: bits below p stay, bits at or above p
// move up by one.  Applied for target positions in ascending order, it
// maps a set id to the index of the set's first amplitude (Section 3).
__device__ __forceinline__ uint64_t insert_zero(uint64_t x, int p) {
    const uint64_t lo = x & ((1ull << p) - 1ull);
    return ((x >> p) << (p + 1)) | lo;
}
__device__ __forceinline__ uint32_t insert_zero32(uint32_t x, int p) {
    const uint32_t lo = x & ((1u << p) - 1u);
    return ((x >> p) << (p + 1)) | lo;
}

template <typename T>
__device__ __forceinline__ T cmul(T m, T x) {
    T r;
    r.x = m.x * x.x - m.y * x.y;
    r.y = m.x * x.y + m.y * x.x;
    return r;
}

// acc += m * x (complex), as four fused multiply-adds
template <typename T>
__device__ __forceinline__ void cmac(T& acc, T m, T x) {
    acc.x = fma(m.x, x.x, acc.x);
    acc.x = fma(-m.y, x.y, acc.x);
    acc.y = fma(m.x, x.y, acc.y);
    acc.y = fma(m.y, x.x, acc.y);
}

// Multiply by i^code without multiplications (Section 4.1: phases +-1, +-i
// are swaps of the real and imaginary parts and negations).
template <typename T>
__device__ __forceinline__ T rot_i(T x, int code) {
    T r;
    switch (code & 3) {
        case 0: r = x; break;
        case 1: r.x = -x.y; r.y = x.x; break;
        case 2: r.x = -x.x; r.y = -x.y; break;
        default: r.x = x.y; r.y = -x.x; break;
    }
    return r;
}

// Error-free transformations on floats (Knuth's TwoSum, FMA-based TwoProd)
// for a two-float accumulator: the "sum-of-two-values" representation that
// Section 4.1 recommends for the norm, in the form of Ogita, Rump and
// Oishi's Sum2 (running sum plus a running sum of the rounding errors).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
struct F2Acc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v) {
        float s, e;
        two_sum(hi, v, s, e);
        hi = s;
        lo += e;
    }
    // add x*x with its product rounding error (one FMA recovers it)
    __device__ __forceinline__ void add_sq(float x) {
        const float p = x * x;
        const float q = fmaf(x, x, -p);
        float s, e;
        two_sum(hi, p, s, e);
        hi = s;
        lo += e + q;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of one double; result valid in thread 0.  blockDim <= 1024.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

}  // namespace qsgb
