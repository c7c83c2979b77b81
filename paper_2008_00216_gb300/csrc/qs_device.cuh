// Device-side helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qsgb {

// Allow a kernel the device's whole opt-in shared memory (minus its static
// shared memory).  The attribute is one value per kernel for the process,
// so every caller sets the same value: launches from concurrent host
// threads with different dynamic sizes cannot undercut each other.  Done
// once per kernel and device (the runtime calls cost microseconds).
bool smem_attr_done(const void* kernel, int device);
void smem_attr_mark(const void* kernel, int device);   // after the attribute is set
template <typename K>
inline cudaError_t allow_max_dynamic_smem(K kernel) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (smem_attr_done(reinterpret_cast<const void*>(kernel), dev)) return cudaSuccess;
    // first callers on several threads may all get here: they set one value
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    int optin = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) smem_attr_mark(reinterpret_cast<const void*>(kernel), dev);
    return e;
}

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

// Gather a 2^L-amplitude tile into shared memory: local index e lives at
// base + rowoff[e >> b] + (e & (2^b - 1)) (rows of 2^b contiguous
// amplitudes).  Each thread issues 8 independent loads before storing any,
// so a block keeps enough loads in flight to cover the HBM latency.  With
// CG the loads bypass L1 (data written by other blocks of the same launch).
template <typename T, bool CG = false>
__device__ __forceinline__ void tile_gather(T* tile, const T* __restrict__ src, uint64_t base, const uint64_t* rowoff,
                                            int b, int L) {
    const uint32_t n = 1u << L, mask = (1u << b) - 1u;
    for (uint32_t e0 = threadIdx.x; e0 < n; e0 += 8u * blockDim.x) {
        T v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t e = e0 + (uint32_t)k * blockDim.x;
            if (e < n) {
                const T* p = src + base + rowoff[e >> b] + (e & mask);
                v[k] = CG ? __ldcg(p) : *p;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t e = e0 + (uint32_t)k * blockDim.x;
            if (e < n) tile[e] = v[k];
        }
    }
}

// The same for two states sharing the tile layout (4 + 4 loads in flight).
template <typename T>
__device__ __forceinline__ void tile_gather2(T* ta, T* tb, const T* __restrict__ a, const T* __restrict__ b_,
                                             uint64_t base, const uint64_t* rowoff, int b, int L) {
    const uint32_t n = 1u << L, mask = (1u << b) - 1u;
    for (uint32_t e0 = threadIdx.x; e0 < n; e0 += 4u * blockDim.x) {
        T va[4], vb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t e = e0 + (uint32_t)k * blockDim.x;
            if (e < n) {
                const uint64_t gi = base + rowoff[e >> b] + (e & mask);
                va[k] = a[gi];
                vb[k] = b_[gi];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t e = e0 + (uint32_t)k * blockDim.x;
            if (e < n) {
                ta[e] = va[k];
                tb[e] = vb[k];
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ T cmul(T m, T x) {
    T r;
    r.x = m.x * x.x - m.y * x.y;
    r.y = m.x * x.y + m.y * x.x;
    return r;
}

// ph times the diagonal entries of `count` gates at index x; gate c has k
// qubits q[0..k) (q[0] the most significant local bit) and its 2^k entries
// at tab[cg[c].tab].
template <typename T, typename X>
__device__ __forceinline__ T cross_phase(const X* cg, int count, const T* tab, uint64_t x, T ph) {
    for (int c = 0; c < count; ++c) {
        uint32_t li = 0;
        for (int i = 0; i < cg[c].k; ++i) li = (li << 1) | (uint32_t)((x >> cg[c].q[i]) & 1);
        ph = cmul(ph, tab[cg[c].tab + li]);
    }
    return ph;
}

// Componentwise a * b + c; for FP32 pairs one packed f32x2 instruction
// (Blackwell), which halves the issue slots of real-by-complex products.
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    const uint64_t ua = (uint64_t)__float_as_uint(a.x) | ((uint64_t)__float_as_uint(a.y) << 32);
    const uint64_t ub = (uint64_t)__float_as_uint(b.x) | ((uint64_t)__float_as_uint(b.y) << 32);
    const uint64_t uc = (uint64_t)__float_as_uint(c.x) | ((uint64_t)__float_as_uint(c.y) << 32);
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(ua), "l"(ub), "l"(uc));
    return make_float2(__uint_as_float((uint32_t)d), __uint_as_float((uint32_t)(d >> 32)));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
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
// complex128: the negations flip sign bits on the integer pipe, leaving the
// FP64 pipe (the scarce one on this GPU) to real arithmetic
__device__ __forceinline__ double flip_sign(double v, bool neg) {
    return __longlong_as_double(__double_as_longlong(v) ^ (neg ? (long long)0x8000000000000000ull : 0ll));
}
template <>
__device__ __forceinline__ double2 rot_i<double2>(double2 x, int code) {
    const int c = code & 3;
    const bool swap = c & 1;
    double2 r;
    r.x = flip_sign(swap ? x.y : x.x, c == 1 || c == 2);
    r.y = flip_sign(swap ? x.x : x.y, c >= 2);
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
        const float p = __fmul_rn(x, x);  // never contracted into the sum below
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
