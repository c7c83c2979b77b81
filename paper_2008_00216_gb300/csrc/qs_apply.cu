// Gate-application kernels for sm_103a: one HBM pass per launch.
//
//   k_dense      dense k <= 4 gate; each thread owns one set (Section 3's
//                2^(n-k) disjoint sets of 2^k amplitudes), or two adjacent
//                sets for complex64 so every access is a 16-byte vector
//                access and a warp touches 512 contiguous bytes per row.
//   k_diag       diagonal gate: a streaming multiply by a phase table over
//                the gate's bits (Section 4.3), multiply-free when every
//                phase is +-1 or +-i (Section 4.1).
//   k_mono       permutation-with-phase gate (NOT/SWAP/iSWAP-like, Section 3
//                "NOT as a swap"), one multiply (or none) per amplitude.
//   k_dense_smem dense 3 <= k <= 6 gate as a small complex GEMM through
//                shared memory (the plain FP32/FP64 CUDA-core path).
//   k_tile       several gates on a 2^L-amplitude tile held in shared memory
//                (the GPU form of Section 5's cache blocking: every gate
//                whose qubits lie in the tile is applied before write-back).
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "qs_device.cuh"
#include "qs_internal.h"
#include "qs_tile.cuh"

namespace qsgb {

static int stream_grid(uint64_t units, int threads) {
    const uint64_t want = (units + threads - 1) / threads;
    const uint64_t cap = (uint64_t)num_sms() * (2048 / threads);
    return (int)std::max<uint64_t>(1, std::min(want, cap));
}

// Kronecker-order offsets: local index l has qubits[0] as its top bit.
static void kron_offsets(int k, const int* qubits, uint64_t* off) {
    for (int l = 0; l < (1 << k); ++l) {
        uint64_t o = 0;
        for (int i = 0; i < k; ++i)
            if ((l >> (k - 1 - i)) & 1) o |= 1ull << qubits[i];
        off[l] = o;
    }
}

static void sorted_targets(int k, const int* qubits, int* sorted) {
    for (int i = 0; i < k; ++i) sorted[i] = qubits[i];
    std::sort(sorted, sorted + k);
}

// ============================================================== k_dense

template <typename R, int K>
struct DenseP {
    typename C2<R>::T m[1 << K][1 << K];
    uint64_t off[1 << K];
    int sorted[K];
    uint64_t units;
};

template <typename R, int K, int VEC>
__global__ void __launch_bounds__(256) k_dense(typename C2<R>::T* __restrict__ psi,
                                               const __grid_constant__ DenseP<R, K> p) {
    using T = typename C2<R>::T;
    constexpr int D = 1 << K;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < p.units; u += stride) {
        uint64_t base = u * VEC;
#pragma unroll
        for (int i = 0; i < K; ++i) base = insert_zero(base, p.sorted[i]);
        if constexpr (VEC == 2 && sizeof(R) == 4) {
            // two adjacent sets (bit 0 is not a target): one float4 per row
            float4 a[D];
#pragma unroll
            for (int l = 0; l < D; ++l) a[l] = *reinterpret_cast<const float4*>(psi + base + p.off[l]);
#pragma unroll
            for (int r = 0; r < D; ++r) {
                float2 o0 = make_float2(0.f, 0.f), o1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int l = 0; l < D; ++l) {
                    const float2 m = p.m[r][l];
                    cmac(o0, m, make_float2(a[l].x, a[l].y));
                    cmac(o1, m, make_float2(a[l].z, a[l].w));
                }
                *reinterpret_cast<float4*>(psi + base + p.off[r]) = make_float4(o0.x, o0.y, o1.x, o1.y);
            }
        } else {
            T a[D];
#pragma unroll
            for (int l = 0; l < D; ++l) a[l] = psi[base + p.off[l]];
#pragma unroll
            for (int r = 0; r < D; ++r) {
                T o;
                o.x = 0;
                o.y = 0;
#pragma unroll
                for (int l = 0; l < D; ++l) cmac(o, p.m[r][l], a[l]);
                psi[base + p.off[r]] = o;
            }
        }
    }
}

template <typename R, int K>
static cudaError_t dense_k(void* psi, int n, const int* qubits, const double* m, cudaStream_t st) {
    using T = typename C2<R>::T;
    constexpr int D = 1 << K;
    DenseP<R, K> p;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            p.m[r][c].x = (R)m[2 * (r * D + c)];
            p.m[r][c].y = (R)m[2 * (r * D + c) + 1];
        }
    kron_offsets(K, qubits, p.off);
    sorted_targets(K, qubits, p.sorted);
    const bool vec2 = sizeof(R) == 4 && p.sorted[0] >= 1;
    p.units = (1ull << (n - K)) >> (vec2 ? 1 : 0);
    const int grid = stream_grid(p.units, 256);
    if constexpr (sizeof(R) == 4) {
        if (vec2) {
            k_dense<R, K, 2><<<grid, 256, 0, st>>>((T*)psi, p);
            return cudaGetLastError();
        }
    }
    k_dense<R, K, 1><<<grid, 256, 0, st>>>((T*)psi, p);
    return cudaGetLastError();
}

cudaError_t launch_dense(void* psi, int n, qs_dtype dt, int k, const int* qubits, const double* m,
                         cudaStream_t st) {
    if (dt == QS_C64) {
        switch (k) {
            case 1: return dense_k<float, 1>(psi, n, qubits, m, st);
            case 2: return dense_k<float, 2>(psi, n, qubits, m, st);
            case 3: return dense_k<float, 3>(psi, n, qubits, m, st);
            case 4: return dense_k<float, 4>(psi, n, qubits, m, st);
        }
    } else {
        switch (k) {
            case 1: return dense_k<double, 1>(psi, n, qubits, m, st);
            case 2: return dense_k<double, 2>(psi, n, qubits, m, st);
            case 3: return dense_k<double, 3>(psi, n, qubits, m, st);
            case 4: return dense_k<double, 4>(psi, n, qubits, m, st);
        }
    }
    return cudaErrorInvalidValue;
}

// ============================================================== k_diag

template <typename R>
struct DiagP {
    typename C2<R>::T ph[64];
    int code[64];      // i^code when the phase is +-1 / +-i
    int q[kMaxK];      // Kronecker order
    int k;
    int mulfree;
    uint64_t units;
};

template <typename R>
__device__ __forceinline__ int local_index(uint64_t j, const int* q, int k) {
    int l = 0;
    for (int i = 0; i < k; ++i) l = (l << 1) | (int)((j >> q[i]) & 1);
    return l;
}

template <typename R, int VEC, bool MF>
__global__ void __launch_bounds__(256) k_diag(typename C2<R>::T* __restrict__ psi,
                                              const __grid_constant__ DiagP<R> p) {
    using T = typename C2<R>::T;
    __shared__ T ph[64];
    __shared__ int code[64];
    if (threadIdx.x < 64) {
        ph[threadIdx.x] = p.ph[threadIdx.x];
        code[threadIdx.x] = p.code[threadIdx.x];
    }
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < p.units; u += stride) {
        const uint64_t j = u * VEC;
        if constexpr (VEC == 2 && sizeof(R) == 4) {
            float4 v = *reinterpret_cast<const float4*>(psi + j);
            float2 a = make_float2(v.x, v.y), b = make_float2(v.z, v.w);
            const int la = local_index<R>(j, p.q, p.k), lb = local_index<R>(j + 1, p.q, p.k);
            if (MF) {
                a = rot_i(a, code[la]);
                b = rot_i(b, code[lb]);
            } else {
                a = cmul(ph[la], a);
                b = cmul(ph[lb], b);
            }
            *reinterpret_cast<float4*>(psi + j) = make_float4(a.x, a.y, b.x, b.y);
        } else {
            T a = psi[j];
            const int l = local_index<R>(j, p.q, p.k);
            a = MF ? rot_i(a, code[l]) : cmul(ph[l], a);
            psi[j] = a;
        }
    }
}

// code c with i^c equal to (re, im) exactly, or -1
static int quarter_code(double re, double im) {
    if (re == 1.0 && im == 0.0) return 0;
    if (re == 0.0 && im == 1.0) return 1;
    if (re == -1.0 && im == 0.0) return 2;
    if (re == 0.0 && im == -1.0) return 3;
    return -1;
}

template <typename R>
static cudaError_t diag_t(void* psi, int n, int k, const int* qubits, const double* m, cudaStream_t st) {
    using T = typename C2<R>::T;
    DiagP<R> p{};
    const int D = 1 << k;
    p.k = k;
    p.mulfree = 1;
    for (int i = 0; i < k; ++i) p.q[i] = qubits[i];
    for (int l = 0; l < 64; ++l) {
        p.ph[l].x = (R)1;
        p.ph[l].y = (R)0;
        p.code[l] = 0;
    }
    for (int l = 0; l < D; ++l) {
        const double re = m[2 * (l * D + l)], im = m[2 * (l * D + l) + 1];
        p.ph[l].x = (R)re;
        p.ph[l].y = (R)im;
        const int c = quarter_code(re, im);
        if (c < 0) p.mulfree = 0;
        p.code[l] = c < 0 ? 0 : c;
    }
    const bool vec2 = sizeof(R) == 4 && n >= 1;
    p.units = (1ull << n) >> (vec2 ? 1 : 0);
    const int grid = stream_grid(p.units, 256);
    if constexpr (sizeof(R) == 4) {
        if (vec2) {
            if (p.mulfree) k_diag<R, 2, true><<<grid, 256, 0, st>>>((T*)psi, p);
            else k_diag<R, 2, false><<<grid, 256, 0, st>>>((T*)psi, p);
            return cudaGetLastError();
        }
    }
    if (p.mulfree) k_diag<R, 1, true><<<grid, 256, 0, st>>>((T*)psi, p);
    else k_diag<R, 1, false><<<grid, 256, 0, st>>>((T*)psi, p);
    return cudaGetLastError();
}

cudaError_t launch_diag(void* psi, int n, qs_dtype dt, int k, const int* qubits, const double* m,
                        cudaStream_t st) {
    if (k < 1 || k > kMaxK) return cudaErrorInvalidValue;
    return dt == QS_C64 ? diag_t<float>(psi, n, k, qubits, m, st) : diag_t<double>(psi, n, k, qubits, m, st);
}

// ============================================================== k_mono

template <typename R, int K>
struct MonoP {
    typename C2<R>::T ph[1 << K];   // nonzero of row r
    int code[1 << K];
    uint64_t off[1 << K];           // destination offset of row r
    uint64_t src[1 << K];           // offset of the source column of row r
    int sorted[K];
    uint64_t units;
    int mulfree;
};

template <typename R, int K, int VEC, bool MF>
__global__ void __launch_bounds__(256) k_mono(typename C2<R>::T* __restrict__ psi,
                                              const __grid_constant__ MonoP<R, K> p) {
    using T = typename C2<R>::T;
    constexpr int D = 1 << K;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < p.units; u += stride) {
        uint64_t base = u * VEC;
#pragma unroll
        for (int i = 0; i < K; ++i) base = insert_zero(base, p.sorted[i]);
        if constexpr (VEC == 2 && sizeof(R) == 4) {
            float4 b[D];
#pragma unroll
            for (int r = 0; r < D; ++r) b[r] = *reinterpret_cast<const float4*>(psi + base + p.src[r]);
#pragma unroll
            for (int r = 0; r < D; ++r) {
                float2 x = make_float2(b[r].x, b[r].y), y = make_float2(b[r].z, b[r].w);
                if (MF) {
                    x = rot_i(x, p.code[r]);
                    y = rot_i(y, p.code[r]);
                } else {
                    x = cmul(p.ph[r], x);
                    y = cmul(p.ph[r], y);
                }
                *reinterpret_cast<float4*>(psi + base + p.off[r]) = make_float4(x.x, x.y, y.x, y.y);
            }
        } else {
            T b[D];
#pragma unroll
            for (int r = 0; r < D; ++r) b[r] = psi[base + p.src[r]];
#pragma unroll
            for (int r = 0; r < D; ++r) psi[base + p.off[r]] = MF ? rot_i(b[r], p.code[r]) : cmul(p.ph[r], b[r]);
        }
    }
}

template <typename R, int K>
static cudaError_t mono_k(void* psi, int n, const int* qubits, const double* m, cudaStream_t st) {
    using T = typename C2<R>::T;
    constexpr int D = 1 << K;
    MonoP<R, K> p;
    uint64_t off[D];
    kron_offsets(K, qubits, off);
    p.mulfree = 1;
    for (int r = 0; r < D; ++r) {
        int c = 0;
        while (c < D && m[2 * (r * D + c)] == 0.0 && m[2 * (r * D + c) + 1] == 0.0) ++c;
        if (c == D) return cudaErrorInvalidValue;
        const double re = m[2 * (r * D + c)], im = m[2 * (r * D + c) + 1];
        p.ph[r].x = (R)re;
        p.ph[r].y = (R)im;
        const int code = quarter_code(re, im);
        if (code < 0) p.mulfree = 0;
        p.code[r] = code < 0 ? 0 : code;
        p.off[r] = off[r];
        p.src[r] = off[c];
    }
    sorted_targets(K, qubits, p.sorted);
    const bool vec2 = sizeof(R) == 4 && p.sorted[0] >= 1;
    p.units = (1ull << (n - K)) >> (vec2 ? 1 : 0);
    const int grid = stream_grid(p.units, 256);
    if constexpr (sizeof(R) == 4) {
        if (vec2) {
            if (p.mulfree) k_mono<R, K, 2, true><<<grid, 256, 0, st>>>((T*)psi, p);
            else k_mono<R, K, 2, false><<<grid, 256, 0, st>>>((T*)psi, p);
            return cudaGetLastError();
        }
    }
    if (p.mulfree) k_mono<R, K, 1, true><<<grid, 256, 0, st>>>((T*)psi, p);
    else k_mono<R, K, 1, false><<<grid, 256, 0, st>>>((T*)psi, p);
    return cudaGetLastError();
}

cudaError_t launch_mono(void* psi, int n, qs_dtype dt, int k, const int* qubits, const double* m,
                        cudaStream_t st) {
#define QS_MONO_CASE(KK)                                                              \
    case KK:                                                                          \
        return dt == QS_C64 ? mono_k<float, KK>(psi, n, qubits, m, st)                \
                            : mono_k<double, KK>(psi, n, qubits, m, st);
    switch (k) {
        QS_MONO_CASE(1)
        QS_MONO_CASE(2)
        QS_MONO_CASE(3)
        QS_MONO_CASE(4)
        QS_MONO_CASE(5)
        QS_MONO_CASE(6)
    }
#undef QS_MONO_CASE
    return cudaErrorInvalidValue;
}

// ============================================================== k_dense_smem

struct SmemP {
    uint64_t off[64];
    int sorted[kMaxK];
    uint64_t nchunks;    // 32 consecutive sets per chunk
    uint64_t nsets;
};

// One CTA of 256 threads: the matrix stays in shared memory; per chunk of
// 32 sets it stages X (2^K x 32), and thread (row group g, column c)
// computes 2^K/8 output rows of column c.
template <typename R, int K>
__global__ void __launch_bounds__(256) k_dense_smem(typename C2<R>::T* __restrict__ psi,
                                                    const typename C2<R>::T* __restrict__ mat,
                                                    const __grid_constant__ SmemP p) {
    using T = typename C2<R>::T;
    constexpr int D = 1 << K;
    constexpr int RPG = D / 8;  // rows per group
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* M = reinterpret_cast<T*>(smem_raw);
    T* X = M + D * D;
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) M[i] = mat[i];
    const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
    for (uint64_t ch = blockIdx.x; ch < p.nchunks; ch += gridDim.x) {
        const uint64_t s = ch * 32 + c;
        const bool live = s < p.nsets;
        uint64_t base = live ? s : 0;
#pragma unroll
        for (int i = 0; i < K; ++i) base = insert_zero(base, p.sorted[i]);
        __syncthreads();  // M loaded / previous chunk's X consumed
        for (int l = g; l < D; l += 8) {
            T v;
            v.x = 0;
            v.y = 0;
            if (live) v = psi[base + p.off[l]];
            X[l * 32 + c] = v;
        }
        __syncthreads();
        T acc[RPG];
#pragma unroll
        for (int r = 0; r < RPG; ++r) {
            acc[r].x = 0;
            acc[r].y = 0;
        }
        for (int l = 0; l < D; ++l) {
            const T x = X[l * 32 + c];
#pragma unroll
            for (int r = 0; r < RPG; ++r) cmac(acc[r], M[(g * RPG + r) * D + l], x);
        }
        if (live) {
#pragma unroll
            for (int r = 0; r < RPG; ++r) psi[base + p.off[g * RPG + r]] = acc[r];
        }
    }
}

template <typename R, int K>
static cudaError_t dense_smem_k(void* psi, int n, const int* qubits, const void* dmat, cudaStream_t st) {
    using T = typename C2<R>::T;
    constexpr int D = 1 << K;
    SmemP p{};
    kron_offsets(K, qubits, p.off);
    sorted_targets(K, qubits, p.sorted);
    p.nsets = 1ull << (n - K);
    p.nchunks = (p.nsets + 31) / 32;
    const size_t smem = sizeof(T) * (D * D + D * 32);
    cudaError_t e = allow_max_dynamic_smem(k_dense_smem<R, K>);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<uint64_t>(p.nchunks, (uint64_t)num_sms() * 4);
    k_dense_smem<R, K><<<grid, 256, smem, st>>>((T*)psi, (const T*)dmat, p);
    return cudaGetLastError();
}

cudaError_t launch_dense_smem(void* psi, int n, qs_dtype dt, int k, const int* qubits, const void* dmat,
                              cudaStream_t st) {
#define QS_SMEM_CASE(KK)                                                              \
    case KK:                                                                          \
        return dt == QS_C64 ? dense_smem_k<float, KK>(psi, n, qubits, dmat, st)       \
                            : dense_smem_k<double, KK>(psi, n, qubits, dmat, st);
    switch (k) {
        QS_SMEM_CASE(3)
        QS_SMEM_CASE(4)
        QS_SMEM_CASE(5)
        QS_SMEM_CASE(6)
    }
#undef QS_SMEM_CASE
    return cudaErrorInvalidValue;
}

// ============================================================== k_tile

struct TileArgs {
    int L;                 // tile qubits
    int b;                 // leading local bits that are global bits 0..b-1
    int ngates;
    int pos[16];           // global bit of local bit i (ascending)
    uint32_t mat_elems;    // complex entries of all the pass's matrices
    uint64_t ntiles;
    int scale_mode;        // 0 none, 1 mag * exp(i pi s / 4), 2 general complex
    int scale_s;
    double scale_mag;      // for mode 1: |scale|, times 1/sqrt(2) when s is odd
    double scale_c[2];
    TileGate g[kMaxTileGates];
};

template <typename R>
__global__ void __launch_bounds__(256) k_tile(typename C2<R>::T* __restrict__ psi,
                                              const typename C2<R>::T* __restrict__ mats,
                                              const __grid_constant__ TileArgs a) {
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [tile: 2^L amplitudes][the pass's matrices][row offsets]
    T* tile = reinterpret_cast<T*>(smem_raw);
    T* smat = tile + (1u << a.L);
    uint64_t* rowoff = reinterpret_cast<uint64_t*>(smat + a.mat_elems);
    const int L = a.L, b = a.b;
    const uint32_t rowlen = 1u << b, nrows = 1u << (L - b);
    for (uint32_t i = threadIdx.x; i < a.mat_elems; i += blockDim.x) smat[i] = mats[i];
    for (uint32_t h = threadIdx.x; h < nrows; h += blockDim.x) {
        uint64_t o = 0;
        for (int i = b; i < L; ++i)
            if ((h >> (i - b)) & 1) o |= 1ull << a.pos[i];
        rowoff[h] = o;
    }
    __syncthreads();
    for (uint64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        uint64_t base = t;
        for (int i = 0; i < L; ++i) base = insert_zero(base, a.pos[i]);
        // load: rows of 2^b contiguous amplitudes
        tile_gather(tile, psi, base, rowoff, b, L);
        __syncthreads();
        for (int gi = 0; gi < a.ngates; ++gi) {
            const TileGate& g = a.g[gi];
            const T* m = smat + g.mat;
            if (g.kind == QS_GATE_DIAGONAL) {
                tile_diag(tile, L, g, m);
            } else if (g.kind == kTileMulfree) {
                tile_mulfree1(tile, L, g, m);
            } else {  // dense or monomial, k <= 4, through registers
                switch (g.k) {
                    case 1: tile_dense<T, 1>(tile, L, g, m); break;
                    case 2: tile_dense<T, 2>(tile, L, g, m); break;
                    case 3: tile_dense<T, 3>(tile, L, g, m); break;
                    case 4: tile_dense<T, 4>(tile, L, g, m); break;
                    default: break;  // excluded by the planner
                }
            }
            __syncthreads();
        }
        if (a.scale_mode == 0) {
            for (uint32_t e = threadIdx.x; e < (1u << L); e += blockDim.x)
                psi[base + rowoff[e >> b] + (e & (rowlen - 1))] = tile[e];
        } else {  // the scalars factored out of the pass's multiply-free gates
            const R mag = (R)a.scale_mag;
            T c;
            c.x = (R)a.scale_c[0];
            c.y = (R)a.scale_c[1];
            for (uint32_t e = threadIdx.x; e < (1u << L); e += blockDim.x) {
                T v = tile[e];
                if (a.scale_mode == 1) {
                    v = rot_i(v, a.scale_s >> 1);
                    if (a.scale_s & 1) {  // times (1 + i) (the 1/sqrt(2) is in mag)
                        const R re = v.x - v.y, im = v.x + v.y;
                        v.x = re;
                        v.y = im;
                    }
                    v.x *= mag;
                    v.y *= mag;
                } else {
                    v = cmul(c, v);
                }
                psi[base + rowoff[e >> b] + (e & (rowlen - 1))] = v;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_tile(void* psi, int n, qs_dtype dt, const Pass& ps, const void* dmats, cudaStream_t st) {
    TileArgs a{};
    a.L = ps.L;
    int b = 0;
    while (b < ps.L && ps.pos[b] == b) ++b;
    a.b = b;
    a.ngates = (int)ps.tgates.size();
    if (a.ngates > kMaxTileGates || ps.L < 1 || ps.L > 13) return cudaErrorInvalidValue;
    for (int i = 0; i < ps.L; ++i) a.pos[i] = ps.pos[i];
    for (int i = 0; i < a.ngates; ++i) a.g[i] = ps.tgates[i];
    a.ntiles = 1ull << (n - ps.L);
    a.mat_elems = (uint32_t)(ps.mats.size() / 2);
    a.scale_mode = ps.scale_mode;
    a.scale_s = ps.scale_s;
    a.scale_mag = ps.scale_mag * ((ps.scale_s & 1) ? 0.70710678118654752440 : 1.0);
    a.scale_c[0] = ps.scale_c[0];
    a.scale_c[1] = ps.scale_c[1];
    const size_t esz = dt == QS_C64 ? 8 : 16;
    const size_t smem = esz * ((1u << ps.L) + a.mat_elems) + sizeof(uint64_t) * (1u << (ps.L - b));
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const int grid = (int)std::min<uint64_t>(a.ntiles, (uint64_t)num_sms() * 8);
    cudaError_t e;
    if (dt == QS_C64) {
        e = allow_max_dynamic_smem(k_tile<float>);
        if (e != cudaSuccess) return e;
        k_tile<float><<<grid, 256, smem, st>>>((float2*)psi, (const float2*)dmats, a);
    } else {
        e = allow_max_dynamic_smem(k_tile<double>);
        if (e != cudaSuccess) return e;
        k_tile<double><<<grid, 256, smem, st>>>((double2*)psi, (const double2*)dmats, a);
    }
    return cudaGetLastError();
}

// ============================================================== init

template <typename T>
__global__ void k_fill(T* __restrict__ psi, uint64_t size, T v, uint64_t one_index, int basis) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < size; j += stride) {
        T x = v;
        if (basis) {
            x.x = (j == one_index) ? 1 : 0;
            x.y = 0;
        }
        psi[j] = x;
    }
}

cudaError_t launch_init_basis(void* psi, int n, qs_dtype dt, uint64_t index, cudaStream_t st) {
    const uint64_t size = 1ull << n;
    const int grid = stream_grid(size, 256);
    if (dt == QS_C64) k_fill<float2><<<grid, 256, 0, st>>>((float2*)psi, size, make_float2(0, 0), index, 1);
    else k_fill<double2><<<grid, 256, 0, st>>>((double2*)psi, size, make_double2(0, 0), index, 1);
    return cudaGetLastError();
}

cudaError_t launch_init_uniform(void* psi, int n, qs_dtype dt, cudaStream_t st) {
    const uint64_t size = 1ull << n;
    const int grid = stream_grid(size, 256);
    const double v = ldexp(1.0, -n / 2) * ((n & 1) ? 0.70710678118654752440 : 1.0);
    if (dt == QS_C64) k_fill<float2><<<grid, 256, 0, st>>>((float2*)psi, size, make_float2((float)v, 0), 0, 0);
    else k_fill<double2><<<grid, 256, 0, st>>>((double2*)psi, size, make_double2(v, 0), 0, 0);
    return cudaGetLastError();
}

}  // namespace qsgb
