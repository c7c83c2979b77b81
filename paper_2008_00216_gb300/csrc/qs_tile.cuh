// Gate application on a tile of 2^L amplitudes held in shared memory, used by
// the tile pass and by the batched kernel.  Local bit i of the tile is some
// global qubit; a gate's qubits are given as local bit positions.
#pragma once

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsgb {

// One-qubit gate with entries in {0, +-1, +-i} (its scalar factored out):
// out0 = u00 a + u01 b, out1 = u10 a + u11 b with each product a swap and
// sign flips (Section 4.1), so a pair costs four additions.
template <typename T>
__device__ __forceinline__ int mulfree_code(T u) {  // -1: zero, else u = i^code
    return (u.x == 0 && u.y == 0) ? -1 : u.x == 1 ? 0 : u.y == 1 ? 1 : u.x == -1 ? 2 : 3;
}
template <typename T>
__device__ __forceinline__ T mulfree_sum(T a, int ca, T b, int cb) {
    if (ca < 0) return rot_i(b, cb);
    if (cb < 0) return rot_i(a, ca);
    const T x = rot_i(a, ca), y = rot_i(b, cb);
    T r;
    r.x = x.x + y.x;
    r.y = x.y + y.y;
    return r;
}
template <typename T>
__device__ __forceinline__ void tile_mulfree1(T* tile, int L, const TileGate& g, const T* m) {
    const int c00 = mulfree_code(m[0]), c01 = mulfree_code(m[1]), c10 = mulfree_code(m[2]), c11 = mulfree_code(m[3]);
    const int q = g.q[0];
    for (uint32_t s = threadIdx.x; s < (1u << (L - 1)); s += blockDim.x) {
        const uint32_t i0 = insert_zero32(s, q), i1 = i0 | (1u << q);
        const T a = tile[i0], b = tile[i1];
        tile[i0] = mulfree_sum(a, c00, b, c01);
        tile[i1] = mulfree_sum(a, c10, b, c11);
    }
}

// dense gate with K <= 4 on the shared tile, one set per thread iteration
template <typename T, int K>
__device__ __forceinline__ void tile_dense(T* tile, int L, const TileGate& g, const T* m) {
    constexpr int D = 1 << K;
    int srt[K];
#pragma unroll
    for (int i = 0; i < K; ++i) srt[i] = g.q[i];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = 0; j + 1 < K - i; ++j)
            if (srt[j] > srt[j + 1]) {
                const int t = srt[j];
                srt[j] = srt[j + 1];
                srt[j + 1] = t;
            }
    uint32_t off[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
        uint32_t o = 0;
#pragma unroll
        for (int i = 0; i < K; ++i)
            if ((l >> (K - 1 - i)) & 1) o |= 1u << g.q[i];
        off[l] = o;
    }
    const uint32_t nsets = 1u << (L - K);
    for (uint32_t s = threadIdx.x; s < nsets; s += blockDim.x) {
        uint32_t base = s;
#pragma unroll
        for (int i = 0; i < K; ++i) base = insert_zero32(base, srt[i]);
        T a[D];
#pragma unroll
        for (int l = 0; l < D; ++l) a[l] = tile[base + off[l]];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            T o;
            o.x = 0;
            o.y = 0;
#pragma unroll
            for (int l = 0; l < D; ++l) cmac(o, m[r * D + l], a[l]);
            tile[base + off[r]] = o;
        }
    }
}

template <typename T>
__device__ __forceinline__ void tile_diag(T* tile, int L, const TileGate& g, const T* m) {
    const int k = g.k, D = 1 << k;
    for (uint32_t e = threadIdx.x; e < (1u << L); e += blockDim.x) {
        int l = 0;
        for (int i = 0; i < k; ++i) l = (l << 1) | ((e >> g.q[i]) & 1);
        tile[e] = cmul(m[l * D + l], tile[e]);
    }
}

}  // namespace qsgb
