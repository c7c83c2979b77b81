// Stage kernels of the adjoint reverse sweep.
//
// The gradient of E = <psi|H|psi> with respect to the angle of a gate
// U_l = exp(-i theta P_l / 2) is Im <lambda_l| P_l |psi_l>, with psi_l and
// lambda_l the forward state and H psi carried back to just after gate l.
// When a run of gates commutes pairwise (disjoint qubits, or all diagonal),
// each of them can be moved to the end of the run, so all of the run's
// gradients come from the same pair (psi, lambda) -- read once -- and the
// run's inverse can then be applied as a few fused passes.  These kernels
// do the two stage steps that are not ordinary gate passes:
//   k_grad_pairs  <lambda|P_g|psi> for up to 16 Pauli generators whose flip
//                 and sign qubits lie in one tile of the state (read only)
//   k_diag_stage  a run of diagonal gates on psi and lambda together: the
//                 Z-type gradients of the run and its inverse, whose phase is
//                 a product of per-8-qubit tables and a few cross gates
#include <stdint.h>

#include <algorithm>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsgb {

namespace {

struct GradPairsArgs {
    int L, b;
    int pos[16];
    uint64_t ntiles;
    int ngen;
    StageGen g[kStageGradGens];
};

// Tile over the qubits pos[0..L-1] (pos[i] = i for i < b: rows of 2^b
// contiguous amplitudes), both states in shared memory.  With
// (P psi)_e = i^ny (-1)^popc((e^px) & pz) psi_(e^px) on local indices, the
// gradient Im <lambda|P|psi> = Im(i^ny S), S = sum_e s_e conj(lambda_e) psi_(e^px),
// needs only one real part of S: Im S for even ny, Re S for odd ny.  A thread
// holds its PER lambda values in registers; per generator it walks them
// (unrolled, one variant per sign kind and part), reading psi_(e^px) from
// shared memory, then the warp adds its sums into per-warp FP64 slots.  The
// block adds its warps in a fixed order and writes Im(i^ny S).
template <typename R, int PER, int SIGN, bool IM>
__device__ __forceinline__ R grad_tile_sum(const typename C2<R>::T* tp, const typename C2<R>::T* lv, uint32_t px,
                                           uint32_t pz, int zb) {
    R acc = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t e = threadIdx.x + 256u * j;
        const uint32_t f = e ^ px;
        const typename C2<R>::T v = tp[f];
        const R t = IM ? lv[j].x * v.y - lv[j].y * v.x : lv[j].x * v.x + lv[j].y * v.y;
        if (SIGN == 0) acc += t;
        else if (SIGN == 1) acc += ((f >> zb) & 1u) ? -t : t;
        else acc += (__popc(f & pz) & 1) ? -t : t;
    }
    return acc;
}

template <typename R, int PER>
__global__ void __launch_bounds__(256) k_grad_pairs(const typename C2<R>::T* __restrict__ psi,
                                                    const typename C2<R>::T* __restrict__ lam,
                                                    const __grid_constant__ GradPairsArgs a,
                                                    double* __restrict__ partials) {
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[8][kStageGradGens];
    const int L = a.L, b = a.b;
    T* tp = reinterpret_cast<T*>(smem_raw);  // psi tile; lambda stays in registers
    uint64_t* rowoff = reinterpret_cast<uint64_t*>(tp + (1u << L));
    for (uint32_t h = threadIdx.x; h < (1u << (L - b)); h += blockDim.x) {
        uint64_t o = 0;
        for (int i = b; i < L; ++i)
            if ((h >> (i - b)) & 1) o |= 1ull << a.pos[i];
        rowoff[h] = o;
    }
    for (int i = threadIdx.x; i < 8 * kStageGradGens; i += blockDim.x) (&red[0][0])[i] = 0.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t mask = (1u << b) - 1u;
    __syncthreads();
    for (uint64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        uint64_t base = t;
        for (int i = 0; i < L; ++i) base = insert_zero(base, a.pos[i]);
        T lv[PER], pv[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {  // all loads in flight before the first store
            const uint32_t e = threadIdx.x + 256u * j;
            const uint64_t gi = base + rowoff[e >> b] + (e & mask);
            pv[j] = psi[gi];
            lv[j] = lam[gi];
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) tp[threadIdx.x + 256u * j] = pv[j];
        __syncthreads();
        for (int g = 0; g < a.ngen; ++g) {
            const uint32_t px = a.g[g].px, pz = a.g[g].pz;
            const bool im = (a.g[g].ny & 1) == 0;
            const int kind = pz == 0 ? 0 : (pz & (pz - 1)) == 0 ? 1 : 2;
            const int zb = kind == 1 ? __ffs(pz) - 1 : 0;
            R acc;
            if (im) {
                acc = kind == 0 ? grad_tile_sum<R, PER, 0, true>(tp, lv, px, pz, zb)
                    : kind == 1 ? grad_tile_sum<R, PER, 1, true>(tp, lv, px, pz, zb)
                                : grad_tile_sum<R, PER, 2, true>(tp, lv, px, pz, zb);
            } else {
                acc = kind == 0 ? grad_tile_sum<R, PER, 0, false>(tp, lv, px, pz, zb)
                    : kind == 1 ? grad_tile_sum<R, PER, 1, false>(tp, lv, px, pz, zb)
                                : grad_tile_sum<R, PER, 2, false>(tp, lv, px, pz, zb);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) red[warp][g] += (double)acc;
        }
        __syncthreads();  // the tiles are overwritten by the next iteration
    }
    __syncthreads();
    for (int g = threadIdx.x; g < a.ngen; g += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][g];  // fixed order: deterministic
        // Im(i^ny S): ny = 0: Im S, 1: Re S, 2: -Im S, 3: -Re S; s holds the part used
        const int q = a.g[g].ny & 3;
        partials[((size_t)a.g[g].slot * gridDim.x + blockIdx.x) * 2] = 0.0;
        partials[((size_t)a.g[g].slot * gridDim.x + blockIdx.x) * 2 + 1] = q >= 2 ? -s : s;
    }
}

constexpr int kDiagMulti = kStageDiagMulti;

struct DiagStageArgs {
    int n;
    int nchunks;              // chunk c holds qubits 8c .. 8c+7 (fewer in the last)
    int nlow, nhigh;          // cross gates with a qubit below 10 / all at or above 10
    int nsingle, nmulti;      // Z generators on one qubit / on several
    int apply;                // 0: gradients only
    uint32_t tab_elems;       // chunk tables, then the cross gates' diagonals
    DiagCross low[kStageDiagCross], high[kStageDiagCross];
    int zbit[kStageDiagGens];     // single-qubit generators: the qubit
    int slot[kStageDiagGens];
    uint64_t mz[kDiagMulti];      // multi-qubit generators: sign mask
    int mslot[kDiagMulti];
};

// Gradients: Im <lambda|Z_g|psi> = sum_x (-1)^popc(x & zm_g) Im(conj(lambda_x) psi_x).
// Inverse: psi_x, lambda_x *= prod_c T_c[bits of chunk c] * prod_cross d_g[its bits].
// For n >= 10 a warp walks blocks of 1024 amplitudes: lane = index bits 0-4,
// step j = bits 5-9, block number = bits >= 10 (coalesced).  A sign on one
// qubit then needs no per-amplitude work: per block the warp reduces the
// total T, the sums U_b over steps with bit b set and W_b over lanes with
// bit b set, and lane 0 adds T - 2 W_b, T - 2 U_b or +-T (block bit) to each
// single-qubit generator's FP64 slot.  Only multi-qubit Z generators are
// summed per amplitude (in R, flushed every 4 blocks).  The phase factors of
// chunk tables 2.. and of cross gates on qubits >= 10 are one constant per
// block.  The block adds its warps' slots in a fixed order.  Below 10 qubits:
// one amplitude per thread, every sign computed directly.
template <typename R>
__global__ void __launch_bounds__(256) k_diag_stage(typename C2<R>::T* __restrict__ psi,
                                                    typename C2<R>::T* __restrict__ lam,
                                                    const typename C2<R>::T* __restrict__ tables,
                                                    const __grid_constant__ DiagStageArgs a,
                                                    double* __restrict__ partials) {
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[8][kStageDiagGens + kDiagMulti];  // per-warp FP64 sums
    T* tab = reinterpret_cast<T*>(smem_raw);
    for (uint32_t i = threadIdx.x; i < a.tab_elems; i += blockDim.x) tab[i] = tables[i];
    for (int i = threadIdx.x; i < 8 * (kStageDiagGens + kDiagMulti); i += blockDim.x) (&red[0][0])[i] = 0.0;
    __syncthreads();
    R pm[kDiagMulti];
#pragma unroll
    for (int g = 0; g < kDiagMulti; ++g) pm[g] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto wsum = [&](R v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    auto flush_multi = [&]() {  // warp-uniform
        if (!a.nmulti) return;
#pragma unroll
        for (int g = 0; g < kDiagMulti; ++g) {
            if (g < a.nmulti) {
                const R v = wsum(pm[g]);
                if (lane == 0) red[warp][kStageDiagGens + g] += (double)v;
                pm[g] = 0;
            }
        }
    };
    auto multi = [&](uint64_t x, R v) {
#pragma unroll
        for (int g = 0; g < kDiagMulti; ++g)
            if (g < a.nmulti) pm[g] += (__popcll(x & a.mz[g]) & 1) ? -v : v;
    };
    if (a.n >= 10) {
        const uint64_t nblk = 1ull << (a.n - 10);
        const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
        int cnt = 0;
        for (uint64_t blk = gw; blk < nblk; blk += nw) {
            const uint64_t x0 = (blk << 10) | (uint64_t)lane;
            T H;  // chunk tables 2.. and cross gates on qubits >= 10
            H.x = 1;
            H.y = 0;
            if (a.apply) {
                for (int c = 2; c < a.nchunks; ++c) H = cmul(H, tab[256 * c + ((x0 >> (8 * c)) & 255)]);
                H = cross_phase(a.high, a.nhigh, tab, x0, H);
            }
            R tsum = 0, u0 = 0, u1 = 0, u2 = 0, u3 = 0, u4 = 0;
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const uint64_t x = x0 | ((uint64_t)j << 5);
                const T p = psi[x], l = lam[x];
                const R v = l.x * p.y - l.y * p.x;  // Im(conj(lambda_x) psi_x)
                tsum += v;
                u0 += (j & 1) ? v : (R)0;
                u1 += (j & 2) ? v : (R)0;
                u2 += (j & 4) ? v : (R)0;
                u3 += (j & 8) ? v : (R)0;
                u4 += (j & 16) ? v : (R)0;
                if (a.nmulti) multi(x, v);
                if (a.apply) {
                    T ph = cmul(tab[x & 255], tab[256 + ((x >> 8) & 255)]);
                    ph = cmul(ph, H);
                    ph = cross_phase(a.low, a.nlow, tab, x, ph);
                    psi[x] = cmul(ph, p);
                    lam[x] = cmul(ph, l);
                }
            }
            if (a.nsingle) {
                const R Tt = wsum(tsum);
                const R U[5] = {wsum(u0), wsum(u1), wsum(u2), wsum(u3), wsum(u4)};
                R W[5];
#pragma unroll
                for (int bb = 0; bb < 5; ++bb) W[bb] = wsum(((lane >> bb) & 1) ? tsum : (R)0);
                if (lane == 0) {
                    for (int g = 0; g < a.nsingle; ++g) {
                        const int zb = a.zbit[g];
                        R c;
                        if (zb < 5) {
                            c = zb == 0 ? W[0] : zb == 1 ? W[1] : zb == 2 ? W[2] : zb == 3 ? W[3] : W[4];
                            c = Tt - 2 * c;
                        } else if (zb < 10) {
                            c = zb == 5 ? U[0] : zb == 6 ? U[1] : zb == 7 ? U[2] : zb == 8 ? U[3] : U[4];
                            c = Tt - 2 * c;
                        } else {
                            c = ((blk >> (zb - 10)) & 1) ? -Tt : Tt;
                        }
                        red[warp][g] += (double)c;
                    }
                }
            }
            if (++cnt == 4) {
                flush_multi();
                cnt = 0;
            }
        }
        flush_multi();
    } else {
        const uint64_t N = 1ull << a.n;
        const uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, xs = (uint64_t)gridDim.x * blockDim.x;
        // one-qubit generators first (reads only): each thread sums its
        // amplitudes, the warp reduces, lane 0 adds -- a fixed order
        for (int g = 0; g < a.nsingle; ++g) {
            R acc = 0;
            for (uint64_t x = x0; x < N; x += xs) {
                const T p = psi[x], l = lam[x];
                const R v = l.x * p.y - l.y * p.x;
                acc += ((x >> a.zbit[g]) & 1) ? -v : v;
            }
            acc = wsum(acc);
            if (lane == 0) red[warp][g] += (double)acc;
        }
        for (uint64_t x = x0; x < N; x += xs) {
            const T p = psi[x], l = lam[x];
            const R v = l.x * p.y - l.y * p.x;
            multi(x, v);
            if (a.apply) {
                T ph = tab[x & 255];
                ph = cross_phase(a.low, a.nlow, tab, x, ph);
                ph = cross_phase(a.high, a.nhigh, tab, x, ph);
                psi[x] = cmul(ph, p);
                lam[x] = cmul(ph, l);
            }
        }
        flush_multi();
    }
    __syncthreads();
    for (int g = threadIdx.x; g < a.nsingle + a.nmulti; g += blockDim.x) {
        const int r = g < a.nsingle ? g : kStageDiagGens + (g - a.nsingle);
        const int slot = g < a.nsingle ? a.slot[g] : a.mslot[g - a.nsingle];
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][r];  // fixed order
        partials[((size_t)slot * gridDim.x + blockIdx.x) * 2] = 0.0;
        partials[((size_t)slot * gridDim.x + blockIdx.x) * 2 + 1] = s;
    }
}

}  // namespace

cudaError_t launch_grad_pairs(const void* psi, const void* lam, int n, qs_dtype dt, int L, const int* pos,
                              const std::vector<StageGen>& gens, double* partials, int nblocks, cudaStream_t st) {
    if (gens.empty() || (int)gens.size() > kStageGradGens || L < 1 || L > 12 || L > n) return cudaErrorInvalidValue;
    GradPairsArgs a{};
    a.L = L;
    int b = 0;
    while (b < L && pos[b] == b) ++b;
    a.b = b;
    for (int i = 0; i < L; ++i) a.pos[i] = pos[i];
    a.ntiles = 1ull << (n - L);
    a.ngen = (int)gens.size();
    for (int i = 0; i < a.ngen; ++i) a.g[i] = gens[i];
    if (L < 8) return cudaErrorInvalidValue;  // a tile is at least one element per thread
    const size_t esz = dt == QS_C64 ? 8 : 16;
    const size_t smem = esz * ((size_t)1 << L) + 8 * ((size_t)1 << (L - b));
    auto go = [&](auto kern, auto* p, auto* l) {
        cudaError_t e = allow_max_dynamic_smem(kern);
        if (e != cudaSuccess) return e;
        kern<<<nblocks, 256, smem, st>>>(p, l, a, partials);
        return cudaGetLastError();
    };
    const float2* pf = (const float2*)psi;
    const float2* lf = (const float2*)lam;
    const double2* pd = (const double2*)psi;
    const double2* ld = (const double2*)lam;
    switch (L) {  // elements per thread and tile = 2^L / 256
        case 8: return dt == QS_C64 ? go(k_grad_pairs<float, 1>, pf, lf) : go(k_grad_pairs<double, 1>, pd, ld);
        case 9: return dt == QS_C64 ? go(k_grad_pairs<float, 2>, pf, lf) : go(k_grad_pairs<double, 2>, pd, ld);
        case 10: return dt == QS_C64 ? go(k_grad_pairs<float, 4>, pf, lf) : go(k_grad_pairs<double, 4>, pd, ld);
        case 11: return dt == QS_C64 ? go(k_grad_pairs<float, 8>, pf, lf) : go(k_grad_pairs<double, 8>, pd, ld);
        case 12: return dt == QS_C64 ? go(k_grad_pairs<float, 16>, pf, lf) : go(k_grad_pairs<double, 16>, pd, ld);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_diag_stage(void* psi, void* lam, int n, qs_dtype dt, int nchunks, const std::vector<DiagCross>& cross,
                              const void* dtables, uint32_t tab_elems, const std::vector<uint64_t>& zmasks,
                              const std::vector<int>& slots, bool apply, double* partials, int nblocks,
                              cudaStream_t st) {
    if (zmasks.size() != slots.size() || nchunks < 1 || nchunks > 8 || (apply && tab_elems > kStageDiagTabElems) ||
        (n >= 10 && nchunks < 2))
        return cudaErrorInvalidValue;
    DiagStageArgs a{};
    a.n = n;
    a.nchunks = nchunks;
    a.apply = apply ? 1 : 0;
    a.tab_elems = apply ? tab_elems : 0;
    if (apply)
        for (const DiagCross& c : cross) {
            bool low = false;
            for (int i = 0; i < c.k; ++i) low = low || c.q[i] < 10;
            if (low) {
                if (a.nlow == kStageDiagCross) return cudaErrorInvalidValue;
                a.low[a.nlow++] = c;
            } else {
                if (a.nhigh == kStageDiagCross) return cudaErrorInvalidValue;
                a.high[a.nhigh++] = c;
            }
        }
    for (size_t g = 0; g < zmasks.size(); ++g) {
        if (__builtin_popcountll(zmasks[g]) == 1) {
            if (a.nsingle == kStageDiagGens) return cudaErrorInvalidValue;
            a.zbit[a.nsingle] = __builtin_ctzll(zmasks[g]);
            a.slot[a.nsingle++] = slots[g];
        } else {
            if (a.nmulti == kDiagMulti) return cudaErrorInvalidValue;
            a.mz[a.nmulti] = zmasks[g];
            a.mslot[a.nmulti++] = slots[g];
        }
    }
    const size_t smem = (dt == QS_C64 ? 8 : 16) * (size_t)a.tab_elems;
    if (dt == QS_C64)
        k_diag_stage<float><<<nblocks, 256, smem, st>>>((float2*)psi, (float2*)lam, (const float2*)dtables, a, partials);
    else
        k_diag_stage<double><<<nblocks, 256, smem, st>>>((double2*)psi, (double2*)lam, (const double2*)dtables, a,
                                                         partials);
    return cudaGetLastError();
}

}  // namespace qsgb
