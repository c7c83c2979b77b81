// Register tile pass: every gate of a tile pass applied to a 2^L-amplitude
// tile held in registers (the GPU form of the paper's cache blocking,
// Section 5.1: all gates whose qubits lie in the tile before write-back).
//
// A 256-thread block holds the tile as 2^RB amplitudes per thread, L = RB + 8
// (complex64: RB = 4, L = 12; complex128: RB = 3, L = 11).  A layout gives
// the tile bit that each lane bit (5), register bit (RB) and warp bit (3)
// stands for.  The tile is loaded and stored in a layout whose lanes are
// tile bits 0..4 (the lowest physical qubits: coalesced rows).  Ops, from a
// program compiled on the host for the pass:
//   RT_GATE   a k-qubit gate (k = 2..RB) whose qubits are register bits
//             0..k-1: each thread applies it to its own 2^(RB-k) sets
//   RT_GATE1  a one-qubit gate on register bit r: within the thread
//   RT_LANE1  a one-qubit gate on lane bit b: the partner amplitude comes
//             from lane ^ (1 << b) with __shfl_xor_sync
//   RT_DIAG   a diagonal gate on any tile bits: each amplitude's phase from
//             its own index, in any layout (no data movement)
//   RT_LAYOUT the tile moves to another layout through shared memory, in a
//             swizzled order chosen per pass so that every layout's warp
//             accesses are free of bank conflicts
// Multiply-free one-qubit gates (entries in {0, +-1, +-i}; Section 4.1) are
// applied with additions and swaps only.  While a tile is processed, the
// next tile's loads are already in flight into a second register set.
#include <stdint.h>

#include <math.h>

#include <algorithm>
#include <type_traits>

#include "qs_device.cuh"
#include "qs_ff.cuh"
#include "qs_internal.h"
#include "qs_tile.cuh"

namespace qsgb {

namespace {

constexpr int kRTThreads = 256;

struct RTArgs {
    RTProgram p;
    int pos[13];          // tile bit i -> qubit
    uint64_t ntiles;
    uint32_t mat_elems;
    int scale_mode, scale_s;
    double scale_mag, scale_c[2];
};

// Complex64 multiply-accumulate in two packed f32x2 FMAs: with the matrix
// entry stored as e = (m.re, m.re, -m.im, m.im) and the swapped amplitude
// vs = (v.im, v.re), acc += m v is acc += e.xy * v + e.zw * vs componentwise.
__device__ __forceinline__ float2 pmac(float2 acc, const float4& e, float2 v, float2 vs) {
    acc = cfma(make_float2(e.x, e.y), v, acc);
    return cfma(make_float2(e.z, e.w), vs, acc);
}
__device__ __forceinline__ float2 swapri(float2 v) { return make_float2(v.y, v.x); }

// one-qubit gate on register bit r: the pairs (j0, j0 | 1 << r) of a thread
template <typename T, int RB, int r>
__device__ __forceinline__ void rt_gate1(T (&v)[1 << RB], const T* m, const float4* m4, int mulfree) {
    if (mulfree) {
        const int c00 = mulfree_code(m[0]), c01 = mulfree_code(m[1]), c10 = mulfree_code(m[2]), c11 = mulfree_code(m[3]);
#pragma unroll
        for (int p = 0; p < (1 << (RB - 1)); ++p) {
            const int j0 = ((p >> r) << (r + 1)) | (p & ((1 << r) - 1)), j1 = j0 | (1 << r);
            const T x = v[j0], y = v[j1];
            v[j0] = mulfree_sum(x, c00, y, c01);
            v[j1] = mulfree_sum(x, c10, y, c11);
        }
    } else if constexpr (std::is_same<T, float2>::value) {
        const float4 e00 = m4[0], e01 = m4[1], e10 = m4[2], e11 = m4[3];
#pragma unroll
        for (int p = 0; p < (1 << (RB - 1)); ++p) {
            const int j0 = ((p >> r) << (r + 1)) | (p & ((1 << r) - 1)), j1 = j0 | (1 << r);
            const float2 x = v[j0], y = v[j1], xs = swapri(x), ys = swapri(y);
            const float2 z = make_float2(0.f, 0.f);
            v[j0] = pmac(pmac(z, e00, x, xs), e01, y, ys);
            v[j1] = pmac(pmac(z, e10, x, xs), e11, y, ys);
        }
    } else {
        const T m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
#pragma unroll
        for (int p = 0; p < (1 << (RB - 1)); ++p) {
            const int j0 = ((p >> r) << (r + 1)) | (p & ((1 << r) - 1)), j1 = j0 | (1 << r);
            const T x = v[j0], y = v[j1];
            T o0 = cmul(m00, x), o1 = cmul(m10, x);
            cmac(o0, m01, y);
            cmac(o1, m11, y);
            v[j0] = o0;
            v[j1] = o1;
        }
    }
}

template <typename T, int RB>
__device__ __forceinline__ void rt_gate1_any(T (&v)[1 << RB], const T* m, const float4* m4, int r, int mulfree) {
    switch (r) {
        case 0: rt_gate1<T, RB, 0>(v, m, m4, mulfree); break;
        case 1: rt_gate1<T, RB, 1>(v, m, m4, mulfree); break;
        case 2: rt_gate1<T, RB, 2>(v, m, m4, mulfree); break;
        default: rt_gate1<T, RB, RB - 1>(v, m, m4, mulfree); break;
    }
}

// k-qubit gate on register bits 0..k-1 (local index = the element's low k
// bits): each thread applies it to its 2^(RB-k) sets; every matrix entry is
// read once per thread (a broadcast shared-memory load)
template <typename T, int RB, int K>
__device__ __forceinline__ void rt_gate(T (&v)[1 << RB], const T* m, const float4* m4) {
    constexpr int D = 1 << K, S = 1 << (RB - K);
    T nv[1 << RB];
    if constexpr (std::is_same<T, float2>::value) {
        float2 vs[1 << RB];
#pragma unroll
        for (int j = 0; j < (1 << RB); ++j) vs[j] = swapri(v[j]);
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float2 acc[S];
#pragma unroll
            for (int s = 0; s < S; ++s) acc[s] = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < D; ++l) {
                const float4 e = m4[r * D + l];
#pragma unroll
                for (int s = 0; s < S; ++s) acc[s] = pmac(acc[s], e, v[(s << K) | l], vs[(s << K) | l]);
            }
#pragma unroll
            for (int s = 0; s < S; ++s) nv[(s << K) | r] = acc[s];
        }
    } else {
#pragma unroll
        for (int r = 0; r < D; ++r) {
            T acc[S];
#pragma unroll
            for (int s = 0; s < S; ++s) acc[s].x = acc[s].y = 0;
#pragma unroll
            for (int l = 0; l < D; ++l) {
                const T mm = m[r * D + l];
#pragma unroll
                for (int s = 0; s < S; ++s) cmac(acc[s], mm, v[(s << K) | l]);
            }
#pragma unroll
            for (int s = 0; s < S; ++s) nv[(s << K) | r] = acc[s];
        }
    }
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) v[j] = nv[j];
}

template <typename T, int RB>
__device__ __forceinline__ void rt_gate_any(T (&v)[1 << RB], const T* m, const float4* m4, int k) {
    if (k == 2) rt_gate<T, RB, 2>(v, m, m4);
    else if (k == 3) rt_gate<T, RB, 3>(v, m, m4);
    else if constexpr (RB >= 4) rt_gate<T, RB, 4>(v, m, m4);
}

template <typename R, int RB>
__global__ void __launch_bounds__(kRTThreads, 2) k_rtile(typename C2<R>::T* __restrict__ psi,
                                                         const typename C2<R>::T* __restrict__ mats,
                                                         const __grid_constant__ RTArgs a) {
    using T = typename C2<R>::T;
    constexpr int PER = 1 << RB, L = RB + 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);   // 2^L: transposes
    T* smat = buf + (1u << L);                 // the pass's matrices
    // complex64: the matrices again as packed-FMA operands (re, re, -im, im)
    float4* smat4 = reinterpret_cast<float4*>(smat + ((a.mat_elems + 1) & ~1u));
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    for (uint32_t i = tid; i < a.mat_elems; i += kRTThreads) {
        const T m = mats[i];
        smat[i] = m;
        if constexpr (std::is_same<T, float2>::value) smat4[i] = make_float4(m.x, m.x, -m.y, m.y);
    }
    __syncthreads();

    // tile bits of this thread's lane and warp in a layout
    auto ebase = [&](const RTLayout& ly) {
        uint32_t e = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) e |= (uint32_t)((lane >> i) & 1) << ly.lane[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) e |= (uint32_t)((wp >> i) & 1) << ly.warp[i];
        return e;
    };
    auto pos_of = [&](uint32_t e) {
        uint32_t p = 0;
#pragma unroll
        for (int i = 0; i < L; ++i) p ^= ((e >> i) & 1) ? (uint32_t)a.p.poscol[i] : 0u;
        return p;
    };
    auto phys_of = [&](uint32_t e) {
        uint64_t x = 0;
#pragma unroll
        for (int i = 0; i < L; ++i) x |= (uint64_t)((e >> i) & 1) << a.pos[i];
        return x;
    };
    // HBM offsets of a thread's elements in layout ly for a tile
    auto tile_base = [&](uint64_t tile) {
        uint64_t base = tile;
#pragma unroll
        for (int i = 0; i < L; ++i) base = insert_zero(base, a.pos[i]);
        return base;
    };
    const RTLayout& ld = a.p.lay[a.p.load_lay];
    const RTLayout& stl = a.p.lay[a.p.store_lay];
    const uint64_t ld_thr = phys_of(ebase(ld)), st_thr = phys_of(ebase(stl));
    uint64_t ld_col[RB], st_col[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) {
        ld_col[i] = 1ull << a.pos[ld.reg[i]];
        st_col[i] = 1ull << a.pos[stl.reg[i]];
    }
    auto gload = [&](T (&v)[PER], uint64_t tile) {
        const uint64_t b = tile_base(tile) | ld_thr;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            uint64_t o = b;
#pragma unroll
            for (int i = 0; i < RB; ++i) o |= ((j >> i) & 1) ? ld_col[i] : 0ull;
            v[j] = psi[o];
        }
    };

    T cur[PER], nxt[PER];
    uint64_t tile = blockIdx.x;
    if (tile < a.ntiles) gload(cur, tile);
    for (; tile < a.ntiles; tile += gridDim.x) {
        const uint64_t tnext = tile + gridDim.x;
        if (tnext < a.ntiles) gload(nxt, tnext);   // in flight while this tile is processed
        int lay = a.p.load_lay;
        for (int o = 0; o < a.p.nops; ++o) {
            const RTOp& op = a.p.ops[o];
            if (op.type == RT_LAYOUT) {
                const RTLayout& A = a.p.lay[lay];
                const RTLayout& Bl = a.p.lay[op.arg];
                __syncthreads();  // earlier readers of buf are done
                {
                    const uint32_t pb = pos_of(ebase(A));
                    uint32_t pc[RB];
#pragma unroll
                    for (int i = 0; i < RB; ++i) pc[i] = a.p.poscol[A.reg[i]];
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        uint32_t p = pb;
#pragma unroll
                        for (int i = 0; i < RB; ++i) p ^= ((j >> i) & 1) ? pc[i] : 0u;
                        buf[p] = cur[j];
                    }
                }
                __syncthreads();
                {
                    const uint32_t pb = pos_of(ebase(Bl));
                    uint32_t pc[RB];
#pragma unroll
                    for (int i = 0; i < RB; ++i) pc[i] = a.p.poscol[Bl.reg[i]];
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        uint32_t p = pb;
#pragma unroll
                        for (int i = 0; i < RB; ++i) p ^= ((j >> i) & 1) ? pc[i] : 0u;
                        cur[j] = buf[p];
                    }
                }
                lay = op.arg;
            } else if (op.type == RT_DIAG) {
                // local index = its lane/warp part | its register part
                const RTLayout& ly = a.p.lay[lay];
                const int k = op.k, D = 1 << k;
                const uint32_t e0 = ebase(ly);
                uint32_t lb = 0;
                for (int i = 0; i < k; ++i) lb |= ((e0 >> op.q[i]) & 1u) << (k - 1 - i);
                uint32_t cm[RB];
#pragma unroll
                for (int m = 0; m < RB; ++m) {
                    cm[m] = 0;
                    for (int i = 0; i < k; ++i)
                        if (ly.reg[m] == op.q[i]) cm[m] = 1u << (k - 1 - i);
                }
                const T* dm = smat + op.mat;
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    uint32_t l = lb;
#pragma unroll
                    for (int m = 0; m < RB; ++m) l |= ((j >> m) & 1) ? cm[m] : 0u;
                    cur[j] = cmul(dm[l * (uint32_t)(D + 1)], cur[j]);
                }
            } else if (op.type == RT_LANE1) {
                const T* m = smat + op.mat;
                const int b = op.arg, sel = (lane >> b) & 1;
                if (op.mulfree) {
                    // out_sel = u[sel][sel] own + u[sel][1-sel] partner, each a phase i^c or 0
                    const int co = mulfree_code(m[sel * 3]), cp = mulfree_code(m[sel ? 2 : 1]);
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        T pv;
                        pv.x = __shfl_xor_sync(0xffffffffu, cur[j].x, 1 << b);
                        pv.y = __shfl_xor_sync(0xffffffffu, cur[j].y, 1 << b);
                        cur[j] = mulfree_sum(cur[j], co, pv, cp);
                    }
                } else if constexpr (std::is_same<T, float2>::value) {
                    const float4 eo = smat4[op.mat + sel * 3], ep = smat4[op.mat + (sel ? 2 : 1)];
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        float2 pv;
                        pv.x = __shfl_xor_sync(0xffffffffu, cur[j].x, 1 << b);
                        pv.y = __shfl_xor_sync(0xffffffffu, cur[j].y, 1 << b);
                        cur[j] = pmac(pmac(make_float2(0.f, 0.f), eo, cur[j], swapri(cur[j])), ep, pv, swapri(pv));
                    }
                } else {
                    const T co = m[sel * 3], cp = m[sel ? 2 : 1];
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        T pv;
                        pv.x = __shfl_xor_sync(0xffffffffu, cur[j].x, 1 << b);
                        pv.y = __shfl_xor_sync(0xffffffffu, cur[j].y, 1 << b);
                        T out = cmul(co, cur[j]);
                        cmac(out, cp, pv);
                        cur[j] = out;
                    }
                }
            } else if (op.type == RT_GATE1) {
                rt_gate1_any<T, RB>(cur, smat + op.mat, smat4 + op.mat, op.arg, op.mulfree);
            } else {  // RT_GATE, k = 2..RB
                rt_gate_any<T, RB>(cur, smat + op.mat, smat4 + op.mat, op.k);
            }
        }
        // store in the store layout (lanes = tile bits 0..4), with the scalar
        // factored out of the pass's multiply-free gates
        {
            const uint64_t b = tile_base(tile) | st_thr;
            const R mag = (R)a.scale_mag;
            T c;
            c.x = (R)a.scale_c[0];
            c.y = (R)a.scale_c[1];
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                uint64_t o = b;
#pragma unroll
                for (int i = 0; i < RB; ++i) o |= ((j >> i) & 1) ? st_col[i] : 0ull;
                T v = cur[j];
                if (a.scale_mode == 1) {
                    v = rot_i(v, a.scale_s >> 1);
                    if (a.scale_s & 1) {  // times (1 + i) (the 1/sqrt(2) is in mag)
                        const R re = v.x - v.y, im = v.x + v.y;
                        v.x = re;
                        v.y = im;
                    }
                    v.x *= mag;
                    v.y *= mag;
                } else if (a.scale_mode == 2) {
                    v = cmul(c, v);
                }
                psi[o] = v;
            }
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) cur[j] = nxt[j];
    }
}

// ---------------------------------------------------------------- complex128
// (float-float helpers: qs_ff.cuh)


template <int RB, int r>
__device__ __forceinline__ void ff_gate1(FFC (&v)[1 << RB], const FFC* m, int mulfree) {
#pragma unroll
    for (int p = 0; p < (1 << (RB - 1)); ++p) {
        const int j0 = ((p >> r) << (r + 1)) | (p & ((1 << r) - 1)), j1 = j0 | (1 << r);
        const FFC x = v[j0], y = v[j1];
        if (mulfree) {
            const int c00 = mulfree_code(m[0].h), c01 = mulfree_code(m[1].h), c10 = mulfree_code(m[2].h),
                      c11 = mulfree_code(m[3].h);
            v[j0] = ff_mulfree_sum(x, c00, y, c01);
            v[j1] = ff_mulfree_sum(x, c10, y, c11);
        } else {
            v[j0] = ff_cmac2(m[0], x, m[1], y);
            v[j1] = ff_cmac2(m[2], x, m[3], y);
        }
    }
}
// A k-qubit gate (k = 2..RB) on register bits 0..k-1.  Its rows run in a
// loop that is not unrolled (unrolled, the gate sizes together overflowed the
// instruction cache and instruction fetch became the top stall); each row's
// outputs go to the thread's own scratch slots in shared memory, read back
// once the gate is done.
template <int RB, int K>
__device__ __forceinline__ void ff_gate(FFC (&v)[1 << RB], const FFC* m, float4* scr) {
    constexpr int D = 1 << K, S = 1 << (RB - K);
#pragma unroll 1
    for (int r = 0; r < D; ++r) {
        FFAcc acc[S];
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = ffa_zero();
        const FFC* mr = m + r * D;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            const FFC mm = mr[l];
#pragma unroll
            for (int s = 0; s < S; ++s) ffa_cmac(acc[s], mm, v[(s << K) | l]);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const FFC o = ffa_get(acc[s]);
            scr[((s << K) | r) * kRTThreads] = make_float4(o.h.x, o.h.y, o.l.x, o.l.y);
        }
    }
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
        const float4 w = scr[j * kRTThreads];
        v[j].h = make_float2(w.x, w.y);
        v[j].l = make_float2(w.z, w.w);
    }
}

template <int RB>
__global__ void __launch_bounds__(kRTThreads, 2) k_rtile_ff(double2* __restrict__ psi, const double2* __restrict__ mats,
                                                            const __grid_constant__ RTArgs a) {
    constexpr int PER = 1 << RB, L = RB + 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* buf = reinterpret_cast<float4*>(smem_raw);            // 2^L: transposes, (h.x, h.y, l.x, l.y)
    float4* scr = buf + (1u << L) + threadIdx.x;                  // PER x kRTThreads: this thread's gate outputs
    FFC* smat = reinterpret_cast<FFC*>(buf + (1u << L) + PER * kRTThreads);   // the pass's matrices, float-float
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    for (uint32_t i = tid; i < a.mat_elems; i += kRTThreads) smat[i] = ff_from(mats[i]);
    __syncthreads();
    auto ebase = [&](const RTLayout& ly) {
        uint32_t e = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) e |= (uint32_t)((lane >> i) & 1) << ly.lane[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) e |= (uint32_t)((wp >> i) & 1) << ly.warp[i];
        return e;
    };
    auto pos_of = [&](uint32_t e) {
        uint32_t p = 0;
#pragma unroll
        for (int i = 0; i < L; ++i) p ^= ((e >> i) & 1) ? (uint32_t)a.p.poscol[i] : 0u;
        return p;
    };
    auto phys_of = [&](uint32_t e) {
        uint64_t x = 0;
#pragma unroll
        for (int i = 0; i < L; ++i) x |= (uint64_t)((e >> i) & 1) << a.pos[i];
        return x;
    };
    auto tile_base = [&](uint64_t tile) {
        uint64_t base = tile;
#pragma unroll
        for (int i = 0; i < L; ++i) base = insert_zero(base, a.pos[i]);
        return base;
    };
    const RTLayout& ld = a.p.lay[a.p.load_lay];
    const RTLayout& stl = a.p.lay[a.p.store_lay];
    const uint64_t ld_thr = phys_of(ebase(ld)), st_thr = phys_of(ebase(stl));
    uint64_t ld_col[RB], st_col[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) {
        ld_col[i] = 1ull << a.pos[ld.reg[i]];
        st_col[i] = 1ull << a.pos[stl.reg[i]];
    }
    auto gload = [&](double2 (&v)[PER], uint64_t tile) {
        const uint64_t b = tile_base(tile) | ld_thr;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            uint64_t o = b;
#pragma unroll
            for (int i = 0; i < RB; ++i) o |= ((j >> i) & 1) ? ld_col[i] : 0ull;
            v[j] = psi[o];
        }
    };
    // the scalar factored out of the pass's multiply-free gates, as float-float
    FFC scale;
    scale.h = make_float2(1.f, 0.f);
    scale.l = make_float2(0.f, 0.f);
    if (a.scale_mode) scale = ff_from(make_double2(a.scale_c[0], a.scale_c[1]));

    double2 nxt[PER];
    FFC cur[PER];
    uint64_t tile = blockIdx.x;
    if (tile < a.ntiles) gload(nxt, tile);
    for (; tile < a.ntiles; tile += gridDim.x) {
#pragma unroll
        for (int j = 0; j < PER; ++j) cur[j] = ff_from(nxt[j]);
        const uint64_t tnext = tile + gridDim.x;
        if (tnext < a.ntiles) gload(nxt, tnext);   // in flight while this tile is processed
        int lay = a.p.load_lay;
        for (int o = 0; o < a.p.nops; ++o) {
            const RTOp& op = a.p.ops[o];
            if (op.type == RT_LAYOUT) {
                const RTLayout& A = a.p.lay[lay];
                const RTLayout& Bl = a.p.lay[op.arg];
                __syncthreads();
                {
                    const uint32_t pb = pos_of(ebase(A));
                    uint32_t pc[RB];
#pragma unroll
                    for (int i = 0; i < RB; ++i) pc[i] = a.p.poscol[A.reg[i]];
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        uint32_t p = pb;
#pragma unroll
                        for (int i = 0; i < RB; ++i) p ^= ((j >> i) & 1) ? pc[i] : 0u;
                        buf[p] = make_float4(cur[j].h.x, cur[j].h.y, cur[j].l.x, cur[j].l.y);
                    }
                }
                __syncthreads();
                {
                    const uint32_t pb = pos_of(ebase(Bl));
                    uint32_t pc[RB];
#pragma unroll
                    for (int i = 0; i < RB; ++i) pc[i] = a.p.poscol[Bl.reg[i]];
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        uint32_t p = pb;
#pragma unroll
                        for (int i = 0; i < RB; ++i) p ^= ((j >> i) & 1) ? pc[i] : 0u;
                        const float4 w = buf[p];
                        cur[j].h = make_float2(w.x, w.y);
                        cur[j].l = make_float2(w.z, w.w);
                    }
                }
                lay = op.arg;
            } else if (op.type == RT_DIAG) {
                const RTLayout& ly = a.p.lay[lay];
                const int k = op.k, D = 1 << k;
                const uint32_t e0 = ebase(ly);
                uint32_t lb = 0;
                for (int i = 0; i < k; ++i) lb |= ((e0 >> op.q[i]) & 1u) << (k - 1 - i);
                uint32_t cm[RB];
#pragma unroll
                for (int m = 0; m < RB; ++m) {
                    cm[m] = 0;
                    for (int i = 0; i < k; ++i)
                        if (ly.reg[m] == op.q[i]) cm[m] = 1u << (k - 1 - i);
                }
                const FFC* dm = smat + op.mat;
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    uint32_t l = lb;
#pragma unroll
                    for (int m = 0; m < RB; ++m) l |= ((j >> m) & 1) ? cm[m] : 0u;
                    cur[j] = ff_cmul(dm[l * (uint32_t)(D + 1)], cur[j]);
                }
            } else if (op.type == RT_LANE1) {
                const FFC* m = smat + op.mat;
                const int b = op.arg, sel = (lane >> b) & 1;
                const FFC co = m[sel * 3], cp = m[sel ? 2 : 1];
                if (op.mulfree) {
                    const int ko = mulfree_code(co.h), kp = mulfree_code(cp.h);
#pragma unroll
                    for (int j = 0; j < PER; ++j) cur[j] = ff_mulfree_sum(cur[j], ko, ff_shfl_xor(cur[j], 1 << b), kp);
                } else {
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        const FFC pv = ff_shfl_xor(cur[j], 1 << b);
                        cur[j] = ff_cmac2(co, cur[j], cp, pv);
                    }
                }
            } else if (op.type == RT_GATE1) {
                const FFC* m = smat + op.mat;
                switch (op.arg) {
                    case 0: ff_gate1<RB, 0>(cur, m, op.mulfree); break;
                    case 1: ff_gate1<RB, 1>(cur, m, op.mulfree); break;
                    default: ff_gate1<RB, RB - 1>(cur, m, op.mulfree); break;
                }
            } else {  // RT_GATE, k = 2..RB
                if (op.k == 2) ff_gate<RB, 2>(cur, smat + op.mat, scr);
                else ff_gate<RB, 3>(cur, smat + op.mat, scr);
            }
        }
        const uint64_t b = tile_base(tile) | st_thr;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            uint64_t o = b;
#pragma unroll
            for (int i = 0; i < RB; ++i) o |= ((j >> i) & 1) ? st_col[i] : 0ull;
            psi[o] = ff_to(a.scale_mode ? ff_cmul(scale, cur[j]) : cur[j]);
        }
    }
}

template <typename R, int RB>
cudaError_t run_rtile(void* psi, const RTArgs& a, const void* dmats, cudaStream_t st) {
    using T = typename C2<R>::T;
    const size_t smem = sizeof(T) * (((size_t)1 << (RB + 8)) + ((a.mat_elems + 1) & ~1u)) +
                        (std::is_same<T, float2>::value ? sizeof(float4) * a.mat_elems : 0);
    cudaError_t e = allow_max_dynamic_smem(k_rtile<R, RB>);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<uint64_t>(a.ntiles, (uint64_t)num_sms() * 2);
    k_rtile<R, RB><<<grid, kRTThreads, smem, st>>>((T*)psi, (const T*)dmats, a);
    return cudaGetLastError();
}

}  // namespace

int rtile_bits(qs_dtype dt) { return dt == QS_C64 ? 12 : 11; }

cudaError_t launch_rtile(void* psi, int n, qs_dtype dt, const Pass& ps, const void* dmats, cudaStream_t st) {
    const int L = rtile_bits(dt);
    if (ps.L != L || n < L || ps.rt.nops < 1 || ps.rt.nops > kRTMaxOps || ps.rt.nlay < 1) return cudaErrorInvalidValue;
    RTArgs a{};
    a.p = ps.rt;
    for (int i = 0; i < L; ++i) a.pos[i] = ps.pos[i];
    a.ntiles = 1ull << (n - L);
    a.mat_elems = (uint32_t)(ps.mats.size() / 2);
    a.scale_mode = ps.scale_mode;
    a.scale_s = ps.scale_s;
    a.scale_mag = ps.scale_mag * ((ps.scale_s & 1) ? 0.70710678118654752440 : 1.0);
    a.scale_c[0] = ps.scale_c[0];
    a.scale_c[1] = ps.scale_c[1];
    if (dt == QS_C64) return run_rtile<float, 4>(psi, a, dmats, st);
    // complex128: float-float arithmetic; the scale as one complex factor
    if (a.scale_mode == 1) {
        const double ang = 0.78539816339744830962 * (double)a.scale_s;   // pi/4 per step
        const double mag = ps.scale_mag;
        a.scale_c[0] = mag * cos(ang);
        a.scale_c[1] = mag * sin(ang);
        a.scale_mode = 2;
    }
    const size_t smem = 16 * ((size_t)1 << 11) + 16 * (size_t)8 * kRTThreads + 16 * (size_t)a.mat_elems;
    cudaError_t e = allow_max_dynamic_smem(k_rtile_ff<3>);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<uint64_t>(a.ntiles, (uint64_t)num_sms() * 2);
    k_rtile_ff<3><<<grid, kRTThreads, smem, st>>>((double2*)psi, (const double2*)dmats, a);
    return cudaGetLastError();
}

}  // namespace qsgb
