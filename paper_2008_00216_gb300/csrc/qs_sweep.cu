// Fused reverse-sweep pass of the adjoint gradient.
//
// The reverse sweep carries psi and lambda = H psi back through the circuit
// one stage of pairwise-commuting gates at a time; the gradient of gate l,
// U_l = exp(-i theta P_l / 2), is Im <lambda_l|P_l|psi_l> with both states
// taken just after the gate.  When every non-diagonal gate of a stage acts on
// one qubit, a tile of the state that holds that qubit can take the gate's
// gradient and inverse on its own, and a diagonal stage needs only each
// amplitude's index.  So a run of such stages is done in a few read/write
// passes over psi and lambda, each running a program of ops on every tile of
// 2^L amplitudes (qubits pos[0..L-1]) held in registers:
//   G1      one-qubit gate on a register bit: its gradient (generator X, Y
//           or Z), then U^dagger on both states
//   DIAG    a diagonal stage: its Z-generator gradients, then its inverse
//           phase (per-8-qubit chunk tables and gates spanning chunks)
//   LAYOUT  bring other tile bits into registers: both states go through a
//           swizzled shared-memory transpose
// Stage members commute, so each G1's gradient may be taken after the
// inverses of the stage's other members.  Per tile, each gradient is one
// value per thread, staged in shared memory and summed over the block in a
// fixed order (in the state's precision within a tile, FP64 across tiles):
// deterministic.
#include <stdint.h>

#include <algorithm>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsgb {

namespace {

constexpr int kThreads = 256;

// L: tile qubits; 2^SW elements per 128-byte row; ROWS: staged gradients
// (one row of kThreads values each, in the state's precision)
template <typename R> struct SweepShape;
template <> struct SweepShape<float> {
    static constexpr int L = kSweepTileC64, SW = 4, ROWS = 16;
};
template <> struct SweepShape<double> {
    static constexpr int L = kSweepTileC128, SW = 3, ROWS = 8;
};

struct SweepArgs {
    int n, nops, ngrad, nlay, nb;
    uint32_t tab_elems;
    uint64_t ntiles;
    int pos[16];
    int lay_a[kSweepMaxLayouts];
    SweepOpRec ops[kSweepMaxOps];
    SweepDiagRec diag[kSweepMaxDiags];
    DiagCross cross[kSweepMaxCross];
    SweepZGen gens[kSweepMaxGens];
    int slot[kSweepMaxGrads];
};

// Tile index of the thread's first element in the layout starting at a: the
// thread bits fill the tile bits outside [a, a + RB).
template <int RB>
__device__ __forceinline__ uint32_t layout_base(uint32_t t, int a) {
    const uint32_t lo = (1u << a) - 1u;
    return (t & lo) | ((t & ~lo) << RB);
}

// Shared-memory slot of tile element e: the low SW bits are XORed with the
// next SW bits, so every layout's warp access is free of bank conflicts.
template <int SW>
__device__ __forceinline__ uint32_t swz(uint32_t e) {
    return e ^ ((e >> SW) & ((1u << SW) - 1u));
}

template <typename T, int L, int SW>
__device__ __forceinline__ void transpose(T* buf, T (&ps)[1 << (L - 8)], T (&ls)[1 << (L - 8)], int a_from, int a_to) {
    constexpr int RB = L - 8, PER = 1 << RB;
    const uint32_t e0 = layout_base<RB>(threadIdx.x, a_from), e1 = layout_base<RB>(threadIdx.x, a_to);
    __syncthreads();  // earlier readers of buf are done
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t s = swz<SW>(e0 + ((uint32_t)j << a_from));
        buf[s] = ps[j];
        buf[(1u << L) + s] = ls[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t s = swz<SW>(e1 + ((uint32_t)j << a_to));
        ps[j] = buf[s];
        ls[j] = buf[(1u << L) + s];
    }
}

// One-qubit gate on register bit r: gradient Im <l|P|p> of the thread's
// pairs (GEN 1 X, 2 Y, 3 Z), then U^dagger (m, row-major) on both states;
// FORM 1: m is real.
template <typename T, int RB, int r, int FORM, int GEN>
__device__ __forceinline__ auto g1(T (&ps)[1 << RB], T (&ls)[1 << RB], const T* __restrict__ m) {
    using R = decltype(T{}.x);
    const T u00 = m[0], u01 = m[1], u10 = m[2], u11 = m[3];
    R acc = 0;
#pragma unroll
    for (int p = 0; p < (1 << (RB - 1)); ++p) {
        const int j0 = ((p >> r) << (r + 1)) | (p & ((1 << r) - 1));
        const int j1 = j0 | (1 << r);
        const T p0 = ps[j0], p1 = ps[j1], l0 = ls[j0], l1 = ls[j1];
        if (GEN == 1) acc += (l0.x * p1.y - l0.y * p1.x) + (l1.x * p0.y - l1.y * p0.x);
        if (GEN == 2) acc += (l1.x * p0.x + l1.y * p0.y) - (l0.x * p1.x + l0.y * p1.y);
        if (GEN == 3) acc += (l0.x * p0.y - l0.y * p0.x) - (l1.x * p1.y - l1.y * p1.x);
        T q0, q1, k0, k1;
        if (FORM == 1) {
            q0.x = u00.x * p0.x + u01.x * p1.x;
            q0.y = u00.x * p0.y + u01.x * p1.y;
            q1.x = u10.x * p0.x + u11.x * p1.x;
            q1.y = u10.x * p0.y + u11.x * p1.y;
            k0.x = u00.x * l0.x + u01.x * l1.x;
            k0.y = u00.x * l0.y + u01.x * l1.y;
            k1.x = u10.x * l0.x + u11.x * l1.x;
            k1.y = u10.x * l0.y + u11.x * l1.y;
        } else {
            q0 = cmul(u00, p0);
            cmac(q0, u01, p1);
            q1 = cmul(u10, p0);
            cmac(q1, u11, p1);
            k0 = cmul(u00, l0);
            cmac(k0, u01, l1);
            k1 = cmul(u10, l0);
            cmac(k1, u11, l1);
        }
        ps[j0] = q0;
        ps[j1] = q1;
        ls[j0] = k0;
        ls[j1] = k1;
    }
    return acc;
}

template <typename T, int RB, int r>
__device__ __forceinline__ auto g1_form(T (&ps)[1 << RB], T (&ls)[1 << RB], const T* m, int form, int gen) {
    if (form) {
        switch (gen) {
            case 1: return g1<T, RB, r, 1, 1>(ps, ls, m);
            case 2: return g1<T, RB, r, 1, 2>(ps, ls, m);
            case 3: return g1<T, RB, r, 1, 3>(ps, ls, m);
            default: return g1<T, RB, r, 1, 0>(ps, ls, m);
        }
    }
    switch (gen) {
        case 1: return g1<T, RB, r, 0, 1>(ps, ls, m);
        case 2: return g1<T, RB, r, 0, 2>(ps, ls, m);
        case 3: return g1<T, RB, r, 0, 3>(ps, ls, m);
        default: return g1<T, RB, r, 0, 0>(ps, ls, m);
    }
}

template <typename T, int RB>
__device__ __forceinline__ auto g1_any(T (&ps)[1 << RB], T (&ls)[1 << RB], const T* m, int r, int form, int gen) {
    static_assert(RB == 3 || RB == 4, "register bits");
    switch (r) {
        case 0: return g1_form<T, RB, 0>(ps, ls, m, form, gen);
        case 1: return g1_form<T, RB, 1>(ps, ls, m, form, gen);
        case 2: return g1_form<T, RB, 2>(ps, ls, m, form, gen);
        default: return g1_form<T, RB, RB - 1>(ps, ls, m, form, gen);
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads, 2) k_sweep_pass(typename C2<R>::T* __restrict__ psi,
                                                            typename C2<R>::T* __restrict__ lam,
                                                            const typename C2<R>::T* __restrict__ mats,
                                                            const typename C2<R>::T* __restrict__ tabs,
                                                            const __grid_constant__ SweepArgs a,
                                                            double* __restrict__ partials) {
    using T = typename C2<R>::T;
    constexpr int L = SweepShape<R>::L, SW = SweepShape<R>::SW, RB = L - 8, PER = 1 << RB;
    constexpr int kRows = SweepShape<R>::ROWS, TPR = kThreads / kRows;  // threads per staged row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);                                    // 2 x 2^L (psi, lambda)
    T* tab = buf + 2 * (1u << L);                                               // a.tab_elems
    R* gs = reinterpret_cast<R*>(tab + a.tab_elems);                            // kRows x kThreads
    double* red = reinterpret_cast<double*>(gs + kRows * kThreads);             // a.ngrad
    uint64_t* xo = reinterpret_cast<uint64_t*>(red + a.ngrad);                  // a.nlay x PER
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < a.tab_elems; i += kThreads) tab[i] = tabs[i];
    for (int i = tid; i < a.ngrad; i += kThreads) red[i] = 0.0;
    for (int i = tid; i < a.nlay * PER; i += kThreads) {  // global offset of register index j per layout
        const int l = i / PER, j = i % PER;
        uint64_t o = 0;
        for (int k = 0; k < RB; ++k)
            if ((j >> k) & 1) o |= 1ull << a.pos[a.lay_a[l] + k];
        xo[i] = o;
    }
    auto global_of = [&](uint32_t e) {  // tile index -> global offset within the tile
        uint64_t x = 0;
        for (int i = 0; i < L; ++i) x |= (uint64_t)((e >> i) & 1u) << a.pos[i];
        return x;
    };
    const uint64_t xg0 = global_of(layout_base<RB>(tid, a.lay_a[0]));
    __syncthreads();

    int gcount = 0;  // gradients produced so far in this tile
    auto flush = [&](int rows) {  // block-uniform: add the staged rows to red
        __syncthreads();
        const int row = tid / TPR, part = tid % TPR;
        R v = 0;
#pragma unroll
        for (int k = 0; k < kThreads / TPR; ++k) v += gs[row * kThreads + part + TPR * k];
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, TPR);
        if (part == 0 && row < rows) red[gcount - rows + row] += (double)v;
        __syncthreads();
    };
    auto stage = [&](R v) {
        gs[(gcount % kRows) * kThreads + tid] = v;
        ++gcount;
        if (gcount % kRows == 0) flush(kRows);
    };

    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        uint64_t base = tile;
        for (int i = 0; i < L; ++i) base = insert_zero(base, a.pos[i]);
        T ps[PER], ls[PER];
        {
            const uint64_t x0 = base | xg0;
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const uint64_t x = x0 | xo[j];
                ps[j] = psi[x];
                ls[j] = lam[x];
            }
        }
        int lay = 0;
        gcount = 0;
        for (int o = 0; o < a.nops; ++o) {
            const SweepOpRec op = a.ops[o];
            if (op.type == SWEEP_LAYOUT) {
                transpose<T, L, SW>(buf, ps, ls, a.lay_a[lay], a.lay_a[op.arg]);
                lay = op.arg;
            } else if (op.type == SWEEP_G1) {
                const R v = g1_any<T, RB>(ps, ls, mats + 4 * op.idx, op.arg, op.form, op.gen);
                if (op.gen) stage(v);
            } else {
                const SweepDiagRec d = a.diag[op.idx];
                const T* dtab = tab + d.tab;
                const uint64_t xt = base | global_of(layout_base<RB>(tid, a.lay_a[lay]));
                const uint64_t* xl = xo + lay * PER;
                // factors that do not depend on the register index
                T pc;
                pc.x = 1;
                pc.y = 0;
                for (int c = 0; c < d.nchunks; ++c)
                    if (!((d.touched >> c) & 1)) pc = cmul(pc, dtab[256 * c + ((xt >> (8 * c)) & 255)]);
                pc = cross_phase(a.cross + d.cross0 + d.nct, d.ncross - d.nct, tab, xt, pc);
                R tsum = 0, u[RB];
#pragma unroll
                for (int i = 0; i < RB; ++i) u[i] = 0;
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    const R t = ls[j].x * ps[j].y - ls[j].y * ps[j].x;  // Im(conj(l) p)
                    tsum += t;
#pragma unroll
                    for (int i = 0; i < RB; ++i)
                        if ((j >> i) & 1) u[i] += t;
                }
                for (int g = 0; g < d.ngen; ++g) {
                    const SweepZGen z = a.gens[d.gen0 + g];
                    R v;
                    if (z.kind == 0) {
                        v = tsum;
                    } else if (z.kind <= RB) {
                        const int i = z.kind - 1;
                        R ui = u[0];
#pragma unroll
                        for (int k = 1; k < RB; ++k) ui = i == k ? u[k] : ui;
                        v = tsum - 2 * ui;
                    } else {
                        v = 0;
#pragma unroll
                        for (int j = 0; j < PER; ++j) {
                            const R t = ls[j].x * ps[j].y - ls[j].y * ps[j].x;
                            v += ((z.jmask >> j) & 1) ? -t : t;
                        }
                    }
                    stage((__popcll(xt & z.mthr) & 1) ? -v : v);
                }
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    const uint64_t x = xt | xl[j];
                    T ph = pc;
                    for (int c = 0; c < d.nchunks; ++c)
                        if ((d.touched >> c) & 1) ph = cmul(ph, dtab[256 * c + ((x >> (8 * c)) & 255)]);
                    ph = cross_phase(a.cross + d.cross0, d.nct, tab, x, ph);
                    ps[j] = cmul(ph, ps[j]);
                    ls[j] = cmul(ph, ls[j]);
                }
            }
        }
        if (lay != 0) transpose<T, L, SW>(buf, ps, ls, a.lay_a[lay], a.lay_a[0]);
        {
            const uint64_t x0 = base | xg0;
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const uint64_t x = x0 | xo[j];
                psi[x] = ps[j];
                lam[x] = ls[j];
            }
        }
        if (gcount % kRows) flush(gcount % kRows);
    }
    __syncthreads();
    for (int s = tid; s < a.ngrad; s += kThreads) {
        const size_t at = ((size_t)a.slot[s] * a.nb + blockIdx.x) * 2;
        partials[at] = 0.0;
        partials[at + 1] = red[s];
    }
}

template <typename R>
size_t sweep_smem(const SweepArgs& a) {
    constexpr int L = SweepShape<R>::L;
    const size_t esz = sizeof(typename C2<R>::T);
    return esz * (2 * ((size_t)1 << L) + a.tab_elems) + sizeof(R) * SweepShape<R>::ROWS * kThreads +
           sizeof(double) * a.ngrad + sizeof(uint64_t) * a.nlay * ((size_t)1 << (L - 8));
}

}  // namespace

int sweep_layouts(qs_dtype dt, int* lay_a) {
    if (dt == QS_C64) {  // L = 12, 4 register bits: tile bits 8-11, 4-7, 0-3
        lay_a[0] = 8;
        lay_a[1] = 4;
        lay_a[2] = 0;
        return 3;
    }
    lay_a[0] = 8;  // L = 11, 3 register bits: 8-10, 5-7, 2-4, 0-2
    lay_a[1] = 5;
    lay_a[2] = 2;
    lay_a[3] = 0;
    return 4;
}

cudaError_t launch_sweep_pass(void* psi, void* lam, int n, qs_dtype dt, const SweepPassDesc& p, const void* dmats,
                              const void* dtabs, double* partials, int nblocks, cudaStream_t st) {
    const int L = dt == QS_C64 ? kSweepTileC64 : kSweepTileC128, RB = L - 8;
    if (p.L != L || n < L || n > kMaxQubits || p.ops.empty() || (int)p.ops.size() > kSweepMaxOps ||
        (int)p.slots.size() > kSweepMaxGrads || (int)p.diags.size() > kSweepMaxDiags ||
        (int)p.cross.size() > kSweepMaxCross || (int)p.gens.size() > kSweepMaxGens ||
        p.tabs.size() / 2 > sweep_tab_budget(dt) || nblocks < 1)
        return cudaErrorInvalidValue;
    SweepArgs a{};
    a.n = n;
    a.nops = (int)p.ops.size();
    a.ngrad = (int)p.slots.size();
    a.nb = nblocks;
    a.tab_elems = (uint32_t)(p.tabs.size() / 2);
    a.ntiles = 1ull << (n - L);
    int lay[kSweepMaxLayouts];
    a.nlay = sweep_layouts(dt, lay);
    if (p.nlay != a.nlay) return cudaErrorInvalidValue;
    for (int l = 0; l < a.nlay; ++l) {
        if (p.lay_a[l] != lay[l]) return cudaErrorInvalidValue;
        a.lay_a[l] = lay[l];
    }
    // every index the kernel follows is checked here
    for (int i = 0; i < L; ++i) {
        if (p.pos[i] < 0 || p.pos[i] >= n || (i > 0 && p.pos[i] <= p.pos[i - 1])) return cudaErrorInvalidValue;
        a.pos[i] = p.pos[i];
    }
    for (int i = 0; i < 5 && i < L; ++i)  // rows of contiguous amplitudes for the coalesced load
        if (p.pos[i] != i) return cudaErrorInvalidValue;
    const uint32_t nmat = (uint32_t)(p.mats.size() / 8);
    int grads = 0;
    for (int o = 0; o < a.nops; ++o) {
        const SweepOpRec& op = p.ops[o];
        if (op.type == SWEEP_LAYOUT) {
            if (op.arg >= a.nlay) return cudaErrorInvalidValue;
        } else if (op.type == SWEEP_G1) {
            if (op.arg >= RB || op.idx >= nmat || op.gen > 3 || op.form > 1) return cudaErrorInvalidValue;
            grads += op.gen != 0;
        } else if (op.type == SWEEP_DIAG) {
            if (op.idx >= p.diags.size()) return cudaErrorInvalidValue;
            const SweepDiagRec& d = p.diags[op.idx];
            if (d.nchunks < 1 || d.nchunks > 8 || 8 * (d.nchunks - 1) >= n || d.nct > d.ncross ||
                (size_t)d.cross0 + d.ncross > p.cross.size() || (size_t)d.gen0 + d.ngen > p.gens.size() ||
                (size_t)d.tab + 256 * (size_t)d.nchunks > a.tab_elems)
                return cudaErrorInvalidValue;
            for (int g = 0; g < d.ngen; ++g)
                if (p.gens[d.gen0 + g].kind > RB + 1) return cudaErrorInvalidValue;
            grads += d.ngen;
        } else {
            return cudaErrorInvalidValue;
        }
        a.ops[o] = op;
    }
    if (grads != a.ngrad) return cudaErrorInvalidValue;
    for (size_t c = 0; c < p.cross.size(); ++c) {
        const DiagCross& x = p.cross[c];
        if (x.k < 1 || x.k > kMaxK || (size_t)x.tab + (1u << x.k) > a.tab_elems) return cudaErrorInvalidValue;
        for (int i = 0; i < x.k; ++i)
            if (x.q[i] >= n) return cudaErrorInvalidValue;
        a.cross[c] = x;
    }
    for (size_t g = 0; g < p.gens.size(); ++g) a.gens[g] = p.gens[g];
    for (size_t d = 0; d < p.diags.size(); ++d) a.diag[d] = p.diags[d];
    for (int s = 0; s < a.ngrad; ++s) {
        if (p.slots[s] < 0) return cudaErrorInvalidValue;
        a.slot[s] = p.slots[s];
    }
    const int grid = (int)std::min<uint64_t>(a.ntiles, (uint64_t)std::min(nblocks, 2 * num_sms()));
    if (dt == QS_C64) {
        cudaError_t e = allow_max_dynamic_smem(k_sweep_pass<float>);
        if (e != cudaSuccess) return e;
        k_sweep_pass<float><<<grid, kThreads, sweep_smem<float>(a), st>>>(
            (float2*)psi, (float2*)lam, (const float2*)dmats, (const float2*)dtabs, a, partials);
    } else {
        cudaError_t e = allow_max_dynamic_smem(k_sweep_pass<double>);
        if (e != cudaSuccess) return e;
        k_sweep_pass<double><<<grid, kThreads, sweep_smem<double>(a), st>>>(
            (double2*)psi, (double2*)lam, (const double2*)dmats, (const double2*)dtabs, a, partials);
    }
    return cudaGetLastError();
}

}  // namespace qsgb
