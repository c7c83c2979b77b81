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
// (one row of kThreads values each, in the state's precision); LAY: the
// register layouts (start of the register range), 0 natural, the last one
// "low" (registers hold qubits 0 .. L-9, where diagonal ops run).
template <typename R> struct SweepShape;
template <> struct SweepShape<float> {
    static constexpr int L = kSweepTileC64, SW = 4, ROWS = 16, NLAY = 3;
    __host__ __device__ static constexpr int lay(int l) { return l == 0 ? 8 : l == 1 ? 4 : 0; }
};
template <> struct SweepShape<double> {
    static constexpr int L = kSweepTileC128, SW = 3, ROWS = 8, NLAY = 4;
    __host__ __device__ static constexpr int lay(int l) { return l == 0 ? 8 : l == 1 ? 5 : l == 2 ? 2 : 0; }
};

struct SweepArgs {
    int n, nops, ngrad, nb, nmat;
    uint32_t tab_elems;
    uint64_t ntiles;
    int pos[16];
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
// next SW bits, so every layout's warp access is free of bank conflicts.  The
// map is linear over XOR, and a thread's elements are e0 | (j << a) with
// disjoint bits, so slot = swz(e0) ^ swz(j << a): one XOR with a constant.
template <int SW>
__host__ __device__ constexpr uint32_t swz(uint32_t e) {
    return e ^ ((e >> SW) & ((1u << SW) - 1u));
}

template <typename T, int L, int SW, int AF, int AT>
__device__ __forceinline__ void transpose_ct(T* buf, T (&ps)[1 << (L - 8)], T (&ls)[1 << (L - 8)]) {
    constexpr int RB = L - 8, PER = 1 << RB;
    const uint32_t s0 = swz<SW>(layout_base<RB>(threadIdx.x, AF)), s1 = swz<SW>(layout_base<RB>(threadIdx.x, AT));
    __syncthreads();  // earlier readers of buf are done
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t s = s0 ^ swz<SW>((uint32_t)j << AF);
        buf[s] = ps[j];
        buf[(1u << L) + s] = ls[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t s = s1 ^ swz<SW>((uint32_t)j << AT);
        ps[j] = buf[s];
        ls[j] = buf[(1u << L) + s];
    }
}

template <typename R, int F>
__device__ __forceinline__ void transpose_from(typename C2<R>::T* buf, typename C2<R>::T (&ps)[1 << (SweepShape<R>::L - 8)],
                                               typename C2<R>::T (&ls)[1 << (SweepShape<R>::L - 8)], int to) {
    using S = SweepShape<R>;
    using T = typename C2<R>::T;
    switch (to) {
        case 0: transpose_ct<T, S::L, S::SW, S::lay(F), S::lay(0)>(buf, ps, ls); break;
        case 1: transpose_ct<T, S::L, S::SW, S::lay(F), S::lay(1)>(buf, ps, ls); break;
        case 2: transpose_ct<T, S::L, S::SW, S::lay(F), S::lay(2)>(buf, ps, ls); break;
        default: transpose_ct<T, S::L, S::SW, S::lay(F), S::lay(S::NLAY - 1)>(buf, ps, ls); break;
    }
}

template <typename R>
__device__ __forceinline__ void transpose_any(typename C2<R>::T* buf, typename C2<R>::T (&ps)[1 << (SweepShape<R>::L - 8)],
                                              typename C2<R>::T (&ls)[1 << (SweepShape<R>::L - 8)], int from, int to) {
    switch (from) {
        case 0: transpose_from<R, 0>(buf, ps, ls, to); break;
        case 1: transpose_from<R, 1>(buf, ps, ls, to); break;
        case 2: transpose_from<R, 2>(buf, ps, ls, to); break;
        default: transpose_from<R, SweepShape<R>::NLAY - 1>(buf, ps, ls, to); break;
    }
}

// sum over the pair of componentwise products: acc += x * y (both lanes)
template <typename T>
__device__ __forceinline__ T dot2(T acc, T x, T y) { return cfma(x, y, acc); }

// complex p += t q, in place
template <typename T, typename C>
__device__ __forceinline__ void shear(T& p, C t, T q) {
    p.x = fma(t.x, q.x, p.x);
    p.x = fma(-t.y, q.y, p.x);
    p.y = fma(t.x, q.y, p.y);
    p.y = fma(t.y, q.x, p.y);
}
// real t (both lanes (t, t)): p += t q, in place
template <typename T>
__device__ __forceinline__ void rshear(T& p, T t, T q) { p = cfma(t, q, p); }

// One-qubit op on register bit r (form V, SweepG1Form): the gradient
// Im <l|P|p> over the thread's pairs, then U^dagger on both states.
template <typename T, int RB, int r, int V>
__device__ __forceinline__ auto g1(T (&ps)[1 << RB], T (&ls)[1 << RB], const T* __restrict__ m, int gen) {
    using R = decltype(T{}.x);
    const T m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3];
    T t0, t1, t2;  // real shears: (z, z), (y, y), (x, x)
    t0.x = t0.y = m0.x;
    t1.x = t1.y = m1.x;
    t2.x = t2.y = m2.x;
    R acc = 0;
    T ya, yb;  // generator Y: sum l1 * p0 and sum l0 * p1, componentwise
    ya.x = ya.y = yb.x = yb.y = 0;
#pragma unroll
    for (int p = 0; p < (1 << (RB - 1)); ++p) {
        const int j0 = ((p >> r) << (r + 1)) | (p & ((1 << r) - 1));
        const int j1 = j0 | (1 << r);
        T& p0 = ps[j0];
        T& p1 = ps[j1];
        T& l0 = ls[j0];
        T& l1 = ls[j1];
        if (V == G1_RSHEAR_Y || (V == G1_DIRECT && gen == 2)) {  // Re(conj(l1) p0) - Re(conj(l0) p1)
            ya = dot2(ya, l1, p0);
            yb = dot2(yb, l0, p1);
        }
        if (V == G1_CSHEAR_X || (V == G1_DIRECT && gen == 1))
            acc += (l0.x * p1.y - l0.y * p1.x) + (l1.x * p0.y - l1.y * p0.x);
        if (V == G1_DIRECT && gen == 3) acc += (l0.x * p0.y - l0.y * p0.x) - (l1.x * p1.y - l1.y * p1.x);
        if (V == G1_RSHEAR || V == G1_RSHEAR_Y || V == G1_RSHEAR_NEG) {
            if (V == G1_RSHEAR_NEG) {
                p1.x = -p1.x;
                p1.y = -p1.y;
                l1.x = -l1.x;
                l1.y = -l1.y;
            }
            rshear(p0, t0, p1);
            rshear(p1, t1, p0);
            rshear(p0, t2, p1);
            rshear(l0, t0, l1);
            rshear(l1, t1, l0);
            rshear(l0, t2, l1);
        } else if (V == G1_CSHEAR || V == G1_CSHEAR_X) {
            shear(p0, m0, p1);
            shear(p1, m1, p0);
            shear(p0, m2, p1);
            shear(l0, m0, l1);
            shear(l1, m1, l0);
            shear(l0, m2, l1);
        } else {
            T q0 = cmul(m0, p0), q1 = cmul(m2, p0), k0 = cmul(m0, l0), k1 = cmul(m2, l0);
            cmac(q0, m1, p1);
            cmac(q1, m3, p1);
            cmac(k0, m1, l1);
            cmac(k1, m3, l1);
            p0 = q0;
            p1 = q1;
            l0 = k0;
            l1 = k1;
        }
    }
    if (V == G1_RSHEAR_Y || (V == G1_DIRECT && gen == 2)) acc = (ya.x + ya.y) - (yb.x + yb.y);
    return acc;
}

template <typename T, int RB, int r>
__device__ __forceinline__ auto g1_form(T (&ps)[1 << RB], T (&ls)[1 << RB], const T* m, int form, int gen) {
    switch (form) {
        case G1_RSHEAR: return g1<T, RB, r, G1_RSHEAR>(ps, ls, m, gen);
        case G1_RSHEAR_Y: return g1<T, RB, r, G1_RSHEAR_Y>(ps, ls, m, gen);
        case G1_RSHEAR_NEG: return g1<T, RB, r, G1_RSHEAR_NEG>(ps, ls, m, gen);
        case G1_CSHEAR: return g1<T, RB, r, G1_CSHEAR>(ps, ls, m, gen);
        case G1_CSHEAR_X: return g1<T, RB, r, G1_CSHEAR_X>(ps, ls, m, gen);
        default: return g1<T, RB, r, G1_DIRECT>(ps, ls, m, gen);
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
    using S = SweepShape<R>;
    constexpr int L = S::L, RB = L - 8, PER = 1 << RB, LOW = S::NLAY - 1;
    constexpr int kRows = S::ROWS, TPR = kThreads / kRows;  // threads per staged row
    static_assert(S::lay(0) == L - RB && S::lay(LOW) == 0, "layouts");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);                                    // 2 x 2^L (psi, lambda)
    T* tab = buf + 2 * (1u << L);                                               // a.tab_elems
    R* gs = reinterpret_cast<R*>(tab + a.tab_elems);                            // kRows x kThreads
    double* red = reinterpret_cast<double*>(gs + kRows * kThreads);             // a.ngrad (even count: 16-byte alignment below)
    uint64_t* xo = reinterpret_cast<uint64_t*>(red + ((a.ngrad + 1) & ~1));    // PER: byte offset of j
    R* dred = reinterpret_cast<R*>(xo + PER);                                   // 8 warps x (6 + RB)
    T* cm = reinterpret_cast<T*>(dred + (kThreads / 32) * (6 + RB));            // 4 x a.nmat coefficients
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < a.tab_elems; i += kThreads) tab[i] = tabs[i];
    for (int i = tid; i < 4 * a.nmat; i += kThreads) cm[i] = mats[i];
    for (int i = tid; i < a.ngrad; i += kThreads) red[i] = 0.0;
    if (tid < PER) {  // natural layout: register bit k is tile bit L - RB + k
        uint64_t o = 0;
        for (int k = 0; k < RB; ++k)
            if ((tid >> k) & 1) o |= 1ull << a.pos[L - RB + k];
        xo[tid] = o * sizeof(T);
    }
    auto global_of = [&](uint32_t e) {  // tile index -> global offset within the tile
        uint64_t x = 0;
        for (int i = 0; i < L; ++i) x |= (uint64_t)((e >> i) & 1u) << a.pos[i];
        return x;
    };
    const uint64_t xg0 = global_of(layout_base<RB>(tid, S::lay(0)));  // the thread's bits, natural layout
    __syncthreads();

    int gdone = 0, srow = 0;  // gradients of this tile already added to red; rows staged since
    auto flush = [&]() {  // block-uniform: add the staged rows to red
        __syncthreads();
        const int row = tid / TPR, part = tid % TPR;
        R v = 0;
#pragma unroll
        for (int k = 0; k < kThreads / TPR; ++k) v += gs[row * kThreads + part + TPR * k];
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, TPR);
        if (part == 0 && row < srow) red[gdone + row] += (double)v;
        gdone += srow;
        srow = 0;
        __syncthreads();
    };
    auto stage = [&](R v) {
        gs[srow * kThreads + tid] = v;
        if (++srow == kRows) flush();
    };

    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        uint64_t base = tile;
        for (int i = 0; i < L; ++i) base = insert_zero(base, a.pos[i]);
        T ps[PER], ls[PER];
        {
            const char* pp = reinterpret_cast<const char*>(psi) + (base | xg0) * sizeof(T);
            const char* pl = reinterpret_cast<const char*>(lam) + (base | xg0) * sizeof(T);
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const uint64_t o = xo[j];
                ps[j] = *reinterpret_cast<const T*>(pp + o);
                ls[j] = *reinterpret_cast<const T*>(pl + o);
            }
        }
        // the next tile of psi and lambda on its way into L2 while this one is processed
        if (tile + gridDim.x < a.ntiles) {
            uint64_t nb = tile + gridDim.x;
            for (int i = 0; i < L; ++i) nb = insert_zero(nb, a.pos[i]);
            const char* pp = reinterpret_cast<const char*>(psi) + (nb | xg0) * sizeof(T);
            const char* pl = reinterpret_cast<const char*>(lam) + (nb | xg0) * sizeof(T);
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pp + xo[j]));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pl + xo[j]));
            }
        }
        int lay = 0;
        gdone = 0;
        for (int o = 0; o < a.nops; ++o) {
            const SweepOpRec op = a.ops[o];
            if (op.type == SWEEP_LAYOUT) {
                transpose_any<R>(buf, ps, ls, lay, op.arg);
                lay = op.arg;
            } else if (op.type == SWEEP_G1) {
                const R v = g1_any<T, RB>(ps, ls, cm + 4 * op.idx, op.arg, op.form, op.gen);
                if (op.gen) stage(v);
            } else {  // DIAG, in the low layout: register index j = bits 0 .. RB-1 of the index
                const SweepDiagRec d = a.diag[op.idx];
                const T* dtab = tab + d.tab;
                const uint64_t xt = base | global_of(layout_base<RB>(tid, 0));
                T pc;  // chunks 1.. and the cross gates without a register qubit
                pc.x = 1;
                pc.y = 0;
                for (int c = 1; c < d.nchunks; ++c) pc = cmul(pc, dtab[256 * c + ((xt >> (8 * c)) & 255)]);
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
                for (int g = 0; g < d.nstaged; ++g) {
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
                if (d.ngen > d.nstaged) {  // block generators: warp sums of S, W_b (lane bits), U_k
                    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
                    for (int i = 0; i < 6 + RB; ++i) {
                        R w = i == 0 ? tsum : i < 6 ? (((lane >> (i - 1)) & 1) ? tsum : (R)0) : u[i < 6 ? 0 : i - 6];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                        if (lane == 0) dred[warp * (6 + RB) + i] = w;
                    }
                    __syncthreads();
                    for (int g = d.nstaged + tid; g < d.ngen; g += kThreads) {
                        const SweepZGen z = a.gens[d.gen0 + g];
                        R S = 0, X = 0;
                        for (int q = 0; q < kThreads / 32; ++q) {  // fixed order
                            const R* wq = dred + q * (6 + RB);
                            S += wq[0];
                            if (z.src >= 1 && z.src <= RB) X += wq[5 + z.src];
                            else if (z.src > RB && z.src <= RB + 5) X += wq[z.src - RB];
                            else if (z.src > RB + 5 && ((q >> (z.src - RB - 6)) & 1)) X += wq[0];
                        }
                        const R v = S - 2 * X;
                        red[z.local] += (double)((__popcll(base & z.mthr) & 1) ? -v : v);
                    }
                    __syncthreads();  // dred is reused by the next diagonal op
                }
                const T* t0 = dtab + (xt & 255);  // chunk 0: the thread's bits, plus j
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    T ph = cmul(pc, t0[j]);
                    if (d.nct) ph = cross_phase(a.cross + d.cross0, d.nct, tab, xt | (uint64_t)j, ph);
                    ps[j] = cmul(ph, ps[j]);
                    ls[j] = cmul(ph, ls[j]);
                }
            }
        }
        if (lay != 0) transpose_any<R>(buf, ps, ls, lay, 0);
        {
            char* pp = reinterpret_cast<char*>(psi) + (base | xg0) * sizeof(T);
            char* pl = reinterpret_cast<char*>(lam) + (base | xg0) * sizeof(T);
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const uint64_t o = xo[j];
                *reinterpret_cast<T*>(pp + o) = ps[j];
                *reinterpret_cast<T*>(pl + o) = ls[j];
            }
        }
        if (srow) flush();
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
           sizeof(double) * ((a.ngrad + 1) & ~1) + sizeof(uint64_t) * ((size_t)1 << (L - 8)) +
           sizeof(R) * (kThreads / 32) * (6 + (L - 8)) + sizeof(typename C2<R>::T) * 4 * a.nmat;
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
    const int nlay = sweep_layouts(dt, lay);
    if (p.nlay != nlay) return cudaErrorInvalidValue;
    for (int l = 0; l < nlay; ++l)
        if (p.lay_a[l] != lay[l]) return cudaErrorInvalidValue;
    // every index the kernel follows is checked here
    for (int i = 0; i < L; ++i) {
        if (p.pos[i] < 0 || p.pos[i] >= n || (i > 0 && p.pos[i] <= p.pos[i - 1])) return cudaErrorInvalidValue;
        a.pos[i] = p.pos[i];
    }
    for (int i = 0; i < RB; ++i)  // diagonal ops: the low layout's registers hold qubits 0 .. RB-1
        if (p.pos[i] != i) return cudaErrorInvalidValue;
    const uint32_t nmat = (uint32_t)(p.mats.size() / 8);
    if (nmat > kSweepMaxOps) return cudaErrorInvalidValue;
    a.nmat = (int)nmat;
    int grads = 0, cur = 0;  // cur: the layout the kernel is in at this op
    for (int o = 0; o < a.nops; ++o) {
        const SweepOpRec& op = p.ops[o];
        if (op.type == SWEEP_LAYOUT) {
            if (op.arg >= nlay) return cudaErrorInvalidValue;
            cur = op.arg;
        } else if (op.type == SWEEP_G1) {
            if (op.arg >= RB || op.idx >= nmat || op.gen > 3 || op.form >= G1_FORMS) return cudaErrorInvalidValue;
            grads += op.gen != 0;
        } else if (op.type == SWEEP_DIAG) {
            if (op.idx >= p.diags.size() || cur != nlay - 1) return cudaErrorInvalidValue;  // the low layout
            const SweepDiagRec& d = p.diags[op.idx];
            if (d.nchunks < 1 || d.nchunks > 8 || 8 * (d.nchunks - 1) >= n || d.nct > d.ncross ||
                (size_t)d.cross0 + d.ncross > p.cross.size() || (size_t)d.gen0 + d.ngen > p.gens.size() ||
                (size_t)d.tab + 256 * (size_t)d.nchunks > a.tab_elems)
                return cudaErrorInvalidValue;
            if (d.nstaged > d.ngen) return cudaErrorInvalidValue;
            for (int g = 0; g < d.ngen; ++g) {
                const SweepZGen& z = p.gens[d.gen0 + g];
                if (g < d.nstaged ? z.kind > RB + 1 : (z.src > RB + 8 || z.local >= p.slots.size()))
                    return cudaErrorInvalidValue;
            }
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
