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
// fixed order: complex64 with error-free TwoSum steps into a (sum, error)
// float pair, FP64 from the tile's sum on across tiles; deterministic.
// Complex64 runs k_sweep_pass<float>; complex128 runs k_sweep_pass_ff, the
// same pass in float-float arithmetic on the FP32 pipe.
#include <stdint.h>

#include <algorithm>

#include "qs_device.cuh"
#include "qs_ff.cuh"
#include "qs_internal.h"

namespace qsgb {

namespace {

constexpr int kThreads = 256;

// L: tile qubits; ROWS: staged gradient rows per bank (one row of kThreads
// values each); lay(l): the register layouts (start of the register range),
// 0 natural, the last one "low" (registers hold qubits 0 .. L-9, where
// diagonal ops run).  float: complex64; double: the complex128 tile of the
// float-float form.
template <typename R> struct SweepShape;
template <> struct SweepShape<float> {
    static constexpr int L = kSweepTileC64, ROWS = 16, NLAY = 3;
    __host__ __device__ static constexpr int lay(int l) { return l == 0 ? 8 : l == 1 ? 4 : 0; }
};
template <> struct SweepShape<double> {
    static constexpr int L = kSweepTileC128, ROWS = 8, NLAY = 4;
    __host__ __device__ static constexpr int lay(int l) { return l == 0 ? 8 : l == 1 ? 5 : l == 2 ? 2 : 0; }
};

struct SweepArgs {
    int n, nops, ngrad, nb, nmat;
    int load_lay, store_lay;   // layouts (0 or 1, both coalesced) the tile is loaded and stored in
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

// Complex64: psi and lambda of one tile element share a 16-byte slot, so a
// transpose moves both with one 128-bit store and one 128-bit load per
// element.  A 128-bit access is served in four phases of 8 lanes; the slot's
// low 3 bits (its 16-byte bank group) are XORed with tile bits 4..6, which
// makes the 8 lanes of every phase hit 8 different groups in all three
// layouts (in layouts 0 and 1 they differ in tile bits 0..2; in layout 2 in
// tile bits 4..6).  Linear over XOR like swz, so a slot is the thread's base
// slot XOR a constant.
__host__ __device__ constexpr uint32_t swz16(uint32_t e) { return e ^ ((e >> 4) & 7u); }

// A transpose needs one barrier, between its writes and its reads.  A slot
// belongs to one tile element, so the slots a thread writes (its elements
// in the current layout) are exactly the slots it alone read in the
// previous transpose, which brought it into this layout (tiles start and
// end in layout 0): no other thread can still be reading them.
template <int L, int AF, int AT>
__device__ __forceinline__ void transpose_pl(float4* buf, float2 (&ps)[1 << (L - 8)], float2 (&ls)[1 << (L - 8)]) {
    constexpr int RB = L - 8, PER = 1 << RB;
    const uint32_t s0 = swz16(layout_base<RB>(threadIdx.x, AF)), s1 = swz16(layout_base<RB>(threadIdx.x, AT));
#pragma unroll
    for (int j = 0; j < PER; ++j)
        buf[s0 ^ swz16((uint32_t)j << AF)] = make_float4(ps[j].x, ps[j].y, ls[j].x, ls[j].y);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const float4 v = buf[s1 ^ swz16((uint32_t)j << AT)];
        ps[j] = make_float2(v.x, v.y);
        ls[j] = make_float2(v.z, v.w);
    }
}

template <typename R, int AF, int AT>
__device__ __forceinline__ void transpose_to(typename C2<R>::T* buf, typename C2<R>::T (&ps)[1 << (SweepShape<R>::L - 8)],
                                             typename C2<R>::T (&ls)[1 << (SweepShape<R>::L - 8)]) {
    using S = SweepShape<R>;
    transpose_pl<S::L, AF, AT>(reinterpret_cast<float4*>(buf), ps, ls);
}

template <typename R, int F>
__device__ __forceinline__ void transpose_from(typename C2<R>::T* buf, typename C2<R>::T (&ps)[1 << (SweepShape<R>::L - 8)],
                                               typename C2<R>::T (&ls)[1 << (SweepShape<R>::L - 8)], int to) {
    using S = SweepShape<R>;
    switch (to) {
        case 0: transpose_to<R, S::lay(F), S::lay(0)>(buf, ps, ls); break;
        case 1: transpose_to<R, S::lay(F), S::lay(1)>(buf, ps, ls); break;
        case 2: transpose_to<R, S::lay(F), S::lay(2)>(buf, ps, ls); break;
        default: transpose_to<R, S::lay(F), S::lay(S::NLAY - 1)>(buf, ps, ls); break;
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

// One-qubit gates of one form on register bits 0 .. RB-1 in that order (they
// commute: one stage), coefficients m, m + 4, ...: one dispatch, and the
// gates' arithmetic in one basic block.  Gradients in g[0 .. RB-1].
template <typename T, int RB, int V>
__device__ __forceinline__ void g1_seq(T (&ps)[1 << RB], T (&ls)[1 << RB], const T* m, int gen,
                                       decltype(T{}.x) (&g)[RB]) {
    g[0] = g1<T, RB, 0, V>(ps, ls, m, gen);
    g[1] = g1<T, RB, 1, V>(ps, ls, m + 4, gen);
    g[2] = g1<T, RB, 2, V>(ps, ls, m + 8, gen);
    if constexpr (RB == 4) g[3] = g1<T, RB, 3, V>(ps, ls, m + 12, gen);
}

template <typename T, int RB>
__device__ __forceinline__ void g1_all(T (&ps)[1 << RB], T (&ls)[1 << RB], const T* m, int form, int gen,
                                       decltype(T{}.x) (&g)[RB]) {
    switch (form) {
        case G1_RSHEAR_Y: g1_seq<T, RB, G1_RSHEAR_Y>(ps, ls, m, gen, g); break;
        case G1_RSHEAR: g1_seq<T, RB, G1_RSHEAR>(ps, ls, m, gen, g); break;
        default: g1_seq<T, RB, G1_CSHEAR_X>(ps, ls, m, gen, g); break;
    }
}

// The sum of row `row` of a bank of staged values (kThreads floats): this
// thread's TPR-strided share with TwoSum steps into a (sum, error) pair, then
// across the row's TPR lanes the same way; the pair enters FP64.
template <int TPR>
__device__ __forceinline__ double row_total(const float* rows, int row, int part) {
    F2Acc v;
#pragma unroll
    for (int k = 0; k < kThreads / TPR; ++k) v.add(rows[row * kThreads + part + TPR * k]);
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, v.hi, o, TPR), l = __shfl_xor_sync(0xffffffffu, v.lo, o, TPR);
        v.add(h);
        v.lo += l;
    }
    return (double)v.hi + (double)v.lo;
}

// complex64 (R = float); complex128 runs k_sweep_pass_ff below
template <typename R>
__global__ void __launch_bounds__(kThreads, 2) k_sweep_pass(typename C2<R>::T* __restrict__ psi,
                                                            typename C2<R>::T* __restrict__ lam,
                                                            const typename C2<R>::T* __restrict__ mats,
                                                            const typename C2<R>::T* __restrict__ tabs,
                                                            const __grid_constant__ SweepArgs a,
                                                            double* __restrict__ partials) {
    using T = typename C2<R>::T;
    static_assert(sizeof(R) == 4, "complex64 only: complex128 runs the float-float form");
    using S = SweepShape<R>;
    constexpr int L = S::L, RB = L - 8, PER = 1 << RB, LOW = S::NLAY - 1;
    constexpr int kRows = S::ROWS, TPR = kThreads / kRows;  // threads per staged row
    static_assert(S::lay(0) == L - RB && S::lay(LOW) == 0, "layouts");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);                                    // 2 x 2^L (psi, lambda)
    T* tab = buf + 2 * (1u << L);                                               // a.tab_elems
    R* gs = reinterpret_cast<R*>(tab + a.tab_elems);                            // 2 banks x kRows x kThreads
    double* red = reinterpret_cast<double*>(gs + 2 * kRows * kThreads);         // a.ngrad (even count: 16-byte alignment below)
    uint64_t* xo = reinterpret_cast<uint64_t*>(red + ((a.ngrad + 1) & ~1));    // 2 x PER: byte offset of j, layouts 0, 1
    R* dred = reinterpret_cast<R*>(xo + 2 * PER);                               // 8 warps x (6 + RB) x (sum, error)
    T* cm = reinterpret_cast<T*>(dred + 2 * (kThreads / 32) * (6 + RB));        // 4 x a.nmat coefficients
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < a.tab_elems; i += kThreads) tab[i] = tabs[i];
    for (int i = tid; i < 4 * a.nmat; i += kThreads) cm[i] = mats[i];
    for (int i = tid; i < a.ngrad; i += kThreads) red[i] = 0.0;
    if (tid < 2 * PER) {  // layout l: register bit k is tile bit lay(l) + k
        const int l = tid / PER, j = tid % PER;
        uint64_t o = 0;
        for (int k = 0; k < RB; ++k)
            if ((j >> k) & 1) o |= 1ull << a.pos[S::lay(l) + k];
        xo[tid] = o * sizeof(T);
    }
    auto global_of = [&](uint32_t e) {  // tile index -> global offset within the tile
        uint64_t x = 0;
        for (int i = 0; i < L; ++i) x |= (uint64_t)((e >> i) & 1u) << a.pos[i];
        return x;
    };
    // the thread's bits in the load and store layouts
    const uint64_t xgl = global_of(layout_base<RB>(tid, S::lay(a.load_lay)));
    const uint64_t xgs = global_of(layout_base<RB>(tid, S::lay(a.store_lay)));
    const uint64_t* xol = xo + PER * a.load_lay;
    const uint64_t* xos = xo + PER * a.store_lay;
    const uint64_t xl0 = global_of(layout_base<RB>(tid, 0));          // the thread's bits, low layout
    auto tile_base = [&](uint64_t t) {
        for (int i = 0; i < L; ++i) t = insert_zero(t, a.pos[i]);
        return t;
    };
    __syncthreads();

    int gdone = 0, srow = 0;  // gradients of this tile already added to red; rows staged since
    // block-uniform: add the staged rows to red.  Complex64: each row's 256
    // values are summed with error-free TwoSum steps into a float pair (sum,
    // rounding errors), so the tile's sum reaches FP64 as if it had been
    // accumulated there.
    // The rows are double-buffered: staging goes on in the other bank while
    // slower threads still read this one, so the flush needs no barrier at
    // its end (the next flush's barrier orders this bank's reuse).
    int bank = 0;
    auto flush = [&]() {
        __syncthreads();
        const int row = tid / TPR, part = tid % TPR;
        const double tot = row_total<TPR>(gs + bank * kRows * kThreads, row, part);
        if (part == 0 && row < srow) red[gdone + row] += tot;
        gdone += srow;
        srow = 0;
        bank ^= 1;
    };
    auto stage = [&](R v) {
        gs[(bank * kRows + srow) * kThreads + tid] = v;
        if (++srow == kRows) flush();
    };

    // the next tile's base: adding the deposited grid stride with the tile
    // bits set to 1 carries straight through them
    uint64_t tmask = 0;
    for (int i = 0; i < L; ++i) tmask |= 1ull << a.pos[i];
    const uint64_t gstep = tile_base(gridDim.x);
    uint64_t base = tile_base(blockIdx.x);
    T ps[PER], ls[PER];
    auto load_tile = [&](uint64_t b) {
        const char* pp = reinterpret_cast<const char*>(psi) + (b | xgl) * sizeof(T);
        const char* pl = reinterpret_cast<const char*>(lam) + (b | xgl) * sizeof(T);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint64_t o = xol[j];
            ps[j] = *reinterpret_cast<const T*>(pp + o);
            ls[j] = *reinterpret_cast<const T*>(pl + o);
        }
    };
    auto prefetch_tile = [&](uint64_t b) {  // into L2, one thread per 128-byte row of the tile
        if ((tid & ((128 / sizeof(T)) - 1)) == 0) {
            const char* pp = reinterpret_cast<const char*>(psi) + (b | xgl) * sizeof(T);
            const char* pl = reinterpret_cast<const char*>(lam) + (b | xgl) * sizeof(T);
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pp + xol[j]));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pl + xol[j]));
            }
        }
    };
    auto next_base = [&](uint64_t b) { return ((b | tmask) + gstep) & ~tmask; };  // tile + gridDim.x, deposited
    // a tile's loads are issued as soon as the previous tile is stored (their
    // latency overlaps that tile's gradient reduction), and the tile after
    // it is prefetched into L2 meanwhile
    if (blockIdx.x < a.ntiles) {
        load_tile(base);
        if (blockIdx.x + gridDim.x < a.ntiles) prefetch_tile(next_base(base));
    }
    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const uint64_t nb = tile + gridDim.x < a.ntiles ? next_base(base) : 0;
        int lay = a.load_lay;
        gdone = 0;
        for (int o = 0; o < a.nops; ++o) {
            const SweepOpRec op = a.ops[o];
            if (op.type == SWEEP_LAYOUT) {
                transpose_any<R>(buf, ps, ls, lay, op.arg);
                lay = op.arg;
            } else if (op.type == SWEEP_G1) {
                const R v = g1_any<T, RB>(ps, ls, cm + 4 * op.idx, op.arg, op.form, op.gen);
                if (op.gen) stage(v);
            } else if (op.type == SWEEP_G1ALL) {
                R g[RB];
                g1_all<T, RB>(ps, ls, cm + 4 * op.idx, op.form, op.gen, g);
                if (op.gen)
#pragma unroll
                    for (int i = 0; i < RB; ++i) stage(g[i]);
            } else {  // DIAG, in the low layout: register index j = bits 0 .. RB-1 of the index
                const SweepDiagRec d = a.diag[op.idx];
                const T* dtab = tab + d.tab;
                const uint64_t xt = base | xl0;
                T pc;  // chunks 1.. and the cross gates without a register qubit
                pc.x = 1;
                pc.y = 0;
                for (int c = 1; c < d.nchunks; ++c) pc = cmul(pc, dtab[256 * c + (256 >> RB) + ((xt >> (8 * c)) & 255)]);
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
                if (d.ngen > d.nstaged) {
                    // block generators: the tile's sums S (all), W_b (thread bit b set)
                    // and U_k (register bit k set) as staged rows of the current bank,
                    // reduced like the gradient rows (TwoSum steps), FP64 per tile
                    constexpr int NB = 1 + 8 + RB;
                    static_assert(NB <= kRows, "basis rows fit a bank");
                    if (srow) flush();  // the current bank is then empty
                    R* rows = gs + bank * kRows * kThreads;
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        const R v = b == 0 ? tsum : b <= 8 ? (((tid >> (b - 1)) & 1) ? tsum : (R)0) : u[b < 9 ? 0 : b - 9];
                        rows[b * kThreads + tid] = v;
                    }
                    __syncthreads();
                    double* tileB = reinterpret_cast<double*>(dred);  // NB totals
                    {  // every thread takes part (rows NB.. hold stale values and are dropped)
                        const int row = tid / TPR, part = tid % TPR;
                        const double tot = row_total<TPR>(rows, row, part);
                        if (part == 0 && row < NB) tileB[row] = tot;
                    }
                    __syncthreads();  // the totals are visible, and the bank's rows are free again
                    for (int g = d.nstaged + tid; g < d.ngen; g += kThreads) {
                        const SweepZGen z = a.gens[d.gen0 + g];
                        double X = 0;
                        if (z.src >= 1 && z.src <= RB) X = tileB[9 + z.src - 1];
                        else if (z.src > RB && z.src <= RB + 8) X = tileB[1 + z.src - RB - 1];
                        const double v = tileB[0] - 2 * X;
                        red[z.local] += (__popcll(base & z.mthr) & 1) ? -v : v;
                    }
                }
                const T* t0 = dtab + ((xt & 255) >> RB) * (PER + 1);  // chunk 0 (padded rows): the thread's row, plus j
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    T ph = cmul(pc, t0[j]);
                    if (d.nct) ph = cross_phase(a.cross + d.cross0, d.nct, tab, xt | (uint64_t)j, ph);
                    ps[j] = cmul(ph, ps[j]);
                    ls[j] = cmul(ph, ls[j]);
                }
            }
        }
        if (lay != a.store_lay) transpose_any<R>(buf, ps, ls, lay, a.store_lay);
        {
            char* pp = reinterpret_cast<char*>(psi) + (base | xgs) * sizeof(T);
            char* pl = reinterpret_cast<char*>(lam) + (base | xgs) * sizeof(T);
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const uint64_t o = xos[j];
                *reinterpret_cast<T*>(pp + o) = ps[j];
                *reinterpret_cast<T*>(pl + o) = ls[j];
            }
        }
        if (tile + gridDim.x < a.ntiles) {
            load_tile(nb);
            if (tile + 2 * (uint64_t)gridDim.x < a.ntiles) prefetch_tile(next_base(nb));
        }
        if (srow) flush();
        base = nb;
    }
    __syncthreads();
    for (int s = tid; s < a.ngrad; s += kThreads) {
        const size_t at = ((size_t)a.slot[s] * a.nb + blockIdx.x) * 2;
        partials[at] = 0.0;
        partials[at + 1] = red[s];
    }
}

// ------------------------------------------------------------ complex128
// The complex128 sweep pass in float-float arithmetic (qs_ff.cuh): psi and
// lambda are held as hi + lo floats in registers, every product and sum runs
// on the FP32 pipe with error-free transformations, and only the loads and
// stores convert to and from FP64.  Tile and layouts as the FP64 form (L = 11,
// 3 register bits).  One-qubit ops take U^dagger's four entries (forms
// G1_FF_REAL / G1_FF_CPLX) and always act on register bit 0: the thread's
// registers are rotated (bit 0 <- bit 1 <- bit 2 <- bit 0) around the op, so
// one copy of the gate code serves every register bit.
struct FFV {
    float h, l;  // a float-float real value
};

// rotate the 8 register elements: new index (j >> 1) | ((j & 1) << 2) takes old j
__device__ __forceinline__ void ff_rotate(FFC (&v)[8]) {
    const FFC t1 = v[1], t2 = v[2], t3 = v[3], t4 = v[4], t5 = v[5], t6 = v[6];
    // old j -> new j': 1->4, 2->1, 3->5, 4->2, 5->6, 6->3 (0 and 7 stay)
    v[4] = t1;
    v[1] = t2;
    v[5] = t3;
    v[2] = t4;
    v[6] = t5;
    v[3] = t6;
}

// S + E += a * b for float-float reals (the ffa_term of qs_ff.cuh)
__device__ __forceinline__ void ffv_term(float& S, float& E, float ah, float al, float bh, float bl) {
    ffa_term(S, E, ah, al, bh, bl);
}

// One-qubit op on register bit 0: the gradient Im <l|P|p> over the thread's
// 4 pairs (generator gen: 1 X, 2 Y, 3 Z), then (p0, p1) <- M (p0, p1) and the
// same for lambda, M = the 4 entries m (real: imaginary parts zero).
template <bool REAL>
__device__ __forceinline__ FFV ff_g1_bit0(FFC (&ps)[8], FFC (&ls)[8], const FFC* m, int gen) {
    float S = 0.f, E = 0.f;
    const FFC m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        FFC& p0 = ps[2 * k];
        FFC& p1 = ps[2 * k + 1];
        FFC& l0 = ls[2 * k];
        FFC& l1 = ls[2 * k + 1];
        if (gen == 2) {  // Re(conj(l1) p0) - Re(conj(l0) p1)
            ffv_term(S, E, l1.h.x, l1.l.x, p0.h.x, p0.l.x);
            ffv_term(S, E, l1.h.y, l1.l.y, p0.h.y, p0.l.y);
            ffv_term(S, E, -l0.h.x, -l0.l.x, p1.h.x, p1.l.x);
            ffv_term(S, E, -l0.h.y, -l0.l.y, p1.h.y, p1.l.y);
        } else if (gen == 1) {  // Im(conj(l0) p1) + Im(conj(l1) p0)
            ffv_term(S, E, l0.h.x, l0.l.x, p1.h.y, p1.l.y);
            ffv_term(S, E, -l0.h.y, -l0.l.y, p1.h.x, p1.l.x);
            ffv_term(S, E, l1.h.x, l1.l.x, p0.h.y, p0.l.y);
            ffv_term(S, E, -l1.h.y, -l1.l.y, p0.h.x, p0.l.x);
        } else if (gen == 3) {  // Im(conj(l0) p0) - Im(conj(l1) p1)
            ffv_term(S, E, l0.h.x, l0.l.x, p0.h.y, p0.l.y);
            ffv_term(S, E, -l0.h.y, -l0.l.y, p0.h.x, p0.l.x);
            ffv_term(S, E, -l1.h.x, -l1.l.x, p1.h.y, p1.l.y);
            ffv_term(S, E, l1.h.y, l1.l.y, p1.h.x, p1.l.x);
        }
        if (REAL) {  // real entries: each output component a two-term sum
            auto rmac = [](const FFC& ma, const FFC& a, const FFC& mb, const FFC& b) {
                const float2 re = ff_dot2(ma.h.x, ma.l.x, a.h.x, a.l.x, mb.h.x, mb.l.x, b.h.x, b.l.x);
                const float2 im = ff_dot2(ma.h.x, ma.l.x, a.h.y, a.l.y, mb.h.x, mb.l.x, b.h.y, b.l.y);
                FFC r;
                r.h = make_float2(re.x, im.x);
                r.l = make_float2(re.y, im.y);
                return r;
            };
            const FFC q0 = rmac(m0, p0, m1, p1), q1 = rmac(m2, p0, m3, p1);
            const FFC k0 = rmac(m0, l0, m1, l1), k1 = rmac(m2, l0, m3, l1);
            p0 = q0;
            p1 = q1;
            l0 = k0;
            l1 = k1;
        } else {
            const FFC q0 = ff_cmac2(m0, p0, m1, p1), q1 = ff_cmac2(m2, p0, m3, p1);
            const FFC k0 = ff_cmac2(m0, l0, m1, l1), k1 = ff_cmac2(m2, l0, m3, l1);
            p0 = q0;
            p1 = q1;
            l0 = k0;
            l1 = k1;
        }
    }
    FFV g;
    g.h = S + E;
    g.l = E - (g.h - S);
    return g;
}

__device__ __forceinline__ FFV ff_g1_any(FFC (&ps)[8], FFC (&ls)[8], const FFC* m, int form, int gen) {
    return form == G1_FF_REAL ? ff_g1_bit0<true>(ps, ls, m, gen) : ff_g1_bit0<false>(ps, ls, m, gen);
}

// psi and lambda of the tile through shared memory (one 16-byte slot per
// element and state, swizzled as the FP64 form); one barrier, as there
__device__ __forceinline__ void ff_transpose(float4* buf, FFC (&ps)[8], FFC (&ls)[8], int af, int at) {
    constexpr int L = kSweepTileC128, SW = 3;
    const uint32_t s0 = swz<SW>(layout_base<3>(threadIdx.x, af)), s1 = swz<SW>(layout_base<3>(threadIdx.x, at));
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t s = s0 ^ swz<SW>((uint32_t)j << af);
        buf[s] = make_float4(ps[j].h.x, ps[j].h.y, ps[j].l.x, ps[j].l.y);
        buf[(1u << L) + s] = make_float4(ls[j].h.x, ls[j].h.y, ls[j].l.x, ls[j].l.y);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t s = s1 ^ swz<SW>((uint32_t)j << at);
        const float4 a = buf[s], b = buf[(1u << L) + s];
        ps[j].h = make_float2(a.x, a.y);
        ps[j].l = make_float2(a.z, a.w);
        ls[j].h = make_float2(b.x, b.y);
        ls[j].l = make_float2(b.z, b.w);
    }
}

// ph times the diagonal entries of `count` gates at index x (float-float tables)
template <typename X>
__device__ __forceinline__ FFC ff_cross_phase(const X* cg, int count, const FFC* tab, uint64_t x, FFC ph) {
    for (int c = 0; c < count; ++c) {
        uint32_t li = 0;
        for (int i = 0; i < cg[c].k; ++i) li = (li << 1) | (uint32_t)((x >> cg[c].q[i]) & 1);
        ph = ff_cmul(ph, tab[cg[c].tab + li]);
    }
    return ph;
}

__global__ void __launch_bounds__(kThreads, 2) k_sweep_pass_ff(double2* __restrict__ psi, double2* __restrict__ lam,
                                                              const double2* __restrict__ mats,
                                                              const double2* __restrict__ tabs,
                                                              const __grid_constant__ SweepArgs a,
                                                              double* __restrict__ partials) {
    constexpr int L = kSweepTileC128, RB = 3, PER = 8;
    constexpr int kRows = 8, TPR = kThreads / kRows;  // staged rows of (hi, lo) gradients, threads per row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* buf = reinterpret_cast<float4*>(smem_raw);                          // 2 x 2^L (psi, lambda)
    FFC* tab = reinterpret_cast<FFC*>(buf + 2 * (1u << L));                     // a.tab_elems
    FFC* cm = tab + a.tab_elems;                                                // 4 x a.nmat
    float* gsh = reinterpret_cast<float*>(cm + 4 * a.nmat);                     // 2 banks x kRows x kThreads
    float* gsl = gsh + 2 * kRows * kThreads;
    float* dred = gsl + 2 * kRows * kThreads;                                   // 8 warps x (6 + RB) x (sum, error)
    double* red = reinterpret_cast<double*>(dred + 2 * (kThreads / 32) * (6 + RB));   // a.ngrad
    uint64_t* xo = reinterpret_cast<uint64_t*>(red + a.ngrad);                  // 2 x PER: byte offset of j, layouts 0, 1
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < a.tab_elems; i += kThreads) tab[i] = ff_from(tabs[i]);
    for (int i = tid; i < 4 * a.nmat; i += kThreads) cm[i] = ff_from(mats[i]);
    for (int i = tid; i < a.ngrad; i += kThreads) red[i] = 0.0;
    if (tid < 2 * PER) {  // layout l: register bit k is tile bit lay(l) + k
        const int l = tid / PER, j = tid % PER;
        uint64_t o = 0;
        for (int k = 0; k < RB; ++k)
            if ((j >> k) & 1) o |= 1ull << a.pos[SweepShape<double>::lay(l) + k];
        xo[tid] = o * sizeof(double2);
    }
    auto global_of = [&](uint32_t e) {
        uint64_t x = 0;
        for (int i = 0; i < L; ++i) x |= (uint64_t)((e >> i) & 1u) << a.pos[i];
        return x;
    };
    auto tile_base = [&](uint64_t t) {
        for (int i = 0; i < L; ++i) t = insert_zero(t, a.pos[i]);
        return t;
    };
    auto lay_a = [](int l) { return SweepShape<double>::lay(l); };   // register ranges 8, 5, 2, 0
    const uint64_t xgl = global_of(layout_base<RB>(tid, lay_a(a.load_lay)));
    const uint64_t xgs = global_of(layout_base<RB>(tid, lay_a(a.store_lay)));
    const uint64_t* xol = xo + PER * a.load_lay;
    const uint64_t* xos = xo + PER * a.store_lay;
    const uint64_t xl0 = global_of(layout_base<RB>(tid, 0));
    __syncthreads();

    int gdone = 0, srow = 0, bank = 0;
    // staged (hi, lo) rows summed with TwoSum steps, FP64 per row (double-
    // buffered banks: no barrier at the end, as in the FP32/FP64 form)
    auto flush = [&]() {
        __syncthreads();
        const int row = tid / TPR, part = tid % TPR;
        const float* bh = gsh + bank * kRows * kThreads;
        const float* bl = gsl + bank * kRows * kThreads;
        F2Acc v;
#pragma unroll
        for (int k = 0; k < kThreads / TPR; ++k) {
            v.add(bh[row * kThreads + part + TPR * k]);
            v.add(bl[row * kThreads + part + TPR * k]);
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) {
            const float h = __shfl_xor_sync(0xffffffffu, v.hi, o, TPR), l = __shfl_xor_sync(0xffffffffu, v.lo, o, TPR);
            v.add(h);
            v.lo += l;
        }
        if (part == 0 && row < srow) red[gdone + row] += (double)v.hi + (double)v.lo;
        gdone += srow;
        srow = 0;
        bank ^= 1;
    };
    auto stage = [&](FFV v) {
        gsh[(bank * kRows + srow) * kThreads + tid] = v.h;
        gsl[(bank * kRows + srow) * kThreads + tid] = v.l;
        if (++srow == kRows) flush();
    };

    // the next tile's base: adding the deposited grid stride with the tile
    // bits set to 1 carries straight through them
    uint64_t tmask = 0;
    for (int i = 0; i < L; ++i) tmask |= 1ull << a.pos[i];
    const uint64_t gstep = tile_base(gridDim.x);
    uint64_t base = tile_base(blockIdx.x);
    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        FFC ps[PER], ls[PER];
        {
            const char* pp = reinterpret_cast<const char*>(psi) + (base | xgl) * sizeof(double2);
            const char* pl = reinterpret_cast<const char*>(lam) + (base | xgl) * sizeof(double2);
            double2 dp[PER], dl[PER];
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                dp[j] = *reinterpret_cast<const double2*>(pp + xol[j]);
                dl[j] = *reinterpret_cast<const double2*>(pl + xol[j]);
            }
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                ps[j] = ff_from(dp[j]);
                ls[j] = ff_from(dl[j]);
            }
        }
        uint64_t nb = 0;
        if (tile + gridDim.x < a.ntiles) {  // the next tile on its way into L2
            nb = ((base | tmask) + gstep) & ~tmask;  // tile + gridDim.x, deposited
            const char* pp = reinterpret_cast<const char*>(psi) + (nb | xgl) * sizeof(double2);
            const char* pl = reinterpret_cast<const char*>(lam) + (nb | xgl) * sizeof(double2);
            if ((tid & 7) == 0) {  // one thread per 128-byte row of the tile
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(pp + xol[j]));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(pl + xol[j]));
                }
            }
        }
        int lay = a.load_lay;
        gdone = 0;
        for (int o = 0; o < a.nops; ++o) {
            const SweepOpRec op = a.ops[o];
            if (op.type == SWEEP_LAYOUT) {
                ff_transpose(buf, ps, ls, lay_a(lay), lay_a(op.arg));
                lay = op.arg;
            } else if (op.type == SWEEP_G1 || op.type == SWEEP_G1ALL) {
                // one call site for every register bit: rotate the gate's bit to 0
                const int pre = op.type == SWEEP_G1 ? op.arg : 0, count = op.type == SWEEP_G1 ? 1 : RB;
                for (int t = 0; t < pre; ++t) {
                    ff_rotate(ps);
                    ff_rotate(ls);
                }
#pragma unroll 1
                for (int i = 0; i < count; ++i) {
                    const FFV g = ff_g1_any(ps, ls, cm + 4 * (op.idx + i), op.form, op.gen);
                    if (op.gen) stage(g);
                    ff_rotate(ps);
                    ff_rotate(ls);
                }
                for (int t = (pre + count) % RB; t != 0 && t < RB; ++t) {
                    ff_rotate(ps);
                    ff_rotate(ls);
                }
            } else {  // DIAG, in the low layout: register index j = bits 0 .. RB-1 of the index
                const SweepDiagRec d = a.diag[op.idx];
                const FFC* dtab = tab + d.tab;
                const uint64_t xt = base | xl0;
                FFC pc;  // chunks 1.. and the cross gates without a register qubit
                pc.h = make_float2(1.f, 0.f);
                pc.l = make_float2(0.f, 0.f);
                for (int c = 1; c < d.nchunks; ++c) pc = ff_cmul(pc, dtab[256 * c + (256 >> RB) + ((xt >> (8 * c)) & 255)]);
                pc = ff_cross_phase(a.cross + d.cross0 + d.nct, d.ncross - d.nct, tab, xt, pc);
                // Im(conj(l) p) per element as float-float, and the sums over
                // the thread's elements (all, and those with register bit i set)
                auto im_lp = [&](int j) {  // Im(conj(l_j) p_j)
                    const float2 v = ff_dot2(ls[j].h.x, ls[j].l.x, ps[j].h.y, ps[j].l.y, -ls[j].h.y, -ls[j].l.y,
                                             ps[j].h.x, ps[j].l.x);
                    return FFV{v.x, v.y};
                };
                float ts = 0.f, te = 0.f, us[RB], ue[RB];
#pragma unroll
                for (int i = 0; i < RB; ++i) us[i] = ue[i] = 0.f;
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    const FFV t = im_lp(j);
                    float s2, e2;
                    two_sum(ts, t.h, s2, e2);
                    ts = s2;
                    te += e2 + t.l;
#pragma unroll
                    for (int i = 0; i < RB; ++i)
                        if ((j >> i) & 1) {
                            two_sum(us[i], t.h, s2, e2);
                            us[i] = s2;
                            ue[i] += e2 + t.l;
                        }
                }
                for (int g = 0; g < d.nstaged; ++g) {
                    const SweepZGen z = a.gens[d.gen0 + g];
                    float S = ts, E = te;  // kind 0: the sum
                    if (z.kind >= 1 && z.kind <= RB) {  // sum - 2 (sum over register bit set)
                        const int i = z.kind - 1;
                        const float uh = i == 0 ? us[0] : i == 1 ? us[1] : us[2];
                        const float ul = i == 0 ? ue[0] : i == 1 ? ue[1] : ue[2];
                        float s2, e2;
                        two_sum(S, -2.f * uh, s2, e2);
                        S = s2;
                        E += e2 - 2.f * ul;
                    } else if (z.kind > RB) {
                        S = 0.f;
                        E = 0.f;
#pragma unroll
                        for (int j = 0; j < PER; ++j) {
                            const float sg = ((z.jmask >> j) & 1) ? -1.f : 1.f;
                            const FFV t = im_lp(j);
                            float s2, e2;
                            two_sum(S, sg * t.h, s2, e2);
                            S = s2;
                            E += e2 + sg * t.l;
                        }
                    }
                    FFV v;
                    v.h = S + E;
                    v.l = E - (v.h - S);
                    if (__popcll(xt & z.mthr) & 1) {
                        v.h = -v.h;
                        v.l = -v.l;
                    }
                    stage(v);
                }
                if (d.ngen > d.nstaged) {  // block generators: warp sums of S, W_b (lane bits), U_k
                    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
                    for (int i = 0; i < 6 + RB; ++i) {
                        const bool on = i == 0 || i >= 6 || ((lane >> (i - 1)) & 1);
                        F2Acc w;
                        w.hi = !on ? 0.f : i < 6 ? ts : us[i - 6];
                        w.lo = !on ? 0.f : i < 6 ? te : ue[i - 6];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const float h = __shfl_xor_sync(0xffffffffu, w.hi, o), l = __shfl_xor_sync(0xffffffffu, w.lo, o);
                            w.add(h);
                            w.lo += l;
                        }
                        if (lane == 0) {
                            dred[2 * (warp * (6 + RB) + i)] = w.hi;
                            dred[2 * (warp * (6 + RB) + i) + 1] = w.lo;
                        }
                    }
                    __syncthreads();
                    for (int g = d.nstaged + tid; g < d.ngen; g += kThreads) {
                        const SweepZGen z = a.gens[d.gen0 + g];
                        double S = 0, X = 0;
                        for (int q = 0; q < kThreads / 32; ++q) {  // fixed order
                            const float* wq = dred + 2 * q * (6 + RB);
                            auto at = [&](int i) { return (double)wq[2 * i] + (double)wq[2 * i + 1]; };
                            S += at(0);
                            if (z.src >= 1 && z.src <= RB) X += at(5 + z.src);
                            else if (z.src > RB && z.src <= RB + 5) X += at(z.src - RB);
                            else if (z.src > RB + 5 && ((q >> (z.src - RB - 6)) & 1)) X += at(0);
                        }
                        const double v = S - 2 * X;
                        red[z.local] += (__popcll(base & z.mthr) & 1) ? -v : v;
                    }
                    __syncthreads();  // dred is reused by the next diagonal op
                }
                const FFC* t0 = dtab + ((xt & 255) >> RB) * (PER + 1);  // chunk 0 (padded rows): the thread's row, plus j
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    FFC ph = ff_cmul(pc, t0[j]);
                    if (d.nct) ph = ff_cross_phase(a.cross + d.cross0, d.nct, tab, xt | (uint64_t)j, ph);
                    ps[j] = ff_cmul(ph, ps[j]);
                    ls[j] = ff_cmul(ph, ls[j]);
                }
            }
        }
        if (lay != a.store_lay) ff_transpose(buf, ps, ls, lay_a(lay), lay_a(a.store_lay));
        {
            char* pp = reinterpret_cast<char*>(psi) + (base | xgs) * sizeof(double2);
            char* pl = reinterpret_cast<char*>(lam) + (base | xgs) * sizeof(double2);
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                *reinterpret_cast<double2*>(pp + xos[j]) = ff_to(ps[j]);
                *reinterpret_cast<double2*>(pl + xos[j]) = ff_to(ls[j]);
            }
        }
        if (srow) flush();
        base = nb;
    }
    __syncthreads();
    for (int s = tid; s < a.ngrad; s += kThreads) {
        const size_t at = ((size_t)a.slot[s] * a.nb + blockIdx.x) * 2;
        partials[at] = 0.0;
        partials[at + 1] = red[s];
    }
}

size_t sweep_smem_ff(const SweepArgs& a) {
    constexpr int L = kSweepTileC128, RB = 3;
    return 16 * (2 * ((size_t)1 << L) + a.tab_elems + 4 * (size_t)a.nmat) + sizeof(float) * 2 * 2 * 8 * kThreads +
           sizeof(float) * 2 * (kThreads / 32) * (6 + RB) + sizeof(double) * (size_t)a.ngrad +
           sizeof(uint64_t) * 2 * ((size_t)1 << RB);
}

template <typename R>
size_t sweep_smem(const SweepArgs& a) {
    constexpr int L = SweepShape<R>::L;
    const size_t esz = sizeof(typename C2<R>::T);
    return esz * (2 * ((size_t)1 << L) + a.tab_elems) + sizeof(R) * 2 * SweepShape<R>::ROWS * kThreads +
           sizeof(double) * ((a.ngrad + 1) & ~1) + sizeof(uint64_t) * 2 * ((size_t)1 << (L - 8)) +
           sizeof(R) * 2 * (kThreads / 32) * (6 + (L - 8)) + sizeof(typename C2<R>::T) * 4 * a.nmat;
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
    if (p.load_lay < 0 || p.load_lay > 1 || p.store_lay < 0 || p.store_lay > 1) return cudaErrorInvalidValue;
    a.load_lay = p.load_lay;
    a.store_lay = p.store_lay;
    int grads = 0, cur = p.load_lay;  // cur: the layout the kernel is in at this op
    for (int o = 0; o < a.nops; ++o) {
        const SweepOpRec& op = p.ops[o];
        if (op.type == SWEEP_LAYOUT) {
            if (op.arg >= nlay) return cudaErrorInvalidValue;
            cur = op.arg;
        } else if (op.type == SWEEP_G1) {
            const bool ff = op.form == G1_FF_REAL || op.form == G1_FF_CPLX;
            if (op.arg >= RB || op.idx >= nmat || op.gen > 3 || op.form >= G1_FORMS || ff != (dt == QS_C128))
                return cudaErrorInvalidValue;
            grads += op.gen != 0;
        } else if (op.type == SWEEP_G1ALL) {
            const bool ok = dt == QS_C128 ? (op.form == G1_FF_REAL || op.form == G1_FF_CPLX)
                                          : (op.form == G1_RSHEAR || op.form == G1_RSHEAR_Y || op.form == G1_CSHEAR_X);
            if ((uint64_t)op.idx + RB > nmat || op.gen > 3 || !ok) return cudaErrorInvalidValue;
            grads += op.gen != 0 ? RB : 0;
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
    } else {  // complex128: the float-float form
        cudaError_t e = allow_max_dynamic_smem(k_sweep_pass_ff);
        if (e != cudaSuccess) return e;
        k_sweep_pass_ff<<<grid, kThreads, sweep_smem_ff(a), st>>>((double2*)psi, (double2*)lam, (const double2*)dmats,
                                                                  (const double2*)dtabs, a, partials);
    }
    return cudaGetLastError();
}

}  // namespace qsgb
