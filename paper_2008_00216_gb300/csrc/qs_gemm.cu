// Dense 6-qubit gates on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// A fused k-qubit gate applies the same 2^k x 2^k complex matrix U to each
// of the 2^(n-k) disjoint sets of 2^k amplitudes (Section 3), i.e. it is the
// product U X with X = 2^k x 2^(n-k).  With real arithmetic:
//   D = [Re U; Im U] (128 x 64)  x  B^T,   B = [re x_s; im x_s] per set s,
//   y_s = (D_re-rows . re-col - D_im-rows . im-col) + i (...).
// A (the gate, split into hi/lo parts) stays resident in tensor memory for
// the whole kernel; B (K-major, K = the gate's 64 local indices, 128-byte
// swizzle) is streamed through shared memory; the accumulator D (128 lanes x
// 64 FP32 columns per tile of 32 sets) is double-buffered in tensor memory.  Precision modes on complex64 states:
//   TF32     one product, operands rounded to TF32
//   3xTF32   A_hi B_hi + A_hi B_lo + A_lo B_hi, hi = TF32(x), lo = x - hi
//   3xBF16   the same split with bfloat16 parts
// all with FP32 accumulation.
//
// One persistent CTA per SM, warp-specialised:
//   warps 0-3  epilogue: tensor memory -> registers -> recombine -> HBM
//   warps 4-11 producer: cp.async gathers of 32 sets x 64 amplitudes
//              (coalesced) several tiles ahead into a raw ring, then the
//              hi/lo split into the swizzled shared-memory stages
//   warp 12    one thread issues the MMAs and commits to mbarriers
// Every mbarrier wait is bounded (about two seconds of clock64); on timeout
// the CTA sets the error flag, drains its MMAs, frees tensor memory, exits.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsgb {
namespace tc {

constexpr int kSets = 32;          // sets (N/2) per tile
constexpr int kRowsB = 2 * kSets;  // B rows: (set, re/im)
constexpr int kStages = 2;         // split, swizzled B stages
constexpr int kEpiWarps = 4, kProdWarps = 8;
constexpr int kProdThreads = 32 * kProdWarps;
constexpr int kMmaWarp = kEpiWarps + kProdWarps;
constexpr int kThreads = 32 * (kMmaWarp + 1);
// tensor memory: A_hi | A_lo (64 columns each for TF32, 32 for packed BF16)
// then two 64-column FP32 accumulators
constexpr int kTmemCols = 256;
constexpr int kTmemD = 128;
constexpr long long kTimeout = 4ll << 30;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: true when the phase completed; false after the timeout (the
// error flag and the CTA's abort flag are set) or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err, volatile int* abort_flag) {
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(b, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kTimeout) {
            atomicExch(err, 1);
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Barrier among the threads of one role (init count = role size), built on an
// mbarrier so a wait is bounded: a role whose member left on an error path
// times out instead of hanging.  The result is made warp-uniform.
__device__ __forceinline__ bool group_sync(uint64_t* bar, uint32_t& phase, int* err, volatile int* abort_flag) {
    mbar_arrive(bar);
    const bool ok = mbar_wait(bar, phase, err, abort_flag);
    phase ^= 1u;
    return __all_sync(0xffffffffu, ok);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO); the leading offset is unused for this layout
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;   // SWIZZLE_128B
    return d;
}

// instruction descriptor: FP32 accumulate, A/B TF32 (kind 0) or BF16
// (kind 1), both K-major, M = 128, N = 64
template <int KIND>
__host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | ((KIND == 0 ? 2u : 1u) << 7) | ((KIND == 0 ? 2u : 1u) << 10) | ((uint32_t)(kRowsB >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// D[tmem] (+)= A[tmem] * B[smem]^T: A is read from tensor memory (row m in
// lane m, K along columns), so only B is streamed from shared memory
template <int KIND>
__device__ __forceinline__ void umma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t acc) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
            "r"(a_tmem), "l"(b), "r"(idesc<0>()), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
            "r"(a_tmem), "l"(b), "r"(idesc<1>()), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void umma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// byte offset of 16-byte chunk `c` of row `r` in a [rows][128 B] swizzled block
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

struct Args {
    uint64_t off[64];   // offset of local index l; the gate's qubits are in
                        // descending order, so local bit b is the b-th lowest target
    int sorted[6];      // target bits ascending
    uint64_t ntiles;    // 2^(n-6) / 32
};

// Q0T: qubit 0 is a target.  Then amplitude pairs (l, l+1), l even, are
// adjacent in memory; otherwise set pairs (s, s+1), s even, are.  Either way
// every gather and write-back moves 16-byte pairs.
template <int SPLITS, int KIND>
struct Layout {
    static constexpr int kAtomsK = KIND == 0 ? 2 : 1;           // 64 K elements
    static constexpr int kBBytes = kAtomsK * kRowsB * 128;       // one B split, one stage
    static constexpr int SPLITS_A = SPLITS == 3 ? 2 : 1;        // stored parts (hi, lo)
    static constexpr int kACols = KIND == 0 ? 64 : 32;          // TMEM columns of one A part
    static constexpr int kB = 0;
    static constexpr int kStageBytes = SPLITS_A * kBBytes;
    static constexpr int kRaw = 6;                               // gathered tiles in flight
    static constexpr int kRawBytes = 32 * 66 * 8;                // [64][32] or [32][66] float2
    static constexpr int kR = kB + kStages * kStageBytes;
    static constexpr int kY = kR + kRaw * kRawBytes;             // [64][34] or [32][66] float2
    static constexpr int kYBytes = 32 * 68 * 8;
    static constexpr int kOff = kY + kYBytes;                    // offsets (64 x u64)
    static constexpr int kBar = kOff + 64 * 8;                   // barriers
    static constexpr int kTotal = kBar + 128;
};

template <int SPLITS, int KIND, bool Q0T>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm6(float2* __restrict__ psi, const float2* __restrict__ U, const __grid_constant__ Args a, int* err) {
    using LY = Layout<SPLITS, KIND>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    uint64_t* full = reinterpret_cast<uint64_t*>(sm + LY::kBar);
    uint64_t* empty = full + kStages;
    uint64_t* dfull = empty + kStages;
    uint64_t* dempty = dfull + 2;
    uint64_t* drain = dempty + 2;
    uint64_t* prodbar = drain + 1;
    uint64_t* epibar = prodbar + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(epibar + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint64_t* soff = reinterpret_cast<uint64_t*>(sm + LY::kOff);
    float2* ystage = reinterpret_cast<float2*>(sm + LY::kY);

    for (int i = threadIdx.x; i < 64; i += blockDim.x) soff[i] = a.off[i];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], kProdThreads);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&dfull[s], 1);
            mbar_init(&dempty[s], 32 * kEpiWarps);
        }
        mbar_init(drain, 1);
        mbar_init(prodbar, kProdThreads);
        mbar_init(epibar, 32 * kEpiWarps);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;

    // ---- A into tensor memory: row m = 32q + 16h + rr holds (h ? Im : Re)
    // U[16q + rr][:], so each epilogue warp owns the real and imaginary rows
    // of 16 outputs.  Warp q writes lanes 32q..32q+31, 16 columns at a time.
    if (warp < kEpiWarps) {
        const int m = threadIdx.x;
        const int r = 16 * (m >> 5) + (m & 15), h = (m >> 4) & 1;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int part = 0; part < LY::SPLITS_A; ++part) {
#pragma unroll
            for (int cb = 0; cb < LY::kACols / 16; ++cb) {
                uint32_t w16[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    if constexpr (KIND == 0) {
                        const int l = 16 * cb + c;
                        const float v = h ? U[r * 64 + l].y : U[r * 64 + l].x;
                        const float hi = tf32_rna(v);
                        w16[c] = __float_as_uint(part == 0 ? hi : tf32_rna(v - hi));
                    } else {  // two bf16 per column, lower K index in the low half
                        const int l = 2 * (16 * cb + c);
                        const float v0 = h ? U[r * 64 + l].y : U[r * 64 + l].x;
                        const float v1 = h ? U[r * 64 + l + 1].y : U[r * 64 + l + 1].x;
                        __nv_bfloat16 b0 = __float2bfloat16_rn(v0), b1 = __float2bfloat16_rn(v1);
                        if (part == 1) {
                            b0 = __float2bfloat16_rn(v0 - __bfloat162float(b0));
                            b1 = __float2bfloat16_rn(v1 - __bfloat162float(b1));
                        }
                        w16[c] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
                    }
                }
                tmem_st16(lane_base + (uint32_t)(part * LY::kACols + 16 * cb), w16);
            }
        }
        tmem_st_wait();
    }
    tc_before();
    __syncthreads();
    tc_after();

    if (warp >= kEpiWarps && warp < kMmaWarp) {
        // ================= producer
        // (1) cp.async gathers tile it+kRaw-1 into a raw ring slot while
        // (2) tile it, already in shared memory, is split and written into
        //     the swizzled stage the MMA reads.
        const int ptid = threadIdx.x - 32 * kEpiWarps, pw = ptid >> 5;
        unsigned char* raw = sm + LY::kR;
        auto issue = [&](uint64_t itx) {
            const uint64_t tt = blockIdx.x + itx * gridDim.x;
            if (tt < a.ntiles) {
                float2* slot = reinterpret_cast<float2*>(raw + (itx % LY::kRaw) * LY::kRawBytes);
                if constexpr (Q0T) {
                    // pairs (l, l+1) of one set; a warp reads one whole set
                    const int lp = ptid & 31;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int jj = (ptid >> 5) + 8 * i;
                        uint64_t base = tt * kSets + jj;
#pragma unroll
                        for (int b = 0; b < 6; ++b) base = insert_zero(base, a.sorted[b]);
                        cp_async16(slot + jj * 66 + 2 * lp, psi + base + soff[2 * lp]);
                    }
                } else {
                    // pairs (s, s+1) of one local index; a warp reads 2 rows
                    const int sp = ptid & 15;
                    uint64_t base = tt * kSets + 2 * sp;
#pragma unroll
                    for (int b = 0; b < 6; ++b) base = insert_zero(base, a.sorted[b]);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int l = (ptid >> 4) + 16 * i;
                        cp_async16(slot + l * 32 + 2 * sp, psi + base + soff[l]);
                    }
                }
            }
            cp_async_commit();  // one group per tile, possibly empty
        };
        for (int p = 0; p < LY::kRaw - 1; ++p) issue((uint64_t)p);
        // conversion unit: (set j, chunk Q of 4 (TF32) or 8 (BF16) local indices)
        const int j = (ptid & 15) + 16 * (pw & 1), lsel = (ptid >> 4) & 1, lg = pw >> 1;
        uint32_t gph = 0;
        for (uint64_t it = 0;; ++it) {
            const uint64_t t = blockIdx.x + it * gridDim.x;
            if (t >= a.ntiles) break;
            issue(it + LY::kRaw - 1);
            cp_async_wait<LY::kRaw - 1>();
            // every producer's copies of tile `it` have landed
            if (!group_sync(prodbar, gph, err, abort_flag)) break;
            const int stage = (int)(it % kStages);
            const uint32_t ph = (uint32_t)((it / kStages) & 1);
            if (!__all_sync(0xffffffffu, mbar_wait(&empty[stage], ph ^ 1, err, abort_flag))) break;
            const float2* rs = reinterpret_cast<const float2*>(raw + (it % LY::kRaw) * LY::kRawBytes);
            auto rawat = [&](int l) { return Q0T ? rs[j * 66 + l] : rs[l * 32 + j]; };
            unsigned char* bst = sm + LY::kB + stage * LY::kStageBytes;
            if constexpr (KIND == 0) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int Q = lsel + 2 * lg + 8 * i;  // 4 consecutive local indices
                    float2 x[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) x[e] = rawat(4 * Q + e);
                    const int atom = Q >> 3, q = Q & 7;
                    float4 rh, ih, rl, il;
                    rh.x = tf32_rna(x[0].x); rh.y = tf32_rna(x[1].x); rh.z = tf32_rna(x[2].x); rh.w = tf32_rna(x[3].x);
                    ih.x = tf32_rna(x[0].y); ih.y = tf32_rna(x[1].y); ih.z = tf32_rna(x[2].y); ih.w = tf32_rna(x[3].y);
                    const uint32_t o_re = atom * (kRowsB * 128) + swz(2 * j, q);
                    const uint32_t o_im = atom * (kRowsB * 128) + swz(2 * j + 1, q);
                    *reinterpret_cast<float4*>(bst + o_re) = rh;
                    *reinterpret_cast<float4*>(bst + o_im) = ih;
                    if constexpr (SPLITS == 3) {
                        rl.x = tf32_rna(x[0].x - rh.x); rl.y = tf32_rna(x[1].x - rh.y);
                        rl.z = tf32_rna(x[2].x - rh.z); rl.w = tf32_rna(x[3].x - rh.w);
                        il.x = tf32_rna(x[0].y - ih.x); il.y = tf32_rna(x[1].y - ih.y);
                        il.z = tf32_rna(x[2].y - ih.z); il.w = tf32_rna(x[3].y - ih.w);
                        *reinterpret_cast<float4*>(bst + LY::kBBytes + o_re) = rl;
                        *reinterpret_cast<float4*>(bst + LY::kBBytes + o_im) = il;
                    }
                }
            } else {
                const int Q = lsel + 2 * lg;  // 8 consecutive local indices
                float2 x[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] = rawat(8 * Q + e);
                uint32_t rh[4], ih[4], rl[4], il[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const __nv_bfloat16 r0 = __float2bfloat16_rn(x[2 * e].x), r1 = __float2bfloat16_rn(x[2 * e + 1].x);
                    const __nv_bfloat16 i0 = __float2bfloat16_rn(x[2 * e].y), i1 = __float2bfloat16_rn(x[2 * e + 1].y);
                    rh[e] = (uint32_t)__bfloat16_as_ushort(r0) | ((uint32_t)__bfloat16_as_ushort(r1) << 16);
                    ih[e] = (uint32_t)__bfloat16_as_ushort(i0) | ((uint32_t)__bfloat16_as_ushort(i1) << 16);
                    if constexpr (SPLITS == 3) {
                        const __nv_bfloat16 a0 = __float2bfloat16_rn(x[2 * e].x - __bfloat162float(r0));
                        const __nv_bfloat16 a1 = __float2bfloat16_rn(x[2 * e + 1].x - __bfloat162float(r1));
                        const __nv_bfloat16 b0 = __float2bfloat16_rn(x[2 * e].y - __bfloat162float(i0));
                        const __nv_bfloat16 b1 = __float2bfloat16_rn(x[2 * e + 1].y - __bfloat162float(i1));
                        rl[e] = (uint32_t)__bfloat16_as_ushort(a0) | ((uint32_t)__bfloat16_as_ushort(a1) << 16);
                        il[e] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
                    }
                }
                const uint32_t o_re = swz(2 * j, Q), o_im = swz(2 * j + 1, Q);
                *reinterpret_cast<uint4*>(bst + o_re) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                *reinterpret_cast<uint4*>(bst + o_im) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                if constexpr (SPLITS == 3) {
                    *reinterpret_cast<uint4*>(bst + LY::kBBytes + o_re) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                    *reinterpret_cast<uint4*>(bst + LY::kBBytes + o_im) = make_uint4(il[0], il[1], il[2], il[3]);
                }
            }
            fence_async_smem();
            mbar_arrive(&full[stage]);
            // raw slot of tile `it` is free for tile it+kRaw
            if (!group_sync(prodbar, gph, err, abort_flag)) break;
        }
        cp_async_wait<0>();  // nothing of ours still in flight at exit
    } else if (warp == kMmaWarp) {
        // ================= MMA issuer
        if (lane == 0) {
            constexpr int ksteps = KIND == 0 ? 8 : 4;
            bool issued = false;
            for (uint64_t it = 0;; ++it) {
                const uint64_t t = blockIdx.x + it * gridDim.x;
                if (t >= a.ntiles) break;
                const int stage = (int)(it % kStages), acc = (int)(it & 1);
                if (!mbar_wait(&full[stage], (uint32_t)((it / kStages) & 1), err, abort_flag)) break;
                if (!mbar_wait(&dempty[acc], (uint32_t)(((it >> 1) & 1) ^ 1), err, abort_flag)) break;
                tc_after();
                const uint32_t b_base = su32(sm + LY::kB + stage * LY::kStageBytes);
                const uint32_t d = tmem + (uint32_t)(kTmemD + acc * kRowsB);
                // products, small terms first: (A_lo, B_hi), (A_hi, B_lo), (A_hi, B_hi)
                constexpr int nprod = SPLITS == 3 ? 3 : 1;
                for (int pr = 0; pr < nprod; ++pr) {
                    const int asel = (SPLITS == 3 && pr == 0) ? 1 : 0;
                    const int bsel = (SPLITS == 3 && pr == 1) ? 1 : 0;
#pragma unroll
                    for (int kk = 0; kk < ksteps; ++kk) {
                        // 8 TMEM columns per K step (8 TF32, or 16 packed BF16)
                        const uint32_t a_t = tmem + (uint32_t)(asel * LY::kACols + 8 * kk);
                        const uint32_t boff = KIND == 0 ? (kk >> 2) * (kRowsB * 128) + (kk & 3) * 32 : kk * 32;
                        umma_ts<KIND>(d, a_t, sdesc(b_base + bsel * LY::kBBytes + boff), (pr > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                umma_commit(&empty[stage]);
                umma_commit(&dfull[acc]);
                issued = true;
            }
            if (issued) {  // drain: wait (bounded, even after an abort) for every MMA issued above
                umma_commit(drain);
                const long long t0 = clock64();
                while (!mbar_try(drain, 0)) {
                    if (clock64() - t0 > kTimeout) {
                        atomicExch(err, 1);
                        break;
                    }
                }
            }
        }
    } else {
        // ================= epilogue: warp q owns TMEM lanes 32q..32q+31 =
        // real rows (lanes 0-15) and imaginary rows (16-31) of outputs
        // r = 16q + (lane & 15)
        const int tid = threadIdx.x;  // 0..127
        const int h = lane >> 4, r = 16 * warp + (lane & 15);
        uint32_t gph = 0;
        for (uint64_t it = 0;; ++it) {
            const uint64_t t = blockIdx.x + it * gridDim.x;
            if (t >= a.ntiles) break;
            const int acc = (int)(it & 1);
            if (!__all_sync(0xffffffffu, mbar_wait(&dfull[acc], (uint32_t)((it >> 1) & 1), err, abort_flag))) break;
            tc_after();
            float v[64];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kTmemD + acc * kRowsB);
#pragma unroll
            for (int c = 0; c < 4; ++c) tmem_ld16(taddr + 16 * c, v + 16 * c);
            tmem_ld_wait();
            tc_before();
            mbar_arrive(&dempty[acc]);
            // lane h=0 (real row) finishes sets 0..15, lane h=1 (imaginary row) sets 16..31
            float w[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) w[c] = __shfl_xor_sync(0xffffffffu, h ? v[c] : v[32 + c], 16);
            float2 y[16];
            if (h == 0) {  // own = Re-row (sets 0..15), w = Im-row columns 0..31
#pragma unroll
                for (int si = 0; si < 16; ++si) {
                    y[si].x = v[2 * si] - w[2 * si + 1];
                    y[si].y = v[2 * si + 1] + w[2 * si];
                }
            } else {       // own = Im-row (sets 16..31), w = Re-row columns 32..63
#pragma unroll
                for (int si = 0; si < 16; ++si) {
                    y[si].x = w[2 * si] - v[32 + 2 * si + 1];
                    y[si].y = w[2 * si + 1] + v[32 + 2 * si];
                }
            }
#pragma unroll
            for (int si = 0; si < 16; ++si) {
                const int s = 16 * h + si;
                if constexpr (Q0T) ystage[s * 66 + r] = y[si];
                else ystage[r * 34 + s] = y[si];
            }
            if (!group_sync(epibar, gph, err, abort_flag)) break;
            // coalesced 16-byte write-back
            if constexpr (Q0T) {
                const int lp = tid & 31;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int s = (tid >> 5) + 4 * i;
                    uint64_t base = t * kSets + s;
#pragma unroll
                    for (int b = 0; b < 6; ++b) base = insert_zero(base, a.sorted[b]);
                    const float4 y2 = *reinterpret_cast<const float4*>(ystage + s * 66 + 2 * lp);
                    *reinterpret_cast<float4*>(psi + base + soff[2 * lp]) = y2;
                }
            } else {
                const int sp = tid & 15;
                uint64_t base = t * kSets + 2 * sp;
#pragma unroll
                for (int b = 0; b < 6; ++b) base = insert_zero(base, a.sorted[b]);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int l = (tid >> 4) + 8 * i;
                    const float4 y2 = *reinterpret_cast<const float4*>(ystage + l * 34 + 2 * sp);
                    *reinterpret_cast<float4*>(psi + base + soff[l]) = y2;
                }
            }
            if (!group_sync(epibar, gph, err, abort_flag)) break;
        }
    }

    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int SPLITS, int KIND, bool Q0T>
static cudaError_t run_q(float2* psi, const float2* U, const Args& a, int* err, cudaStream_t st) {
    using LY = Layout<SPLITS, KIND>;
    const int smem = LY::kTotal + 1024;  // slack to align the base to 1024 bytes
    cudaError_t e = cudaFuncSetAttribute(k_gemm6<SPLITS, KIND, Q0T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<uint64_t>(a.ntiles, (uint64_t)num_sms());
    k_gemm6<SPLITS, KIND, Q0T><<<grid, kThreads, smem, st>>>(psi, U, a, err);
    return cudaGetLastError();
}

template <int SPLITS, int KIND>
static cudaError_t run(float2* psi, const float2* U, const Args& a, int* err, cudaStream_t st) {
    return a.sorted[0] == 0 ? run_q<SPLITS, KIND, true>(psi, U, a, err, st)
                            : run_q<SPLITS, KIND, false>(psi, U, a, err, st);
}

}  // namespace tc

bool gemm_supported(int n, int k) { return k == 6 && n >= 11; }

cudaError_t launch_gemm(void* psi, int n, int k, const int* qubits, const void* dmat, int precision, int* err,
                        cudaStream_t st) {
    if (!gemm_supported(n, k)) return cudaErrorInvalidValue;
    for (int i = 0; i + 1 < 6; ++i)  // the planner hands over descending qubit lists
        if (qubits[i] <= qubits[i + 1]) return cudaErrorInvalidValue;
    tc::Args a{};
    for (int l = 0; l < 64; ++l) {
        uint64_t o = 0;
        for (int i = 0; i < 6; ++i)
            if ((l >> (5 - i)) & 1) o |= 1ull << qubits[i];
        a.off[l] = o;
    }
    for (int i = 0; i < 6; ++i) a.sorted[i] = qubits[i];
    std::sort(a.sorted, a.sorted + 6);
    a.ntiles = (1ull << (n - 6)) / tc::kSets;
    float2* p = (float2*)psi;
    const float2* U = (const float2*)dmat;
    switch (precision) {
        case QS_PREC_TF32: return tc::run<1, 0>(p, U, a, err, st);
        case QS_PREC_3XTF32: return tc::run<3, 0>(p, U, a, err, st);
        case QS_PREC_3XBF16: return tc::run<3, 1>(p, U, a, err, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qsgb
