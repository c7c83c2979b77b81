// Dense 6-qubit gates on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// A fused k-qubit gate applies the same 2^k x 2^k complex matrix U to each
// of the 2^(n-k) disjoint sets of 2^k amplitudes (Section 3), i.e. it is the
// product U X with X = 2^k x 2^(n-k).  With real arithmetic:
//   D = [Re U; Im U] (128 x 64)  x  B^T,   B = [re x_s; im x_s] per set s,
//   y_s = (D_top re - D_bot im) + i (D_top im + D_bot re).
// Both operands are K-major (K = the gate's 64 local indices) with the
// 128-byte swizzle; the accumulator D (128 lanes x 64 fp32 columns per tile
// of 32 sets) lives in tensor memory.  Precision modes on complex64 states:
//   TF32     one product, operands rounded to TF32
//   3xTF32   A_hi B_hi + A_hi B_lo + A_lo B_hi, hi = TF32(x), lo = x - hi
//   3xBF16   the same split with bfloat16 parts
// all with FP32 accumulation.
//
// One persistent CTA per SM, warp-specialised:
//   warps 0-3  epilogue: tensor memory -> registers -> recombine -> HBM
//   warps 4-7  producer: gather 32 sets x 64 amplitudes (coalesced), split,
//              write swizzled shared-memory stages
//   warp 8     one thread issues the MMAs and commits to mbarriers
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
constexpr int kStages = 3;
constexpr int kThreads = 288;
constexpr int kTmemCols = 128;     // two accumulators of 64 columns
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
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

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

template <int KIND>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc<0>()), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc<1>()), "r"(acc)
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

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of 16-byte chunk `c` of row `r` in a [rows][128 B] swizzled block
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

struct Args {
    uint64_t off[64];   // offset of local index l (Kronecker order)
    int sorted[6];      // target bits ascending
    uint64_t ntiles;    // 2^(n-6) / 32
};

template <int SPLITS, int KIND>
struct Layout {
    static constexpr int kAtomsK = KIND == 0 ? 2 : 1;           // 64 K elements
    static constexpr int kABytes = kAtomsK * 128 * 128;          // one A split
    static constexpr int kBBytes = kAtomsK * kRowsB * 128;       // one B split, one stage
    static constexpr int SPLITS_A = SPLITS == 3 ? 2 : 1;        // stored parts (hi, lo)
    static constexpr int kA = 0;
    static constexpr int kB = kA + SPLITS_A * kABytes;
    static constexpr int kStageBytes = SPLITS_A * kBBytes;
    static constexpr int kX = kB + kStages * kStageBytes;        // Im-row exchange, 64 x 65 floats
    static constexpr int kY = kX + 64 * 65 * 4;                  // output staging, 64 x 34 float2
    static constexpr int kOff = kY + 64 * 34 * 8;                // offsets (64 x u64)
    static constexpr int kBar = kOff + 64 * 8;                   // barriers
    static constexpr int kTotal = kBar + 128;
};

template <int SPLITS, int KIND>
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
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint64_t* soff = reinterpret_cast<uint64_t*>(sm + LY::kOff);
    float* xbuf = reinterpret_cast<float*>(sm + LY::kX);
    float2* ystage = reinterpret_cast<float2*>(sm + LY::kY);

    // ---- A = [Re U; Im U] split into hi (and lo) parts, swizzled K-major
    for (int idx = threadIdx.x; idx < 128 * 64; idx += blockDim.x) {
        const int m = idx >> 6, l = idx & 63;
        const float v = m < 64 ? U[m * 64 + l].x : U[(m - 64) * 64 + l].y;
        if constexpr (KIND == 0) {
            const float hi = tf32_rna(v);
            const int atom = l >> 5, kin = l & 31;
            const uint32_t o = atom * (128 * 128) + swz(m, kin >> 2) + (kin & 3) * 4;
            *reinterpret_cast<float*>(sm + LY::kA + o) = hi;
            if constexpr (SPLITS == 3) *reinterpret_cast<float*>(sm + LY::kA + LY::kABytes + o) = tf32_rna(v - hi);
        } else {
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            const uint32_t o = swz(m, l >> 3) + (l & 7) * 2;
            *reinterpret_cast<__nv_bfloat16*>(sm + LY::kA + o) = hi;
            if constexpr (SPLITS == 3)
                *reinterpret_cast<__nv_bfloat16*>(sm + LY::kA + LY::kABytes + o) =
                    __float2bfloat16_rn(v - __bfloat162float(hi));
        }
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) soff[i] = a.off[i];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 128);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&dfull[s], 1);
            mbar_init(&dempty[s], 128);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= 4 && warp < 8) {
        // ================= producer
        const int pw = warp - 4;
        const int j = (lane & 15) + 16 * (pw & 1), lsel = lane >> 4, lg = pw >> 1;
        for (uint64_t it = 0;; ++it) {
            const uint64_t t = blockIdx.x + it * gridDim.x;
            if (t >= a.ntiles) break;
            const int stage = (int)(it % kStages);
            const uint32_t ph = (uint32_t)((it / kStages) & 1);
            if (!mbar_wait(&empty[stage], ph ^ 1, err, abort_flag)) break;
            uint64_t base = t * kSets + j;
#pragma unroll
            for (int i = 0; i < 6; ++i) base = insert_zero(base, a.sorted[i]);
            unsigned char* bst = sm + LY::kB + stage * LY::kStageBytes;
            if constexpr (KIND == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int Q = lsel + 2 * lg + 4 * i;  // chunk of 4 consecutive local indices
                    float2 x[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) x[e] = psi[base + soff[4 * Q + e]];
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
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int Q = lsel + 2 * lg + 4 * i;  // chunk of 8 consecutive local indices
                    float2 x[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) x[e] = psi[base + soff[8 * Q + e]];
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
            }
            fence_async_smem();
            mbar_arrive(&full[stage]);
        }
    } else if (warp == 8) {
        // ================= MMA issuer
        if (lane == 0) {
            const uint32_t a_base = su32(sm + LY::kA);
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
                const uint32_t d = tmem + (uint32_t)(acc * kRowsB);
                // products, small terms first: (A_lo, B_hi), (A_hi, B_lo), (A_hi, B_hi)
                constexpr int nprod = SPLITS == 3 ? 3 : 1;
                for (int pr = 0; pr < nprod; ++pr) {
                    const int asel = (SPLITS == 3 && pr == 0) ? 1 : 0;
                    const int bsel = (SPLITS == 3 && pr == 1) ? 1 : 0;
#pragma unroll
                    for (int kk = 0; kk < ksteps; ++kk) {
                        const uint32_t aoff = KIND == 0 ? (kk >> 2) * (128 * 128) + (kk & 3) * 32 : kk * 32;
                        const uint32_t boff = KIND == 0 ? (kk >> 2) * (kRowsB * 128) + (kk & 3) * 32 : kk * 32;
                        umma<KIND>(d, sdesc(a_base + asel * LY::kABytes + aoff), sdesc(b_base + bsel * LY::kBBytes + boff),
                                   (pr > 0 || kk > 0) ? 1u : 0u);
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
        // ================= epilogue (warps 0-3 own TMEM lanes 32w .. 32w+31)
        const int tid = threadIdx.x;  // 0..127
        for (uint64_t it = 0;; ++it) {
            const uint64_t t = blockIdx.x + it * gridDim.x;
            if (t >= a.ntiles) break;
            const int acc = (int)(it & 1);
            if (!mbar_wait(&dfull[acc], (uint32_t)((it >> 1) & 1), err, abort_flag)) break;
            tc_after();
            float v[64];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * kRowsB);
#pragma unroll
            for (int c = 0; c < 4; ++c) tmem_ld16(taddr + 16 * c, v + 16 * c);
            tmem_ld_wait();
            tc_before();
            mbar_arrive(&dempty[acc]);
            if (warp >= 2) {  // rows of Im U: hand them to the Re U rows
                const int r = tid - 64;
#pragma unroll
                for (int c = 0; c < 64; ++c) xbuf[r * 65 + c] = v[c];
            }
            named_sync(1, 128);
            if (warp < 2) {
                const int r = tid;
#pragma unroll
                for (int s = 0; s < kSets; ++s) {
                    float2 y;
                    y.x = v[2 * s] - xbuf[r * 65 + 2 * s + 1];
                    y.y = v[2 * s + 1] + xbuf[r * 65 + 2 * s];
                    ystage[r * 34 + s] = y;
                }
            }
            named_sync(1, 128);
            // coalesced write-back: thread owns set j, rows l = tid/32 + 4i
            const int j = tid & 31;
            uint64_t base = t * kSets + j;
#pragma unroll
            for (int i = 0; i < 6; ++i) base = insert_zero(base, a.sorted[i]);
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int l = (tid >> 5) + 4 * i;
                psi[base + soff[l]] = ystage[l * 34 + j];
            }
            named_sync(1, 128);
        }
    }

    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int SPLITS, int KIND>
static cudaError_t run(float2* psi, const float2* U, const Args& a, int* err, cudaStream_t st) {
    using LY = Layout<SPLITS, KIND>;
    const int smem = LY::kTotal + 1024;  // slack to align the base to 1024 bytes
    cudaError_t e = cudaFuncSetAttribute(k_gemm6<SPLITS, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<uint64_t>(a.ntiles, (uint64_t)num_sms());
    k_gemm6<SPLITS, KIND><<<grid, kThreads, smem, st>>>(psi, U, a, err);
    return cudaGetLastError();
}

}  // namespace tc

bool gemm_supported(int n, int k) { return k == 6 && n >= 11; }

cudaError_t launch_gemm(void* psi, int n, int k, const int* qubits, const void* dmat, int precision, int* err,
                        cudaStream_t st) {
    if (!gemm_supported(n, k)) return cudaErrorInvalidValue;
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
