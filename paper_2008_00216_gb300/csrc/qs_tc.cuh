// Building blocks of the tensor-core passes (tcgen05, sm_103a): mbarrier
// waits with a bound, tensor-memory loads/stores, MMA issue and commit,
// shared-memory matrix descriptors, cp.async, the TF32 rounding and the
// power-of-two scaling of the FP16 split.  Inline PTX only.
#ifndef QS_TC_CUH
#define QS_TC_CUH

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "qs_device.cuh"

namespace qsgb {
namespace tc {

constexpr int kN = 128;                    // MMA N: gate rows (r, Re/Im)
constexpr long long kTimeout = 4ll << 30;  // bounded waits: about two seconds of clock64

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
// The same test, but the thread may be suspended until the phase completes
// or about 20 us pass (a waiting warp then takes no issue slots from the
// warps doing work on its scheduler).
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}
// Bounded wait: true when the phase completed; false after the timeout (the
// error flag and the CTA's abort flag are set) or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err, volatile int* abort_flag) {
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_sleep(b, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kTimeout) {
            atomicExch(err, 1);
            *abort_flag = 1;
            return false;
        }
    }
}

// named barrier among `count` threads (whole warps)
__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
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

// instruction descriptor: FP32 accumulate, A/B TF32 (kind 0), BF16 (kind
// 1) or FP16 (kind 2), both K-major, M = 128, N = kN
template <int KIND>
__host__ __device__ constexpr uint32_t ab_format() {
    return KIND == 0 ? 2u : KIND == 1 ? 1u : 0u;
}
template <int KIND>
__host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | (ab_format<KIND>() << 7) | (ab_format<KIND>() << 10) | ((uint32_t)(kN >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// D[tmem] (+)= A[tmem] * B[smem]^T: A (the state tile) is read from tensor
// memory (row m in lane m, K along columns), B (the gate) from shared memory
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
            "r"(a_tmem), "l"(b), "r"(idesc<KIND>()), "r"(acc)
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

// x rounded to TF32 (10 explicit mantissa bits), to nearest with ties away
// from zero: add half of the lowest kept bit to the magnitude, clear the 13
// dropped bits (a carry into the exponent is the correct result).  Same as
// cvt.rna.tf32.f32 for finite x, in two integer operations.
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// FP16 scaling: the power-of-two exponent e that brings a largest magnitude
// m into [2^14, 2^15) (m * 2^e stays below FP16's 65504), within
// [-113, 126] so that 2^e and 2^-e are normal floats (FP32 subnormal maxima
// are treated as 2^-126); 0 for m = 0.
__device__ __forceinline__ int fp16_scale_exp(float m) {
    if (!(m > 0.f)) return 0;
    int ex = (int)((__float_as_uint(m) >> 23) & 0xFFu) - 127;   // floor(log2 m) for normal m
    if (ex < -126) ex = -126;
    return min(126, max(-113, 14 - ex));
}
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((uint32_t)(127 + e) << 23); }

// index of the first amplitude of set x (zero bits inserted at the targets)
__device__ __forceinline__ uint64_t set_base(uint64_t x, const int* sorted) {
#pragma unroll
    for (int b = 0; b < 6; ++b) x = insert_zero(x, sorted[b]);
    return x;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Programmatic dependent launch: the tensor-core passes are launched so that
// their prologue (barriers, tensor memory, the gate in shared memory) may
// overlap the previous kernel's last CTAs.  Every thread waits here for the
// previous grid's completion and memory before it touches a state, then
// lets the next pass be scheduled (its CTAs only start where an SM frees up).
__device__ __forceinline__ void pdl_wait_then_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// launch `kernel` with programmatic stream serialisation allowed
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// byte offset of 16-byte chunk `c` of row `r` in a [rows][128 B] swizzled block
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

}  // namespace tc
}  // namespace qsgb

#endif  // QS_TC_CUH
