// Dense 6-qubit gates on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// A fused k-qubit gate applies the same 2^k x 2^k complex matrix U to each
// of the 2^(n-k) disjoint sets of 2^k amplitudes (Section 3), i.e. it is the
// product Y = X U^T with X = the 2^(n-k) x 2^k matrix whose rows are the
// sets.  In real arithmetic, for a tile of 64 sets:
//   D = A G^T,  A = [re x_s ; im x_s] (128 rows: set s, re/im; K = the 64
//   local indices),  G = [Re U row r ; Im U row r] (128 rows n = 2r + h),
//   y_s[r] = (D[s,re][2r] - D[s,im][2r+1]) + i (D[s,im][2r] + D[s,re][2r+1]).
// The state tile is the A operand and lives in tensor memory: producers
// write it there from registers (tcgen05.st), so the state never passes
// through shared memory on its way in.  The gate (split into hi/lo parts)
// is the B operand, resident in shared memory (128-byte swizzle, K-major)
// for the whole kernel.  D (128 lanes x 128 FP32 columns) is read back by
// the epilogue, which combines real and imaginary rows with one exchange
// between lane pairs and stores each set's outputs straight to HBM.
// Precision modes on complex64 states:
//   TF32     one product, operands rounded to TF32
//   3xTF32   A_lo G_hi + A_hi G_lo + A_hi G_hi, hi = TF32(x), lo = x - hi
//   3xBF16   the same split with bfloat16 parts
//   3xFP16   the same split with IEEE half parts (11-bit significands like
//            TF32, at the 16-bit MMA rate).  FP16's exponent range is
//            narrow, so every set's amplitudes are scaled by a power of two
//            2^e_s that brings their largest magnitude to [2^14, 2^15), and
//            the gate by 2^e_G likewise; the epilogue multiplies each
//            output by 2^-(e_s + e_G).  Power-of-two scaling is exact, so
//            the split keeps its ~22 bits whatever the state's magnitude.
// all with FP32 accumulation.
//
// One persistent CTA per SM, warp-specialised:
//   warps 0-3  epilogue: warp q owns TMEM lanes 32q..32q+31 (sets 16q..16q+15)
//   warps 4-11 producer: warp w owns the lanes of quadrant w % 4 and half of
//              the local indices; it gathers them with cp.async (16-byte
//              pairs, coalesced) several tiles ahead into its own slice of a
//              shared-memory ring, then rounds/splits them into tensor memory
//   warp 12    one thread issues the MMAs and commits to mbarriers
// Tensor memory: two A buffers (hi | lo) and two accumulators, 512 columns.
// Every mbarrier wait is bounded (about two seconds of clock64); on timeout
// the CTA sets the error flag, drains its MMAs, frees tensor memory, exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>

#include "qs_device.cuh"
#include "qs_internal.h"
#include "qs_tc.cuh"

namespace qsgb {
namespace tc {

constexpr int kSets = 64;          // sets per tile: TMEM lane 32q + 16c + j = (set 16q + j, re/im c)
constexpr int kEpiWarps = 4, kProdWarps = 8;
constexpr int kMmaWarp = kEpiWarps + kProdWarps;
constexpr int kThreads = 32 * (kMmaWarp + 1);
constexpr int kTmemCols = 512;
constexpr int kTmemABuf = 128;     // columns per A buffer (hi | lo)
constexpr int kTmemD = 256;        // two accumulators of kN columns

struct Args {
    uint64_t off[64];   // offset of local index l; the gate's qubits are in
                        // descending order, so local bit b is the b-th lowest target
    int sorted[6];      // target bits ascending
    uint64_t ntiles;    // 2^(n-6) / 64
    int inject;         // testing: block 0's first producer warp skips its first arrival
    int swap_p;         // > 0: writes exchange index bits 0 and swap_p (two of the set bits)
    int store_mode;     // 0: 8-byte stores (pairs when qubit 0 is a target); 1: qubit 1 a target
                        // and 0 not, lane pairs exchange; 2: qubits 0 and 1 targets, 32-byte stores
    int sidx[4];        // slot position bit of set bit a (a < 4) in a producer's raw slice
    int lidx[5];        // slot position bit of local bit b (b < 5)
    uint64_t hoff[5];   // amplitude offset of slot position bits 4..8
    int wsw[5];         // swizzle: slot bit 4 + h set flips slot bits 1..3 by wsw[h]
};

template <int SPLITS, int KIND>
struct Layout {
    static constexpr int SPLITS_A = SPLITS == 3 ? 2 : 1;        // stored parts (hi, lo)
    static constexpr int kACols = KIND == 0 ? 64 : 32;          // TMEM columns of one A part
    static constexpr int kAtomsK = KIND == 0 ? 2 : 1;           // 128-byte atoms along K
    static constexpr int kGBytes = kAtomsK * kN * 128;          // one gate part
    static constexpr int kG = 0;
    static constexpr int kRaw = 4;                               // gathered tiles in flight
    // one producer warp's slice of a raw slot: 16 sets x 32 local indices,
    // 32 memory lines of 16 amplitudes (float2)
    static constexpr int kWarpRaw = 512 * 8;
    static constexpr int kSlot = kProdWarps * kWarpRaw;
    static constexpr int kR = kG + SPLITS_A * kGBytes;
    // FP16: per-set scale exponents of the 4 most recent tiles, and the two
    // producer warps' half-row maxima of a quadrant
    static constexpr int kScale = kR + kRaw * kSlot;
    static constexpr int kBar = kScale + (KIND == 2 ? 4 * 64 * 4 + 2 * 2 * 64 * 4 + 64 : 0);   // barriers
    static constexpr int kTotal = kBar + 128;
};

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    tmem_ld16(taddr, v);
    tmem_ld16(taddr + 16, v + 16);
}

template <int SPLITS, int KIND, bool Q0T>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm6(float2* __restrict__ psi, const float2* __restrict__ U, const __grid_constant__ Args a, int* err) {
    using LY = Layout<SPLITS, KIND>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base by pointer arithmetic on the shared array, so the
    // compiler keeps the accesses below in the shared window (LDS/STS)
    unsigned char* sm = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    uint64_t* afull = reinterpret_cast<uint64_t*>(sm + LY::kBar);
    uint64_t* aempty = afull + 2;
    uint64_t* dfull = aempty + 2;
    uint64_t* dempty = dfull + 2;
    uint64_t* drain = dempty + 2;
    uint64_t* sfull = drain + 1;       // FP16: a tile's set scales written (4 slots)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sfull + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    unsigned int* gmax_slot = reinterpret_cast<unsigned int*>(tmem_slot + 2);
    int* escale = reinterpret_cast<int*>(sm + LY::kScale);                 // [4 tiles][64 sets]
    float* hmax = reinterpret_cast<float*>(sm + LY::kScale + 4 * 64 * 4);   // [2 parities][2 halves][64 sets]

    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&afull[b], kProdWarps);
            mbar_init(&aempty[b], 1);
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], kEpiWarps);
        }
        mbar_init(drain, 1);
        for (int i = 0; i < 4; ++i) mbar_init(&sfull[i], 4);
        *abort_flag = 0;
        *gmax_slot = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // FP16: the gate's largest magnitude sets its scale 2^eG
    int eG = 0;
    if constexpr (KIND == 2) {
        __syncthreads();
        float mx = 0.f;
        for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
            const float2 u = U[idx];
            mx = fmaxf(mx, fmaxf(fabsf(u.x), fabsf(u.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(gmax_slot, __float_as_uint(mx));   // non-negative floats order as integers
        __syncthreads();
        eG = fp16_scale_exp(__uint_as_float(*gmax_slot));
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // ---- the gate into shared memory: row n = 2r + h holds (h ? Im : Re) U[r][:],
    // hi part then lo part, K-major with the 128-byte swizzle
    for (int idx = threadIdx.x; idx < kN * 64; idx += blockDim.x) {
        const int n = idx >> 6, k = idx & 63, r = n >> 1, h = n & 1;
        const float v = h ? U[r * 64 + k].y : U[r * 64 + k].x;
        if constexpr (KIND == 0) {
            const uint32_t o = (uint32_t)((k >> 5) * (kN * 128)) + swz(n, (k & 31) >> 2) + 4u * (uint32_t)(k & 3);
            const float hi = tf32_round(v);
            *reinterpret_cast<float*>(sm + LY::kG + o) = hi;
            if constexpr (SPLITS == 3) *reinterpret_cast<float*>(sm + LY::kG + LY::kGBytes + o) = tf32_round(v - hi);
        } else if constexpr (KIND == 1) {
            const uint32_t o = swz(n, k >> 3) + 2u * (uint32_t)(k & 7);
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            *reinterpret_cast<__nv_bfloat16*>(sm + LY::kG + o) = hi;
            if constexpr (SPLITS == 3)
                *reinterpret_cast<__nv_bfloat16*>(sm + LY::kG + LY::kGBytes + o) = __float2bfloat16_rn(v - __bfloat162float(hi));
        } else {
            const uint32_t o = swz(n, k >> 3) + 2u * (uint32_t)(k & 7);
            const float vs = v * exp2i(eG);
            const __half hi = __float2half_rn(vs);
            *reinterpret_cast<__half*>(sm + LY::kG + o) = hi;
            if constexpr (SPLITS == 3) *reinterpret_cast<__half*>(sm + LY::kG + LY::kGBytes + o) = __float2half_rn(vs - __half2float(hi));
        }
    }
    fence_async_smem();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait_then_release();  // the state is the previous pass's output

    if (warp >= kEpiWarps && warp < kMmaWarp) {
        // ================= producer: TMEM quadrant q, local indices 32kh..32kh+31
        const int pw = warp - kEpiWarps, q = warp & 3, kh = pw >> 2;
        const int j = lane & 15, c = lane >> 4;  // this lane's TMEM row: set 16q + j, part c
        unsigned char* slice = sm + LY::kR + pw * LY::kWarpRaw;
        // The warp's slice of a tile (16 sets x 32 local indices = 512
        // amplitudes) is gathered by 128-byte memory lines: every amplitude
        // index bit 0..3 is one of the slice's bits (a low set bit or a low
        // target), so the slice is 32 whole lines.  Copy i: lanes 8u..8u+7
        // move line 4i + u, 16 bytes each (index bits 1..3 = lane & 7), into
        // 128 contiguous bytes of the warp's raw slot -- one memory request
        // per line, whatever the targets.  Slot position of slice element
        // (set j, local kl): low 4 bits = index bits 0..3, high 5 bits = the
        // other slice bits (a.sidx, a.lidx give each slice bit's position).
        uint64_t goff[8];
        int gdst[8];
        {
            const int u = lane >> 3, piece = lane & 7;
            const uint64_t fixed = set_base((uint64_t)(16 * q), a.sorted) + a.off[32 * kh] + (uint64_t)(piece << 1);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int L = 4 * i + u;
                uint64_t hp = 0;
#pragma unroll
                for (int h = 0; h < 5; ++h) hp += ((L >> h) & 1) ? a.hoff[h] : 0ull;
                goff[i] = fixed + hp;
                int wl = 0;
#pragma unroll
                for (int h = 0; h < 5; ++h) wl ^= ((L >> h) & 1) ? a.wsw[h] : 0;
                gdst[i] = L * 16 + ((2 * piece) ^ (wl << 1));   // swizzled: see rswz
            }
        }
        // slot position of (set j, local kl) = rp_lo[kl & 3] ^ rp_hi[kl >> 2], after
        // the swizzle rswz(p) = p ^ (XOR of wsw[h] over slot bits 4 + h of p) << 1:
        // chosen per pass so the 16 sets a warp reads at once fall into distinct
        // bank groups; bit 0 stays (16-byte pairs stay whole), each line maps
        // onto itself, and rswz is linear, so parts combine by XOR
        auto rswz = [&](uint32_t p) {
            int w = 0;
#pragma unroll
            for (int h = 0; h < 5; ++h) w ^= ((p >> (4 + h)) & 1) ? a.wsw[h] : 0;
            return p ^ ((uint32_t)w << 1);
        };
        uint32_t rp_lo[4], rp_hi[8];
        {
            uint32_t pj = 0;
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2) pj |= (uint32_t)((j >> s2) & 1) << a.sidx[s2];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                rp_lo[i] = rswz(pj | ((i & 1) ? 1u << a.lidx[0] : 0u) | ((i & 2) ? 1u << a.lidx[1] : 0u));
#pragma unroll
            for (int i = 0; i < 8; ++i)
                rp_hi[i] = rswz(((i & 1) ? 1u << a.lidx[2] : 0u) | ((i & 2) ? 1u << a.lidx[3] : 0u) |
                                ((i & 4) ? 1u << a.lidx[4] : 0u));
        }
        auto issue = [&](uint64_t itx) {
            const uint64_t tt = blockIdx.x + itx * gridDim.x;
            if (tt < a.ntiles) {
                float2* dstp = reinterpret_cast<float2*>(slice + (itx % LY::kRaw) * LY::kSlot);
                const float2* src = psi + set_base(tt * kSets, a.sorted);
#pragma unroll
                for (int i = 0; i < 8; ++i) cp_async16(dstp + gdst[i], src + goff[i]);
            }
            cp_async_commit();  // one group per tile, possibly empty
        };
        for (int p = 0; p < LY::kRaw - 1; ++p) issue((uint64_t)p);
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        for (uint64_t it = 0;; ++it) {
            const uint64_t t = blockIdx.x + it * gridDim.x;
            if (t >= a.ntiles) break;
            issue(it + LY::kRaw - 1);
            cp_async_wait<LY::kRaw - 1>();
            __syncwarp();  // the warp's copies of tile `it` are visible to all its lanes
            const int b = (int)(it & 1);
            const float2* rs = reinterpret_cast<const float2*>(slice + (it % LY::kRaw) * LY::kSlot);
            float v[32];  // part c of x[set][32kh + kl], kl = 0..31
#pragma unroll
            for (int kl = 0; kl < 32; ++kl) {
                const float2 xv = rs[rp_lo[kl & 3] ^ rp_hi[kl >> 2]];
                v[kl] = c ? xv.y : xv.x;
            }
            // (the raw slot is warp-private: it was read before the wait below)
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&aempty[b], (uint32_t)(((it >> 1) & 1) ^ 1), err, abort_flag));
            float sc = 1.f;
            if constexpr (KIND == 2) {
                // the set's scale: largest magnitude over both parts (lanes c = 0, 1)
                // and both halves of K (the other producer warp of this quadrant,
                // through shared memory and a named barrier of the pair); the pair
                // also agrees on stopping, so both always pass the same barriers
                float m = 0.f;
#pragma unroll
                for (int e = 0; e < 32; ++e) m = fmaxf(m, fabsf(v[e]));
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
                float* hm = hmax + (int)(it & 1) * 128;                                // [half][set]
                int* okf = reinterpret_cast<int*>(hmax + 256) + (int)(it & 1) * 8;     // [half][quadrant]
                if (c == 0) hm[kh * 64 + 16 * q + j] = m;
                if (lane == 0) okf[kh * 4 + q] = ok ? 1 : 0;
                named_bar_sync(1 + q, 64);
                m = fmaxf(m, hm[(kh ^ 1) * 64 + 16 * q + j]);
                if (!(ok && okf[(kh ^ 1) * 4 + q] != 0)) break;
                const int e = fp16_scale_exp(m);
                sc = exp2i(e);
                if (kh == 0) {
                    if (c == 0) escale[(int)(it & 3) * 64 + 16 * q + j] = e;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sfull[it & 3]);
                }
            } else {
                if (!ok) break;
            }
            tc_after();
            const uint32_t acol = lane_base + (uint32_t)(b * kTmemABuf);
            if constexpr (KIND == 0) {
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    uint32_t hw[16], lw[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float hi = tf32_round(v[16 * hf + e]);
                        hw[e] = __float_as_uint(hi);
                        if constexpr (SPLITS == 3) lw[e] = __float_as_uint(tf32_round(v[16 * hf + e] - hi));
                    }
                    tmem_st16(acol + (uint32_t)(32 * kh + 16 * hf), hw);
                    if constexpr (SPLITS == 3) tmem_st16(acol + (uint32_t)(LY::kACols + 32 * kh + 16 * hf), lw);
                }
            } else if constexpr (KIND == 1) {  // two bf16 per column, lower K index in the low half
                uint32_t hw[16], lw[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
                    hw[e] = *reinterpret_cast<const uint32_t*>(&hb);
                    if constexpr (SPLITS == 3) {
                        const float2 hf = __bfloat1622float2(hb);
                        const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
                        lw[e] = *reinterpret_cast<const uint32_t*>(&lb);
                    }
                }
                tmem_st16(acol + (uint32_t)(16 * kh), hw);
                if constexpr (SPLITS == 3) tmem_st16(acol + (uint32_t)(LY::kACols + 16 * kh), lw);
            } else {  // two scaled halves per column, lower K index in the low half
                uint32_t hw[16], lw[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const float x0 = v[2 * e] * sc, x1 = v[2 * e + 1] * sc;
                    const __half2 hh = __floats2half2_rn(x0, x1);
                    hw[e] = *reinterpret_cast<const uint32_t*>(&hh);
                    if constexpr (SPLITS == 3) {
                        const float2 hf = __half22float2(hh);
                        const __half2 lh = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
                        lw[e] = *reinterpret_cast<const uint32_t*>(&lh);
                    }
                }
                tmem_st16(acol + (uint32_t)(16 * kh), hw);
                if constexpr (SPLITS == 3) tmem_st16(acol + (uint32_t)(LY::kACols + 16 * kh), lw);
            }
            tmem_st_wait();
            tc_before();
            __syncwarp();  // all lanes' tensor-memory writes done; raw slot `it` free again
            // (testing: a withheld arrival makes the MMA issuer's wait run out)
            const bool withhold = a.inject && blockIdx.x == 0 && it == 0 && pw == 0;
            if (lane == 0 && !withhold) mbar_arrive(&afull[b]);
        }
        cp_async_wait<0>();  // nothing of ours still in flight at exit
    } else if (warp == kMmaWarp) {
        // ================= MMA issuer
        if (lane == 0) {
            constexpr int ksteps = KIND == 0 ? 8 : 4;
            const uint32_t g_base = su32(sm + LY::kG);
            bool issued = false;
            for (uint64_t it = 0;; ++it) {
                const uint64_t t = blockIdx.x + it * gridDim.x;
                if (t >= a.ntiles) break;
                const int b = (int)(it & 1);
                const uint32_t ph = (uint32_t)((it >> 1) & 1);
                if (!mbar_wait(&afull[b], ph, err, abort_flag)) break;
                if (!mbar_wait(&dempty[b], ph ^ 1, err, abort_flag)) break;
                tc_after();
                const uint32_t d = tmem + (uint32_t)(kTmemD + b * kN);
                // products, small terms first: (A_lo, G_hi), (A_hi, G_lo), (A_hi, G_hi)
                constexpr int nprod = SPLITS == 3 ? 3 : 1;
#pragma unroll
                for (int pr = 0; pr < nprod; ++pr) {
                    const int asel = (SPLITS == 3 && pr == 0) ? 1 : 0;
                    const int gsel = (SPLITS == 3 && pr == 1) ? 1 : 0;
#pragma unroll
                    for (int kk = 0; kk < ksteps; ++kk) {
                        // 8 TMEM columns per K step (8 TF32, or 16 packed BF16)
                        const uint32_t a_t = tmem + (uint32_t)(b * kTmemABuf + asel * LY::kACols + 8 * kk);
                        const uint32_t goff = KIND == 0 ? (kk >> 2) * (kN * 128) + (kk & 3) * 32 : kk * 32;
                        umma_ts<KIND>(d, a_t, sdesc(g_base + gsel * LY::kGBytes + goff), (pr > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                umma_commit(&aempty[b]);
                umma_commit(&dfull[b]);
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
        // ================= epilogue: warp q reads TMEM lanes 32q..32q+31;
        // lane (c, j) holds row (set 16q + j, part c) of D.  Per chunk of 16
        // outputs r, the real-part lane finishes the first 8, the imaginary-
        // part lane the last 8, after one exchange of 16 values.
        const int q = warp, j = lane & 15, c = lane >> 4;
        for (uint64_t it = 0;; ++it) {
            const uint64_t t = blockIdx.x + it * gridDim.x;
            if (t >= a.ntiles) break;
            const int b = (int)(it & 1);
            if (!__all_sync(0xffffffffu, mbar_wait(&dfull[b], (uint32_t)((it >> 1) & 1), err, abort_flag))) break;
            tc_after();
            float unscale = 1.f, unscale_g = 1.f;
            if constexpr (KIND == 2) {  // undo the set's and the gate's power-of-two scales
                if (!__all_sync(0xffffffffu, mbar_wait(&sfull[it & 3], (uint32_t)((it >> 2) & 1), err, abort_flag))) break;
                unscale = exp2i(-escale[(int)(it & 3) * 64 + 16 * q + j]);
                unscale_g = exp2i(-eG);
            }
            uint64_t sb = set_base(t * kSets + (uint64_t)(16 * q + j), a.sorted);
            if (!Q0T && a.swap_p > 0) {  // the tile's footprint maps onto itself: in place
                const uint64_t dbit = (sb ^ (sb >> a.swap_p)) & 1u;
                sb ^= dbit | (dbit << a.swap_p);
            }
            float2* dst = psi + sb;
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kTmemD + b * kN);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                float d[32];  // d[2rr + h] = D[row][2(16ch + rr) + h]
                tmem_ld32(taddr + (uint32_t)(32 * ch), d);
                tmem_ld_wait();
                if (ch == 3) {  // the accumulator is free for tile it+2
                    tc_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&dempty[b]);
                }
                float rcv[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) rcv[e] = __shfl_xor_sync(0xffffffffu, c ? d[e] : d[16 + e], 16);
                float2 y[8];
#pragma unroll
                for (int rr = 0; rr < 8; ++rr) {
                    if (c == 0) {  // own: D[re][.]; partner: D[im][.] of outputs 16ch + rr
                        y[rr].x = d[2 * rr] - rcv[2 * rr + 1];
                        y[rr].y = rcv[2 * rr] + d[2 * rr + 1];
                    } else {       // own: D[im][.]; partner: D[re][.] of outputs 16ch + 8 + rr
                        y[rr].x = rcv[2 * rr] - d[16 + 2 * rr + 1];
                        y[rr].y = d[16 + 2 * rr] + rcv[2 * rr + 1];
                    }
                    if constexpr (KIND == 2) {  // two steps: the product of the scales may leave FP32's range
                        y[rr].x = (y[rr].x * unscale) * unscale_g;
                        y[rr].y = (y[rr].y * unscale) * unscale_g;
                    }
                }
                if constexpr (Q0T) {
                    if (a.store_mode == 2) {
                        // qubits 0 and 1 both targets: outputs r..r+3 are 32
                        // contiguous bytes, one 256-bit store each (full sectors)
#pragma unroll
                        for (int rr = 0; rr < 8; rr += 4) {
                            const uint64_t o = c ? a.off[16 * ch + 8 + rr] : a.off[16 * ch + rr];
                            asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(dst + o),
                                         "f"(y[rr].x), "f"(y[rr].y), "f"(y[rr + 1].x), "f"(y[rr + 1].y), "f"(y[rr + 2].x),
                                         "f"(y[rr + 2].y), "f"(y[rr + 3].x), "f"(y[rr + 3].y)
                                         : "memory");
                        }
                    } else {
                        // pairs (r, r+1) are adjacent amplitudes
#pragma unroll
                        for (int rr = 0; rr < 8; rr += 2) {
                            const uint64_t o = c ? a.off[16 * ch + 8 + rr] : a.off[16 * ch + rr];
                            *reinterpret_cast<float4*>(dst + o) = make_float4(y[rr].x, y[rr].y, y[rr + 1].x, y[rr + 1].y);
                        }
                    }
                } else if (a.store_mode == 1) {
                    // qubit 1 a target, qubit 0 not: the 32 bytes of sets (s, s+1) x
                    // outputs (r, r+1) sit in lanes j, j+1; one exchange lets each
                    // lane store 16 bytes, so every instruction writes full sectors
                    const bool odd = (j & 1) != 0;
#pragma unroll
                    for (int rr = 0; rr < 8; rr += 2) {
                        const float2 send = odd ? y[rr] : y[rr + 1];
                        float2 got;
                        got.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
                        got.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
                        const int r = 16 * ch + 8 * c + rr;
                        // one store instruction for both lanes of the pair
                        float2* const p = odd ? dst - 1 + a.off[r + 1] : dst + a.off[r];
                        const float4 val = odd ? make_float4(got.x, got.y, y[rr + 1].x, y[rr + 1].y)
                                               : make_float4(y[rr].x, y[rr].y, got.x, got.y);
                        *reinterpret_cast<float4*>(p) = val;
                    }
                } else {
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr) {
                        const uint64_t o = c ? a.off[16 * ch + 8 + rr] : a.off[16 * ch + rr];
                        dst[o] = y[rr];
                    }
                }
            }
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
    cudaError_t e = allow_max_dynamic_smem(k_gemm6<SPLITS, KIND, Q0T>);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<uint64_t>(a.ntiles, (uint64_t)num_sms());
    e = launch_pdl(k_gemm6<SPLITS, KIND, Q0T>, dim3(grid), dim3(kThreads), (size_t)smem, st, psi, U, a, err);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int SPLITS, int KIND>
static cudaError_t run(float2* psi, const float2* U, const Args& a, int* err, cudaStream_t st) {
    return a.sorted[0] == 0 ? run_q<SPLITS, KIND, true>(psi, U, a, err, st)
                            : run_q<SPLITS, KIND, false>(psi, U, a, err, st);
}

}  // namespace tc

// at least one tile of 64 sets
bool gemm_supported(int n, int k) { return k == 6 && n >= 12; }

cudaError_t launch_gemm(void* psi, int n, int k, const int* qubits, const void* dmat, int precision, int* err,
                        cudaStream_t st, int inject, int swap_p) {
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
    a.inject = inject ? 1 : 0;
    a.swap_p = -1;
    a.store_mode = 0;
    if (swap_p >= 0) {  // bit 0 and swap_p must be among the set bits 0..3 (the 4 lowest non-targets)
        uint64_t tmask = 0;
        for (int i = 0; i < 6; ++i) tmask |= 1ull << qubits[i];
        int rank = 0, found = -1;
        for (int b = 0; b < n && rank < 4; ++b) {
            if ((tmask >> b) & 1) continue;
            if (b == swap_p) found = rank;
            ++rank;
        }
        if (tmask & 1 || found < 1) return cudaErrorInvalidValue;
        a.swap_p = swap_p;
    }
    {
        uint64_t tmask = 0;
        for (int i = 0; i < 6; ++i) tmask |= 1ull << qubits[i];
        if ((tmask & 3) == 3 && ((uintptr_t)psi & 31) == 0) a.store_mode = 2;
        else if ((tmask & 3) == 2 && a.swap_p < 0) a.store_mode = 1;
        // a producer's slice: set bits 0..3 (the 4 lowest non-targets) and
        // local bits 0..4 (the 5 lowest targets); index bits 0..3 keep their
        // place, the other 5 slice bits take slot position bits 4..8
        int np[4], cnt = 0;
        for (int b = 0; b < n && cnt < 4; ++b)
            if (!((tmask >> b) & 1)) np[cnt++] = b;
        int hi = 4;
        for (int s2 = 0; s2 < 4; ++s2) {
            if (np[s2] < 4) a.sidx[s2] = np[s2];
            else {
                a.sidx[s2] = hi;
                a.hoff[hi - 4] = 1ull << np[s2];
                ++hi;
            }
        }
        for (int l = 0; l < 5; ++l) {
            if (a.sorted[l] < 4) a.lidx[l] = a.sorted[l];
            else {
                a.lidx[l] = hi;
                a.hoff[hi - 4] = 1ull << a.sorted[l];
                ++hi;
            }
        }
        if (hi != 9) return cudaErrorInvalidValue;   // cannot happen: bits 0..3 are slice bits
        // swizzle: give each set bit held in a high slot bit a flip of bits 1..3
        // outside the span of the set bits already placed (bank group = slot
        // bits 0..3), so the 16 sets of a warp's read spread over the banks
        for (int h = 0; h < 5; ++h) a.wsw[h] = 0;
        uint32_t span[16] = {0};
        int nspan = 1;  // span of the placed bank-group vectors (starts with 0)
        auto add = [&](uint32_t v) {
            bool in = false;
            for (int i = 0; i < nspan; ++i) in |= span[i] == v;
            if (in) return false;
            for (int i = 0, m = nspan; i < m; ++i) span[nspan++] = span[i] ^ v;
            return true;
        };
        for (int s2 = 0; s2 < 4; ++s2)
            if (a.sidx[s2] < 4) add(1u << a.sidx[s2]);
        for (int s2 = 0; s2 < 4; ++s2) {
            if (a.sidx[s2] < 4) continue;
            for (int w = 1; w < 8; ++w)
                if (add((uint32_t)w << 1)) {
                    a.wsw[a.sidx[s2] - 4] = w;
                    break;
                }
        }
    }
    float2* p = (float2*)psi;
    const float2* U = (const float2*)dmat;
    switch (precision) {
        case QS_PREC_TF32: return tc::run<1, 0>(p, U, a, err, st);
        case QS_PREC_3XTF32: return tc::run<3, 0>(p, U, a, err, st);
        case QS_PREC_3XBF16: return tc::run<3, 1>(p, U, a, err, st);
        case QS_PREC_3XFP16: return tc::run<3, 2>(p, U, a, err, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qsgb
