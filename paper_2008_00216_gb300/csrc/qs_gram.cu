// Gradients of fused blocks on the tensor cores (tcgen05, sm_103a).
//
// The adjoint gradient of gate l, U_l = exp(-i theta_l P_l / 2), is
// Im <lambda_l|P_l|psi_l> with psi_l, lambda_l the two states just after the
// gate (the reverse sweep).  When the sweep undoes a whole fused block
// B = U_m ... U_1 on six qubits T at once (a group of the commuting-reorder
// fusion of Sections 4.2-4.5), every gradient inside it
// still follows from the two states taken before B^dagger is applied: with
// x_s, y_s the 64 amplitudes of psi and lambda over T in set s,
//   M = sum_s x_s y_s^dagger                      (64 x 64, all sets)
//   <lambda_l|P_l|psi_l> = tr(P_l M_l),  M_m = M,  M_{l-1} = U_l^dagger M_l U_l
// (psi_l = W^dagger psi, lambda_l = W^dagger lambda, W = U_m ... U_{l+1}).
// M is a product of two state-sized operands contracted over the sets, a
// GEMM: k_gram6 computes it with 3xTF32 tcgen05 MMAs, both operands staged
// in shared memory; k_gram_reduce sums the CTAs' parts in FP64 in a fixed
// order; k_block_grads runs the recursion over each block's gates (one CTA
// per block) and writes the gradients.
//
// k_gram6, per stage of 32 sets (K = 32 TF32 = one 128-byte swizzle row):
//   A (128 rows r = 2l + c: part c of psi's local index l) and
//   B (the same rows for lambda), each split into hi = TF32(v) and
//   lo = TF32(v - hi), K-major with the 128-byte swizzle;
//   D (128 x 128 FP32 in tensor memory) += A_lo B_hi^T + A_hi B_lo^T + A_hi B_hi^T
//   Re M[l][l'] = D[2l][2l'] + D[2l+1][2l'+1],  Im M[l][l'] = D[2l+1][2l'] - D[2l][2l'+1].
// One persistent CTA per SM, warp-specialised:
//   warps 0-3   epilogue: warp q owns tensor-memory lanes 32q..32q+31
//   warps 4-19  producers: warp w copies 8 local indices of psi (w < 12) or
//               lambda (rows of 32 sets) with cp.async into a raw ring kRaw
//               stages ahead, then splits its own rows into the operands
//   warp 20     one thread issues the MMAs
// Two accumulators alternate every kFlush stages; the epilogue adds each
// finished one into the CTA's FP64 part of M, so no FP32 sum runs over more
// than 2048 sets.  Every mbarrier wait is bounded (about two seconds of
// clock64); on timeout the CTA sets the error flag, drains its MMAs, frees
// tensor memory and exits.  Launched with programmatic dependent launch: the
// prologue runs while the previous pass finishes (pdl_wait_then_release).
#include <stdint.h>

#include <algorithm>

#include "qs_device.cuh"
#include "qs_internal.h"
#include "qs_tc.cuh"

namespace qsgb {
namespace gram {

using namespace tc;

constexpr int kKSets = 32;                    // sets per stage
constexpr int kStages = 2;                    // operand stages (split, swizzled)
constexpr int kRaw = 3;                       // raw stages in flight (cp.async)
constexpr int kEpiWarps = 4, kProdWarps = 16;
constexpr int kMmaWarp = kEpiWarps + kProdWarps;
constexpr int kThreads = 32 * (kMmaWarp + 1);
constexpr int kPart = 128 * 128;              // bytes of one operand part: 128 rows x 128 bytes
constexpr int kStage = 4 * kPart;             // psi hi, psi lo, lambda hi, lambda lo
constexpr int kRawStage = 128 * 256;          // 128 rows of 32 sets (complex64), 8 rows per producer warp
constexpr int kRawOff = kStages * kStage;
constexpr int kBar = kRawOff + kRaw * kRawStage;
constexpr int kSmem = kBar + 256;
constexpr int kTmemCols = 256;                // two accumulators of 128 columns
constexpr int kFlush = 64;                    // stages per accumulator period
constexpr int kMElems = 2 * 64 * 64;          // one M in FP64: Re rows, then Im rows

struct Args {
    uint64_t off[64];   // amplitude offset of local index l (local bit b = the b-th lowest target)
    int sorted[6];      // targets ascending
    uint64_t ntiles;    // 2^(n-6) / 32
};

__device__ __forceinline__ void umma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc<0>()), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    tmem_ld16(taddr, v);
    tmem_ld16(taddr + 16, v + 16);
}

// W = 2^w: the w lowest qubits are not targets, so W consecutive sets are
// adjacent amplitudes; a lane copies W of them at once (32 / W lanes per
// row, W rows per warp instruction).  W = 0: qubit 0 is a target (local
// bit 0), so rows 2i and 2i + 1 of a set are adjacent amplitudes: a lane
// copies that pair (raw layout [row pair][set][2]) and converts as W = 1.
// W = 3: qubits 0..2 are targets, so a warp's 8 rows of a set are 64
// adjacent bytes, four lanes' copies (raw layout [set][8 rows], 16-byte
// chunks swizzled by the set so that a lane per set reads them without
// conflicts); converts as W = 1.
template <int W>
__global__ void __launch_bounds__(kThreads, 1)
    k_gram6(const float2* __restrict__ psi, const float2* __restrict__ lam, const __grid_constant__ Args a,
            double* __restrict__ ws, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kBar);
    uint64_t* empty = full + kStages;
    uint64_t* dfull = empty + kStages;
    uint64_t* dempty = dfull + 2;
    uint64_t* drain = dempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], kProdWarps);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], kEpiWarps);
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
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait_then_release();  // psi and lambda are the previous passes' outputs
    // this CTA's stages: tiles blockIdx.x + it * gridDim.x, it < my
    const uint64_t my = a.ntiles > blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t nper = (my + kFlush - 1) / kFlush;

    if (warp >= kEpiWarps && warp < kMmaWarp) {
        // ================= producers: 8 local indices of one state
        const int pw = warp - kEpiWarps;
        const float2* src = pw < 8 ? psi : lam;
        const int l0 = (pw & 7) * 8;
        const uint32_t part = pw < 8 ? 0u : 2u * kPart;
        constexpr int WC = (W == 0 || W == 3) ? 1 : W;  // sets per lane in the conversion
        constexpr int LPR = 32 / WC, NLD = 8 / WC;  // lanes per row, rows per lane
        const int rsub = lane / LPR, s0 = (lane % LPR) * WC;  // row within a copy, first set
        // raw layout: [stage][warp][row 0..7][32 sets] complex64 (256-byte rows)
        auto raw_at = [&](int slot, int row) {
            return sm + kRawOff + slot * kRawStage + pw * 2048 + row * 256 + s0 * 8;
        };
        auto copy = [&](uint64_t it) {  // the warp's rows of stage it, into raw slot it % kRaw
            if (it < my) {
                const uint64_t t = blockIdx.x + it * gridDim.x;
                const float2* p = src + set_base(t * kKSets + (uint64_t)s0, a.sorted);
                const int slot = (int)(it % kRaw);
                if constexpr (W == 3) {  // per set, the warp's 8 rows are 64 adjacent bytes: 4 lanes, 16 each
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int ss = 8 * i + (lane >> 2), c = lane & 3;
                        const float2* g = src + set_base(t * kKSets + (uint64_t)ss, a.sorted) + a.off[l0] + 2 * c;
                        unsigned char* d =
                            sm + kRawOff + slot * kRawStage + pw * 2048 + ss * 64 + ((c ^ ((ss >> 1) & 3)) << 4);
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(d)), "l"(g) : "memory");
                    }
                } else if constexpr (W == 0) {  // rows 2i, 2i + 1 of set `lane`: 16 adjacent bytes
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(
                                         sm + kRawOff + slot * kRawStage + pw * 2048 + i * 512 + lane * 16)),
                                     "l"(p + a.off[l0 + 2 * i])
                                     : "memory");
                } else {
#pragma unroll
                    for (int i = 0; i < NLD; ++i) {
                        const int row = W * i + rsub;
                        const float2* g = p + a.off[l0 + row];
                        if constexpr (W == 2)
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(raw_at(slot, row))),
                                         "l"(g)
                                         : "memory");
                        else
                            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(su32(raw_at(slot, row))),
                                         "l"(g)
                                         : "memory");
                    }
                }
            }
            cp_async_commit();  // one group per stage, empty past the end
        };
        auto put = [&](uint64_t it) {
            const int st = (int)(it % kStages);
            const uint64_t u = it / kStages;
            cp_async_wait<kRaw - 1>();  // this lane's copies of stage it are done
            __syncwarp();               // and the other lanes' (each warp reads only its own rows)
            float v[NLD][2 * WC];
            const int slot = (int)(it % kRaw);
            if constexpr (W == 3) {  // lane = set; chunk c holds rows 2c, 2c + 1 (swizzled by set)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float4 x = *reinterpret_cast<const float4*>(sm + kRawOff + slot * kRawStage + pw * 2048 +
                                                                      lane * 64 + ((c ^ ((lane >> 1) & 3)) << 4));
                    v[2 * c][0] = x.x;
                    v[2 * c][1] = x.y;
                    v[2 * c + 1][0] = x.z;
                    v[2 * c + 1][1] = x.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < NLD; ++i) {
                    const unsigned char* q = W == 0 ? sm + kRawOff + slot * kRawStage + pw * 2048 + (i >> 1) * 512 + lane * 16 + (i & 1) * 8
                                                    : raw_at(slot, WC * i + rsub);
                    if constexpr (W == 2) {
                        const float4 x = *reinterpret_cast<const float4*>(q);
                        v[i][0] = x.x;
                        v[i][1] = x.y;
                        v[i][2] = x.z;
                        v[i][3] = x.w;
                    } else {
                        const float2 x = *reinterpret_cast<const float2*>(q);
                        v[i][0] = x.x;
                        v[i][1] = x.y;
                    }
                }
            }
            if (u > 0 && !mbar_wait(&empty[st], (uint32_t)((u - 1) & 1), err, abort_flag)) return false;
            unsigned char* hi = sm + st * kStage + part;
            unsigned char* lo = hi + kPart;
#pragma unroll
            for (int i = 0; i < NLD; ++i) {
                const int r = 2 * (l0 + WC * i + rsub);  // the real row; r + 1 the imaginary
                const uint32_t o = swz(r, s0 >> 2) + 4u * (uint32_t)(s0 & 3);
                const uint32_t o1 = swz(r + 1, s0 >> 2) + 4u * (uint32_t)(s0 & 3);
                float rh[WC], rl[WC], ih[WC], il[WC];
#pragma unroll
                for (int e = 0; e < WC; ++e) {
                    rh[e] = tf32_round(v[i][2 * e]);
                    rl[e] = tf32_round(v[i][2 * e] - rh[e]);
                    ih[e] = tf32_round(v[i][2 * e + 1]);
                    il[e] = tf32_round(v[i][2 * e + 1] - ih[e]);
                }
                if constexpr (WC == 1) {
                    *reinterpret_cast<float*>(hi + o) = rh[0];
                    *reinterpret_cast<float*>(lo + o) = rl[0];
                    *reinterpret_cast<float*>(hi + o1) = ih[0];
                    *reinterpret_cast<float*>(lo + o1) = il[0];
                } else {
                    *reinterpret_cast<float2*>(hi + o) = make_float2(rh[0], rh[1]);
                    *reinterpret_cast<float2*>(lo + o) = make_float2(rl[0], rl[1]);
                    *reinterpret_cast<float2*>(hi + o1) = make_float2(ih[0], ih[1]);
                    *reinterpret_cast<float2*>(lo + o1) = make_float2(il[0], il[1]);
                }
            }
            fence_async_smem();
            __syncwarp();  // also: every lane has read raw slot it % kRaw before it is refilled
            if (lane == 0) mbar_arrive(&full[st]);
            return true;
        };
        for (int it = 0; it < kRaw - 1; ++it) copy((uint64_t)it);
        for (uint64_t it = 0; it < my; ++it) {
            copy(it + kRaw - 1);
            if (!put(it)) break;
        }
        cp_async_wait<0>();  // nothing of ours in flight at exit
    } else if (warp == kMmaWarp) {
        // ================= MMA issuer
        if (lane == 0) {
            bool issued = false;
            for (uint64_t it = 0; it < my; ++it) {
                const int st = (int)(it % kStages);
                const uint64_t u = it / kStages, per = it / kFlush;
                const int acc = (int)(per & 1);
                const bool first = (it % kFlush) == 0;
                if (first && per >= 2 && !mbar_wait(&dempty[acc], (uint32_t)(((per - 2) >> 1) & 1), err, abort_flag))
                    break;
                if (!mbar_wait(&full[st], (uint32_t)(u & 1), err, abort_flag)) break;
                tc_after();
                const uint32_t d = tmem + (uint32_t)(128 * acc);
                const uint32_t base = su32(sm + st * kStage);
                // products, small terms first: (A_lo, B_hi), (A_hi, B_lo), (A_hi, B_hi)
#pragma unroll
                for (int pr = 0; pr < 3; ++pr) {
                    const uint32_t aoff = pr == 0 ? (uint32_t)kPart : 0u;
                    const uint32_t boff = 2u * kPart + (pr == 1 ? (uint32_t)kPart : 0u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_ss(d, sdesc(base + aoff + 32u * kk), sdesc(base + boff + 32u * kk),
                                (first && pr == 0 && kk == 0) ? 0u : 1u);
                }
                umma_commit(&empty[st]);
                if ((it % kFlush) == kFlush - 1 || it + 1 == my) umma_commit(&dfull[acc]);
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
        // ================= epilogue: lane holds row m = 32q + lane of D, i.e.
        // part c = m & 1 of local index l = m >> 1; with its partner lane
        // (m ^ 1) it forms row l of Re M (c = 0) or Im M (c = 1)
        const int q = warp, m = 32 * q + lane, l = m >> 1, c = m & 1;
        double* dst = ws + (size_t)blockIdx.x * kMElems + (size_t)c * 4096 + (size_t)l * 64;
        for (uint64_t per = 0; per < nper; ++per) {
            const int acc = (int)(per & 1);
            if (!__all_sync(0xffffffffu, mbar_wait(&dfull[acc], (uint32_t)((per >> 1) & 1), err, abort_flag))) break;
            tc_after();
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 * acc);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                float d[32];  // d[2e + c'] = D[m][2(16ch + e) + c']
                tmem_ld32(taddr + (uint32_t)(32 * ch), d);
                tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const float pd = __shfl_xor_sync(0xffffffffu, d[2 * e + 1], 1);  // partner's D[m^1][2l'+1]
                    const double v = c == 0 ? (double)d[2 * e] + (double)pd : (double)d[2 * e] - (double)pd;
                    const int lp = 16 * ch + e;
                    dst[lp] = per == 0 ? v : dst[lp] + v;
                }
            }
            tc_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[acc]);
        }
    }

    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// M = the sum of the CTAs' parts, FP64, in a fixed order: a block takes 32
// entries of one Gram matrix (blockIdx.y); its 8 warps sum every 8th part
// (coalesced rows of 32), then one warp adds the 8 partial sums in order.
constexpr int kRedParts = 8;
__global__ void __launch_bounds__(32 * kRedParts) k_gram_reduce(const double* __restrict__ ws_all, int parts,
                                                                 size_t slot_elems, double* __restrict__ M_all) {
    __shared__ double acc[kRedParts][32];
    const double* ws = ws_all + slot_elems * blockIdx.y;
    double* M = M_all + (size_t)kMElems * blockIdx.y;
    const int o = blockIdx.x * 32 + (threadIdx.x & 31), g = threadIdx.x >> 5;
    double s0 = 0.0, s1 = 0.0;
    int b = g;
    for (; b + kRedParts < parts; b += 2 * kRedParts) {
        s0 += ws[(size_t)b * kMElems + o];
        s1 += ws[(size_t)(b + kRedParts) * kMElems + o];
    }
    if (b < parts) s0 += ws[(size_t)b * kMElems + o];
    acc[g][threadIdx.x & 31] = s0 + s1;
    __syncthreads();
    if (g == 0) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kRedParts; ++k) t += acc[k][threadIdx.x];
        M[o] = t;
    }
}

// One CTA per block: M (FP64 from k_gram_reduce) to FP32 in shared memory,
// then the block's gates from the last to the first: the gradient of a
// gate with a generator, tr(P M) = i^ny sum_j (-1)^popc(j & zmask) M[j][j ^ xmask],
// then M <- U^dagger M U.  Per gate, the local index maps (gate index of
// each local index, the local index of each gate index) and U are
// tabulated in shared memory first.  A gate on d = 2^k indices updates M
// in d x d blocks (rows base_r | loc(a), columns base_c | loc(b)), each
// owned by one thread: in place, one pass; diagonal gates elementwise.
constexpr int kGradThreads = 512;

template <int D>
__device__ __forceinline__ void block_update(float2 (*Ms)[65], const float2* Us, const int* loc, int r0, int c0) {
    float2 x[D][D], t[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) x[a][b] = Ms[r0 | loc[a]][c0 | loc[b]];
    // t = U^dagger x: t[a][b] = sum_e conj(U[e][a]) x[e][b]
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < D; ++e) {
                const float2 u = Us[e * D + a], v = x[e][b];
                s.x += u.x * v.x + u.y * v.y;
                s.y += u.x * v.y - u.y * v.x;
            }
            t[a][b] = s;
        }
    // x = t U: x[a][b] = sum_e t[a][e] U[e][b]
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < D; ++e) {
                const float2 u = Us[e * D + b], v = t[a][e];
                s.x += v.x * u.x - v.y * u.y;
                s.y += v.x * u.y + v.y * u.x;
            }
            Ms[r0 | loc[a]][c0 | loc[b]] = s;
        }
}

__global__ void __launch_bounds__(kGradThreads) k_block_grads(const double* __restrict__ Mall,
                                                                const BlockGradGate* __restrict__ gates,
                                                                const int* __restrict__ gate0,
                                                                const float2* __restrict__ mats,
                                                                double* __restrict__ sums) {
    extern __shared__ float2 gsm[];
    float2 (*Ms)[65] = reinterpret_cast<float2 (*)[65]>(gsm);            // M, rows padded
    float2 (*Ts)[65] = reinterpret_cast<float2 (*)[65]>(gsm + 64 * 65);  // U^dagger M (gates on 3+ qubits)
    float2* Us = gsm + 2 * 64 * 65;                                      // U (up to 64 x 64)
    __shared__ int gi_of[64], base_of[64], loc_of[64], blk_of[64];
    const int slot = blockIdx.x, tid = threadIdx.x;
    const double* Mg = Mall + (size_t)slot * kMElems;
    for (int i = tid; i < 4096; i += kGradThreads) Ms[i >> 6][i & 63] = make_float2((float)Mg[i], (float)Mg[4096 + i]);
    __syncthreads();
    for (int gi = gate0[slot]; gi < gate0[slot + 1]; ++gi) {
        const int k = gates[gi].k, d = 1 << k, param = gates[gi].param, diag = gates[gi].diag, flags = gates[gi].flags;
        const uint32_t moff = gates[gi].moff;
        // tables and U (M is not touched in this phase), and the gradient
        if (tid < 64) {
            int li = 0, gm = 0;
            for (int t = 0; t < k; ++t) {
                const int b = gates[gi].lb[t];
                li = (li << 1) | ((tid >> b) & 1);
                gm |= 1 << b;
            }
            gi_of[tid] = li;
            base_of[tid] = tid & ~gm;
            if (tid < d) {
                int x = 0;
                for (int t = 0; t < k; ++t)
                    if ((tid >> (k - 1 - t)) & 1) x |= 1 << gates[gi].lb[t];
                loc_of[tid] = x;
            }
            // the tid-th index with the gate's bits zero (64 / d of them)
            if (tid < 64 / d) {
                int x = 0, src = 0;
                for (int b = 0; b < 6; ++b) {
                    if ((gm >> b) & 1) continue;
                    if ((tid >> src) & 1) x |= 1 << b;
                    ++src;
                }
                blk_of[tid] = x;
            }
        } else if (tid < 128 && !(flags & kGradNoUpdate)) {
            const int e = tid - 64;
            if (diag)  // diagonal entries
                Us[e] = mats[moff + (size_t)(e < d ? e : 0) * ((flags & kGradCompactDiag) ? 1 : d + 1)];
        }
        if (!diag && !(flags & kGradNoUpdate))
            for (int e = tid; e < d * d; e += kGradThreads) Us[e] = mats[moff + e];
        if (param >= 0 && tid >= 128 && tid < 160) {
            const int ln = tid - 128;
            const int xm = gates[gi].xmask, zm = gates[gi].zmask, ny = gates[gi].ny;
            float2 v = make_float2(0.f, 0.f);
            for (int j = ln; j < 64; j += 32) {
                const float2 x = Ms[j][j ^ xm];
                const float sg = (__popc(j & zm) & 1) ? -1.f : 1.f;
                v.x += sg * x.x;
                v.y += sg * x.y;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
            }
            if (ln == 0) {  // Im(i^ny v)
                const int r = ny & 3;
                const float g = r == 0 ? v.y : r == 1 ? v.x : r == 2 ? -v.y : -v.x;
                sums[2 * (size_t)param] = 0.0;
                sums[2 * (size_t)param + 1] = (double)g;
            }
        }
        __syncthreads();  // tables and U written; the gradient has read M
        if (flags & kGradNoUpdate) continue;
        if (diag) {  // M[i][j] <- conj(u_i) M[i][j] u_j
            for (int e = tid; e < 4096; e += kGradThreads) {
                const int i = e >> 6, j = e & 63;
                const float2 ui = Us[gi_of[i]], uj = Us[gi_of[j]], x = Ms[i][j];
                const float2 y = make_float2(ui.x * x.x + ui.y * x.y, ui.x * x.y - ui.y * x.x);
                Ms[i][j] = make_float2(y.x * uj.x - y.y * uj.y, y.x * uj.y + y.y * uj.x);
            }
        } else if (d == 2 || d == 4) {
            const int nb = 64 / d;
            for (int e = tid; e < nb * nb; e += kGradThreads) {
                const int r0 = blk_of[e / nb], c0 = blk_of[e % nb];
                if (d == 2) block_update<2>(Ms, Us, loc_of, r0, c0);
                else block_update<4>(Ms, Us, loc_of, r0, c0);
            }
        } else {
            // T = U^dagger M: T[i][j] = sum_a conj(U[a][lo(i)]) M[base(i) | loc(a)][j]
            for (int e = tid; e < 4096; e += kGradThreads) {
                const int i = e >> 6, j = e & 63, lo = gi_of[i], r0 = base_of[i];
                float2 s2 = make_float2(0.f, 0.f);
                for (int a2 = 0; a2 < d; ++a2) {
                    const float2 u = Us[a2 * d + lo], x = Ms[r0 | loc_of[a2]][j];
                    s2.x += u.x * x.x + u.y * x.y;
                    s2.y += u.x * x.y - u.y * x.x;
                }
                Ts[i][j] = s2;
            }
            __syncthreads();
            // M = T U: M[i][j] = sum_a T[i][base(j) | loc(a)] U[a][lo(j)]
            for (int e = tid; e < 4096; e += kGradThreads) {
                const int i = e >> 6, j = e & 63, lo = gi_of[j], c0 = base_of[j];
                float2 s2 = make_float2(0.f, 0.f);
                for (int a2 = 0; a2 < d; ++a2) {
                    const float2 u = Us[a2 * d + lo], x = Ts[i][c0 | loc_of[a2]];
                    s2.x += x.x * u.x - x.y * u.y;
                    s2.y += x.x * u.y + x.y * u.x;
                }
                Ms[i][j] = s2;
            }
        }
        __syncthreads();  // M is complete; the tables may be rewritten
    }
}

}  // namespace gram

bool gram_supported(int n) { return n >= 12; }

static int gram_grid(int n) { return (int)std::min<uint64_t>((1ull << (n - 6)) / gram::kKSets, (uint64_t)num_sms()); }

// one part per CTA of the n-qubit Gram kernel's grid
size_t gram_workspace_elems(int n) { return (size_t)gram_grid(n) * gram::kMElems; }

cudaError_t launch_gram(const void* psi, const void* lam, int n, const int* targets, double* ws, int* err,
                        cudaStream_t st) {
    if (!gram_supported(n)) return cudaErrorInvalidValue;
    for (int i = 0; i + 1 < 6; ++i)  // descending target list
        if (targets[i] <= targets[i + 1]) return cudaErrorInvalidValue;
    gram::Args a{};
    for (int l = 0; l < 64; ++l) {
        uint64_t o = 0;
        for (int i = 0; i < 6; ++i)
            if ((l >> (5 - i)) & 1) o |= 1ull << targets[i];
        a.off[l] = o;
    }
    for (int i = 0; i < 6; ++i) a.sorted[i] = targets[i];
    std::sort(a.sorted, a.sorted + 6);
    a.ntiles = (1ull << (n - 6)) / gram::kKSets;
    const int grid = gram_grid(n);
    // the lowest target bounds how many consecutive sets are adjacent amplitudes
    auto run = [&](auto kern) {
        cudaError_t r = allow_max_dynamic_smem(kern);
        if (r != cudaSuccess) return r;
        return tc::launch_pdl(kern, dim3(grid), dim3(gram::kThreads), (size_t)(gram::kSmem + 1024), st, (const float2*)psi,
                          (const float2*)lam, a, ws, err);
    };
    // (16-byte copies measured faster than 32-byte loads or 256-byte bulk copies here)
    // 16-byte copies need 16-byte aligned states (a wrapped buffer may be 8-byte aligned only)
    const bool a16 = (((uintptr_t)psi | (uintptr_t)lam) & 15) == 0;
    cudaError_t e = !a16                ? run(gram::k_gram6<1>)
                    : a.sorted[0] >= 1  ? run(gram::k_gram6<2>)
                    : a.sorted[2] == 2  ? run(gram::k_gram6<3>)   // targets 0, 1, 2 (ascending, distinct)
                                        : run(gram::k_gram6<0>);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_gram_reduce(const double* ws, int n, int nslots, double* Mall, cudaStream_t st) {
    if (nslots <= 0) return cudaSuccess;
    const dim3 grid(gram::kMElems / 32, (unsigned)nslots);
    gram::k_gram_reduce<<<grid, 32 * gram::kRedParts, 0, st>>>(ws, gram_grid(n), gram_workspace_elems(n), Mall);
    return cudaGetLastError();
}

cudaError_t launch_block_grads(const double* Mall, int nslots, const BlockGradGate* gates, const int* gate0,
                               const void* mats, double* sums, cudaStream_t st) {
    if (nslots <= 0) return cudaSuccess;
    const int smem = (2 * 64 * 65 + 64 * 64) * (int)sizeof(float2);
    cudaError_t e = allow_max_dynamic_smem(gram::k_block_grads);
    if (e != cudaSuccess) return e;
    gram::k_block_grads<<<nslots, gram::kGradThreads, smem, st>>>(Mall, gates, gate0, (const float2*)mats, sums);
    return cudaGetLastError();
}

}  // namespace qsgb
