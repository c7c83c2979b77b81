// Tensor tile pass: up to two dense 6-qubit blocks per HBM round trip on
// the tcgen05 tensor cores (sm_103a), split 3xFP16 arithmetic.
//
// A tile is the 2^12 amplitudes whose indices agree outside 12 tile qubits
// (physical bits s_0 < ... < s_11, with s_0 = 0 and s_1 = 1 so every tile is
// made of 32-byte runs).  Every block of the pass acts on 6 of the tile
// qubits, so the blocks can be applied to the tile one after the other while
// it stays in shared memory -- the paper's cache blocking (Section 5.1:
// several gates per pass over memory), with the gates of Section 3 applied
// as products on the tensor cores.  For block b, the tile is the 64 x 64
// complex matrix X_b whose rows are the 64 sets over the other 6 tile qubits
// M_b and whose columns are the block's local index over its qubits K_b;
// the block replaces it by X_b U_b^T exactly as in the one-block pass
// (state rows in tensor memory as the MMA's A operand, the gate's real
// 128 x 128 form in shared memory as B, 3 products hi*hi + hi*lo + lo*hi of
// FP16 parts with per-set power-of-two scales).  Between blocks the
// epilogue writes the block's outputs back into the tile in shared memory
// and the producers read them in the next block's row/column split: a
// transpose through shared memory, never through HBM.
//
// Shared-memory tile layout: tile-local index t (bit i <-> tile qubit i) is
// stored at float2 slot pos(t), a GF(2)-linear bijection chosen on the host
// per pass: bit 0 of t stays bit 0 of pos (16-byte pairs for the loads), the
// next three bits of pos (the bank group of an 8-byte access) are linear
// combinations of tile bits chosen so that, for every block, the 16 sets a
// warp touches at once (the block's 4 lowest row qubits) fall into 16
// distinct bank groups -- conflict-free for both the producers' reads and
// the epilogue's writes of every block of the pass.
//
// One persistent CTA per SM, warp-specialised (18 warps):
//   warps 0-7   epilogue: TMEM lanes of quadrant e % 4, half e / 4 of the
//               outputs; block b < last: outputs back into the tile; last
//               block: straight to HBM
//   warps 8-15  producers: read the tile in block b's layout, scale/split to
//               FP16, store to tensor memory
//   warp 16     MMA issuer (one thread)
//   warp 17     loader: cp.async of the next tiles into free tile slots
// Work items are (tile, block) pairs, three tiles interleaved: for each
// group of three tiles, block 0 of each, then block 1 of each, so the
// transpose of one tile overlaps the MMAs of the others; four tile slots let
// the loaders fetch the next tile while three are in the block chain.
// Every mbarrier wait is bounded; on timeout the CTA sets the error flag, its roles stop,
// the MMAs drain and tensor memory is freed.
#include <stdint.h>

#include <algorithm>

#include "qs_device.cuh"
#include "qs_internal.h"
#include "qs_tc.cuh"

namespace qsgb {
namespace tc {

constexpr int kTTMaxBlocks = kTTileMaxBlocks;
constexpr int kTTSlots = 4;               // tile slots (32 KB each): tile i in slot i % 4
constexpr int kTTGroup = 3;               // tiles interleaved in the block chain (one slot loads ahead)
constexpr int kTTAmps = 4096;             // amplitudes per tile
constexpr int kTTEpi = 8, kTTProd = 8, kTTLoad = 1;
constexpr int kTTMma = kTTEpi + kTTProd;  // warp 16
constexpr int kTTLoad0 = kTTMma + 1;      // warp 17
constexpr int kTTThreads = 32 * (kTTLoad0 + kTTLoad);
constexpr int kTTTmemCols = 512;
constexpr int kTTAcols = 64;              // one A buffer: FP16 hi (32 columns) | lo (32)
constexpr int kTTD = 256;                 // accumulators at columns 256 and 384

struct TTLayout {
    static constexpr int kGPart = kN * 128;                  // one FP16 gate part: 128 rows x 64 K
    static constexpr int kG = 0;                             // [block][hi, lo]
    static constexpr int kSlot0 = kG + kTTMaxBlocks * 2 * kGPart;
    static constexpr int kSlotBytes = kTTAmps * 8;
    static constexpr int kPosK = kSlot0 + kTTSlots * kSlotBytes;   // u16 [block][64]
    static constexpr int kPosM = kPosK + kTTMaxBlocks * 64 * 2;    // u16 [block][64]
    static constexpr int kPhysK = kPosM + kTTMaxBlocks * 64 * 2;   // u64 [block][64]
    static constexpr int kPhysM = kPhysK + kTTMaxBlocks * 64 * 8;  // u64 [block][64]
    static constexpr int kLoadW = kPhysM + kTTMaxBlocks * 64 * 8;  // u64 phys [64], then u16 pos [64]
    static constexpr int kScale = kLoadW + 64 * 8 + 64 * 2;        // int [4][64] set scale exponents
    static constexpr int kHmax = kScale + 4 * 64 * 4;              // float [2][2][64], then int ok [2][8]
    static constexpr int kBar = kHmax + 2 * 2 * 64 * 4 + 64;
    static constexpr int kTotal = kBar + 256;
};


struct TTArgs {
    TTileDesc d;
    int mbit[kTTMaxBlocks][6];   // block b: tile bit of set-index bit i (the other 6, ascending)
    uint64_t ntiles;             // 2^(n-12)
};

// first amplitude of tile tn: zero bits inserted at the 12 tile qubits
__device__ __forceinline__ uint64_t tile_base(uint64_t tn, const int* s) {
#pragma unroll
    for (int i = 0; i < 12; ++i) tn = insert_zero(tn, s[i]);
    return tn;
}

__global__ void __launch_bounds__(kTTThreads, 1)
    k_ttile(float2* __restrict__ psi, const float2* __restrict__ U, const __grid_constant__ TTArgs a, int* err) {
    using LY = TTLayout;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base by pointer arithmetic on the shared array, so the
    // compiler keeps every access below in the shared window (LDS/STS)
    unsigned char* sm = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = a.d.nb;

    uint64_t* slot_full = reinterpret_cast<uint64_t*>(sm + LY::kBar);  // loaders' copies landed [3]
    uint64_t* slot_empty = slot_full + kTTSlots;                        // producers done with a tile [4]
    uint64_t* epi_done = slot_empty + kTTSlots;                         // block outputs back in the tile [4]
    uint64_t* afull = epi_done + kTTSlots;
    uint64_t* aempty = afull + 2;
    uint64_t* dfull = aempty + 2;
    uint64_t* dempty = dfull + 2;
    uint64_t* sfull = dempty + 2;                                       // set scales written [4]
    uint64_t* drain = sfull + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    unsigned int* gmax = reinterpret_cast<unsigned int*>(tmem_slot + 2);  // [kTTMaxBlocks]
    int* eGs = reinterpret_cast<int*>(gmax + kTTMaxBlocks);                  // [kTTMaxBlocks]
    uint16_t* posK = reinterpret_cast<uint16_t*>(sm + LY::kPosK);
    uint16_t* posM = reinterpret_cast<uint16_t*>(sm + LY::kPosM);
    uint64_t* physK = reinterpret_cast<uint64_t*>(sm + LY::kPhysK);
    uint64_t* physM = reinterpret_cast<uint64_t*>(sm + LY::kPhysM);
    uint64_t* physW = reinterpret_cast<uint64_t*>(sm + LY::kLoadW);
    uint16_t* posW = reinterpret_cast<uint16_t*>(sm + LY::kLoadW + 64 * 8);
    int* escale = reinterpret_cast<int*>(sm + LY::kScale);
    float* hmax = reinterpret_cast<float*>(sm + LY::kHmax);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kTTSlots; ++i) {
            mbar_init(&slot_full[i], 32 * kTTLoad);   // one cp.async arrival per loader thread
            mbar_init(&slot_empty[i], kTTProd);
            mbar_init(&epi_done[i], kTTEpi);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&afull[b], kTTProd);
            mbar_init(&aempty[b], 1);
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], kTTEpi);
        }
        for (int i = 0; i < 4; ++i) mbar_init(&sfull[i], 4);
        mbar_init(drain, 1);
        *abort_flag = 0;
        for (int b = 0; b < kTTMaxBlocks; ++b) gmax[b] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // index tables: slot positions and HBM offsets of every local index and
    // every set of each block, and of the loaders' pair groups
    for (int idx = threadIdx.x; idx < kTTMaxBlocks * 64; idx += blockDim.x) {
        const int b = idx >> 6, x = idx & 63;
        uint32_t pk = 0, pm = 0;
        uint64_t fk = 0, fm = 0;
        if (b < nb) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                if ((x >> i) & 1) {
                    pk ^= a.d.poscol[a.d.kbit[b][i]];
                    fk |= 1ull << a.d.s[a.d.kbit[b][i]];
                    pm ^= a.d.poscol[a.mbit[b][i]];
                    fm |= 1ull << a.d.s[a.mbit[b][i]];
                }
            }
        }
        posK[idx] = (uint16_t)pk;
        posM[idx] = (uint16_t)pm;
        physK[idx] = fk;
        physM[idx] = fm;
    }
    if (threadIdx.x < 64) {  // pair group w: tile bits 6..11 from the bits of w
        uint32_t p = 0;
        uint64_t f = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i)
            if ((threadIdx.x >> i) & 1) {
                p ^= a.d.poscol[6 + i];
                f |= 1ull << a.d.s[6 + i];
            }
        posW[threadIdx.x] = (uint16_t)p;
        physW[threadIdx.x] = f;
    }
    __syncthreads();
    // each gate's largest magnitude sets its power-of-two scale 2^eG[b]
    {
        for (int b = 0; b < nb; ++b) {
            float mx = 0.f;
            for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
                const float2 u = U[b * 4096 + idx];
                mx = fmaxf(mx, fmaxf(fabsf(u.x), fabsf(u.y)));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) atomicMax(&gmax[b], __float_as_uint(mx));   // non-negative floats order as integers
        }
    }
    __syncthreads();
    if (threadIdx.x < kTTMaxBlocks) eGs[threadIdx.x] = fp16_scale_exp(__uint_as_float(gmax[threadIdx.x]));
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTTTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the gates into shared memory: block b, row n = 2r + h = (h ? Im : Re)
    // U_b[r][:] scaled by 2^eG[b], FP16 hi then lo part, K-major, 128-byte swizzle
    for (int idx = threadIdx.x; idx < nb * kN * 64; idx += blockDim.x) {
        const int b = idx / (kN * 64), rem = idx % (kN * 64);
        const int n = rem >> 6, k = rem & 63, r = n >> 1, h = n & 1;
        const float2 u = U[b * 4096 + r * 64 + k];
        const float vs = (h ? u.y : u.x) * exp2i(eGs[b]);
        const uint32_t o = (uint32_t)(LY::kG + b * 2 * LY::kGPart) + swz(n, k >> 3) + 2u * (uint32_t)(k & 7);
        const __half hi = __float2half_rn(vs);
        *reinterpret_cast<__half*>(sm + o) = hi;
        *reinterpret_cast<__half*>(sm + o + LY::kGPart) = __float2half_rn(vs - __half2float(hi));
    }
    fence_async_smem();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;
    float2* const slot0 = reinterpret_cast<float2*>(sm + LY::kSlot0);

    // Work items: groups of three consecutive tiles of this CTA (tile i is
    // blockIdx.x + i * gridDim.x, held in slot i % 4, whose i / 4-th use it
    // is); per group, block 0 of each tile, then block 1 of each.  Every role
    // walks this sequence; v counts the items a role has processed (buffers
    // and phases follow it).  The loaders walk the tiles in order.
    auto group_size = [&](uint64_t g) -> int {
        int cnt = 0;
        while (cnt < kTTGroup && blockIdx.x + (kTTGroup * g + cnt) * gridDim.x < a.ntiles) ++cnt;
        return cnt;
    };

    if (warp >= kTTEpi && warp < kTTMma) {
        // ================= producers: quadrant q, local indices 32kh..32kh+31
        const int pw = warp - kTTEpi, q = warp & 3, kh = pw >> 2;
        const int j = lane & 15, c = lane >> 4, set = 16 * q + j;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        uint32_t epi_par = 0;   // bit sl: parity of the next epi_done phase of slot sl
        uint32_t v = 0;
        bool stop = false;
        for (uint64_t g = 0; !stop; ++g) {
            const int cnt = group_size(g);
            if (!cnt) break;
            for (int b = 0; b < nb && !stop; ++b) {
                for (int w = 0; w < cnt; ++w, ++v) {
                    const uint64_t ti = kTTGroup * g + w;
                    const int sl = (int)(ti % kTTSlots);
                    // the tile's data: loaded (block 0) or the previous block's outputs
                    bool ok = b == 0 ? mbar_wait(&slot_full[sl], (uint32_t)((ti / kTTSlots) & 1), err, abort_flag)
                                     : mbar_wait(&epi_done[sl], (epi_par >> sl) & 1u, err, abort_flag);
                    if (b > 0) epi_par ^= 1u << sl;
                    const float2* slot = slot0 + sl * kTTAmps;
                    // slot position of (set, k) = posM(set) ^ posK(k), posK linear in
                    // the bits of k: one XOR per element from the block's columns
                    uint32_t kc[5];
#pragma unroll
                    for (int i = 0; i < 5; ++i) kc[i] = posK[b * 64 + (1 << i)];
                    uint32_t o[32];  // positions of part c of X_b[set][32kh + kl]
                    o[0] = posM[b * 64 + set] ^ (kh ? (uint32_t)posK[b * 64 + 32] : 0u);
#pragma unroll
                    for (int bit = 0; bit < 5; ++bit)
#pragma unroll
                        for (int i = 0; i < (1 << bit); ++i) o[(1 << bit) + i] = o[i] ^ kc[bit];
                    float x[32];
#pragma unroll
                    for (int kl = 0; kl < 32; ++kl) {
                        const float2 xv = slot[o[kl]];
                        x[kl] = c ? xv.y : xv.x;
                    }
                    const int buf = (int)(v & 1);
                    ok = __all_sync(0xffffffffu, ok) &&
                         __all_sync(0xffffffffu, mbar_wait(&aempty[buf], ((v >> 1) & 1) ^ 1, err, abort_flag));
                    // the set's scale: both parts, both halves of K (the pair of
                    // producer warps of this quadrant agree through shared memory
                    // and a named barrier, and also agree on stopping)
                    float m = 0.f;
#pragma unroll
                    for (int e = 0; e < 32; ++e) m = fmaxf(m, fabsf(x[e]));
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
                    float* hm = hmax + (int)(v & 1) * 128;
                    int* okf = reinterpret_cast<int*>(hmax + 256) + (int)(v & 1) * 8;
                    if (c == 0) hm[kh * 64 + set] = m;
                    if (lane == 0) okf[kh * 4 + q] = ok ? 1 : 0;
                    named_bar_sync(1 + q, 64);
                    m = fmaxf(m, hm[(kh ^ 1) * 64 + set]);
                    if (!(ok && okf[(kh ^ 1) * 4 + q] != 0)) {
                        stop = true;
                        break;
                    }
                    const int e = fp16_scale_exp(m);
                    const float sc = exp2i(e);
                    if (kh == 0) {
                        if (c == 0) escale[(int)(v & 3) * 64 + set] = e;
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sfull[v & 3]);
                    }
                    tc_after();
                    uint32_t hw[16], lw[16];
#pragma unroll
                    for (int e2 = 0; e2 < 16; ++e2) {
                        const float x0 = x[2 * e2] * sc, x1 = x[2 * e2 + 1] * sc;
                        const __half2 hh = __floats2half2_rn(x0, x1);
                        hw[e2] = *reinterpret_cast<const uint32_t*>(&hh);
                        const float2 hf = __half22float2(hh);
                        const __half2 lh = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
                        lw[e2] = *reinterpret_cast<const uint32_t*>(&lh);
                    }
                    const uint32_t acol = lane_base + (uint32_t)(buf * kTTAcols);
                    tmem_st16(acol + (uint32_t)(16 * kh), hw);
                    tmem_st16(acol + (uint32_t)(32 + 16 * kh), lw);
                    tmem_st_wait();
                    tc_before();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(&afull[buf]);
                        if (b == nb - 1) mbar_arrive(&slot_empty[sl]);   // this warp is done with the tile
                    }
                }
            }
        }
    } else if (warp == kTTMma) {
        // ================= MMA issuer
        if (lane == 0) {
            uint32_t v = 0;
            bool issued = false, stop = false;
            for (uint64_t g = 0; !stop; ++g) {
                const int cnt = group_size(g);
                if (!cnt) break;
                for (int b = 0; b < nb && !stop; ++b) {
                    const uint32_t g_base = su32(sm + LY::kG + b * 2 * LY::kGPart);
                    for (int w = 0; w < cnt; ++w, ++v) {
                        const int buf = (int)(v & 1);
                        const uint32_t ph = (v >> 1) & 1;
                        if (!mbar_wait(&afull[buf], ph, err, abort_flag) || !mbar_wait(&dempty[buf], ph ^ 1, err, abort_flag)) {
                            stop = true;
                            break;
                        }
                        tc_after();
                        const uint32_t d = tmem + (uint32_t)(kTTD + buf * kN);
                        // products, small terms first: (A_lo, G_hi), (A_hi, G_lo), (A_hi, G_hi)
#pragma unroll
                        for (int pr = 0; pr < 3; ++pr) {
                            const int asel = pr == 0 ? 1 : 0, gsel = pr == 1 ? 1 : 0;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint32_t a_t = tmem + (uint32_t)(buf * kTTAcols + asel * 32 + 8 * kk);
                                umma_ts<2>(d, a_t, sdesc(g_base + gsel * LY::kGPart + kk * 32), (pr > 0 || kk > 0) ? 1u : 0u);
                            }
                        }
                        umma_commit(&aempty[buf]);
                        umma_commit(&dfull[buf]);
                        issued = true;
                    }
                }
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
    } else if (warp >= kTTLoad0) {
        // ================= loader: 32 threads, 64 pairs (16 bytes) each per tile
        const int tau = threadIdx.x - 32 * kTTLoad0;   // tile bits 1..5 of the pairs it moves
        uint32_t pt = 0;
        uint64_t ft = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i)
            if ((tau >> i) & 1) {
                pt ^= a.d.poscol[1 + i];
                ft |= 1ull << a.d.s[1 + i];
            }
        for (uint64_t ti = 0;; ++ti) {
            const uint64_t tn = blockIdx.x + ti * gridDim.x;
            if (tn >= a.ntiles) break;
            const int sl = (int)(ti % kTTSlots);
            if (!mbar_wait(&slot_empty[sl], (uint32_t)((ti / kTTSlots) & 1) ^ 1u, err, abort_flag)) break;
            const float2* src = psi + tile_base(tn, a.d.s) + ft;
            float2* dst = slot0 + sl * kTTAmps;
#pragma unroll 8
            for (int kw = 0; kw < 64; ++kw) cp_async16(dst + (pt ^ posW[kw]), src + physW[kw]);
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(&slot_full[sl])) : "memory");
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else {
        // ================= epilogue: warp e reads TMEM lanes 32q..32q+31 (q = e % 4),
        // accumulator columns 64hc..64hc+63 (hc = e / 4): outputs 32hc..32hc+31
        const int q = warp & 3, hc = warp >> 2, j = lane & 15, c = lane >> 4, set = 16 * q + j;
        uint32_t v = 0;
        bool stop = false;
        for (uint64_t g = 0; !stop; ++g) {
            const int cnt = group_size(g);
            if (!cnt) break;
            for (int b = 0; b < nb && !stop; ++b) {
                const bool last = b == nb - 1;
                const float ug = exp2i(-eGs[b]);
                for (int w = 0; w < cnt; ++w, ++v) {
                    const int buf = (int)(v & 1);
                    if (!__all_sync(0xffffffffu, mbar_wait(&dfull[buf], (v >> 1) & 1, err, abort_flag)) ||
                        !__all_sync(0xffffffffu, mbar_wait(&sfull[v & 3], (v >> 2) & 1, err, abort_flag))) {
                        stop = true;
                        break;
                    }
                    tc_after();
                    const float us = exp2i(-escale[(int)(v & 3) * 64 + set]);
                    const uint64_t ti = kTTGroup * g + w;
                    const int sl = (int)(ti % kTTSlots);
                    const uint64_t tn = blockIdx.x + ti * gridDim.x;
                    // output r = 16ch + 8c + rr: slot position posM(set) ^ posK(r) and
                    // HBM offset physM(set) + physK(r), both linear in the bits of r
                    float2* const out_hbm = psi + (last ? tile_base(tn, a.d.s) + physM[b * 64 + set] : 0);
                    float2* const out_slot = slot0 + sl * kTTAmps;
                    const uint32_t pbase = posM[b * 64 + set] ^ (c ? (uint32_t)posK[b * 64 + 8] : 0u);
                    const uint64_t fbase = c ? physK[b * 64 + 8] : 0ull;
                    uint32_t pr_[8];
                    uint64_t fr_[8];
                    pr_[0] = 0;
                    fr_[0] = 0;
#pragma unroll
                    for (int bit = 0; bit < 3; ++bit) {
                        const uint32_t pc = posK[b * 64 + (1 << bit)];
                        const uint64_t fc = physK[b * 64 + (1 << bit)];
#pragma unroll
                        for (int i = 0; i < (1 << bit); ++i) {
                            pr_[(1 << bit) + i] = pr_[i] ^ pc;
                            fr_[(1 << bit) + i] = fr_[i] | fc;
                        }
                    }
                    const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kTTD + buf * kN);
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        const int ch = 2 * hc + cc;
                        float d[32];  // d[2rr + h] = D[row][2(16ch + rr) + h]
                        tmem_ld16(taddr + (uint32_t)(32 * ch), d);
                        tmem_ld16(taddr + (uint32_t)(32 * ch + 16), d + 16);
                        tmem_ld_wait();
                        if (cc == 1) {  // this warp is done with the accumulator (free for item v + 2)
                            tc_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&dempty[buf]);
                        }
                        float rcv[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) rcv[e] = __shfl_xor_sync(0xffffffffu, c ? d[e] : d[16 + e], 16);
#pragma unroll
                        for (int rr = 0; rr < 8; ++rr) {
                            float2 y;
                            if (c == 0) {  // own: D[re][.]; partner: D[im][.] of output 16ch + rr
                                y.x = d[2 * rr] - rcv[2 * rr + 1];
                                y.y = rcv[2 * rr] + d[2 * rr + 1];
                            } else {       // own: D[im][.]; partner: D[re][.] of output 16ch + 8 + rr
                                y.x = rcv[2 * rr] - d[16 + 2 * rr + 1];
                                y.y = d[16 + 2 * rr] + rcv[2 * rr + 1];
                            }
                            y.x = (y.x * us) * ug;   // two steps: the product of the scales may leave FP32's range
                            y.y = (y.y * us) * ug;
                            if (last) out_hbm[fbase | physK[b * 64 + 16 * ch] | fr_[rr]] = y;
                            else out_slot[pbase ^ posK[b * 64 + 16 * ch] ^ pr_[rr]] = y;
                        }
                    }
                    if (!last) {  // the block's outputs are in the tile: the next block may read it
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&epi_done[sl]);
                    }
                }
            }
        }
    }

    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTTTmemCols) : "memory");
}

}  // namespace tc
}  // namespace qsgb

namespace qsgb {

bool ttile_supported(int n) { return n >= 12; }

cudaError_t launch_ttile(void* psi, int n, const TTileDesc& d, const void* dmat, int* err, cudaStream_t st) {
    using namespace tc;
    if (!ttile_supported(n) || d.nb < 1 || d.nb > kTTMaxBlocks) return cudaErrorInvalidValue;
    if (d.s[0] != 0 || d.s[1] != 1) return cudaErrorInvalidValue;
    for (int i = 1; i < 12; ++i)
        if (d.s[i] <= d.s[i - 1] || d.s[i] >= n) return cudaErrorInvalidValue;
    // the slot positions must be a bijection of the 12 tile bits with bit 0 fixed
    {
        uint16_t basis[12];
        int rank = 0;
        for (int i = 0; i < 12; ++i) {  // Gaussian elimination over GF(2)
            uint16_t x = d.poscol[i];
            for (int r = 0; r < rank; ++r)
                if ((x ^ basis[r]) < x) x ^= basis[r];
            if (!x || x >= 4096) return cudaErrorInvalidValue;
            basis[rank++] = x;
            std::sort(basis, basis + rank, [](uint16_t p, uint16_t q) { return p > q; });
        }
        if (d.poscol[0] != 1) return cudaErrorInvalidValue;
        for (int i = 1; i < 12; ++i)
            if (d.poscol[i] & 1) return cudaErrorInvalidValue;
    }
    TTArgs a{};
    a.d = d;
    for (int b = 0; b < d.nb; ++b) {
        uint32_t used = 0;
        for (int i = 0; i < 6; ++i) {
            if (d.kbit[b][i] < 0 || d.kbit[b][i] >= 12 || ((used >> d.kbit[b][i]) & 1)) return cudaErrorInvalidValue;
            used |= 1u << d.kbit[b][i];
        }
        int m = 0;
        for (int t = 0; t < 12; ++t)
            if (!((used >> t) & 1)) a.mbit[b][m++] = t;
    }
    a.ntiles = 1ull << (n - 12);
    const int smem = TTLayout::kTotal + 1024;  // slack to align the base to 1024 bytes
    cudaError_t e = allow_max_dynamic_smem(k_ttile);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<uint64_t>(a.ntiles, (uint64_t)num_sms());
    k_ttile<<<grid, kTTThreads, smem, st>>>((float2*)psi, (const float2*)dmat, a, err);
    return cudaGetLastError();
}

}  // namespace qsgb
