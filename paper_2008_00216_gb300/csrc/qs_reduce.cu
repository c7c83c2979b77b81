// Reductions over the state (norm, Pauli expectations, inner products),
// H|psi> for a Pauli sum, and the adjoint-gradient tile pass.
//
// Every reduction runs on a fixed grid of reduce_blocks() CTAs; each CTA
// writes one FP64 partial and a single CTA adds the partials in a fixed
// order, so results are deterministic run to run.  Complex64 amplitudes are
// accumulated per thread with a two-float compensated sum (Section 4.1's
// "sum-of-two-values"); complex128 ones in FP64.
#include <algorithm>
#include <map>
#include <vector>

#include "qs_device.cuh"
#include "qs_internal.h"
#include "qs_tile.cuh"

namespace qsgb {

int reduce_blocks() { return num_sms() * 4; }

// ------------------------------------------------------------------ finalize

// out[row] = sum over cols of partials[row*cols + c] (complex when `cplx`)
__global__ void k_sum_rows(const double* __restrict__ partials, int cols, int cplx, double* __restrict__ out) {
    __shared__ double sh[32];
    const int row = blockIdx.x;
    for (int part = 0; part < (cplx ? 2 : 1); ++part) {
        double s = 0.0;
        for (int c = threadIdx.x; c < cols; c += blockDim.x)
            s += partials[((size_t)row * cols + c) * (cplx ? 2 : 1) + part];
        s = block_sum(s, sh);
        if (threadIdx.x == 0) out[row * (cplx ? 2 : 1) + part] = s;
    }
}

cudaError_t launch_sum_partials(const double* partials, int rows, int cols, double* out, cudaStream_t st) {
    k_sum_rows<<<rows, 256, 0, st>>>(partials, cols, 1, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ norm

template <typename R>
__global__ void __launch_bounds__(256) k_norm(const typename C2<R>::T* __restrict__ psi, uint64_t size,
                                              double* __restrict__ partial) {
    __shared__ double sh[32];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double v;
    if constexpr (sizeof(R) == 4) {
        F2Acc acc;
        const float4* p4 = reinterpret_cast<const float4*>(psi);
        for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < size / 2; u += stride) {
            const float4 x = p4[u];
            acc.add_sq(x.x);
            acc.add_sq(x.y);
            acc.add_sq(x.z);
            acc.add_sq(x.w);
        }
        if ((size & 1) && blockIdx.x == 0 && threadIdx.x == 0) {  // n = 0 only
            acc.add_sq(psi[size - 1].x);
            acc.add_sq(psi[size - 1].y);
        }
        v = acc.value();
    } else {
        double s = 0.0;
        for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < size; u += stride) {
            const double2 x = psi[u];
            s = fma(x.x, x.x, s);
            s = fma(x.y, x.y, s);
        }
        v = s;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

cudaError_t launch_norm(const void* psi, int n, qs_dtype dt, double* scratch, double* result, cudaStream_t st) {
    const int nb = reduce_blocks();
    const uint64_t size = 1ull << n;
    if (dt == QS_C64) k_norm<float><<<nb, 256, 0, st>>>((const float2*)psi, size, scratch);
    else k_norm<double><<<nb, 256, 0, st>>>((const double2*)psi, size, scratch);
    k_sum_rows<<<1, 256, 0, st>>>(scratch, nb, 0, result);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ partial sums

// result[0] (+)= the sum of cols partials, in a fixed order
__global__ void k_accumulate(const double* __restrict__ partials, int cols, double* __restrict__ result, int set) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) s += partials[c];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) result[0] = set ? s : result[0] + s;
}

cudaError_t launch_accumulate(const double* partials, int cols, double* result, bool set, cudaStream_t st) {
    k_accumulate<<<1, 256, 0, st>>>(partials, cols, result, set ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ <a|b>

template <typename R>
__global__ void __launch_bounds__(256) k_inner(const typename C2<R>::T* __restrict__ a,
                                               const typename C2<R>::T* __restrict__ b, uint64_t size,
                                               double* __restrict__ partial) {
    __shared__ double sh[32];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double vr, vi;
    if constexpr (sizeof(R) == 4) {
        F2Acc ar, ai;
        for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < size; j += stride) {
            const float2 x = a[j], y = b[j];
            ar.add(x.x * y.x);
            ar.add(x.y * y.y);
            ai.add(x.x * y.y);
            ai.add(-x.y * y.x);
        }
        vr = ar.value();
        vi = ai.value();
    } else {
        double sr = 0.0, si = 0.0;
        for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < size; j += stride) {
            const double2 x = a[j], y = b[j];
            sr = fma(x.x, y.x, sr);
            sr = fma(x.y, y.y, sr);
            si = fma(x.x, y.y, si);
            si = fma(-x.y, y.x, si);
        }
        vr = sr;
        vi = si;
    }
    vr = block_sum(vr, sh);
    vi = block_sum(vi, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = vr;
        partial[2 * blockIdx.x + 1] = vi;
    }
}

cudaError_t launch_inner(const void* a, const void* b, int n, qs_dtype dt, double* scratch, double* result,
                         cudaStream_t st) {
    const int nb = reduce_blocks();
    const uint64_t size = 1ull << n;
    if (dt == QS_C64) k_inner<float><<<nb, 256, 0, st>>>((const float2*)a, (const float2*)b, size, scratch);
    else k_inner<double><<<nb, 256, 0, st>>>((const double2*)a, (const double2*)b, size, scratch);
    k_sum_rows<<<1, 256, 0, st>>>(scratch, nb, 1, result);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ adjoint tile pass

// A single-qubit unit (local bit q) with a parameter: accumulate
// <lambda|P|psi> and apply U^dagger to psi and lambda in the same sweep --
// the thread holds both amplitudes of each pair of both states.  P is the
// unit's Pauli letter: flip fx (X, Y), sign fz (Z, Y), ny factors of i.
// Matrix structure of a single-qubit U^dagger, chosen on the host: general
// complex, diagonal (RZ-like: one complex multiply per amplitude) or real
// (RY-like: two real multiplies per output component).
enum { ADJ1_DENSE = 0, ADJ1_DIAG = 1, ADJ1_REAL = 2 };

template <typename T, typename R, int FORM>
__device__ __forceinline__ void adj_1q_grad_apply_f(T* tp, T* tl, int L, int q, const T* m, int fx, int fz, int ny,
                                                    R& zr, R& zi) {
    const T m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
    for (uint32_t s = threadIdx.x; s < (1u << (L - 1)); s += blockDim.x) {
        const uint32_t i0 = insert_zero32(s, q), i1 = i0 | (1u << q);
        const T a0 = tp[i0], a1 = tp[i1], b0 = tl[i0], b1 = tl[i1];
        // (P a)_e = i^ny (-1)^((e ^ fx) & fz) a_(e ^ fx), e = bit q of the index
        const T p0 = rot_i(fx ? a1 : a0, ny + 2 * (fx & fz));
        const T p1 = rot_i(fx ? a0 : a1, ny + 2 * ((1 ^ fx) & fz));
        zr += b0.x * p0.x + b0.y * p0.y + b1.x * p1.x + b1.y * p1.y;
        zi += b0.x * p0.y - b0.y * p0.x + b1.x * p1.y - b1.y * p1.x;
        T o0, o1, c0, c1;
        if constexpr (FORM == ADJ1_DIAG) {
            o0 = cmul(m00, a0);
            o1 = cmul(m11, a1);
            c0 = cmul(m00, b0);
            c1 = cmul(m11, b1);
        } else if constexpr (FORM == ADJ1_REAL) {
            o0.x = m00.x * a0.x + m01.x * a1.x;
            o0.y = m00.x * a0.y + m01.x * a1.y;
            o1.x = m10.x * a0.x + m11.x * a1.x;
            o1.y = m10.x * a0.y + m11.x * a1.y;
            c0.x = m00.x * b0.x + m01.x * b1.x;
            c0.y = m00.x * b0.y + m01.x * b1.y;
            c1.x = m10.x * b0.x + m11.x * b1.x;
            c1.y = m10.x * b0.y + m11.x * b1.y;
        } else {
            o0.x = o0.y = o1.x = o1.y = 0;
            cmac(o0, m00, a0); cmac(o0, m01, a1); cmac(o1, m10, a0); cmac(o1, m11, a1);
            c0.x = c0.y = c1.x = c1.y = 0;
            cmac(c0, m00, b0); cmac(c0, m01, b1); cmac(c1, m10, b0); cmac(c1, m11, b1);
        }
        tp[i0] = o0;
        tp[i1] = o1;
        tl[i0] = c0;
        tl[i1] = c1;
    }
}

// Single-qubit unit with a parameter: accumulate <lambda|P|psi> and apply
// U^dagger to psi and lambda in the same sweep (the thread holds both
// amplitudes of each pair of both states).  P's letter: flip fx (X, Y),
// sign fz (Z, Y), ny factors of i.
template <typename T, typename R>
__device__ __forceinline__ void adj_1q_grad_apply(T* tp, T* tl, int L, int q, const T* m, int form, int fx, int fz,
                                                  int ny, R& zr, R& zi) {
    if (form == ADJ1_DIAG) adj_1q_grad_apply_f<T, R, ADJ1_DIAG>(tp, tl, L, q, m, fx, fz, ny, zr, zi);
    else if (form == ADJ1_REAL) adj_1q_grad_apply_f<T, R, ADJ1_REAL>(tp, tl, L, q, m, fx, fz, ny, zr, zi);
    else adj_1q_grad_apply_f<T, R, ADJ1_DENSE>(tp, tl, L, q, m, fx, fz, ny, zr, zi);
}

// diagonal U^dagger on both tiles in one sweep; phases +-1 / +-i (CZ, S,
// Z, ...) are applied as swaps and negations without multiplications
template <typename T>
__device__ __forceinline__ void adj_diag_both(T* tp, T* tl, int L, const TileGate& g, const T* m, bool mulfree) {
    const int k = g.k, D = 1 << k;
    for (uint32_t e = threadIdx.x; e < (1u << L); e += blockDim.x) {
        int l = 0;
        for (int i = 0; i < k; ++i) l = (l << 1) | ((e >> g.q[i]) & 1);
        const T ph = m[l * D + l];
        if (mulfree) {
            const int code = ph.x == 1 ? 0 : ph.y == 1 ? 1 : ph.x == -1 ? 2 : 3;
            tp[e] = rot_i(tp[e], code);
            tl[e] = rot_i(tl[e], code);
        } else {
            tp[e] = cmul(ph, tp[e]);
            tl[e] = cmul(ph, tl[e]);
        }
    }
}

struct AdjTileArgs {
    int L, b, ngates;
    int pos[16];
    uint32_t mat_elems;
    uint64_t ntiles;
    AdjTileGate g[kMaxTileGates];
};

template <typename R>
__global__ void __launch_bounds__(256) k_adj_tile(typename C2<R>::T* __restrict__ psi, typename C2<R>::T* __restrict__ lam,
                                                  const typename C2<R>::T* __restrict__ mats,
                                                  const __grid_constant__ AdjTileArgs a, double* __restrict__ partials) {
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = a.L, b = a.b;
    T* tp = reinterpret_cast<T*>(smem_raw);        // psi tile
    T* tl = tp + (1u << L);                         // lambda tile
    T* smat = tl + (1u << L);
    uint64_t* rowoff = reinterpret_cast<uint64_t*>(smat + a.mat_elems);
    // the double2 accumulators need 16-byte alignment: round the offset up
    double2* acc = reinterpret_cast<double2*>((reinterpret_cast<uintptr_t>(rowoff + (1u << (L - b))) + 15) &
                                              ~(uintptr_t)15);
    const uint32_t rowlen = 1u << b;
    for (uint32_t i = threadIdx.x; i < a.mat_elems; i += blockDim.x) smat[i] = mats[i];
    for (uint32_t h = threadIdx.x; h < (1u << (L - b)); h += blockDim.x) {
        uint64_t o = 0;
        for (int i = b; i < L; ++i)
            if ((h >> (i - b)) & 1) o |= 1ull << a.pos[i];
        rowoff[h] = o;
    }
    for (int i = threadIdx.x; i < 8 * a.ngates; i += blockDim.x) acc[i] = make_double2(0.0, 0.0);
    __syncthreads();
    for (uint64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        uint64_t base = t;
        for (int i = 0; i < L; ++i) base = insert_zero(base, a.pos[i]);
        tile_gather2(tp, tl, psi, lam, base, rowoff, b, L);
        __syncthreads();
        for (int gi = 0; gi < a.ngates; ++gi) {
            const AdjTileGate& ag = a.g[gi];
            const TileGate& g = ag.g;
            const T* m = smat + g.mat;
            if (ag.slot >= 0 && g.k == 1) {
                // fused: gradient and U^dagger in one sweep, one barrier
                const int q = g.q[0];
                R zr = 0, zi = 0;
                adj_1q_grad_apply<T, R>(tp, tl, L, q, m, ag.form, (ag.px >> q) & 1, (ag.pz >> q) & 1, ag.ny, zr, zi);
                const double sr = warp_sum((double)zr), si = warp_sum((double)zi);
                if ((threadIdx.x & 31) == 0) {
                    double2& w = acc[gi * 8 + (threadIdx.x >> 5)];
                    w.x += sr;
                    w.y += si;
                }
                __syncthreads();
                continue;
            }
            if (ag.slot >= 0) {
                // <lambda| P |psi> on this tile: (P psi)_e = i^ny (-1)^popc((e^px) & pz) psi_{e^px};
                // warp-reduced into this warp's accumulator (no block barrier)
                R zr = 0, zi = 0;
                for (uint32_t e = threadIdx.x; e < (1u << L); e += blockDim.x) {
                    const uint32_t f = e ^ ag.px;
                    const T v = rot_i(tp[f], ag.ny + 2 * (__popc(f & ag.pz) & 1));
                    const T l = tl[e];
                    zr += l.x * v.x + l.y * v.y;
                    zi += l.x * v.y - l.y * v.x;
                }
                const double sr = warp_sum((double)zr), si = warp_sum((double)zi);
                if ((threadIdx.x & 31) == 0) {
                    double2& w = acc[gi * 8 + (threadIdx.x >> 5)];
                    w.x += sr;
                    w.y += si;
                }
                __syncthreads();  // psi/lambda reads above finish before the gate rewrites them
            }
            if (g.kind == QS_GATE_DIAGONAL) {
                adj_diag_both(tp, tl, L, g, m, ag.mulfree != 0);
            } else {
                switch (g.k) {
                    case 1: tile_dense<T, 1>(tp, L, g, m); tile_dense<T, 1>(tl, L, g, m); break;
                    case 2: tile_dense<T, 2>(tp, L, g, m); tile_dense<T, 2>(tl, L, g, m); break;
                    case 3: tile_dense<T, 3>(tp, L, g, m); tile_dense<T, 3>(tl, L, g, m); break;
                    case 4: tile_dense<T, 4>(tp, L, g, m); tile_dense<T, 4>(tl, L, g, m); break;
                    default: break;
                }
            }
            __syncthreads();
        }
        for (uint32_t e = threadIdx.x; e < (1u << L); e += blockDim.x) {
            const uint64_t gi = base + rowoff[e >> b] + (e & (rowlen - 1));
            psi[gi] = tp[e];
            lam[gi] = tl[e];
        }
        __syncthreads();
    }
    __syncthreads();
    for (int gi = threadIdx.x; gi < a.ngates; gi += blockDim.x) {
        const int slot = a.g[gi].slot;
        if (slot < 0) continue;
        double sr = 0.0, si = 0.0;
        for (int w = 0; w < 8; ++w) {  // fixed order: deterministic
            sr += acc[gi * 8 + w].x;
            si += acc[gi * 8 + w].y;
        }
        partials[((size_t)slot * gridDim.x + blockIdx.x) * 2] = sr;
        partials[((size_t)slot * gridDim.x + blockIdx.x) * 2 + 1] = si;
    }
}

cudaError_t launch_adjoint_tile(void* psi, void* lam, int n, qs_dtype dt, int L, const int* pos,
                                const std::vector<AdjTileGate>& gates, const void* dmats, size_t mat_elems,
                                double* partials, int nblocks, cudaStream_t st) {
    if ((int)gates.size() > kMaxTileGates || L < 1 || L > 13) return cudaErrorInvalidValue;
    AdjTileArgs a{};
    a.L = L;
    int b = 0;
    while (b < L && pos[b] == b) ++b;
    a.b = b;
    a.ngates = (int)gates.size();
    for (int i = 0; i < L; ++i) a.pos[i] = pos[i];
    for (int i = 0; i < a.ngates; ++i) a.g[i] = gates[i];
    a.mat_elems = (uint32_t)mat_elems;
    a.ntiles = 1ull << (n - L);
    const size_t esz = dt == QS_C64 ? 8 : 16;
    const size_t smem = esz * (2 * (1u << L) + mat_elems) + sizeof(uint64_t) * (1u << (L - b)) + 16 +
                        sizeof(double2) * 8 * a.ngates;   // one accumulator per warp (8 warps)
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    cudaError_t e;
    if (dt == QS_C64) {
        e = allow_max_dynamic_smem(k_adj_tile<float>);
        if (e != cudaSuccess) return e;
        k_adj_tile<float><<<nblocks, 256, smem, st>>>((float2*)psi, (float2*)lam, (const float2*)dmats, a, partials);
    } else {
        e = allow_max_dynamic_smem(k_adj_tile<double>);
        if (e != cudaSuccess) return e;
        k_adj_tile<double><<<nblocks, 256, smem, st>>>((double2*)psi, (double2*)lam, (const double2*)dmats, a,
                                                        partials);
    }
    return cudaGetLastError();
}

}  // namespace qsgb
