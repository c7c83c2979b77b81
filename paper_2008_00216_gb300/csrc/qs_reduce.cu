// Reductions over the state (norm, Pauli expectations, inner products),
// H|psi> for a Pauli sum, and the adjoint-gradient gate step.
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

// ------------------------------------------------------------------ <psi|P|psi>

struct PauliGroupP {
    uint64_t xmask;
    int f0;        // lowest flipped bit (pairs are visited once)
    int nterms;
    double coeff[32];
    uint64_t zmask[32];
    int ny[32];
    uint64_t units;
};

// For the pair (y, y^F) with bit f0 of y clear and z = conj(psi_y) psi_{y^F},
// the two contributions of a term with sign s(x) = (-1)^popc(x & Z) sum to
// i^ny [s(y^F) z + s(y) conj(z)], whose real part is taken.
template <typename R>
__global__ void __launch_bounds__(256) k_pauli_group(const typename C2<R>::T* __restrict__ psi,
                                                     const __grid_constant__ PauliGroupP p,
                                                     double* __restrict__ partial) {
    using T = typename C2<R>::T;
    __shared__ double sh[32];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    if (p.xmask == 0) {
        for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < p.units; y += stride) {
            const T a = psi[y];
            const double pr = (double)(a.x * a.x + a.y * a.y);
            double w = 0.0;
            for (int t = 0; t < p.nterms; ++t) w += (__popcll(y & p.zmask[t]) & 1) ? -p.coeff[t] : p.coeff[t];
            acc = fma(w, pr, acc);
        }
    } else {
        for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < p.units; u += stride) {
            const uint64_t y = insert_zero(u, p.f0), y2 = y ^ p.xmask;
            const T a = psi[y], b = psi[y2];
            const double zr = (double)(a.x * b.x + a.y * b.y);   // conj(a) b
            const double zi = (double)(a.x * b.y - a.y * b.x);
            for (int t = 0; t < p.nterms; ++t) {
                const double s1 = (__popcll(y & p.zmask[t]) & 1) ? -1.0 : 1.0;
                const double s2 = (__popcll(y2 & p.zmask[t]) & 1) ? -1.0 : 1.0;
                double re;
                switch (p.ny[t] & 3) {
                    case 0: re = (s1 + s2) * zr; break;
                    case 1: re = -(s2 - s1) * zi; break;
                    case 2: re = -(s1 + s2) * zr; break;
                    default: re = (s2 - s1) * zi; break;
                }
                acc = fma(p.coeff[t], re, acc);
            }
        }
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void k_accumulate(const double* __restrict__ partials, int cols, double* __restrict__ result) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) s += partials[c];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) result[0] += s;
}

cudaError_t launch_pauli_group(const void* psi, int n, qs_dtype dt, uint64_t xmask, const qs_pauli_sum::Term* terms,
                               int nterms, double* scratch, double* result, cudaStream_t st) {
    if (nterms < 1 || nterms > 32) return cudaErrorInvalidValue;
    PauliGroupP p{};
    p.xmask = xmask;
    p.f0 = xmask ? __builtin_ctzll(xmask) : -1;
    p.nterms = nterms;
    for (int t = 0; t < nterms; ++t) {
        p.coeff[t] = terms[t].coeff;
        p.zmask[t] = terms[t].zmask;
        p.ny[t] = terms[t].ny;
    }
    p.units = xmask ? (1ull << (n - 1)) : (1ull << n);
    const int nb = reduce_blocks();
    if (dt == QS_C64) k_pauli_group<float><<<nb, 256, 0, st>>>((const float2*)psi, p, scratch);
    else k_pauli_group<double><<<nb, 256, 0, st>>>((const double2*)psi, p, scratch);
    k_accumulate<<<1, 256, 0, st>>>(scratch, nb, result);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ out = H psi

struct HP {
    int ngroups;
    int accumulate;
    uint64_t xmask[48];
    int first[49];        // terms of group g: [first[g], first[g+1])
    double coeff[96];
    uint64_t zmask[96];
    int ny[96];
    uint64_t size;
};

template <typename R>
__global__ void __launch_bounds__(256) k_apply_pauli(const typename C2<R>::T* __restrict__ psi,
                                                     typename C2<R>::T* __restrict__ out,
                                                     const __grid_constant__ HP p) {
    using T = typename C2<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < p.size; y += stride) {
        double accr = 0.0, acci = 0.0;
        if (p.accumulate) {
            const T o = out[y];
            accr = o.x;
            acci = o.y;
        }
        for (int g = 0; g < p.ngroups; ++g) {
            const uint64_t x = y ^ p.xmask[g];
            // w = sum_t c_t i^ny (-1)^popc(x & Z_t)
            double wr = 0.0, wi = 0.0;
            for (int t = p.first[g]; t < p.first[g + 1]; ++t) {
                const double c = (__popcll(x & p.zmask[t]) & 1) ? -p.coeff[t] : p.coeff[t];
                switch (p.ny[t] & 3) {
                    case 0: wr += c; break;
                    case 1: wi += c; break;
                    case 2: wr -= c; break;
                    default: wi -= c; break;
                }
            }
            const T a = psi[x];
            accr += wr * (double)a.x - wi * (double)a.y;
            acci += wr * (double)a.y + wi * (double)a.x;
        }
        T o;
        o.x = (R)accr;
        o.y = (R)acci;
        out[y] = o;
    }
}

cudaError_t launch_apply_pauli_sum(const void* psi, void* out, int n, qs_dtype dt, const qs_pauli_sum& h,
                                   cudaStream_t st) {
    std::map<uint64_t, std::vector<qs_pauli_sum::Term>> groups;
    for (const auto& t : h.terms) groups[t.xmask].push_back(t);
    std::vector<std::pair<uint64_t, std::vector<qs_pauli_sum::Term>>> gl(groups.begin(), groups.end());
    const uint64_t size = 1ull << n;
    int gi = 0;
    bool first_launch = true;
    while (gi < (int)gl.size() || first_launch) {
        HP p{};
        p.size = size;
        p.accumulate = first_launch ? 0 : 1;
        int nt = 0;
        while (gi < (int)gl.size() && p.ngroups < 48 && nt + (int)gl[gi].second.size() <= 96) {
            p.xmask[p.ngroups] = gl[gi].first;
            p.first[p.ngroups] = nt;
            for (const auto& t : gl[gi].second) {
                p.coeff[nt] = t.coeff;
                p.zmask[nt] = t.zmask;
                p.ny[nt] = t.ny;
                ++nt;
            }
            ++p.ngroups;
            ++gi;
        }
        p.first[p.ngroups] = nt;
        if (p.ngroups == 0 && gi < (int)gl.size()) return cudaErrorInvalidValue;  // one group > 96 terms
        const int nb = reduce_blocks() * 2;
        if (dt == QS_C64) k_apply_pauli<float><<<nb, 256, 0, st>>>((const float2*)psi, (float2*)out, p);
        else k_apply_pauli<double><<<nb, 256, 0, st>>>((const double2*)psi, (double2*)out, p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        first_launch = false;
    }
    return cudaSuccess;
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

// ------------------------------------------------------------------ adjoint step

template <typename R, int K>
struct AdjP {
    typename C2<R>::T u[1 << K][1 << K];   // U^dagger
    uint64_t off[1 << K];
    uint64_t psrc[1 << K];                  // (P psi)_r = i^pcode[r] psi[base + psrc[r]]
    int pcode[1 << K];
    int sorted[K];
    int has_param;
    int slot;
    uint64_t units;
};

template <typename R, int K>
__global__ void __launch_bounds__(256) k_adjoint(typename C2<R>::T* __restrict__ psi,
                                                 typename C2<R>::T* __restrict__ lam,
                                                 const __grid_constant__ AdjP<R, K> p,
                                                 double* __restrict__ partials) {
    using T = typename C2<R>::T;
    constexpr int D = 1 << K;
    __shared__ double sh[32];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double zr = 0.0, zi = 0.0;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < p.units; u += stride) {
        uint64_t base = u;
#pragma unroll
        for (int i = 0; i < K; ++i) base = insert_zero(base, p.sorted[i]);
        T a[D], l[D];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            a[r] = psi[base + p.off[r]];
            l[r] = lam[base + p.off[r]];
        }
        if (p.has_param) {
            // <lambda| P |psi> over this set
#pragma unroll
            for (int r = 0; r < D; ++r) {
                const T pp = rot_i(psi[base + p.psrc[r]], p.pcode[r]);
                zr += (double)(l[r].x * pp.x + l[r].y * pp.y);
                zi += (double)(l[r].x * pp.y - l[r].y * pp.x);
            }
        }
#pragma unroll
        for (int r = 0; r < D; ++r) {
            T o1, o2;
            o1.x = o1.y = o2.x = o2.y = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                cmac(o1, p.u[r][c], a[c]);
                cmac(o2, p.u[r][c], l[c]);
            }
            psi[base + p.off[r]] = o1;
            lam[base + p.off[r]] = o2;
        }
    }
    if (p.has_param) {
        zr = block_sum(zr, sh);
        zi = block_sum(zi, sh);
        if (threadIdx.x == 0) {
            partials[((size_t)p.slot * gridDim.x + blockIdx.x) * 2] = zr;
            partials[((size_t)p.slot * gridDim.x + blockIdx.x) * 2 + 1] = zi;
        }
    }
}

template <typename R, int K>
static cudaError_t adjoint_k(void* psi, void* lam, int n, const int* qubits, const double* udag,
                             const double* pauli, double* partials, int slot, cudaStream_t st) {
    using T = typename C2<R>::T;
    constexpr int D = 1 << K;
    AdjP<R, K> p{};
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            p.u[r][c].x = (R)udag[2 * (r * D + c)];
            p.u[r][c].y = (R)udag[2 * (r * D + c) + 1];
        }
    for (int l = 0; l < D; ++l) {
        uint64_t o = 0;
        for (int i = 0; i < K; ++i)
            if ((l >> (K - 1 - i)) & 1) o |= 1ull << qubits[i];
        p.off[l] = o;
    }
    p.has_param = pauli != nullptr && slot >= 0;
    p.slot = slot;
    if (p.has_param) {
        for (int r = 0; r < D; ++r) {
            int c = 0;
            while (c < D - 1 && pauli[2 * (r * D + c)] == 0.0 && pauli[2 * (r * D + c) + 1] == 0.0) ++c;
            const double re = pauli[2 * (r * D + c)], im = pauli[2 * (r * D + c) + 1];
            p.pcode[r] = re == 1.0 ? 0 : im == 1.0 ? 1 : re == -1.0 ? 2 : 3;
            p.psrc[r] = p.off[c];
        }
    }
    for (int i = 0; i < K; ++i) p.sorted[i] = qubits[i];
    std::sort(p.sorted, p.sorted + K);
    p.units = 1ull << (n - K);
    k_adjoint<R, K><<<reduce_blocks(), 256, 0, st>>>((T*)psi, (T*)lam, p, partials);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_gate(void* psi, void* lam, int n, qs_dtype dt, int k, const int* qubits,
                                const double* udag, const double* pauli, double* partials, int slot,
                                cudaStream_t st) {
#define QS_ADJ_CASE(KK)                                                                           \
    case KK:                                                                                      \
        return dt == QS_C64 ? adjoint_k<float, KK>(psi, lam, n, qubits, udag, pauli, partials, slot, st) \
                            : adjoint_k<double, KK>(psi, lam, n, qubits, udag, pauli, partials, slot, st);
    switch (k) {
        QS_ADJ_CASE(1)
        QS_ADJ_CASE(2)
        QS_ADJ_CASE(3)
        QS_ADJ_CASE(4)
    }
#undef QS_ADJ_CASE
    return cudaErrorInvalidValue;
}

}  // namespace qsgb
