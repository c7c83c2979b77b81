// One pass for a cluster of diagonal gates of any width.
//
// Section 4.2 clusters gates of a kind; diagonal gates (T, CZ, ...) commute,
// so a whole cluster is one phase per amplitude, applied in one memory pass
// (Section 4.3: a CZ layer as a parity of bitmask matches, a T layer as a
// popcount mod 8).  Here the phase is a product of tables: one per 8-qubit
// chunk of the index (the FP64 product of the cluster's gates that lie in
// that chunk) and one per gate spanning two chunks.  When every entry is an
// eighth root of unity exp(i pi m / 4) the tables hold the integers m, the
// kernel adds them mod 8 and multiplies by exp(i pi m / 4) as a rotation by
// i^(m/2) plus, for odd m, (re - im, re + im) / sqrt(2): no general complex
// multiply, which keeps complex128 off the slow FP64 pipe.
#include <stdint.h>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsgb {

namespace {

struct WideArgs {
    int n;
    int nchunks;
    int nlow, nhigh;                  // cross gates with a qubit below 10 / all at or above 10
    uint32_t tab_elems;
    DiagCross low[kWideDiagCross], high[kWideDiagCross];
};

template <typename T, bool ROOT8>
struct Phase;
template <typename T>
struct Phase<T, false> {  // a complex factor
    T v;
    __device__ __forceinline__ static Phase one() {
        Phase p;
        p.v.x = 1;
        p.v.y = 0;
        return p;
    }
    __device__ __forceinline__ void mul(const T& t) { v = cmul(v, t); }
    __device__ __forceinline__ void mul(const Phase& o) { v = cmul(v, o.v); }
    __device__ __forceinline__ T apply(T a) const { return cmul(v, a); }
};
template <typename T>
struct Phase<T, true> {  // an exponent m of exp(i pi m / 4)
    int m;
    __device__ __forceinline__ static Phase one() {
        Phase p;
        p.m = 0;
        return p;
    }
    __device__ __forceinline__ void mul(const T& t) { m += (int)t.x; }
    __device__ __forceinline__ void mul(const Phase& o) { m += o.m; }
    __device__ __forceinline__ T apply(T a) const {
        const int e = m & 7;
        T r = rot_i(a, e >> 1);
        if (e & 1) {
            using R = decltype(a.x);
            const R s = (R)0.70710678118654752440;
            const R re = (r.x - r.y) * s, im = (r.x + r.y) * s;
            r.x = re;
            r.y = im;
        }
        return r;
    }
};

template <typename T, bool ROOT8>
__device__ __forceinline__ void cross_mul(Phase<T, ROOT8>& ph, const DiagCross* cg, int count, const T* tab, uint64_t x) {
    for (int c = 0; c < count; ++c) {
        uint32_t li = 0;
        for (int i = 0; i < cg[c].k; ++i) li = (li << 1) | (uint32_t)((x >> cg[c].q[i]) & 1);
        ph.mul(tab[cg[c].tab + li]);
    }
}

// For n >= 10 a warp walks blocks of 1024 amplitudes (lane = index bits 0-4,
// step = bits 5-9, block number = bits >= 10; coalesced): the factors of
// chunk tables 2.. and of cross gates on qubits >= 10 are one constant per
// block, so an amplitude needs two table lookups and the low cross gates.
template <typename R, bool ROOT8>
__global__ void __launch_bounds__(256) k_diag_wide(typename C2<R>::T* __restrict__ psi,
                                                   const typename C2<R>::T* __restrict__ tables,
                                                   const __grid_constant__ WideArgs a) {
    using T = typename C2<R>::T;
    using P = Phase<T, ROOT8>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    for (uint32_t i = threadIdx.x; i < a.tab_elems; i += blockDim.x) tab[i] = tables[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (a.n >= 10) {
        const uint64_t nblk = 1ull << (a.n - 10);
        const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
        for (uint64_t blk = gw; blk < nblk; blk += nw) {
            const uint64_t x0 = (blk << 10) | (uint64_t)lane;
            P H = P::one();
            for (int c = 2; c < a.nchunks; ++c) H.mul(tab[256 * c + ((x0 >> (8 * c)) & 255)]);
            cross_mul(H, a.high, a.nhigh, tab, x0);
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const uint64_t x = x0 | ((uint64_t)j << 5);
                const T v = psi[x];
                P ph = H;
                ph.mul(tab[x & 255]);
                ph.mul(tab[256 + ((x >> 8) & 255)]);
                cross_mul(ph, a.low, a.nlow, tab, x);
                psi[x] = ph.apply(v);
            }
        }
    } else {
        const uint64_t N = 1ull << a.n;
        for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
            P ph = P::one();
            for (int c = 0; c < a.nchunks; ++c) ph.mul(tab[256 * c + ((x >> (8 * c)) & 255)]);
            cross_mul(ph, a.low, a.nlow, tab, x);
            cross_mul(ph, a.high, a.nhigh, tab, x);
            psi[x] = ph.apply(psi[x]);
        }
    }
}

}  // namespace

cudaError_t launch_diag_wide(void* psi, int n, qs_dtype dt, const WideDiag& w, const void* dtables, cudaStream_t st) {
    if (w.nchunks != (n + 7) / 8 || w.tab_elems > kWideDiagTabElems || w.tab_elems < 256u * w.nchunks)
        return cudaErrorInvalidValue;
    WideArgs a{};
    a.n = n;
    a.nchunks = w.nchunks;
    a.tab_elems = w.tab_elems;
    for (const DiagCross& c : w.cross) {
        bool low = false;
        for (int i = 0; i < c.k; ++i) low = low || c.q[i] < 10;
        if (low) {
            if (a.nlow == kWideDiagCross) return cudaErrorInvalidValue;
            a.low[a.nlow++] = c;
        } else {
            if (a.nhigh == kWideDiagCross) return cudaErrorInvalidValue;
            a.high[a.nhigh++] = c;
        }
    }
    const int threads = 256;
    const uint64_t units = n >= 10 ? (1ull << (n - 10)) * 32 : (1ull << n);  // threads with work
    const int grid = (int)std::min<uint64_t>((units + threads - 1) / threads, (uint64_t)num_sms() * 8);
    const size_t smem = (dt == QS_C64 ? 8 : 16) * (size_t)w.tab_elems;
    if (dt == QS_C64) {
        if (w.root8) k_diag_wide<float, true><<<grid, threads, smem, st>>>((float2*)psi, (const float2*)dtables, a);
        else k_diag_wide<float, false><<<grid, threads, smem, st>>>((float2*)psi, (const float2*)dtables, a);
    } else {
        if (w.root8) k_diag_wide<double, true><<<grid, threads, smem, st>>>((double2*)psi, (const double2*)dtables, a);
        else k_diag_wide<double, false><<<grid, threads, smem, st>>>((double2*)psi, (const double2*)dtables, a);
    }
    return cudaGetLastError();
}

}  // namespace qsgb
