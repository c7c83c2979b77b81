// One pass for a cluster of diagonal gates of any width.
//
// Section 4.2 clusters gates of a kind; diagonal gates (T, CZ, ...) commute,
// so a whole cluster is one phase per amplitude, applied in one memory pass
// (Section 4.3: a CZ layer as a parity of bitmask matches, a T layer as a
// popcount mod 8).  Here the phase is a product of tables: one per chunk of
// index bits (the FP64 product of the cluster's gates that lie in that
// chunk) and one per gate spanning two chunks.  General phases: complex
// tables over 8-bit chunks.  When every entry is an eighth root of unity
// exp(i pi m / 4) (T, S, Z, CZ, ...): byte tables of the integers m over
// 10-bit chunks; the kernel adds them mod 8 and multiplies by
// exp(i pi m / 4) as a rotation by i^(m/2) plus, for odd m,
// (re - im, re + im) / sqrt(2): no general complex multiply, which keeps
// complex128 off the slow FP64 pipe.
#include <stdint.h>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsgb {

namespace {

struct WideArgs {
    int n;
    int nchunks;
    int nlow, nhigh;                  // cross gates with a qubit below 10 / all at or above 10
    int nmixed;                       // exponent tables: cross gates with exactly one qubit below 10
    uint32_t tab_elems;
    DiagCross low[kWideDiagCross], high[kWideDiagCross], mixed[kWideDiagCross];
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

// Exponent tables, 10-bit chunks (one byte per entry in shared memory).  A
// warp walks blocks of 1024 amplitudes (lane = index bits 0-4, step = bits
// 5-9, block = bits >= 10).  Per block: the tables of chunks 1.. and the
// gates on qubits >= 10 give a constant; a gate with exactly one qubit a
// below 10 gives a constant plus d * x_a, and the d's are added bit-sliced
// into three 10-bit masks (coefficient bits 1, 2, 4).  Per amplitude:
// T_0[x & 1023] + popc(x & C0) + 2 popc(x & C1) + 4 popc(x & C2) (+ gates
// with two or more qubits below 10 that span chunks, evaluated directly).
template <typename R>
__global__ void __launch_bounds__(256) k_diag_wide_root8(typename C2<R>::T* __restrict__ psi,
                                                         const typename C2<R>::T* __restrict__ tables,
                                                         const __grid_constant__ WideArgs a) {
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint8_t* tab = smem_raw;
    for (uint32_t i = threadIdx.x; i < a.tab_elems; i += blockDim.x) tab[i] = (uint8_t)((int)tables[i].x & 7);
    __syncthreads();
    using P = Phase<T, true>;
    auto cross_exp = [&](const DiagCross& cg, uint64_t x) {
        uint32_t li = 0;
        for (int i = 0; i < cg.k; ++i) li = (li << 1) | (uint32_t)((x >> cg.q[i]) & 1);
        return (int)tab[cg.tab + li];
    };
    const int lane = threadIdx.x & 31;
    if (a.n >= 10) {
        const uint64_t nblk = 1ull << (a.n - 10);
        const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
        for (uint64_t blk = gw; blk < nblk; blk += nw) {
            const uint64_t x0 = blk << 10;
            int H = 0;
            for (int c = 1; c < a.nchunks; ++c) H += tab[1024 * c + ((x0 >> (10 * c)) & 1023)];
            for (int c = 0; c < a.nhigh; ++c) H += cross_exp(a.high[c], x0);
            uint32_t C0 = 0, C1 = 0, C2 = 0;  // bit-sliced 3-bit coefficients of the low qubits
            for (int c = 0; c < a.nmixed; ++c) {
                const DiagCross& cg = a.mixed[c];
                int lowq = 0;
                for (int i = 0; i < cg.k; ++i)
                    if (cg.q[i] < 10) lowq = cg.q[i];
                const int e0 = cross_exp(cg, x0), e1 = cross_exp(cg, x0 | (1ull << lowq));
                H += e0;
                const int d = (e1 - e0) & 7;
                const uint32_t A = (uint32_t)(d & 1) << lowq, B = (uint32_t)((d >> 1) & 1) << lowq,
                               Cc = (uint32_t)((d >> 2) & 1) << lowq;
                const uint32_t c1 = C0 & A;
                C0 ^= A;
                const uint32_t s1 = C1 ^ B ^ c1, c2 = (C1 & B) | (C1 & c1) | (B & c1);
                C1 = s1;
                C2 ^= Cc ^ c2;
            }
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const uint64_t x = x0 | ((uint64_t)j << 5) | (uint64_t)lane;
                const uint32_t xl = (uint32_t)x & 1023u;
                P ph;
                ph.m = H + tab[xl] + __popc(xl & C0) + 2 * __popc(xl & C1) + 4 * __popc(xl & C2);
                for (int c = 0; c < a.nlow; ++c) ph.m += cross_exp(a.low[c], x);
                psi[x] = ph.apply(psi[x]);
            }
        }
    } else {  // one chunk: bits below 10
        const uint64_t N = 1ull << a.n;
        for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
            P ph;
            ph.m = tab[x & 1023];
            psi[x] = ph.apply(psi[x]);
        }
    }
}

}  // namespace

cudaError_t launch_diag_wide(void* psi, int n, qs_dtype dt, const WideDiag& w, const void* dtables, cudaStream_t st) {
    const int cb = w.root8 ? 10 : 8;
    if (w.chunk_bits != cb || w.nchunks != (n + cb - 1) / cb ||
        w.tab_elems > (w.root8 ? kWideDiagRoot8Elems : kWideDiagTabElems) || w.tab_elems < (1u << cb) * w.nchunks)
        return cudaErrorInvalidValue;
    WideArgs a{};
    a.n = n;
    a.nchunks = w.nchunks;
    a.tab_elems = w.tab_elems;
    for (const DiagCross& c : w.cross) {
        int nlow = 0;
        for (int i = 0; i < c.k; ++i) nlow += c.q[i] < 10;
        DiagCross* list;
        int* cnt;
        if (nlow == 0) {
            list = a.high;
            cnt = &a.nhigh;
        } else if (nlow == 1 && w.root8) {
            list = a.mixed;
            cnt = &a.nmixed;
        } else {
            list = a.low;
            cnt = &a.nlow;
        }
        if (*cnt == kWideDiagCross) return cudaErrorInvalidValue;
        list[(*cnt)++] = c;
    }
    const int threads = 256;
    const uint64_t units = n >= 10 ? (1ull << (n - 10)) * 32 : (1ull << n);  // threads with work
    const int grid = (int)std::min<uint64_t>((units + threads - 1) / threads, (uint64_t)num_sms() * 8);
    if (w.root8) {
        const size_t smem = w.tab_elems;  // bytes
        if (dt == QS_C64) k_diag_wide_root8<float><<<grid, threads, smem, st>>>((float2*)psi, (const float2*)dtables, a);
        else k_diag_wide_root8<double><<<grid, threads, smem, st>>>((double2*)psi, (const double2*)dtables, a);
    } else {
        const size_t smem = (dt == QS_C64 ? 8 : 16) * (size_t)w.tab_elems;
        if (dt == QS_C64) k_diag_wide<float, false><<<grid, threads, smem, st>>>((float2*)psi, (const float2*)dtables, a);
        else k_diag_wide<double, false><<<grid, threads, smem, st>>>((double2*)psi, (const double2*)dtables, a);
    }
    return cudaGetLastError();
}

}  // namespace qsgb
