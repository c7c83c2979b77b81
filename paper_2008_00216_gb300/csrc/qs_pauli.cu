// Pauli sums on the state: out = H psi and <psi|H|psi>, tile by tile.
//
// H = sum_t c_t P_t, P_t |x> = i^ny (-1)^popc(x & z_t) |x ^ f_t> (f: X or Y
// positions, z: Z or Y positions).  Terms are grouped by flip mask f; group
// g adds w_g(x) psi_x to out_y, x = y ^ f_g, w_g(x) = sum c_t i^ny
// (-1)^popc(x & z_t).  A pass gathers tiles of 2^L amplitudes of psi (the
// qubits pos[0..L-1]) into shared memory and applies every group whose flip
// mask lies in the tile, so each pass reads psi once, and the groups of a
// typical Hamiltonian (single-qubit X terms, ZZ couplings) need
// ceil((n - b) / (L - b)) passes instead of one read per group.  The
// diagonal group (f = 0) rides on the first pass: its Z terms inside one
// 8-qubit chunk are summed into per-chunk tables built in shared memory.
// Modes: write out, add into out, or the expectation's per-block partial
// sums of Re(conj(psi_y) (H_pass psi)_y) (compensated two-float sums for
// complex64, FP64 across tiles and blocks).
#include <stdint.h>

#include <algorithm>
#include <map>
#include <vector>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsgb {

namespace {

constexpr int kPTGroups = 64;
constexpr int kPTTerms = 160;
constexpr int kPTChunks = 5;  // n <= 40

struct PauliTileArgs {
    int L, b, mode;            // mode 0: out = ..., 1: out += ..., 2: expectation partials
    int ngroups, dg;           // dg: the diagonal group, or -1
    int nchunks;
    uint64_t ntiles;
    int pos[16];
    uint32_t flip[kPTGroups];  // local flip mask
    uint64_t gflip[kPTGroups]; // global flip mask
    int first[kPTGroups + 1];  // terms of group g
    int loop0[kPTGroups];      // first term summed per element (the diagonal group's tabled terms come first)
    double wc[kPTGroups][2];   // groups whose terms have no Z: the constant weight
    float wcf[kPTGroups][2];   // the same in FP32 (complex64 states)
    uint8_t wconst[kPTGroups];
    uint8_t gread[kPTGroups];  // flip mask wider than a tile: the partner is read from global memory
    double coeff[kPTTerms];
    float coeff_f[kPTTerms];
    uint64_t zmask[kPTTerms];
    uint8_t ny[kPTTerms];
    int8_t chunk[kPTTerms];    // diagonal group: chunk of a term in one chunk (its sum is tabled), else -1
};

template <typename R>
__device__ __forceinline__ void term_weight(R& wr, R& wi, R c, int ny, uint64_t x, uint64_t z) {
    const R v = (__popcll(x & z) & 1) ? -c : c;
    switch (ny & 3) {
        case 0: wr += v; break;
        case 1: wi += v; break;
        case 2: wr -= v; break;
        default: wi -= v; break;
    }
}

// PER = 2^L / 256 tile elements per thread (e = threadIdx.x + 256 k), each
// with its own accumulator; the groups are the outer loop, so a group's
// parameters are read once per tile.  PER = 1 also serves tiles below 256
// elements (threads past the tile idle).
template <typename R, int PER>
__global__ void __launch_bounds__(256) k_pauli_tile(const typename C2<R>::T* __restrict__ psi,
                                                    typename C2<R>::T* __restrict__ out,
                                                    const __grid_constant__ PauliTileArgs a,
                                                    double* __restrict__ partial) {
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sh[32];
    T* tile = reinterpret_cast<T*>(smem_raw);                                       // 2^L
    uint64_t* rowoff = reinterpret_cast<uint64_t*>(tile + (1u << a.L));             // 2^(L-b)
    R* wtab = reinterpret_cast<R*>(rowoff + (1u << (a.L - a.b)));                   // nchunks x 256
    const int L = a.L, b = a.b;
    for (uint32_t h = threadIdx.x; h < (1u << (L - b)); h += blockDim.x) {
        uint64_t o = 0;
        for (int i = b; i < L; ++i)
            if ((h >> (i - b)) & 1) o |= 1ull << a.pos[i];
        rowoff[h] = o;
    }
    if (a.dg >= 0) {  // per-chunk sums of the diagonal group's one-chunk terms
        for (int i = threadIdx.x; i < a.nchunks * 256; i += blockDim.x) {
            const int c = i >> 8;
            const uint64_t x = (uint64_t)(i & 255) << (8 * c);
            R w = 0;
            for (int t = a.first[a.dg]; t < a.first[a.dg + 1]; ++t)
                if (a.chunk[t] == c) {
                    const R ct = sizeof(R) == 4 ? (R)a.coeff_f[t] : (R)a.coeff[t];
                    w += (__popcll(x & a.zmask[t]) & 1) ? -ct : ct;
                }
            wtab[i] = w;
        }
    }
    __syncthreads();
    const uint32_t mask = (1u << b) - 1u, ne = 1u << L;
    F2Acc e2;
    double e1 = 0.0;
    for (uint64_t tidx = blockIdx.x; tidx < a.ntiles; tidx += gridDim.x) {
        uint64_t base = tidx;
        for (int i = 0; i < L; ++i) base = insert_zero(base, a.pos[i]);
        tile_gather(tile, psi, base, rowoff, b, L);
        __syncthreads();
        auto elem = [&](int k) { return threadIdx.x + 256u * (uint32_t)k; };
        auto gidx = [&](uint32_t e) { return base + rowoff[e >> b] + (e & mask); };
        auto live = [&](int k) { return PER > 1 || elem(k) < ne; };  // a tile below 256 elements
        auto coef = [&](int t) { return sizeof(R) == 4 ? (R)a.coeff_f[t] : (R)a.coeff[t]; };
        T acc[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            acc[k].x = acc[k].y = 0;
            if (a.mode == 1 && live(k)) acc[k] = out[gidx(elem(k))];
        }
        for (int g = 0; g < a.ngroups; ++g) {
            const uint32_t fl = a.flip[g];
            const uint64_t gf = a.gflip[g];
            if (a.wconst[g] && !a.gread[g]) {  // weight c i^ny: the common case (X, Y strings without Z)
                const R wr = sizeof(R) == 4 ? (R)a.wcf[g][0] : (R)a.wc[g][0];
                const R wi = sizeof(R) == 4 ? (R)a.wcf[g][1] : (R)a.wc[g][1];
                const uint32_t tf = threadIdx.x ^ (fl & 255u), fh = fl >> 8;
                if (wi == 0) {
                    T w2;
                    w2.x = w2.y = wr;
#pragma unroll
                    for (int k = 0; k < PER; ++k)
                        if (live(k)) acc[k] = cfma(w2, tile[tf + (((uint32_t)k ^ fh) << 8)], acc[k]);
                } else {
#pragma unroll
                    for (int k = 0; k < PER; ++k) {
                        if (!live(k)) continue;
                        const T v = tile[tf + (((uint32_t)k ^ fh) << 8)];
                        acc[k].x += wr * v.x - wi * v.y;
                        acc[k].y += wr * v.y + wi * v.x;
                    }
                }
                continue;
            }
            const int t0 = a.loop0[g], t1 = a.first[g + 1];
            const bool diag = g == a.dg, rd = a.gread[g];
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                if (!live(k)) continue;
                const uint32_t e = elem(k);
                const uint64_t x = gidx(e) ^ gf;
                R wr = 0, wi = 0;
                if (diag)
                    for (int c = 0; c < a.nchunks; ++c) wr += wtab[256 * c + ((x >> (8 * c)) & 255)];
                for (int t = t0; t < t1; ++t) term_weight(wr, wi, coef(t), a.ny[t], x, a.zmask[t]);
                const T v = rd ? psi[x] : tile[e ^ fl];
                acc[k].x += wr * v.x - wi * v.y;
                acc[k].y += wr * v.y + wi * v.x;
            }
        }
        if (a.mode == 2) {
            R es = 0;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                if (!live(k)) continue;
                const T p = tile[elem(k)];
                es += p.x * acc[k].x + p.y * acc[k].y;  // Re(conj(psi_y) (H psi)_y)
            }
            if constexpr (sizeof(R) == 4) e2.add(es);
            else e1 += es;
        } else {
#pragma unroll
            for (int k = 0; k < PER; ++k)
                if (live(k)) out[gidx(elem(k))] = acc[k];
        }
        __syncthreads();  // the tile is overwritten next
    }
    if (a.mode == 2) {
        double v = sizeof(R) == 4 ? e2.value() : e1;
        v = block_sum(v, sh);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

// The passes for h on n qubits: tiles of L qubits that hold the b lowest
// qubits (rows of 2^b contiguous amplitudes) and the flip qubits of as many
// groups as fit.
std::vector<PauliTileArgs> plan_pauli(const qs_pauli_sum& h, int n, qs_dtype dt, int* err) {
    *err = 0;
    std::map<uint64_t, std::vector<qs_pauli_sum::Term>> gm;
    for (const auto& t : h.terms) gm[t.xmask].push_back(t);
    const int L = std::min(n, dt == QS_C64 ? 12 : 11), b = std::min(n, 5);
    const int nchunks = (n + 7) / 8;
    // split groups with more terms than one pass holds
    struct G { uint64_t f; std::vector<qs_pauli_sum::Term> t; };
    std::vector<G> groups;
    for (auto& kv : gm)
        for (size_t at = 0; at < kv.second.size(); at += kPTTerms / 2) {
            G g{kv.first, {}};
            g.t.assign(kv.second.begin() + at, kv.second.begin() + std::min(kv.second.size(), at + kPTTerms / 2));
            groups.push_back(std::move(g));
        }
    std::vector<char> done(groups.size(), 0);
    std::vector<PauliTileArgs> passes;
    size_t left = groups.size();
    do {
        PauliTileArgs a{};
        a.L = L;
        a.b = b;
        a.mode = passes.empty() ? 0 : 1;
        a.dg = -1;
        a.nchunks = nchunks;
        a.ntiles = 1ull << (n - L);
        uint64_t Q = (1ull << b) - 1;
        int nt = 0;
        std::vector<size_t> mine;
        std::vector<char> wide(groups.size(), 0);
        for (size_t g = 0; g < groups.size(); ++g) {
            if (done[g]) continue;
            // a flip mask that fits no tile rides on any pass, its partners read from global memory
            wide[g] = __builtin_popcountll(((1ull << b) - 1) | groups[g].f) > L;
            if ((!wide[g] && __builtin_popcountll(Q | groups[g].f) > L) || a.ngroups == kPTGroups ||
                nt + (int)groups[g].t.size() > kPTTerms)
                continue;
            if (groups[g].f == 0 && a.dg >= 0) continue;  // one diagonal group per pass
            if (!wide[g]) Q |= groups[g].f;
            mine.push_back(g);
            done[g] = 1;
            --left;
            if (groups[g].f == 0) a.dg = a.ngroups;
            a.ngroups++;
            nt += (int)groups[g].t.size();
        }
        if (mine.empty() && left) {  // cannot happen: a pass takes at least one group
            *err = 1;
            return {};
        }
        for (int q = 0; q < n && __builtin_popcountll(Q) < L; ++q) Q |= 1ull << q;
        int local_of[64], np = 0;
        for (int q = 0; q < n; ++q)
            if ((Q >> q) & 1) {
                local_of[q] = np;
                a.pos[np++] = q;
            }
        nt = 0;
        for (int k = 0; k < (int)mine.size(); ++k) {
            const G& g = groups[mine[k]];
            a.gflip[k] = g.f;
            a.gread[k] = wide[mine[k]];
            for (int q = 0; q < n && !a.gread[k]; ++q)
                if ((g.f >> q) & 1) a.flip[k] |= 1u << local_of[q];
            a.first[k] = nt;
            bool noz = true;
            double wr = 0, wi = 0;
            std::vector<qs_pauli_sum::Term> ts = g.t;
            auto one_chunk = [](const qs_pauli_sum::Term& t) {
                return t.zmask && (__builtin_ctzll(t.zmask) >> 3) == ((63 - __builtin_clzll(t.zmask)) >> 3);
            };
            if (g.f == 0) std::stable_partition(ts.begin(), ts.end(), one_chunk);
            a.loop0[k] = nt;
            for (const auto& t : ts) {
                a.coeff[nt] = t.coeff;
                a.coeff_f[nt] = (float)t.coeff;
                a.zmask[nt] = t.zmask;
                a.ny[nt] = (uint8_t)(t.ny & 3);
                a.chunk[nt] = -1;
                if (g.f == 0 && one_chunk(t)) {
                    a.chunk[nt] = (int8_t)(__builtin_ctzll(t.zmask) >> 3);
                    a.loop0[k] = nt + 1;  // tabled: not summed per element
                }
                noz = noz && t.zmask == 0;
                const double v = t.coeff;
                switch (t.ny & 3) {
                    case 0: wr += v; break;
                    case 1: wi += v; break;
                    case 2: wr -= v; break;
                    default: wi -= v; break;
                }
                ++nt;
            }
            a.wconst[k] = noz ? 1 : 0;
            a.wc[k][0] = wr;
            a.wc[k][1] = wi;
            a.wcf[k][0] = (float)wr;
            a.wcf[k][1] = (float)wi;
        }
        a.first[mine.size()] = nt;
        passes.push_back(a);
    } while (left);
    return passes;
}

template <typename R>
size_t pauli_smem(const PauliTileArgs& a) {
    return sizeof(typename C2<R>::T) * ((size_t)1 << a.L) + 8 * ((size_t)1 << (a.L - a.b)) +
           sizeof(R) * 256 * (size_t)a.nchunks;
}

template <typename R>
cudaError_t launch_pass(const void* psi, void* out, const PauliTileArgs& a, double* partial, int grid,
                        cudaStream_t st) {
    using T = typename C2<R>::T;
    const size_t smem = pauli_smem<R>(a);
    switch (a.L) {
        case 12:  // complex64 only (complex128 tiles hold 2^11 amplitudes)
            if constexpr (sizeof(R) == 4) k_pauli_tile<R, 16><<<grid, 256, smem, st>>>((const T*)psi, (T*)out, a, partial);
            else return cudaErrorInvalidValue;
            break;
        case 11: k_pauli_tile<R, 8><<<grid, 256, smem, st>>>((const T*)psi, (T*)out, a, partial); break;
        case 10: k_pauli_tile<R, 4><<<grid, 256, smem, st>>>((const T*)psi, (T*)out, a, partial); break;
        case 9: k_pauli_tile<R, 2><<<grid, 256, smem, st>>>((const T*)psi, (T*)out, a, partial); break;
        default: k_pauli_tile<R, 1><<<grid, 256, smem, st>>>((const T*)psi, (T*)out, a, partial); break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply_pauli_sum(const void* psi, void* out, int n, qs_dtype dt, const qs_pauli_sum& h,
                                   cudaStream_t st) {
    if (n > 8 * kPTChunks) return cudaErrorInvalidValue;
    int err = 0;
    std::vector<PauliTileArgs> passes = plan_pauli(h, n, dt, &err);
    if (err) return cudaErrorInvalidValue;
    for (const PauliTileArgs& a : passes) {
        const int grid = (int)std::min<uint64_t>(a.ntiles, (uint64_t)reduce_blocks());
        cudaError_t e = dt == QS_C64 ? launch_pass<float>(psi, out, a, nullptr, grid, st)
                                     : launch_pass<double>(psi, out, a, nullptr, grid, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_expectation(const void* psi, int n, qs_dtype dt, const qs_pauli_sum& h, double* scratch,
                               double* result, cudaStream_t st) {
    if (n > 8 * kPTChunks) return cudaErrorInvalidValue;
    int err = 0;
    std::vector<PauliTileArgs> passes = plan_pauli(h, n, dt, &err);
    if (err) return cudaErrorInvalidValue;
    const int nb = reduce_blocks();
    for (size_t i = 0; i < passes.size(); ++i) {
        PauliTileArgs& a = passes[i];
        a.mode = 2;
        // every block writes its partial (blocks without tiles write 0)
        cudaError_t e = dt == QS_C64 ? launch_pass<float>(psi, nullptr, a, scratch, nb, st)
                                     : launch_pass<double>(psi, nullptr, a, scratch, nb, st);
        if (e != cudaSuccess) return e;
        e = launch_accumulate(scratch, nb, result, i == 0, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qsgb
