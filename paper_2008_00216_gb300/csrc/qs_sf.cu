// Schroedinger-Feynman amplitudes (the paper's hybrid mode, Sections 1 and
// 6: the qubits split into two halves simulated Schroedinger-style, the gates
// across the cut summed over Feynman paths).
//
// Each gate across the cut, a two-qubit matrix M on (a, b) with a in half A
// and b in half B, is written as M = sum_k X_k (x) Y_k: M realigned as the
// 4 x 4 matrix R[(i_a, j_a), (i_b, j_b)] = M[(i_a i_b), (j_a j_b)] is split
// into rank-one terms by elimination with full pivoting (R = sum_k x_k y_k^T,
// r = rank R <= 4 terms; CZ gives 2, fSim 4).  A path picks one term per
// crossing gate; half A then runs its own gates and the X_k of the path in
// circuit order, half B likewise, and
//   <x|U|0> = sum over paths <x_A|psi_A(path)> <x_B|psi_B(path)>.
// Every path's two half states are computed by the batched hot path (one
// persistent launch per half for all paths), and one kernel sums the
// products over paths in FP64 for the requested indices.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsgb {
namespace {

using cd = std::complex<double>;

// M (4 x 4, Kronecker order (first, second)) = sum_k X_k (x) Y_k, X_k on the
// first qubit, Y_k on the second; returns the number of terms.
int split_two_qubit(const std::vector<double>& m, std::vector<cd>& xs, std::vector<cd>& ys) {
    cd R[4][4];
    double mx = 0;
    for (int i0 = 0; i0 < 2; ++i0)
        for (int i1 = 0; i1 < 2; ++i1)
            for (int j0 = 0; j0 < 2; ++j0)
                for (int j1 = 0; j1 < 2; ++j1) {
                    const int r = i0 * 2 + i1, c = j0 * 2 + j1;
                    const cd v(m[2 * (r * 4 + c)], m[2 * (r * 4 + c) + 1]);
                    R[i0 * 2 + j0][i1 * 2 + j1] = v;
                    mx = std::max(mx, std::abs(v));
                }
    xs.clear();
    ys.clear();
    int terms = 0;
    for (; terms < 4; ++terms) {
        int pr = 0, pc = 0;
        double best = 0;
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c)
                if (std::abs(R[r][c]) > best) {
                    best = std::abs(R[r][c]);
                    pr = r;
                    pc = c;
                }
        if (best <= 1e-14 * mx) break;
        const cd piv = R[pr][pc];
        cd x[4], y[4];
        for (int r = 0; r < 4; ++r) x[r] = R[r][pc];
        for (int c = 0; c < 4; ++c) y[c] = R[pr][c] / piv;
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) R[r][c] -= x[r] * y[c];
        for (int r = 0; r < 4; ++r) xs.push_back(x[r]);   // X_k[i][j] = x[2i + j]
        for (int c = 0; c < 4; ++c) ys.push_back(y[c]);   // Y_k[i][j] = y[2i + j]
    }
    return terms;
}

template <typename T>
__global__ void __launch_bounds__(256) k_sf_combine(const T* __restrict__ sa, const T* __restrict__ sb,
                                                    const uint64_t* __restrict__ offa, const uint64_t* __restrict__ offb,
                                                    uint64_t paths, const uint64_t* __restrict__ idx, uint64_t count,
                                                    uint64_t amask, int n, double* __restrict__ out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = idx[i];
        uint64_t xa = 0, xb = 0;
        int ka = 0, kb = 0;
        for (int q = 0; q < n; ++q) {
            const uint64_t bit = (x >> q) & 1;
            if ((amask >> q) & 1) xa |= bit << ka++;
            else xb |= bit << kb++;
        }
        double re = 0, im = 0;
        for (uint64_t p = 0; p < paths; ++p) {
            const T va = sa[offa[p] + xa], vb = sb[offb[p] + xb];
            re += (double)va.x * (double)vb.x - (double)va.y * (double)vb.y;
            im += (double)va.x * (double)vb.y + (double)va.y * (double)vb.x;
        }
        out[2 * i] = re;
        out[2 * i + 1] = im;
    }
}

struct CircuitSet {  // owns the half circuits of every path
    std::vector<qs_circuit*> c;
    ~CircuitSet() {
        for (qs_circuit* x : c) qs_circuit_destroy(x);
    }
};

}  // namespace
}  // namespace qsgb

using namespace qsgb;

extern "C" qs_status qs_sf_amplitudes(const qs_circuit* c, uint64_t part_a, qs_dtype dt, const uint64_t* indices,
                                      uint64_t count, void* stream, double* out, uint64_t* num_paths) {
    if (!c) return fail(QS_ERR_ARG, "null circuit");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_ERR_ARG, "bad dtype");
    const int n = c->n;
    const uint64_t all = n >= 64 ? ~0ull : (1ull << n) - 1;
    if (part_a & ~all) return fail(QS_ERR_ARG, "part A names qubits outside the circuit");
    const int na = __builtin_popcountll(part_a), nb = n - na;
    if (na < 1 || nb < 1) return fail(QS_ERR_ARG, "both halves need at least one qubit");
    if (na > 30 || nb > 30) return fail(QS_ERR_UNSUPPORTED, "a half of more than 30 qubits");
    if (count && (!indices || !out)) return fail(QS_ERR_ARG, "null indices or output");
    for (uint64_t i = 0; i < count; ++i)
        if (indices[i] > all) return fail(QS_ERR_ARG, "index %llu out of range", (unsigned long long)indices[i]);
    int local[64];  // qubit -> index within its half
    {
        int ka = 0, kb = 0;
        for (int q = 0; q < n; ++q) local[q] = ((part_a >> q) & 1) ? ka++ : kb++;
    }
    // the crossing gates and their splittings
    struct Cross {
        int gate, terms, qa, qb;
        std::vector<cd> xa, yb;   // factors on the A and on the B qubit
    };
    std::vector<Cross> cross;
    uint64_t paths = 1;
    for (int gi = 0; gi < (int)c->gates.size(); ++gi) {
        const GateRec& g = c->gates[gi];
        if (g.k == 0) return fail(QS_ERR_ARG, "circuit holds a fused cluster; pass the gates themselves");
        uint64_t supp = 0;
        for (int i = 0; i < g.k; ++i) supp |= 1ull << g.qubits[i];
        if (!(supp & part_a) || !(supp & ~part_a)) continue;
        if (g.k != 2) return fail(QS_ERR_UNSUPPORTED, "gate %d crosses the cut on %d qubits (two at most)", gi, g.k);
        Cross x;
        x.gate = gi;
        std::vector<cd> f0, f1;   // factors on qubits[0], on qubits[1]
        x.terms = split_two_qubit(g.m, f0, f1);
        const bool first_in_a = (part_a >> g.qubits[0]) & 1;
        x.qa = first_in_a ? g.qubits[0] : g.qubits[1];
        x.qb = first_in_a ? g.qubits[1] : g.qubits[0];
        x.xa = first_in_a ? f0 : f1;
        x.yb = first_in_a ? f1 : f0;
        if (x.terms == 0) x.terms = 1, x.xa.assign(4, cd(0)), x.yb.assign(4, cd(0));   // the zero gate
        paths *= (uint64_t)x.terms;
        if (paths > (1ull << 16)) return fail(QS_ERR_UNSUPPORTED, "more than 65536 paths across the cut");
        cross.push_back(std::move(x));
    }
    if (num_paths) *num_paths = paths;
    if (!count) return QS_OK;
    // every path's two half circuits
    CircuitSet ca, cb;
    std::vector<int> term_of(c->gates.size(), -1);
    std::vector<int> cross_of(c->gates.size(), -1);
    for (size_t i = 0; i < cross.size(); ++i) cross_of[cross[i].gate] = (int)i;
    for (uint64_t p = 0; p < paths; ++p) {
        qs_circuit *a = nullptr, *b = nullptr;
        qs_status st = qs_circuit_create(na, &a);
        if (st != QS_OK) return st;
        ca.c.push_back(a);
        st = qs_circuit_create(nb, &b);
        if (st != QS_OK) return st;
        cb.c.push_back(b);
        uint64_t rest = p;  // mixed-radix digits: the term of each crossing gate
        for (size_t i = 0; i < cross.size(); ++i) {
            term_of[cross[i].gate] = (int)(rest % (uint64_t)cross[i].terms);
            rest /= (uint64_t)cross[i].terms;
        }
        for (int gi = 0; gi < (int)c->gates.size(); ++gi) {
            const GateRec& g = c->gates[gi];
            const int ci = cross_of[gi];
            if (ci < 0) {
                int qs[kMaxK];
                for (int i = 0; i < g.k; ++i) qs[i] = local[g.qubits[i]];
                st = qs_circuit_add(((part_a >> g.qubits[0]) & 1) ? a : b, qs, g.k, g.m.data());
                if (st != QS_OK) return st;
                continue;
            }
            const Cross& x = cross[ci];
            const int t = term_of[gi];
            double ma[8], mb[8];
            for (int e = 0; e < 4; ++e) {
                ma[2 * e] = x.xa[4 * t + e].real();
                ma[2 * e + 1] = x.xa[4 * t + e].imag();
                mb[2 * e] = x.yb[4 * t + e].real();
                mb[2 * e + 1] = x.yb[4 * t + e].imag();
            }
            int qa = local[x.qa], qb = local[x.qb];
            st = qs_circuit_add(a, &qa, 1, ma);
            if (st != QS_OK) return st;
            st = qs_circuit_add(b, &qb, 1, mb);
            if (st != QS_OK) return st;
        }
    }
    // both halves of every path in one batched launch each
    cudaStream_t s = (cudaStream_t)stream;
    qs_options opt;
    qs_options_default(&opt);
    opt.k_max = 3;
    qs_batch *ba = nullptr, *bb = nullptr;
    qs_status st = qs_batch_create(ca.c.data(), (int)paths, dt, &opt, &ba);
    if (st != QS_OK) return st;
    st = qs_batch_create(cb.c.data(), (int)paths, dt, &opt, &bb);
    if (st != QS_OK) {
        qs_batch_destroy(ba);
        return st;
    }
    std::vector<uint64_t> offa(paths + 1), offb(paths + 1);
    qs_batch_layout(ba, offa.data());
    qs_batch_layout(bb, offb.data());
    const size_t esz = dt == QS_C64 ? 8 : 16;
    void *da = nullptr, *db = nullptr, *dofa = nullptr, *dofb = nullptr, *didx = nullptr, *dout = nullptr;
    cudaError_t e = cudaMallocAsync(&da, offa[paths] * esz, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&db, offb[paths] * esz, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&dofa, paths * 8, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&dofb, paths * 8, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&didx, count * 8, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&dout, count * 16, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dofa, offa.data(), paths * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dofb, offb.data(), paths * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(didx, indices, count * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        st = qs_batch_run(ba, da, s);
        if (st == QS_OK) st = qs_batch_run(bb, db, s);
        if (st == QS_OK) {
            const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((count + 255) / 256, (uint64_t)num_sms() * 8));
            if (dt == QS_C64)
                k_sf_combine<float2><<<grid, 256, 0, s>>>((const float2*)da, (const float2*)db, (const uint64_t*)dofa,
                                                          (const uint64_t*)dofb, paths, (const uint64_t*)didx, count,
                                                          part_a, n, (double*)dout);
            else
                k_sf_combine<double2><<<grid, 256, 0, s>>>((const double2*)da, (const double2*)db, (const uint64_t*)dofa,
                                                           (const uint64_t*)dofb, paths, (const uint64_t*)didx, count,
                                                           part_a, n, (double*)dout);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, count * 16, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
    }
    for (void* ptr : {da, db, dofa, dofb, didx, dout})
        if (ptr) cudaFreeAsync(ptr, s);
    if (st == QS_OK) st = qs_batch_sync(ba);   // reports a bounded-wait timeout of either launch
    if (st == QS_OK) st = qs_batch_sync(bb);
    qs_batch_destroy(ba);
    qs_batch_destroy(bb);
    if (e != cudaSuccess) return cuda_fail(e, "Schroedinger-Feynman amplitudes");
    return st;
}
