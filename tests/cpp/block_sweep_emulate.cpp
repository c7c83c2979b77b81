// Host-logic check of the complex64 block adjoint sweep, on the CPU.
//
// The library's planner (build_block_sweep: fusion groups, block products,
// the Gram qubits of each block and its gates as recursion records in Gram
// coordinates, with merged diagonal runs) runs as it does before a GPU
// sweep; the device steps are redone here in FP64: per block, last first,
// the Gram matrix M = sum_s psi_s lambda_s^dagger over the block's six
// qubits, the gradient kernel's walk over the block's records (gradient
// Im tr(P M), then M <- U^dagger M U), then B^dagger on both states.
//
// argv: circuit file, psi file, lambda file (complex128, little endian),
// and optionally "known": the planner then takes the groups' block
// products formed beforehand (as the streamed forward hands them over).
// Circuit file: "n" on the first line, then one gate per line:
//   R k q_0 .. q_{k-1} param paulis theta     (exp(-i theta P / 2))
//   F k q_0 .. q_{k-1} m_0 .. m_{2 4^k - 1}    (row-major, interleaved)
// Prints the gradient of each parameter, one per line.
#include <complex>
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>

#include "qs_adjoint_host.cpp"

using Cd = std::complex<double>;
using namespace qsgb;

static void apply_block(std::vector<Cd>& v, int n, const GateRec& g) {
    const int k = g.k, d = 1 << k;
    uint64_t mask = 0;
    for (int t = 0; t < k; ++t) mask |= 1ull << g.qubits[t];
    std::vector<Cd> in(d);
    for (size_t b = 0; b < (1ull << n); ++b) {
        if (b & mask) continue;
        auto at = [&](int l) {
            size_t idx = b;
            for (int t = 0; t < k; ++t)
                if ((l >> (k - 1 - t)) & 1) idx |= 1ull << g.qubits[t];
            return idx;
        };
        for (int l = 0; l < d; ++l) in[l] = v[at(l)];
        for (int r = 0; r < d; ++r) {
            Cd s = 0;
            for (int l = 0; l < d; ++l) s += Cd(g.m[2 * (r * d + l)], g.m[2 * (r * d + l) + 1]) * in[l];
            v[at(r)] = s;
        }
    }
}

static std::vector<Cd> read_state(const char* path, int n) {
    std::vector<Cd> v(1ull << n);
    std::ifstream f(path, std::ios::binary);
    f.read(reinterpret_cast<char*>(v.data()), (std::streamsize)(v.size() * sizeof(Cd)));
    if (!f) throw std::runtime_error("short state file");
    return v;
}

int main(int argc, char** argv) {
    if (argc != 4 && argc != 5) return 2;
    const bool known_blocks = argc == 5 && std::string(argv[4]) == "known";
    std::ifstream cf(argv[1]);
    int n = 0;
    cf >> n;
    qs_circuit* c = nullptr;
    if (qs_circuit_create(n, &c) != QS_OK) return 3;
    std::string kind;
    int nparams = 0;
    while (cf >> kind) {
        int k = 0;
        cf >> k;
        std::vector<int> q(k);
        for (int& x : q) cf >> x;
        if (kind == "R") {
            int param = 0;
            std::string paulis;
            double theta = 0;
            cf >> param >> paulis >> theta;
            if (qs_circuit_add_rotation(c, q.data(), k, paulis.c_str(), param, theta) != QS_OK) return 4;
            nparams = std::max(nparams, param + 1);
        } else {
            std::vector<double> m(2u << (2 * k));
            for (double& x : m) cf >> x;
            if (qs_circuit_add(c, q.data(), k, m.data()) != QS_OK) return 5;
        }
    }
    std::vector<Cd> psi = read_state(argv[2], n), lam = read_state(argv[3], n);
    qs_options fast;
    qs_options_default(&fast);
    fast.k_max = 6;
    fast.precision = QS_PREC_3XTF32;
    fast.fusion_effort = 1;
    BlockSweep bs;
    std::vector<GateRec> known;
    if (known_blocks) {
        std::vector<std::vector<int>> groups;
        if (fuse_each(n, c->gates, 6, fast.fusion_effort, c->fuse_cache.get(),
                      [&](std::vector<int>&& g) { groups.push_back(std::move(g)); }) != QS_OK)
            return 8;
        known.resize(groups.size());
        for (size_t i = 0; i < groups.size(); ++i) block_product(n, c->gates, groups[i], known[i]);
    }
    if (build_block_sweep(*c, n, fast, bs, known_blocks ? &known : nullptr) != QS_OK) return 6;
    if (known_blocks && !known.empty() && !known[0].m.empty()) return 9;  // the planner must have taken them over
    std::vector<double> grad(nparams, 0.0);
    std::vector<int> seen(nparams, 0);
    for (size_t i = 0; i < bs.blocks.size(); ++i) {
        const int sl = bs.slot[i];
        if (sl >= 0) {
            const auto& T = bs.targets[sl];
            uint64_t tm = 0;
            for (int qq : T) tm |= 1ull << qq;
            std::vector<Cd> M(4096, 0.0);
            for (size_t b = 0; b < (1ull << n); ++b) {
                if (b & tm) continue;
                Cd x[64], y[64];
                for (int l = 0; l < 64; ++l) {
                    size_t idx = b;
                    for (int t = 0; t < 6; ++t)
                        if ((l >> (5 - t)) & 1) idx |= 1ull << T[t];
                    x[l] = psi[idx];
                    y[l] = lam[idx];
                }
                for (int l = 0; l < 64; ++l)
                    for (int l2 = 0; l2 < 64; ++l2) M[l * 64 + l2] += x[l] * std::conj(y[l2]);
            }
            for (int gi = bs.gate0[sl]; gi < bs.gate0[sl + 1]; ++gi) {
                const BlockGradGate& G = bs.gates[gi];
                const int d = 1 << G.k;
                auto U = [&](int r, int col) {
                    const float* f = bs.gmats.data();
                    if (G.flags & kGradCompactDiag)
                        return r == col ? Cd(f[2 * (G.moff + r)], f[2 * (G.moff + r) + 1]) : Cd(0.0, 0.0);
                    return Cd(f[2 * (G.moff + r * d + col)], f[2 * (G.moff + r * d + col) + 1]);
                };
                if (G.param >= 0) {
                    Cd v = 0;
                    for (int j = 0; j < 64; ++j)
                        v += ((__builtin_popcount(j & G.zmask) & 1) ? -1.0 : 1.0) * M[j * 64 + (j ^ G.xmask)];
                    for (int r = 0; r < (G.ny & 3); ++r) v *= Cd(0.0, 1.0);
                    grad[G.param] = v.imag();
                    seen[G.param]++;
                }
                if (G.flags & kGradNoUpdate) continue;
                int gm = 0;
                for (int t = 0; t < G.k; ++t) gm |= 1 << G.lb[t];
                std::vector<int> loc(d);
                for (int a = 0; a < d; ++a) {
                    int x = 0;
                    for (int t = 0; t < G.k; ++t)
                        if ((a >> (G.k - 1 - t)) & 1) x |= 1 << G.lb[t];
                    loc[a] = x;
                }
                for (int r0 = 0; r0 < 64; ++r0) {
                    if (r0 & gm) continue;
                    for (int c0 = 0; c0 < 64; ++c0) {
                        if (c0 & gm) continue;
                        std::vector<Cd> x(d * d), t(d * d);
                        for (int a = 0; a < d; ++a)
                            for (int b2 = 0; b2 < d; ++b2) x[a * d + b2] = M[(r0 | loc[a]) * 64 + (c0 | loc[b2])];
                        for (int a = 0; a < d; ++a)
                            for (int b2 = 0; b2 < d; ++b2) {
                                Cd s = 0;
                                for (int e = 0; e < d; ++e) s += std::conj(U(e, a)) * x[e * d + b2];
                                t[a * d + b2] = s;
                            }
                        for (int a = 0; a < d; ++a)
                            for (int b2 = 0; b2 < d; ++b2) {
                                Cd s = 0;
                                for (int e = 0; e < d; ++e) s += t[a * d + e] * U(e, b2);
                                M[(r0 | loc[a]) * 64 + (c0 | loc[b2])] = s;
                            }
                    }
                }
            }
        }
        GateRec inv;
        conj_transpose(bs.blocks[i], inv);
        apply_block(psi, n, inv);
        apply_block(lam, n, inv);
    }
    for (int p = 0; p < nparams; ++p)
        if (seen[p] != 1) {
            std::fprintf(stderr, "parameter %d has %d gradient records\n", p, seen[p]);
            return 7;
        }
    for (double g : grad) std::printf("%.17g\n", g);
    return 0;
}
