// Host side of the adjoint gradient: the reverse sweep's planning (stages of
// commuting gates, fused sweep passes, stage kernels, tile segments) and the
// C ABI entry points qs_adjoint_gradient / qs_adjoint_gradient_batch.  Device
// work goes through the launchers in the .cu files.
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <complex>
#include <string>
#include <thread>
#include <vector>

#include "qs_internal.h"

using namespace qsgb;

// The reverse sweep visits the gates last to first.  A maximal run of
// pairwise-commuting gates (disjoint qubits, or all diagonal with diagonal
// generators) is a stage: every gate of the run can be moved to the run's
// end, so all of its gradients Im <lambda|P|psi> come from the current
// (psi, lambda), after which the run's inverse is applied.
//   stages whose non-diagonal gates act on one qubit (n >= the fused tile):
//                 fused sweep passes (k_sweep_pass), several consecutive
//                 stages per read/write pass over psi and lambda
// Other stages of at least kStageMin gates:
//   all diagonal  one k_diag_stage pass over psi and lambda (gradients, then
//                 the inverse as per-8-qubit phase tables and cross gates)
//   otherwise     read-only k_grad_pairs passes for the gradients, then the
//                 inverse as a fused plan (6-qubit blocks) on each state
// Shorter runs are merged into segments that take the per-gate tile sweep
// (k_adj_tile: each gate's gradient, then its inverse, in shared memory).
namespace {

constexpr int kStageMin = 8;

struct SweepUnit {
    int fwd = 0;               // index of the gate in the circuit
    uint64_t qm = 0;
    bool diag = false;         // diagonal, and its generator (if any) is diagonal
};

struct AdjPass {
    int L = 0;
    int pos[16] = {0};
    std::vector<AdjTileGate> tg;
    std::vector<double> mats;  // U^dagger, interleaved
    size_t mat0 = 0;
};

struct GradLaunch {
    int L = 0;
    int pos[16] = {0};
    std::vector<StageGen> gens;
};

struct DiagLaunch {
    int nchunks = 0;
    std::vector<DiagCross> cross;
    size_t tab0 = 0;           // element offset in the tables buffer
    uint32_t tab_elems = 0;
    std::vector<uint64_t> zm;
    std::vector<int> slots;
    bool apply = false;
};

struct SweepOp {
    int type = 0;              // 0 tile pass, 1 gradient pass, 2 diagonal stage, 3 plan on both states,
                               // 4 fused sweep pass
    int index = 0;
};

// A stage for the fused sweep pass: its non-diagonal one-qubit gates and its
// diagonal gates (circuit indices).
struct FusedStage {
    std::vector<int> one;
    std::vector<int> diag;
};

}  // namespace

struct AdjointSweep {
    std::vector<AdjPass> tile;
    std::vector<GradLaunch> grad;
    std::vector<DiagLaunch> diag;
    std::vector<SweepPassDesc> fused;
    std::vector<qs_plan*> plans;
    std::vector<SweepOp> ops;
    std::vector<double> allm, tables;
    double* partials = nullptr;
    double* sums = nullptr;
    void* dmats = nullptr;
    void* dtables = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<char> hostm, hostt;   // kept until the stream has consumed them
    void release() {
        if (stream) {
            cudaStreamSynchronize(stream);
            if (partials) cudaFreeAsync(partials, stream);
            if (sums) cudaFreeAsync(sums, stream);
            if (dmats) cudaFreeAsync(dmats, stream);
            if (dtables) cudaFreeAsync(dtables, stream);
        }
        partials = sums = nullptr;
        dmats = dtables = nullptr;
        for (qs_plan* p : plans) qs_plan_destroy(p);
        plans.clear();
    }
};

static void conj_transpose(const GateRec& g, GateRec& u) {
    u = g;
    const int d = 1 << g.k;
    for (int r = 0; r < d; ++r)
        for (int col = 0; col < d; ++col) {
            u.m[2 * (r * d + col)] = g.m[2 * (col * d + r)];
            u.m[2 * (r * d + col) + 1] = -g.m[2 * (col * d + r) + 1];
        }
    u.kind = classify_matrix(g.k, u.m.data());
}

// t[j] (j = 0 .. 255, the bits of the 8-qubit chunk c0) times the diagonal
// entry of u that j's bits select; u's qubits all lie in the chunk
static void scale_chunk_table(std::complex<double>* t, const GateRec& u, int c0) {
    const int k = u.k, d = 1 << k;
    double er[1 << kMaxK], ei[1 << kMaxK];
    int sh[kMaxK];
    for (int l = 0; l < d; ++l) {
        er[l] = u.m[2 * (l * d + l)];
        ei[l] = u.m[2 * (l * d + l) + 1];
    }
    for (int i = 0; i < k; ++i) sh[i] = u.qubits[i] - 8 * c0;
    auto scale = [&](auto index) {
        for (int j = 0; j < 256; ++j) {
            const int l = index(j);
            const double ar = t[j].real(), ai = t[j].imag();
            t[j] = std::complex<double>(ar * er[l] - ai * ei[l], ar * ei[l] + ai * er[l]);
        }
    };
    if (k == 1)
        scale([&](int j) { return (j >> sh[0]) & 1; });
    else if (k == 2)
        scale([&](int j) { return (((j >> sh[0]) & 1) << 1) | ((j >> sh[1]) & 1); });
    else
        scale([&](int j) {
            int l = 0;
            for (int i = 0; i < k; ++i) l = (l << 1) | ((j >> sh[i]) & 1);
            return l;
        });
}

static bool generator_diagonal(const GateRec& g) {
    for (int i = 0; g.param >= 0 && i < g.k; ++i)
        if (g.paulis[i] == 'X' || g.paulis[i] == 'Y') return false;
    return true;
}

// Tile-sweep passes for the gates `rev` (circuit indices in sweep order,
// i.e. the reverse of a valid circuit order); runs of fixed gates are fused
// to <= 4 qubits first.  Appended to sw.tile / sw.ops.
static qs_status add_tile_segment(const qs_circuit& c, const std::vector<int>& rev, int n, qs_dtype dt,
                                  AdjointSweep& sw) {
    std::vector<GateRec> fwd;
    const int cnt = (int)rev.size();
    for (int l = cnt - 1; l >= 0;) {
        const GateRec& g0 = c.gates[rev[l]];
        if (g0.param >= 0) {
            fwd.push_back(g0);
            --l;
            continue;
        }
        std::vector<GateRec> run;
        while (l >= 0 && c.gates[rev[l]].param < 0) run.push_back(c.gates[rev[l--]]);
        std::vector<GateRec> blocks;
        qs_status st = fuse_gates(n, run, 4, blocks);
        if (st != QS_OK) return st;
        fwd.insert(fwd.end(), blocks.begin(), blocks.end());
    }
    std::vector<GateRec> units;
    std::vector<int> appl_kind;
    for (int l = (int)fwd.size() - 1; l >= 0; --l) {
        const GateRec& g = fwd[l];
        if (g.k > 4 && g.kind != QS_GATE_DIAGONAL)
            return fail(QS_ERR_UNSUPPORTED, "adjoint tile sweep supports dense gates on up to 4 qubits");
        GateRec u;
        conj_transpose(g, u);
        appl_kind.push_back(u.kind);
        if (!generator_diagonal(g)) u.kind = QS_GATE_DENSE;  // generator mixes amplitudes
        units.push_back(std::move(u));
    }
    const int L = auto_tile_qubits(n, dt);
    const int lowb = std::min(dt == QS_C64 ? 5 : 4, L);
    std::vector<std::vector<int>> groups = group_for_tiles(units, L, lowb, 3072);
    for (const auto& gr : groups) {
        AdjPass ap;
        uint64_t S = (1ull << lowb) - 1;
        for (int u : gr)
            for (int i = 0; i < units[u].k; ++i) S |= 1ull << units[u].qubits[i];
        for (int q = 0; q < n && __builtin_popcountll(S) < L; ++q) S |= 1ull << q;
        int local_of[kMaxQubits];
        for (int q = 0; q < n; ++q)
            if ((S >> q) & 1) {
                local_of[q] = ap.L;
                ap.pos[ap.L++] = q;
            }
        for (int u : gr) {
            const GateRec& g = units[u];
            AdjTileGate a{};
            a.g.k = (uint8_t)g.k;
            a.g.kind = (uint8_t)appl_kind[u];
            for (int i = 0; i < g.k; ++i) a.g.q[i] = (uint8_t)local_of[g.qubits[i]];
            a.g.mat = (uint32_t)(ap.mats.size() / 2);
            ap.mats.insert(ap.mats.end(), g.m.begin(), g.m.end());
            if (appl_kind[u] == QS_GATE_DIAGONAL) {  // all phases +-1 / +-i: no multiplies
                a.mulfree = 1;
                const int d = 1 << g.k;
                for (int r = 0; r < d; ++r) {
                    const double re = g.m[2 * (r * d + r)], im = g.m[2 * (r * d + r) + 1];
                    const bool q = (re == 0.0 && (im == 1.0 || im == -1.0)) || (im == 0.0 && (re == 1.0 || re == -1.0));
                    if (!q) a.mulfree = 0;
                }
            }
            if (g.k == 1) {
                bool real = true;
                for (int i = 0; i < 4; ++i) real = real && g.m[2 * i + 1] == 0.0;
                a.form = appl_kind[u] == QS_GATE_DIAGONAL ? 1 : real ? 2 : 0;
            }
            a.slot = g.param;
            for (int i = 0; g.param >= 0 && i < g.k; ++i) {
                const uint32_t bit = 1u << local_of[g.qubits[i]];
                if (g.paulis[i] == 'X' || g.paulis[i] == 'Y') a.px |= bit;
                if (g.paulis[i] == 'Z' || g.paulis[i] == 'Y') a.pz |= bit;
                if (g.paulis[i] == 'Y') a.ny++;
            }
            ap.tg.push_back(a);
        }
        ap.mat0 = sw.allm.size() / 2;
        sw.allm.insert(sw.allm.end(), ap.mats.begin(), ap.mats.end());
        sw.ops.push_back({0, (int)sw.tile.size()});
        sw.tile.push_back(std::move(ap));
    }
    return QS_OK;
}

// Gradient passes for the parameterised gates among `gates` (generators on
// global qubits): batches of <= kStageGradGens whose qubits fit one tile.
static void add_gradient_passes(const std::vector<const GateRec*>& gates, int n, qs_dtype dt, AdjointSweep& sw) {
    const int L = std::min(n, dt == QS_C64 ? 12 : 11);
    const int lowb = std::min(dt == QS_C64 ? 5 : 4, L);
    const uint64_t low = (1ull << lowb) - 1;
    struct G { uint64_t x, z; int ny, slot; };
    std::vector<G> gens;
    for (const GateRec* g : gates) {
        if (g->param < 0) continue;
        G e{0, 0, 0, g->param};
        for (int i = 0; i < g->k; ++i) {
            const uint64_t bit = 1ull << g->qubits[i];
            if (g->paulis[i] == 'X' || g->paulis[i] == 'Y') e.x |= bit;
            if (g->paulis[i] == 'Z' || g->paulis[i] == 'Y') e.z |= bit;
            if (g->paulis[i] == 'Y') e.ny++;
        }
        gens.push_back(e);
    }
    // group by the highest qubit touched, so neighbours share a tile
    std::stable_sort(gens.begin(), gens.end(), [](const G& a, const G& b) {
        const uint64_t ma = a.x | a.z, mb = b.x | b.z;
        return (ma ? 63 - __builtin_clzll(ma) : -1) > (mb ? 63 - __builtin_clzll(mb) : -1);
    });
    size_t i = 0;
    while (i < gens.size()) {
        uint64_t S = low;
        std::vector<G> batch;
        while (i < gens.size() && (int)batch.size() < kStageGradGens &&
               __builtin_popcountll(S | gens[i].x | gens[i].z) <= L) {
            S |= gens[i].x | gens[i].z;
            batch.push_back(gens[i++]);
        }
        for (int q = 0; q < n && __builtin_popcountll(S) < L; ++q) S |= 1ull << q;
        GradLaunch gl;
        int local_of[kMaxQubits];
        for (int q = 0; q < n; ++q)
            if ((S >> q) & 1) {
                local_of[q] = gl.L;
                gl.pos[gl.L++] = q;
            }
        for (const G& e : batch) {
            StageGen sg{0, 0, e.ny, e.slot};
            for (int q = 0; q < n; ++q) {
                if ((e.x >> q) & 1) sg.px |= 1u << local_of[q];
                if ((e.z >> q) & 1) sg.pz |= 1u << local_of[q];
            }
            gl.gens.push_back(sg);
        }
        sw.ops.push_back({1, (int)sw.grad.size()});
        sw.grad.push_back(std::move(gl));
    }
}

// A run of diagonal gates: its Z-generator gradients and its inverse.
static void add_diag_stage(const std::vector<const GateRec*>& gates, int n, AdjointSweep& sw) {
    const int nchunks = (n + 7) / 8;
    DiagLaunch dl;
    dl.nchunks = nchunks;
    std::vector<std::complex<double>> tab(256 * (size_t)nchunks, 1.0), cross;
    for (const GateRec* g : gates) {
        GateRec u;
        conj_transpose(*g, u);
        const int k = u.k, d = 1 << k;
        const int c0 = u.qubits[0] >> 3;
        bool one_chunk = true;
        for (int i = 1; i < k; ++i) one_chunk = one_chunk && (u.qubits[i] >> 3) == c0;
        if (one_chunk) {
            scale_chunk_table(tab.data() + 256 * c0, u, c0);
        } else {
            DiagCross x{};
            x.k = (uint8_t)k;
            for (int i = 0; i < k; ++i) x.q[i] = (uint8_t)u.qubits[i];
            x.tab = (uint32_t)(256 * nchunks + cross.size());
            for (int l = 0; l < d; ++l) cross.emplace_back(u.m[2 * (l * d + l)], u.m[2 * (l * d + l) + 1]);
            dl.cross.push_back(x);
        }
        if (g->param >= 0) {
            uint64_t zm = 0;
            for (int i = 0; i < g->k; ++i)
                if (g->paulis[i] == 'Z') zm |= 1ull << g->qubits[i];
            dl.zm.push_back(zm);
            dl.slots.push_back(g->param);
        }
    }
    tab.insert(tab.end(), cross.begin(), cross.end());
    dl.tab0 = sw.tables.size() / 2;
    dl.tab_elems = (uint32_t)tab.size();
    for (const auto& z : tab) {
        sw.tables.push_back(z.real());
        sw.tables.push_back(z.imag());
    }
    dl.apply = true;
    sw.ops.push_back({2, (int)sw.diag.size()});
    sw.diag.push_back(std::move(dl));
}

// Cost of a stage's diagonal gates as one DIAG op of a fused pass: table
// entries, gates spanning two 8-qubit chunks, Z generators.
struct DiagCost {
    uint32_t tab = 0;
    int cross = 0, gens = 0;
};
static DiagCost fused_diag_cost(const qs_circuit& c, const std::vector<int>& diag, int n, int RB) {
    DiagCost dc;
    if (diag.empty()) return dc;
    dc.tab = 256u * (uint32_t)((n + 7) / 8) + (256u >> RB);  // chunk 0 padded (see compile_fused_diag)
    for (int gi : diag) {
        const GateRec& g = c.gates[gi];
        bool one_chunk = true;
        for (int i = 1; i < g.k; ++i) one_chunk = one_chunk && (g.qubits[i] >> 3) == (g.qubits[0] >> 3);
        if (!one_chunk) {
            dc.cross++;
            dc.tab += 1u << g.k;
        }
        dc.gens += g.param >= 0;
    }
    return dc;
}

// The DIAG op of `diag` for a pass (tile p.pos) whose registers hold the
// global qubits `rq[0..RB)` (register bit k = rq[k], thread bit b = tile bit
// RB + b): chunk tables and cross gates of the members' inverses appended to
// p.tabs / p.cross, Z generators to p.gens.  Block-summed generators get
// gradient slots numbered in `block_slots` (placed after the staged ones).
static void compile_fused_diag(const qs_circuit& c, const std::vector<int>& diag, int n, const int* rq, int RB,
                               SweepPassDesc& p, std::vector<int>& block_slots) {
    const int nchunks = (n + 7) / 8;
    uint64_t rmask = 0;
    for (int k = 0; k < RB; ++k) rmask |= 1ull << rq[k];
    SweepDiagRec d{};
    d.nchunks = (uint8_t)nchunks;
    d.tab = (uint32_t)(p.tabs.size() / 2);
    std::vector<std::complex<double>> tab(256 * (size_t)nchunks, 1.0);
    struct Cross { DiagCross x; std::vector<std::complex<double>> e; bool touched; };
    std::vector<Cross> cross;
    for (int gi : diag) {
        GateRec u;
        conj_transpose(c.gates[gi], u);
        const int k = u.k, dd = 1 << k, c0 = u.qubits[0] >> 3;
        bool one_chunk = true, touched = false;
        for (int i = 0; i < k; ++i) {
            one_chunk = one_chunk && (u.qubits[i] >> 3) == c0;
            touched = touched || ((rmask >> u.qubits[i]) & 1);
        }
        if (one_chunk) {
            scale_chunk_table(tab.data() + 256 * c0, u, c0);
        } else {
            Cross x{};
            x.x.k = (uint8_t)k;
            for (int i = 0; i < k; ++i) x.x.q[i] = (uint8_t)u.qubits[i];
            for (int l = 0; l < dd; ++l) x.e.emplace_back(u.m[2 * (l * dd + l)], u.m[2 * (l * dd + l) + 1]);
            x.touched = touched;
            cross.push_back(std::move(x));
        }
    }
    // Chunk 0 is read with the register bits (qubits 0 .. RB-1) as its low
    // index bits and thread bits above them: each row of 2^RB entries is
    // padded by one, so the lanes of a warp, which read different rows at
    // the same column, fall in different shared-memory banks.
    {
        const int per = 1 << RB;
        std::vector<std::complex<double>> padded;
        padded.reserve(tab.size() + (256 >> RB));
        for (int r = 0; r < (256 >> RB); ++r) {
            padded.insert(padded.end(), tab.begin() + r * per, tab.begin() + (r + 1) * per);
            padded.push_back(1.0);
        }
        padded.insert(padded.end(), tab.begin() + 256, tab.end());
        tab.swap(padded);
    }
    // the gates that hold a register qubit first: the kernel looks those up per amplitude
    std::stable_partition(cross.begin(), cross.end(), [](const Cross& x) { return x.touched; });
    d.cross0 = (uint16_t)p.cross.size();
    for (const Cross& x : cross) {
        d.nct += x.touched;
        DiagCross dc = x.x;
        dc.tab = (uint32_t)(p.tabs.size() / 2 + tab.size());
        tab.insert(tab.end(), x.e.begin(), x.e.end());
        p.cross.push_back(dc);
        d.ncross++;
    }
    for (const auto& z : tab) {
        p.tabs.push_back(z.real());
        p.tabs.push_back(z.imag());
    }
    // generators with at most one tile bit are summed per block (S - 2X);
    // the others per thread, staged like the one-qubit gradients
    d.gen0 = (uint16_t)p.gens.size();
    uint64_t tmask = 0;
    int tile_bit[kMaxQubits];
    for (int i = 0; i < p.L; ++i) {
        tmask |= 1ull << p.pos[i];
        tile_bit[p.pos[i]] = i;
    }
    std::vector<SweepZGen> staged, block;
    for (int gi : diag) {
        const GateRec& g = c.gates[gi];
        if (g.param < 0) continue;
        uint64_t zm = 0;
        for (int i = 0; i < g.k; ++i)
            if (g.paulis[i] == 'Z') zm |= 1ull << g.qubits[i];
        SweepZGen z{};
        const uint64_t zin = zm & tmask;
        if (__builtin_popcountll(zin) <= 1) {
            z.mthr = zm & ~tmask;
            z.src = 0;
            if (zin) {
                const int bit = tile_bit[__builtin_ctzll(zin)];
                z.src = (uint8_t)(bit < RB ? 1 + bit : RB + 1 + (bit - RB));  // register bit, or thread bit
            }
            z.local = (uint16_t)block_slots.size();
            block_slots.push_back(g.param);
            block.push_back(z);
            continue;
        }
        z.src = kZStaged;
        z.mthr = zm & ~rmask;
        uint32_t zr = 0;  // register bits of the mask
        for (int k = 0; k < RB; ++k)
            if ((zm >> rq[k]) & 1) zr |= 1u << k;
        if (zr == 0) {
            z.kind = 0;
        } else if ((zr & (zr - 1)) == 0) {
            z.kind = (uint8_t)(__builtin_ctz(zr) + 1);
        } else {
            z.kind = (uint8_t)(RB + 1);
            for (int j = 0; j < (1 << RB); ++j)
                if (__builtin_popcount(j & zr) & 1) z.jmask |= (uint16_t)(1u << j);
        }
        staged.push_back(z);
        p.slots.push_back(g.param);
    }
    d.nstaged = (uint8_t)staged.size();
    d.ngen = (uint8_t)(staged.size() + block.size());
    p.gens.insert(p.gens.end(), staged.begin(), staged.end());
    p.gens.insert(p.gens.end(), block.begin(), block.end());
    p.ops.push_back({SWEEP_DIAG, 0, 0, 0, (uint32_t)p.diags.size()});
    p.diags.push_back(d);
}

// Form and coefficients (4 complex) of a one-qubit op of the fused pass for
// U^dagger = `u` and generator `gen` (0 none, 1 X, 2 Y, 3 Z).  A phase
// common to psi and lambda cancels in every Im <lambda|P|psi>, and the states
// are work states, so U^dagger / sqrt(det) = M = [[a, -conj(b)], [b, conj(a)]]
// (sign chosen so that Re a >= 0) can stand for it.  M is then three shears,
// p0 += z p1, p1 += y p0, p0 += x p1 with y = b, x = (a - 1) / b,
// z = (conj(a) - 1) / b, each done in place; real M (rotations, and
// reflections after negating p1) keeps real coefficients.  Shears are used
// when |x|, |z| <= 2 (always for rotations with Re a >= 0, whose |x| =
// tan(angle / 4) <= 1); otherwise the four entries are applied directly.
static int g1_coefficients(const GateRec& u, int gen, double* c8) {
    using C = std::complex<double>;
    const C m00(u.m[0], u.m[1]), m01(u.m[2], u.m[3]), m10(u.m[4], u.m[5]), m11(u.m[6], u.m[7]);
    for (int i = 0; i < 8; ++i) c8[i] = u.m[i];
    bool real = true;
    for (int i = 0; i < 4; ++i) real = real && u.m[2 * i + 1] == 0.0;
    auto put = [&](C z, C y, C x) {
        const C v[4] = {z, y, x, C(0.0)};
        for (int i = 0; i < 4; ++i) {
            c8[2 * i] = v[i].real();
            c8[2 * i + 1] = v[i].imag();
        }
    };
    if (real) {
        const double det = (m00 * m11 - m01 * m10).real();
        const bool refl = det < 0;
        // rotation part: U^dagger = R diag(1, -1) for a reflection
        double a = m00.real(), b = m10.real();
        const double r01 = refl ? -m01.real() : m01.real(), r11 = refl ? -m11.real() : m11.real();
        if (std::abs(std::abs(det) - 1.0) > 1e-12 || std::abs(r01 + b) > 1e-12 || std::abs(r11 - a) > 1e-12)
            return G1_DIRECT;  // not orthogonal (cannot happen for a unitary)
        if (a < 0) {  // -R: the common sign
            a = -a;
            b = -b;
        }
        const double x = b == 0.0 ? 0.0 : (a - 1.0) / b;  // b = 0: R = I
        if (std::abs(x) > 2.0) return G1_DIRECT;
        if (gen != 0 && (refl || gen != 2)) return G1_DIRECT;
        put(C(x), C(b), C(x));
        return refl ? G1_RSHEAR_NEG : gen == 2 ? G1_RSHEAR_Y : G1_RSHEAR;
    }
    if (gen != 0 && gen != 1) return G1_DIRECT;
    C ph = std::sqrt(m00 * m11 - m01 * m10);
    C a = m00 / ph, b = m10 / ph;
    if (a.real() < 0) {
        a = -a;
        b = -b;
    }
    if (std::abs(b) < 1e-9) return G1_DIRECT;
    const C x = (a - 1.0) / b, z = (std::conj(a) - 1.0) / b;
    if (std::abs(x) > 2.0 || std::abs(z) > 2.0) return G1_DIRECT;
    put(z, b, x);
    return gen == 1 ? G1_CSHEAR_X : G1_CSHEAR;
}

// A run of stages whose non-diagonal gates act on one qubit, as fused sweep
// passes.  Each pass's tile holds the lowest qubits (rows of 128 contiguous
// bytes) and up to L - 4 (complex64) or L - 3 (complex128) others, taken as
// the pending stage's one-qubit gates need them.  A pass finishes the current stage's one-qubit gates
// whose qubits fit, and while a stage completes it carries on into the next
// one (its diagonal op, then its one-qubit gates), so a layered circuit
// needs about (qubits - 4) / 8 passes per layer.
static qs_status add_fused_run(const qs_circuit& c, const std::vector<FusedStage>& run, int n, qs_dtype dt,
                               AdjointSweep& sw) {
    // low rows of 128 bytes (16 complex64 / 8 complex128 amplitudes): full
    // sectors, and the diagonal ops' register qubits 0 .. RB-1 among them
    const int L = dt == QS_C64 ? kSweepTileC64 : kSweepTileC128, RB = L - 8, lowb = dt == QS_C64 ? 4 : 3;
    int lay_a[kSweepMaxLayouts];
    const int nlay = sweep_layouts(dt, lay_a);
    const uint32_t budget = sweep_tab_budget(dt);
    struct Step {
        int stage;
        bool diag;
        std::vector<int> gates;
    };
    struct PassPlan {
        uint64_t Q;
        std::vector<Step> steps;
    };
    std::vector<PassPlan> plans;
    size_t si = 0;
    std::vector<int> rem = run.empty() ? std::vector<int>() : run[0].one;
    bool diag_done = run.empty() || run[0].diag.empty();
    while (si < run.size()) {
        PassPlan pp{(1ull << lowb) - 1, {}};
        int highs = L - lowb, nops = 0, ngrad = 0, ndiag = 0, ncross = 0, ngens = 0;
        uint32_t tabs = 0;
        for (;;) {
            Step st{(int)si, false, {}};
            if (!diag_done) {
                const DiagCost dc = fused_diag_cost(c, run[si].diag, n, RB);
                if (ndiag + 1 > kSweepMaxDiags || tabs + dc.tab > budget || ncross + dc.cross > kSweepMaxCross ||
                    ngens + dc.gens > kSweepMaxGens || ngrad + dc.gens > kSweepMaxGrads ||
                    nops + 1 + nlay > kSweepMaxOps)
                    break;
                ndiag++;
                tabs += dc.tab;
                ncross += dc.cross;
                ngens += dc.gens;
                ngrad += dc.gens;
                nops += 1;
                st.diag = true;
                diag_done = true;
            }
            std::vector<int> keep;
            for (int gi : rem) {
                const int q = c.gates[gi].qubits[0];
                const bool in = (pp.Q >> q) & 1;
                const int gr = c.gates[gi].param >= 0;
                if ((in || highs > 0) && nops + 1 + nlay <= kSweepMaxOps && ngrad + gr <= kSweepMaxGrads) {
                    if (!in) {
                        pp.Q |= 1ull << q;
                        --highs;
                    }
                    st.gates.push_back(gi);
                    nops++;
                    ngrad += gr;
                } else {
                    keep.push_back(gi);
                }
            }
            rem.swap(keep);
            nops += nlay;  // layout changes of this step
            if (st.diag || !st.gates.empty()) pp.steps.push_back(std::move(st));
            if (!rem.empty()) break;
            if (++si == run.size()) break;
            rem = run[si].one;
            diag_done = run[si].diag.empty();
        }
        if (pp.steps.empty()) return fail(QS_ERR_UNSUPPORTED, "fused sweep pass: a stage does not fit one pass");
        plans.push_back(std::move(pp));
    }
    for (PassPlan& pp : plans) {
        SweepPassDesc p;
        p.L = L;
        p.nlay = nlay;
        for (int l = 0; l < nlay; ++l) p.lay_a[l] = lay_a[l];
        for (int q = 0; q < n && __builtin_popcountll(pp.Q) < L; ++q) pp.Q |= 1ull << q;
        int local_of[kMaxQubits];
        int npos = 0;
        for (int q = 0; q < n; ++q)
            if ((pp.Q >> q) & 1) {
                local_of[q] = npos;
                p.pos[npos++] = q;
            }
        auto layout_of = [&](int bit) {
            for (int l = 0; l < nlay; ++l)
                if (bit >= lay_a[l] && bit < lay_a[l] + RB) return l;
            return 0;
        };
        // diagonal ops run in the last ("low") layout, whose registers hold
        // qubits 0 .. RB-1; each step's gates are grouped by layout, the
        // current one first and the one the next step starts in last
        const int low = nlay - 1;
        // the tile is loaded and stored in layout 0 or 1 (both coalesced): start
        // in 1 when the first step's gates all sit there, store in the layout
        // the pass ends in when that is 0 or 1
        int cur = 0;
        if (!pp.steps.empty() && !pp.steps[0].diag) {
            bool has0 = false, has1 = false;
            for (int gi : pp.steps[0].gates) {
                const int l = layout_of(local_of[c.gates[gi].qubits[0]]);
                has0 = has0 || l == 0;
                has1 = has1 || l == 1;
            }
            if (has1 && !has0) cur = 1;
        }
        p.load_lay = cur;
        std::vector<int> block_slots;
        for (size_t k = 0; k < pp.steps.size(); ++k) {
            const Step& st = pp.steps[k];
            if (st.diag) {
                if (cur != low) {
                    p.ops.push_back({SWEEP_LAYOUT, (uint8_t)low, 0, 0, 0});
                    cur = low;
                }
                int rq[8];
                for (int b = 0; b < RB; ++b) rq[b] = p.pos[lay_a[low] + b];
                compile_fused_diag(c, run[st.stage].diag, n, rq, RB, p, block_slots);
            }
            std::vector<int> order{cur};
            if (k + 1 < pp.steps.size()) {
                const int last = pp.steps[k + 1].diag ? low : 0;
                for (int l = 0; l < nlay; ++l)
                    if (l != cur && l != last) order.push_back(l);
                if (last != cur) order.push_back(last);
            } else {  // the final step: end in a layout the tile can be stored from
                for (int l = nlay - 1; l >= 2; --l)
                    if (l != cur) order.push_back(l);
                for (int l = 0; l < 2; ++l)
                    if (l != cur) order.push_back(l);
            }
            struct G1Op {
                SweepOpRec op;
                double c8[8];
                int param;
            };
            for (int l : order) {
                std::vector<G1Op> gl;  // this step's gates on the layout's register bits
                for (int gi : st.gates) {
                    const GateRec& g = c.gates[gi];
                    const int bit = local_of[g.qubits[0]];
                    if (layout_of(bit) != l) continue;
                    GateRec u;
                    conj_transpose(g, u);
                    G1Op e{};
                    e.op = SweepOpRec{SWEEP_G1, (uint8_t)(bit - lay_a[l]), 0, 0, 0};
                    e.param = -1;
                    if (g.param >= 0) {
                        const char P = g.paulis[0];
                        e.op.gen = P == 'X' ? 1 : P == 'Y' ? 2 : P == 'Z' ? 3 : 0;
                        if (e.op.gen) e.param = g.param;
                    }
                    if (dt == QS_C128) {  // float-float pass: U^dagger's four entries
                        bool real = true;
                        for (int i = 0; i < 8; ++i) {
                            e.c8[i] = u.m[i];
                            real = real && (i % 2 == 0 || u.m[i] == 0.0);
                        }
                        e.op.form = (uint8_t)(real ? G1_FF_REAL : G1_FF_CPLX);
                    } else {
                        e.op.form = (uint8_t)g1_coefficients(u, e.op.gen, e.c8);
                    }
                    gl.push_back(e);
                }
                if (gl.empty()) continue;
                if (l != cur) {
                    p.ops.push_back({SWEEP_LAYOUT, (uint8_t)l, 0, 0, 0});
                    cur = l;
                }
                // one gate of one form on every register bit: a single op (the
                // gates commute, so bit order is as good as circuit order)
                bool all = (int)gl.size() == RB;
                unsigned bits = 0;
                for (const G1Op& e : gl) {
                    all = all && e.op.form == gl[0].op.form && e.op.gen == gl[0].op.gen;
                    bits |= 1u << e.op.arg;
                }
                const int f0 = gl[0].op.form;
                all = all && bits == (1u << RB) - 1 &&
                      (f0 == G1_RSHEAR || f0 == G1_RSHEAR_Y || f0 == G1_CSHEAR_X || f0 == G1_FF_REAL || f0 == G1_FF_CPLX);
                if (all) {
                    std::sort(gl.begin(), gl.end(), [](const G1Op& x, const G1Op& y) { return x.op.arg < y.op.arg; });
                    p.ops.push_back({SWEEP_G1ALL, 0, (uint8_t)f0, gl[0].op.gen, (uint32_t)(p.mats.size() / 8)});
                }
                for (G1Op& e : gl) {
                    e.op.idx = (uint32_t)(p.mats.size() / 8);
                    p.mats.insert(p.mats.end(), e.c8, e.c8 + 8);
                    if (e.param >= 0) p.slots.push_back(e.param);
                    if (!all) p.ops.push_back(e.op);
                }
            }
        }
        p.store_lay = cur <= 1 ? cur : 0;
        for (const SweepDiagRec& d : p.diags)  // block generators' slots follow the staged ones
            for (int g = d.nstaged; g < d.ngen; ++g) p.gens[d.gen0 + g].local += (uint16_t)p.slots.size();
        p.slots.insert(p.slots.end(), block_slots.begin(), block_slots.end());
        p.mat0 = sw.allm.size() / 2;
        sw.allm.insert(sw.allm.end(), p.mats.begin(), p.mats.end());
        p.tab0 = sw.tables.size() / 2;
        sw.tables.insert(sw.tables.end(), p.tabs.begin(), p.tabs.end());
        sw.ops.push_back({4, (int)sw.fused.size()});
        sw.fused.push_back(std::move(p));
    }
    return QS_OK;
}

// Host phase: stages, segments and every launch's arguments.  Stages are
// formed by the scan of Section 4.5 over the reversed gate list: from the
// first unplaced gate, a later gate joins when it commutes with every member
// and with every gate skipped so far (disjoint qubits, or both diagonal);
// a skipped gate obstructs its qubits.
static qs_status build_reverse_sweep(const qs_circuit& c, int n, qs_dtype dt, const qs_options& fast,
                                     cudaStream_t stream, AdjointSweep& sw) {
    const int G = (int)c.gates.size();
    std::vector<SweepUnit> units;  // reverse order
    for (int l = G - 1; l >= 0; --l) {
        const GateRec& g = c.gates[l];
        SweepUnit u;
        u.fwd = l;
        for (int i = 0; i < g.k; ++i) u.qm |= 1ull << g.qubits[i];
        GateRec ud;
        conj_transpose(g, ud);
        u.diag = ud.kind == QS_GATE_DIAGONAL && generator_diagonal(g);
        units.push_back(u);
    }
    const int nchunks = (n + 7) / 8;
    auto crosses = [&](const SweepUnit& u) {
        const GateRec& g = c.gates[u.fwd];
        for (int q = 1; q < g.k; ++q)
            if ((g.qubits[q] >> 3) != (g.qubits[0] >> 3)) return true;
        return false;
    };
    const uint64_t all = n >= 64 ? ~0ull : (1ull << n) - 1;
    std::vector<char> placed(units.size(), 0);
    std::vector<qs_circuit> invs;  // inverse of each general stage, planned at the end
    std::vector<int> segment;  // pending tile-sweep gates (circuit indices, sweep order)
    auto flush_segment = [&]() -> qs_status {
        if (segment.empty()) return QS_OK;
        qs_status st = add_tile_segment(c, segment, n, dt, sw);
        segment.clear();
        return st;
    };
    std::vector<FusedStage> run;  // pending stages for the fused sweep passes
    auto flush_run = [&]() -> qs_status {
        if (run.empty()) return QS_OK;
        qs_status st = add_fused_run(c, run, n, dt, sw);
        run.clear();
        return st;
    };
    const int fused_L = dt == QS_C64 ? kSweepTileC64 : kSweepTileC128;
    for (size_t s0 = 0; s0 < units.size(); ++s0) {
        if (placed[s0]) continue;
        std::vector<size_t> stage{s0};
        placed[s0] = 1;
        uint64_t st_any = units[s0].diag ? 0 : units[s0].qm, st_diag = units[s0].diag ? units[s0].qm : 0;
        uint64_t bl_any = 0, bl_diag = 0;
        bool all_diag = units[s0].diag;
        // Z generators on one qubit / on several, as one diagonal-stage launch counts them
        auto zkind = [&](const SweepUnit& u) {
            const GateRec& g = c.gates[u.fwd];
            if (g.param < 0) return 0;
            int z = 0;
            for (int i = 0; i < g.k; ++i) z += g.paulis[i] == 'Z';
            return z == 1 ? 1 : 2;
        };
        int nsingle = zkind(units[s0]) == 1, nmulti = zkind(units[s0]) == 2, ncross = crosses(units[s0]);
        size_t entries = 256 * (size_t)nchunks + (ncross ? (1u << c.gates[units[s0].fwd].k) : 0);
        int scanned = 0;
        for (size_t j = s0 + 1; j < units.size() && scanned < 4096; ++j) {
            if (placed[j]) continue;
            ++scanned;
            const SweepUnit& u = units[j];
            const bool with_skipped = (u.qm & bl_any) == 0 && (u.diag || (u.qm & bl_diag) == 0);
            const bool with_stage = (u.qm & st_any) == 0 && (u.diag || (u.qm & st_diag) == 0);
            bool join = with_skipped && with_stage;
            if (join && all_diag && u.diag) {  // capacity of one diagonal-stage launch
                const int zk = zkind(u);
                const bool cr = crosses(u);
                const size_t ent = cr ? (1u << c.gates[u.fwd].k) : 0;
                if (nsingle + (zk == 1) > kStageDiagGens || nmulti + (zk == 2) > kStageDiagMulti ||
                    ncross + (int)cr > kStageDiagCross || entries + ent > kStageDiagTabElems)
                    join = false;
                else {
                    nsingle += zk == 1;
                    nmulti += zk == 2;
                    ncross += cr;
                    entries += ent;
                }
            }
            if (join) {
                stage.push_back(j);
                placed[j] = 1;
                if (u.diag) st_diag |= u.qm;
                else st_any |= u.qm;
                all_diag = all_diag && u.diag;
            } else if (u.diag) {
                bl_diag |= u.qm;
            } else {
                bl_any |= u.qm;
            }
            if ((bl_any & all) == all) break;  // every qubit obstructed: nothing more can join
        }
        // fused sweep passes take a stage whose non-diagonal members act on one qubit
        FusedStage fs;
        bool fused_ok = n >= fused_L;
        for (size_t j : stage) {
            const GateRec& g = c.gates[units[j].fwd];
            if (units[j].diag) fs.diag.push_back(units[j].fwd);
            else if (g.k == 1) fs.one.push_back(units[j].fwd);
            else fused_ok = false;
        }
        if (fused_ok) {
            const DiagCost dc = fused_diag_cost(c, fs.diag, n, fused_L - 8);
            fused_ok = dc.tab <= sweep_tab_budget(dt) && dc.cross <= kSweepDiagCross && dc.gens <= kSweepDiagGens;
        }
        if (fused_ok) {
            qs_status fst = flush_segment();
            if (fst != QS_OK) return fst;
            run.push_back(std::move(fs));
            continue;
        }
        {
            qs_status fst = flush_run();
            if (fst != QS_OK) return fst;
        }
        // the gradient tile pass needs 2^8 amplitudes (one per thread)
        if ((int)stage.size() < kStageMin || (!all_diag && n < 8)) {
            for (size_t j : stage) segment.push_back(units[j].fwd);
            continue;
        }
        qs_status fst = flush_segment();
        if (fst != QS_OK) return fst;
        std::vector<const GateRec*> gates;
        for (size_t j : stage) gates.push_back(&c.gates[units[j].fwd]);
        if (all_diag) {
            add_diag_stage(gates, n, sw);
        } else {
            add_gradient_passes(gates, n, dt, sw);
            qs_circuit inv;
            inv.n = n;
            for (const GateRec* g : gates) {  // sweep order; the members commute
                GateRec u;
                conj_transpose(*g, u);
                u.param = -1;
                u.paulis[0] = 0;
                inv.gates.push_back(std::move(u));
            }
            sw.ops.push_back({3, (int)invs.size()});
            invs.push_back(std::move(inv));
        }
    }
    qs_status st = flush_segment();
    if (st == QS_OK) st = flush_run();
    if (st != QS_OK) return st;
    // the stages' inverse plans are independent: fused on host threads
    sw.plans.assign(invs.size(), nullptr);
    std::vector<qs_status> sts(invs.size(), QS_OK);
    std::vector<std::string> msgs(invs.size());
    std::atomic<size_t> next(0);
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned cap = set_host_thread_cap(0);
    set_host_thread_cap(cap);
    auto worker = [&]() {
        cudaSetDevice(dev);
        set_host_thread_cap(cap);
        for (size_t i = next++; i < invs.size(); i = next++) {
            sts[i] = plan_create_on(&invs[i], dt, &fast, stream, &sw.plans[i]);
            if (sts[i] != QS_OK) msgs[i] = qs_last_error();
        }
    };
    const size_t nthreads = std::min<size_t>((size_t)host_threads(8), invs.size());
    std::vector<std::thread> pool;
    for (size_t t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    for (size_t i = 0; i < invs.size(); ++i)
        if (sts[i] != QS_OK) return fail(sts[i], "stage plan: %s", msgs[i].c_str());
    return QS_OK;
}

// ------------------------------------------------------------ block sweep
// Complex64 gradients on the tensor cores (qs_gram.cu).  The sweep undoes
// the forward's fused blocks one at a time, B^dagger on psi and on lambda as
// tensor-core passes, and every gradient inside a block comes from its Gram
// matrix M = sum_s psi_s lambda_s^dagger over the block's six qubits, taken
// just before: <lambda_l|P_l|psi_l> = tr(P_l M_l) with M_l = W^dagger M W, W
// the block's gates after gate l (the reverse sweep, one block per step; the
// blocks are the fusion groups of Sections 4.2-4.5, so their reverse order is
// a valid reverse order of the circuit).
struct BlockSweep {
    std::vector<GateRec> blocks;              // the forward blocks B, last first
    std::vector<Pass> passes;                 // their B^dagger passes, in the same order
    qs_plan* inv = nullptr;                   // those passes, uploaded
    std::vector<int> slot;                    // per pass: Gram slot, or -1 (no generator in the block)
    std::vector<std::array<int, 6>> targets;  // per slot: the Gram's six qubits, descending
    std::vector<BlockGradGate> gates;         // per slot: the block's gates, last to first
    std::vector<int> gate0;                   // slot ranges (slots + 1)
    std::vector<float> gmats;                 // complex64 gate matrices
    void release() {
        if (inv) qs_plan_destroy(inv);
        inv = nullptr;
    }
};

// Plan the block sweep; QS_ERR_UNSUPPORTED when a group is not one block of
// at most six qubits (wide diagonal clusters), so the stage sweep is used.
// known (optional): the groups' block products, already formed by the
// streamed forward (taken over when there is one per group).
static qs_status build_block_sweep(const qs_circuit& c, int n, const qs_options& fast, BlockSweep& bs,
                                   std::vector<GateRec>* known = nullptr) {
    std::vector<std::vector<int>> groups;
    qs_status st = fuse_each(n, c.gates, 6, fast.fusion_effort, c.fuse_cache.get(),
                             [&](std::vector<int>&& g) { groups.push_back(std::move(g)); });
    if (st != QS_OK) return st;
    const size_t G = groups.size();
    std::vector<GateRec> blocks(G);
    const bool reuse = known && known->size() == G;
    if (reuse) blocks.swap(*known);
    std::vector<Pass> fwd_inv(G);
    std::vector<char> bad(G, 0);
    std::atomic<size_t> next(0);
    auto work = [&]() {
        for (size_t i = next++; i < G; i = next++) {
            if (!reuse) block_product(n, c.gates, groups[i], blocks[i]);
            if (blocks[i].k == 0) {
                bad[i] = 1;
                continue;
            }
            GateRec binv;
            conj_transpose(blocks[i], binv);
            single_block_pass(n, QS_C64, fast, binv, fwd_inv[i]);
            factor_tile_scalars(fwd_inv[i]);
        }
    };
    {
        const size_t nt = std::min<size_t>(host_threads(4), G);
        std::vector<std::thread> pool;
        for (size_t t = 1; t < nt; ++t) pool.emplace_back(work);
        work();
        for (auto& th : pool) th.join();
    }
    for (size_t i = 0; i < G; ++i)
        if (bad[i]) return QS_ERR_UNSUPPORTED;
    bs.passes.reserve(G);
    bs.gate0.assign(1, 0);
    for (size_t r = 0; r < G; ++r) {
        const size_t i = G - 1 - r;  // the sweep runs the blocks last to first
        const std::vector<int>& g = groups[i];
        std::vector<int> members;
        if (g[0] < 0) members.push_back(-1 - g[0]);
        else members = g;
        bool has_param = false;
        for (int gi : members) has_param = has_param || c.gates[gi].param >= 0;
        bs.passes.push_back(std::move(fwd_inv[i]));
        if (!has_param) {
            bs.slot.push_back(-1);
            continue;
        }
        // Gram qubits: the block's, then the highest others (low qubits stay
        // set bits, so a set's neighbours are adjacent amplitudes)
        uint64_t used = 0;
        for (int t = 0; t < blocks[i].k; ++t) used |= 1ull << blocks[i].qubits[t];
        for (int q = n - 1; q >= 0 && __builtin_popcountll(used) < 6; --q) used |= 1ull << q;
        std::array<int, 6> T{};
        int cnt = 0;
        for (int q = n - 1; q >= 0; --q)
            if ((used >> q) & 1) T[cnt++] = q;
        bs.slot.push_back((int)bs.targets.size());
        bs.targets.push_back(T);
        // The block's gates last to first.  A run of diagonal gates with
        // diagonal generators commutes, and its generators with every update
        // inside it, so all its gradients come from the M at the run's end,
        // followed by one elementwise update with the run's product.
        auto record = [&](const GateRec& gr) {
            BlockGradGate bg{};
            bg.k = gr.k;
            for (int t = 0; t < gr.k; ++t) {
                int pos = 0;
                while (T[pos] != gr.qubits[t]) ++pos;
                bg.lb[t] = 5 - pos;
            }
            bg.param = gr.param;
            if (gr.param >= 0)
                for (int t = 0; t < gr.k; ++t) {
                    const char pc = gr.paulis[t];
                    if (pc == 'X' || pc == 'Y') bg.xmask |= 1 << bg.lb[t];
                    if (pc == 'Y' || pc == 'Z') bg.zmask |= 1 << bg.lb[t];
                    bg.ny += pc == 'Y';
                }
            bg.diag = gr.kind == QS_GATE_DIAGONAL;
            return bg;
        };
        auto push_full = [&](BlockGradGate bg, const GateRec& gr) {
            bg.moff = (uint32_t)(bs.gmats.size() / 2);
            for (double v : gr.m) bs.gmats.push_back((float)v);
            bs.gates.push_back(bg);
        };
        std::vector<const GateRec*> run;  // the current run, in sweep order
        // last: the run ends the block, and no update after it is read
        auto flush_run = [&](bool last) {
            if (run.empty()) return;
            if (run.size() == 1 && !last) {
                push_full(record(*run[0]), *run[0]);
            } else {
                std::vector<std::complex<double>> prod(64, 1.0);
                for (const GateRec* g : run) {
                    BlockGradGate bg = record(*g);
                    const int d = 1 << g->k;
                    for (int j = 0; j < 64; ++j) {
                        int li = 0;
                        for (int t = 0; t < g->k; ++t) li = (li << 1) | ((j >> bg.lb[t]) & 1);
                        const double er = g->m[2 * (li * d + li)], ei = g->m[2 * (li * d + li) + 1];
                        prod[j] = std::complex<double>(prod[j].real() * er - prod[j].imag() * ei,
                                                       prod[j].real() * ei + prod[j].imag() * er);
                    }
                    if (g->param >= 0) {  // its gradient now; its update with the run's
                        bg.flags = kGradNoUpdate;
                        bg.moff = 0;
                        bs.gates.push_back(bg);
                    }
                }
                if (!last) {
                    BlockGradGate bg{};
                    bg.k = 6;
                    for (int t = 0; t < 6; ++t) bg.lb[t] = 5 - t;  // gate index = local index
                    bg.param = -1;
                    bg.diag = 1;
                    bg.flags = kGradCompactDiag;
                    bg.moff = (uint32_t)(bs.gmats.size() / 2);
                    for (const auto& z : prod) {
                        bs.gmats.push_back((float)z.real());
                        bs.gmats.push_back((float)z.imag());
                    }
                    bs.gates.push_back(bg);
                }
            }
            run.clear();
        };
        for (size_t m = members.size(); m-- > 0;) {
            const GateRec& gr = c.gates[members[m]];
            BlockGradGate bg = record(gr);
            if (bg.diag && bg.xmask == 0) {
                run.push_back(&gr);
                continue;
            }
            flush_run(false);
            if (m == 0) bg.flags = kGradNoUpdate;  // the block's first gate: nothing reads M after it
            if (bg.param >= 0 || m != 0) push_full(bg, gr);
        }
        flush_run(true);
        bs.gate0.push_back((int)bs.gates.size());
    }
    for (size_t r = 0; r < G; ++r) bs.blocks.push_back(std::move(blocks[G - 1 - r]));
    return QS_OK;
}

// Device phase: per block, its Gram matrix (when it has generators), then
// B^dagger on both states; finally every block's gradients into sums.  All
// device memory is one allocation from the library's pool and all host data
// one copy through pinned staging, so the host enqueues the sweep without
// waiting for the forward still running on the stream.
namespace {
thread_local PinnedStage t_sweep_stage;
}

static qs_status run_block_sweep(BlockSweep& bs, const qs_options& fast, qs_state* psi, qs_state* lam, double* sums,
                                 cudaStream_t sm) {
    const int nslots = (int)bs.targets.size();
    const int npass = (int)bs.passes.size();
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    // layout: [pass matrices | gates | gate0 | gate matrices] (uploaded), [M | Gram parts] (device only)
    size_t mats_elems = 0;
    for (Pass& ps : bs.passes) {
        ps.dev_offset = mats_elems;
        mats_elems += ps.mats.size() / 2;
    }
    const size_t o_gates = up(mats_elems * 8), o_gate0 = o_gates + up(sizeof(BlockGradGate) * bs.gates.size());
    const size_t o_gmats = o_gate0 + up(sizeof(int) * bs.gate0.size());
    const size_t host_bytes = o_gmats + up(sizeof(float) * bs.gmats.size());
    const size_t o_M = host_bytes, o_ws = o_M + up(sizeof(double) * 8192 * (size_t)nslots);
    const size_t total = o_ws + sizeof(double) * gram_workspace_elems(psi->n) * (size_t)nslots;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = t_sweep_stage.reserve(host_bytes, dev);
    if (e != cudaSuccess) return cuda_fail(e, "sweep staging");
    char* hp = t_sweep_stage.p;
    {
        float* f = reinterpret_cast<float*>(hp);
        size_t at = 0;
        for (const Pass& ps : bs.passes)
            for (double v : ps.mats) f[at++] = (float)v;
    }
    std::copy(bs.gates.begin(), bs.gates.end(), reinterpret_cast<BlockGradGate*>(hp + o_gates));
    std::copy(bs.gate0.begin(), bs.gate0.end(), reinterpret_cast<int*>(hp + o_gate0));
    std::copy(bs.gmats.begin(), bs.gmats.end(), reinterpret_cast<float*>(hp + o_gmats));
    char* base = nullptr;
    e = lib_malloc_async(reinterpret_cast<void**>(&base), total, sm);
    if (e != cudaSuccess) return cuda_fail(e, "block sweep memory");
    e = cudaMemcpyAsync(base, hp, host_bytes, cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess) e = cudaEventRecord(t_sweep_stage.done, sm);  // the staging is free once this passes
    if (e != cudaSuccess) {
        cudaFreeAsync(base, sm);
        return cuda_fail(e, "block sweep upload");
    }
    // the inverse passes as a plan over the uploaded matrices (not owned by it)
    bs.inv = new (std::nothrow) qs_plan;
    if (!bs.inv) {
        cudaFreeAsync(base, sm);
        return fail(QS_ERR_OOM, "host allocation failed");
    }
    bs.inv->n = psi->n;
    bs.inv->dt = QS_C64;
    bs.inv->opt = fast;
    bs.inv->device = dev;
    bs.inv->passes = std::move(bs.passes);
    bs.inv->dev_mats = base;
    bs.inv->dev_elems = mats_elems;
    double* Mall = reinterpret_cast<double*>(base + o_M);
    double* ws = reinterpret_cast<double*>(base + o_ws);
    qs_status st = QS_OK;
    for (int i = 0; i < npass && e == cudaSuccess && st == QS_OK; ++i) {
        const int sl = bs.slot[i];
        if (sl >= 0)
            e = launch_gram(psi->data, lam->data, psi->n, bs.targets[sl].data(),
                            ws + gram_workspace_elems(psi->n) * (size_t)sl, psi->errflag, sm);
        if (e != cudaSuccess) break;
        if (i + 1 == npass) break;  // the first block's inverse: nothing reads the states after it
        st = qs_plan_execute_range(psi, bs.inv, i, 1);
        if (st == QS_OK) st = qs_plan_execute_range(lam, bs.inv, i, 1);
    }
    if (e == cudaSuccess && st == QS_OK && nslots) {
        e = launch_gram_reduce(ws, psi->n, nslots, Mall, sm);
        if (e == cudaSuccess)
            e = launch_block_grads(Mall, nslots, reinterpret_cast<const BlockGradGate*>(base + o_gates),
                                   reinterpret_cast<const int*>(base + o_gate0), base + o_gmats, sums, sm);
    }
    cudaFreeAsync(base, sm);
    bs.inv->dev_mats = nullptr;  // freed above, in stream order
    if (st != QS_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "block sweep");
    return QS_OK;
}

// Device phase: one upload of the tile-sweep matrices and the phase tables,
// then every launch in order on the states' stream.
static qs_status run_reverse_sweep(AdjointSweep& sw, qs_state* psi, qs_state* lam, int nb, int rows, cudaStream_t sm) {
    sw.stream = sm;
    const size_t esz = psi->amp_bytes();
    auto convert = [&](const std::vector<double>& v, std::vector<char>& out) {
        out.resize(v.size() / 2 * esz);
        for (size_t i = 0; i < v.size(); ++i) {
            if (psi->dt == QS_C64) ((float*)out.data())[i] = (float)v[i];
            else ((double*)out.data())[i] = v[i];
        }
    };
    convert(sw.allm, sw.hostm);
    convert(sw.tables, sw.hostt);
    QS_CUDA(cudaMallocAsync(&sw.partials, sizeof(double) * 2 * nb * (size_t)rows, sm));
    QS_CUDA(cudaMallocAsync(&sw.sums, sizeof(double) * 2 * rows, sm));
    QS_CUDA(cudaMallocAsync(&sw.dmats, std::max<size_t>(sw.hostm.size(), 16), sm));
    QS_CUDA(cudaMallocAsync(&sw.dtables, std::max<size_t>(sw.hostt.size(), 16), sm));
    QS_CUDA(cudaMemsetAsync(sw.partials, 0, sizeof(double) * 2 * nb * (size_t)rows, sm));
    if (!sw.hostm.empty()) QS_CUDA(cudaMemcpyAsync(sw.dmats, sw.hostm.data(), sw.hostm.size(), cudaMemcpyHostToDevice, sm));
    if (!sw.hostt.empty()) QS_CUDA(cudaMemcpyAsync(sw.dtables, sw.hostt.data(), sw.hostt.size(), cudaMemcpyHostToDevice, sm));
    for (const SweepOp& op : sw.ops) {
        cudaError_t e = cudaSuccess;
        if (op.type == 0) {
            const AdjPass& ap = sw.tile[op.index];
            const void* dm = (const char*)sw.dmats + ap.mat0 * esz;
            e = launch_adjoint_tile(psi->data, lam->data, psi->n, psi->dt, ap.L, ap.pos, ap.tg, dm, ap.mats.size() / 2,
                                    sw.partials, nb, sm);
        } else if (op.type == 1) {
            const GradLaunch& gl = sw.grad[op.index];
            e = launch_grad_pairs(psi->data, lam->data, psi->n, psi->dt, gl.L, gl.pos, gl.gens, sw.partials, nb, sm);
        } else if (op.type == 2) {
            const DiagLaunch& dl = sw.diag[op.index];
            e = launch_diag_stage(psi->data, lam->data, psi->n, psi->dt, dl.nchunks, dl.cross,
                                  (const char*)sw.dtables + dl.tab0 * esz, dl.tab_elems, dl.zm, dl.slots, dl.apply,
                                  sw.partials, nb, sm);
        } else if (op.type == 4) {
            const SweepPassDesc& fp = sw.fused[op.index];
            e = launch_sweep_pass(psi->data, lam->data, psi->n, psi->dt, fp, (const char*)sw.dmats + fp.mat0 * esz,
                                  (const char*)sw.dtables + fp.tab0 * esz, sw.partials, nb, sm);
        } else {
            qs_status st = qs_plan_execute(psi, sw.plans[op.index]);
            if (st == QS_OK) st = qs_plan_execute(lam, sw.plans[op.index]);
            if (st != QS_OK) return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "adjoint sweep launch");
    }
    return QS_OK;
}

extern "C" {

qs_status qs_adjoint_gradient(qs_circuit* c, const double* theta, int num_params, const qs_pauli_sum* h,
                              qs_state* psi, qs_state* lam, double* energy, double* grad) {
    if (!c || !h || !psi || !lam || !energy || (num_params > 0 && !grad))
        return fail(QS_ERR_ARG, "null argument");
    qs_status st = check_state(psi);
    if (st != QS_OK) return st;
    st = check_state(lam);
    if (st != QS_OK) return st;
    if (psi->n != c->n || lam->n != c->n || h->n != c->n || psi->dt != lam->dt)
        return fail(QS_ERR_ARG, "circuit, states and Hamiltonian disagree on n or dtype");
    if (psi->data == lam->data) return fail(QS_ERR_ARG, "psi and lambda must be distinct");
    if (num_params != c->num_params)
        return fail(QS_ERR_ARG, "circuit has %d parameters, %d given", c->num_params, num_params);
    {
        std::vector<char> seen(c->num_params, 0);
        for (const GateRec& g : c->gates)
            if (g.param >= 0) {
                if (seen[g.param]) return fail(QS_ERR_UNSUPPORTED, "parameter %d is shared by several gates", g.param);
                seen[g.param] = 1;
            }
    }
    if (num_params) {
        st = qs_circuit_set_params(c, theta, num_params);
        if (st != QS_OK) return st;
    }
    cudaStream_t sm = psi->stream;
    if (lam->stream != sm) return fail(QS_ERR_ARG, "psi and lambda must share a stream");
    // forward: psi = U |0>, with the fastest exact plan (6-qubit blocks, on
    // the tensor cores for complex64)
    qs_options fast;
    qs_options_default(&fast);
    if (psi->dt == QS_C64 && gemm_supported(psi->n, 6)) {
        fast.k_max = 6;
        fast.precision = QS_PREC_3XTF32;
    } else if (psi->dt == QS_C128) {
        fast.k_max = 3;  // blocks the float-float register tile applies (up to its 3 register bits)
    }
    // the full block search (fewer blocks); its grouping is cached on the
    // circuit, so repeated gradients (new angles, same gates) skip it
    fast.fusion_effort = 1;
    // The forward and lambda are enqueued first while the reverse sweep is
    // planned on a host thread of its own (it reads only the gate list; plan
    // memory is stream-ordered, so nothing here synchronises).
    AdjointSweep sw;
    struct Releaser {  // on every return, after the planner thread has joined
        AdjointSweep& s;
        ~Releaser() { s.release(); }
    } releaser{sw};
    qs_status sweep_st = QS_OK;
    std::string sweep_msg;
    struct Joiner {
        std::thread t;
        ~Joiner() {
            if (t.joinable()) t.join();
        }
    } planner;
    // complex64 with tensor-core blocks: the block sweep (gradients from Gram
    // matrices); otherwise, or when a group is not a block of at most six
    // qubits, the stage sweep
    BlockSweep bsw;
    struct BlockReleaser {
        BlockSweep& s;
        ~BlockReleaser() { s.release(); }
    } block_releaser{bsw};
    bool use_blocks = false;
    std::vector<GateRec> fwd_blocks;  // the forward's block products (kept when the sweep is planned here)
    auto plan_sweep = [&]() {
        if (psi->dt == QS_C64 && fast.k_max == 6 && gram_supported(psi->n)) {
            sweep_st = build_block_sweep(*c, psi->n, fast, bsw, &fwd_blocks);
            if (sweep_st == QS_OK) {
                use_blocks = true;
                return;
            }
            bsw = BlockSweep();
            if (sweep_st != QS_ERR_UNSUPPORTED) {
                sweep_msg = qs_last_error();
                return;
            }
        }
        sweep_st = build_reverse_sweep(*c, psi->n, psi->dt, fast, sm, sw);
        if (sweep_st != QS_OK) sweep_msg = qs_last_error();
    };
    // (with the host threads capped at one, as inside a batch of gradients
    // that run in parallel, it is planned here after the forward is enqueued)
    const bool own_thread = host_threads(2) >= 2;
    if (own_thread) {
        int dev = 0;
        cudaGetDevice(&dev);
        const unsigned cap = set_host_thread_cap(0);
        set_host_thread_cap(cap);
        planner.t = std::thread([&, dev, cap]() {
            cudaSetDevice(dev);  // the caller's device and thread cap hold on this thread too
            set_host_thread_cap(cap);
            plan_sweep();
        });
    }
    if (fast.k_max == 6) {  // on the tensor cores: fused and run together (the GPU starts at once)
        cudaError_t le = launch_init_basis(psi->data, psi->n, psi->dt, 0, sm);
        if (le != cudaSuccess) return cuda_fail(le, "init");
        st = apply_streamed(psi, c, fast, own_thread ? nullptr : &fwd_blocks);
        if (st != QS_OK) return st;
    } else {
        qs_plan* fwd = nullptr;
        st = plan_create_on(c, psi->dt, &fast, sm, &fwd);
        if (st != QS_OK) return st;
        cudaError_t le = launch_init_basis(psi->data, psi->n, psi->dt, 0, sm);
        if (le != cudaSuccess) {
            qs_plan_destroy(fwd);
            return cuda_fail(le, "init");
        }
        st = qs_plan_execute(psi, fwd);
        qs_plan_destroy(fwd);  // freed in stream order, after the forward passes
        if (st != QS_OK) return st;
    }
    // lambda = H psi; E = <psi|lambda>
    QS_CUDA(launch_apply_pauli_sum(psi->data, lam->data, psi->n, psi->dt, *h, sm));
    double* res = result_area(psi);
    QS_CUDA(launch_inner(psi->data, lam->data, psi->n, psi->dt, psi->scratch, res, sm));
    if (own_thread) planner.t.join();
    else plan_sweep();
    if (sweep_st != QS_OK) return fail(sweep_st, "%s", sweep_msg.c_str());
    const int rows = std::max(num_params, 1);
    double* sums = nullptr;  // (Re, Im) <lambda|P|psi> per parameter
    cudaError_t e = cudaSuccess;
    if (use_blocks) {
        QS_CUDA(cudaMallocAsync(&sums, sizeof(double) * 2 * rows, sm));
        e = cudaMemsetAsync(sums, 0, sizeof(double) * 2 * rows, sm);
        st = e == cudaSuccess ? run_block_sweep(bsw, fast, psi, lam, sums, sm) : cuda_fail(e, "block sweep");
        if (st != QS_OK) {
            cudaFreeAsync(sums, sm);
            return st;
        }
    } else {
        const int nb = reduce_blocks();
        st = run_reverse_sweep(sw, psi, lam, nb, rows, sm);
        if (st != QS_OK) {
            sw.release();
            return st;
        }
        e = launch_sum_partials(sw.partials, rows, nb, sw.sums, sm);
        sums = sw.sums;
    }
    std::vector<double> host(2 * rows + 2);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host.data(), sums, sizeof(double) * 2 * rows, cudaMemcpyDeviceToHost, sm);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host.data() + 2 * rows, res, sizeof(double) * 2, cudaMemcpyDeviceToHost, sm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
    if (use_blocks) cudaFreeAsync(sums, sm);
    sw.release();
    bsw.release();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint sweep");
    st = check_device_flag(psi);
    if (st != QS_OK) return st;
    st = check_device_flag(lam);
    if (st != QS_OK) return st;
    *energy = host[2 * rows];
    for (int p = 0; p < num_params; ++p) grad[p] = host[2 * p + 1];  // Im <lambda|P|psi>
    return QS_OK;
}

qs_status qs_adjoint_gradient_batch(int count, qs_circuit* const* circuits, const double* const* thetas,
                                    const int* num_params, const qs_pauli_sum* const* hams,
                                    qs_state* const* psi, qs_state* const* lam, double* energies,
                                    double* const* grads) {
    if (count < 0) return fail(QS_ERR_ARG, "negative count");
    if (count == 0) return QS_OK;
    if (!circuits || !thetas || !num_params || !hams || !psi || !lam || !energies || !grads)
        return fail(QS_ERR_ARG, "null array");
    {  // distinct circuits (their parameters are set) and distinct states
        std::vector<const void*> objs, mem;
        for (int i = 0; i < count; ++i) {
            if (!circuits[i] || !psi[i] || !lam[i]) return fail(QS_ERR_ARG, "null entry %d", i);
            objs.push_back(circuits[i]);
            mem.push_back(psi[i]->data);
            mem.push_back(lam[i]->data);
        }
        std::sort(objs.begin(), objs.end());
        std::sort(mem.begin(), mem.end());
        if (std::adjacent_find(objs.begin(), objs.end()) != objs.end())
            return fail(QS_ERR_ARG, "a circuit appears twice in the batch");
        if (std::adjacent_find(mem.begin(), mem.end()) != mem.end())
            return fail(QS_ERR_ARG, "a state appears twice in the batch");
    }
    std::vector<qs_status> status(count, QS_OK);
    std::vector<std::string> msg(count);
    std::atomic<int> next(0);
    auto worker = [&]() {
        const unsigned prev = set_host_thread_cap(1);  // the gradients themselves run in parallel
        for (int i = next++; i < count; i = next++) {
            cudaSetDevice(psi[i]->device);
            status[i] = qs_adjoint_gradient(circuits[i], thetas[i], num_params[i], hams[i], psi[i], lam[i],
                                            &energies[i], grads[i]);
            if (status[i] != QS_OK) msg[i] = qs_last_error();
        }
        set_host_thread_cap(prev);
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nthreads = std::min(count, (int)std::min(16u, hw));
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    for (int i = 0; i < count; ++i)
        if (status[i] != QS_OK) return fail(status[i], "gradient %d: %s", i, msg[i].c_str());
    return QS_OK;
}

}  // extern "C"
