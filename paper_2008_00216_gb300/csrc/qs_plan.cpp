// Host-side planning: gate classification, rotation matrices, gate fusion
// with commuting reorder, and grouping of fused blocks into passes.
//
// Fusion and pass formation are the same scan (Section 4.5, "Gate clustering
// by reordering"): start at the first unplaced gate and walk forward; a later
// gate joins the current group when it commutes with every gate skipped so
// far -- disjoint qubits, or both diagonal (Sections 4.2 and 4.3) -- and the
// group's qubit set stays within its bound.  A skipped gate marks its qubits
// obstructed.  The paper's "same kind" test is replaced by "fits in the
// group's qubit bound": k_max qubits for a fused matrix (whose FP64 product
// replaces the group, as in Eq. 2's coalescing), or the tile's qubit count
// for a shared-memory pass that applies the group's blocks one after another.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <deque>
#include <functional>
#include <thread>
#include <unordered_map>

#include "qs_internal.h"

namespace qsgb {

using cd = std::complex<double>;

int classify_matrix(int k, const double* m) {
    const int d = 1 << k;
    bool diag = true, mono = true;
    for (int r = 0; r < d; ++r) {
        int nz = 0;
        for (int c = 0; c < d; ++c) {
            const double re = m[2 * (r * d + c)], im = m[2 * (r * d + c) + 1];
            if (re != 0.0 || im != 0.0) {
                ++nz;
                if (r != c) diag = false;
            }
        }
        if (nz != 1) mono = false;
    }
    if (mono) {  // columns must also hold exactly one nonzero
        for (int c = 0; c < d && mono; ++c) {
            int nz = 0;
            for (int r = 0; r < d; ++r)
                if (m[2 * (r * d + c)] != 0.0 || m[2 * (r * d + c) + 1] != 0.0) ++nz;
            if (nz != 1) mono = false;
        }
    }
    if (diag && mono) return QS_GATE_DIAGONAL;
    if (mono) return QS_GATE_MONOMIAL;
    return QS_GATE_DENSE;
}

static void pauli_1q(char c, cd p[2][2]) {
    p[0][0] = p[0][1] = p[1][0] = p[1][1] = 0.0;
    switch (c) {
        case 'X': p[0][1] = 1.0; p[1][0] = 1.0; break;
        case 'Y': p[0][1] = cd(0, -1); p[1][0] = cd(0, 1); break;
        case 'Z': p[0][0] = 1.0; p[1][1] = -1.0; break;
        default: p[0][0] = 1.0; p[1][1] = 1.0; break;
    }
}

void pauli_matrix(int k, const char* paulis, double* m) {
    const int d = 1 << k;
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            cd v = 1.0;
            for (int i = 0; i < k; ++i) {  // paulis[0] is the most significant local bit
                cd p[2][2];
                pauli_1q(paulis[i], p);
                const int br = (r >> (k - 1 - i)) & 1, bc = (c >> (k - 1 - i)) & 1;
                v *= p[br][bc];
            }
            m[2 * (r * d + c)] = v.real();
            m[2 * (r * d + c) + 1] = v.imag();
        }
}

void rotation_matrix(int k, const char* paulis, double theta, double* m) {
    // exp(-i theta P / 2) = cos(theta/2) I - i sin(theta/2) P, since P^2 = I
    const int d = 1 << k;
    pauli_matrix(k, paulis, m);
    const double c = cos(0.5 * theta), s = sin(0.5 * theta);
    for (int r = 0; r < d; ++r)
        for (int col = 0; col < d; ++col) {
            const double pr = m[2 * (r * d + col)], pi = m[2 * (r * d + col) + 1];
            // -i s (pr + i pi) = s pi - i s pr
            double re = s * pi, im = -s * pr;
            if (r == col) re += c;
            m[2 * (r * d + col)] = re;
            m[2 * (r * d + col) + 1] = im;
        }
}

static inline uint64_t qmask(const GateRec& g) {
    if (g.k == 0) return g.wide_mask;  // a wide diagonal cluster
    uint64_t m = 0;
    for (int i = 0; i < g.k; ++i) m |= 1ull << g.qubits[i];
    return m;
}

// Multiply gate g (on its qubits) into the block matrix acc = R + i I
// (real and imaginary parts apart, row-major D x D, so the column loops
// vectorise) whose local bit b corresponds to qubit bq[K-1-b] (bq listed
// most significant first): acc <- E(g) acc.  For each row set r (the gate's
// bits zero) the 2^k rows r | l mix as (g.m) x (those rows), for all D
// columns at once; complex products are written out in real arithmetic.
static void apply_into_block(const GateRec& g, int K, const int* bq, double* R, double* I) {
    const int D = 1 << K, d = 1 << g.k;
    int lpos[kMaxK];  // local bit of each gate qubit
    for (int i = 0; i < g.k; ++i) {
        lpos[i] = -1;
        for (int j = 0; j < K; ++j)
            if (bq[j] == g.qubits[i]) lpos[i] = K - 1 - j;
    }
    uint64_t gmask = 0;
    for (int i = 0; i < g.k; ++i) gmask |= 1ull << lpos[i];
    int rowof[1 << kMaxK];  // offset of local gate index l within a row set
    for (int l = 0; l < d; ++l) {
        int idx = 0;
        for (int i = 0; i < g.k; ++i)
            if ((l >> (g.k - 1 - i)) & 1) idx |= 1 << lpos[i];
        rowof[l] = idx;
    }
    const double* m = g.m.data();
    if (g.kind == QS_GATE_DIAGONAL) {  // scale each row by its diagonal entry
        for (int r = 0; r < D; ++r) {
            int l = 0;
            for (int i = 0; i < g.k; ++i) l = (l << 1) | ((r >> lpos[i]) & 1);
            const double mr = m[2 * (l * d + l)], mi = m[2 * (l * d + l) + 1];
            if (mr == 1.0 && mi == 0.0) continue;
            double* xr = R + (size_t)r * D;
            double* xi = I + (size_t)r * D;
            for (int c = 0; c < D; ++c) {
                const double a = xr[c], b = xi[c];
                xr[c] = mr * a - mi * b;
                xi[c] = mr * b + mi * a;
            }
        }
        return;
    }
    if (g.k == 1) {  // in place: each row pair (r, r | bit) mixes as a 2 x 2
        const double m00r = m[0], m00i = m[1], m01r = m[2], m01i = m[3];
        const double m10r = m[4], m10i = m[5], m11r = m[6], m11i = m[7];
        const int bit = 1 << lpos[0];
        for (int r = 0; r < D; ++r) {
            if (r & bit) continue;
            double* __restrict__ r0 = R + (size_t)r * D;
            double* __restrict__ i0 = I + (size_t)r * D;
            double* __restrict__ r1 = R + (size_t)(r | bit) * D;
            double* __restrict__ i1 = I + (size_t)(r | bit) * D;
            for (int c = 0; c < D; ++c) {
                const double ar = r0[c], ai = i0[c], br = r1[c], bi = i1[c];
                r0[c] = (m00r * ar - m00i * ai) + (m01r * br - m01i * bi);
                i0[c] = (m00r * ai + m00i * ar) + (m01r * bi + m01i * br);
                r1[c] = (m10r * ar - m10i * ai) + (m11r * br - m11i * bi);
                i1[c] = (m10r * ai + m10i * ar) + (m11r * bi + m11i * br);
            }
        }
        return;
    }
    thread_local std::vector<double> inr, ini;
    inr.resize((size_t)d * D);
    ini.resize((size_t)d * D);
    for (int r = 0; r < D; ++r) {
        if (r & gmask) continue;
        for (int l = 0; l < d; ++l) {
            const size_t row = (size_t)(r | rowof[l]) * D;
            std::copy(R + row, R + row + D, inr.begin() + (size_t)l * D);
            std::copy(I + row, I + row + D, ini.begin() + (size_t)l * D);
        }
        for (int lo = 0; lo < d; ++lo) {
            double* __restrict__ outr = R + (size_t)(r | rowof[lo]) * D;
            double* __restrict__ outi = I + (size_t)(r | rowof[lo]) * D;
            for (int c = 0; c < D; ++c) {
                outr[c] = 0.0;
                outi[c] = 0.0;
            }
            for (int li = 0; li < d; ++li) {
                const double mr = m[2 * (lo * d + li)], mi = m[2 * (lo * d + li) + 1];
                const double* __restrict__ xr = inr.data() + (size_t)li * D;
                const double* __restrict__ xi = ini.data() + (size_t)li * D;
                for (int c = 0; c < D; ++c) {
                    outr[c] += mr * xr[c] - mi * xi[c];
                    outi[c] += mr * xi[c] + mi * xr[c];
                }
            }
        }
    }
}

// One greedy scan from the first unplaced gate; returns the indices taken.
// `bound` limits popcount(init_mask | taken qubits); `max_dense_k` bounds
// the size of non-diagonal members (diagonal ones may use up to kMaxK).
static std::vector<int> scan_group(const std::vector<GateRec>& g, std::vector<char>& placed,
                                   int start, uint64_t init_mask, int bound, int window,
                                   int max_dense_k = kMaxK,
                                   const std::function<bool(const GateRec&)>* accept = nullptr) {
    std::vector<int> taken;
    uint64_t support = init_mask | qmask(g[start]);
    taken.push_back(start);
    placed[start] = 1;
    uint64_t blocked_any = 0, blocked_diag = 0;
    int scanned = 0;
    for (int j = start + 1; j < (int)g.size() && scanned < window; ++j) {
        if (placed[j]) continue;
        ++scanned;
        const uint64_t gm = qmask(g[j]);
        const bool gdiag = g[j].kind == QS_GATE_DIAGONAL;
        const bool commutes = (gm & blocked_any) == 0 && (gdiag || (gm & blocked_diag) == 0);
        const bool fits = __builtin_popcountll(support | gm) <= bound &&
                          (gdiag || g[j].k <= max_dense_k);
        if (commutes && fits && (!accept || (*accept)(g[j]))) {
            taken.push_back(j);
            placed[j] = 1;
            support |= gm;
        } else if (gdiag) {
            blocked_diag |= gm;
        } else {
            blocked_any |= gm;
        }
        // nothing more can join: the support is full and fully obstructed
        if (__builtin_popcountll(support) >= bound && (support & ~blocked_any) == 0) break;
    }
    return taken;
}

// The gates as the block search reads them: qubit masks, diagonal flags and
// whether a gate may join a block at all, in flat arrays.
struct GateView {
    std::vector<uint64_t> m;
    std::vector<uint8_t> diag, ok;
    std::vector<int> idx;  // the gate's index in the circuit
    uint64_t allq = 0;     // the qubits of the circuit
};

// The scan of Section 4.5 with the block's qubit set S fixed, over `v` (the
// unplaced gates after `start`, in order): take every gate whose qubits lie
// in S and that commutes with the gates skipped so far (disjoint qubits, or
// both diagonal); a skipped gate obstructs its qubits.  With `ext`, also collect the qubits that each
// reachable gate outside S would add (keeping |S| <= kmax).
static int absorb_scan(const GateView& v, int start, uint64_t S, std::vector<int>* taken, std::vector<uint64_t>* ext,
                       int kmax) {
    int count = 1;
    if (taken) taken->push_back(start);
    uint64_t blocked_any = 0, blocked_diag = 0;
    const int G = (int)v.m.size();
    for (int j = 0; j < G; ++j) {
        const uint64_t gm = v.m[j];
        const bool gdiag = v.diag[j];
        const bool commutes = (gm & blocked_any) == 0 && (gdiag || (gm & blocked_diag) == 0);
        const bool ok = v.ok[j];
        if (commutes && ok && (gm & ~S) == 0) {
            ++count;
            if (taken) taken->push_back(v.idx[j]);
            continue;
        }
        if (ext && commutes && ok && __builtin_popcountll(S | gm) <= kmax) ext->push_back(gm & ~S);
        if (gdiag) blocked_diag |= gm;
        else blocked_any |= gm;
        // every qubit of S (of the circuit, for extensions) obstructed by a
        // non-diagonal gate: no later gate can join or extend
        if ((ext ? (v.allq & ~blocked_any) : (S & ~blocked_any)) == 0) break;
    }
    return count;
}

// Open-addressing map from a nonzero qubit set to an int (linear probing).
struct SetMap {
    std::vector<uint64_t> keys;
    std::vector<int> vals;
    size_t used = 0;
    explicit SetMap(size_t cap = 1024) : keys(cap, 0), vals(cap, 0) {}
    static size_t hash(uint64_t k) { return (size_t)((k * 0x9E3779B97F4A7C15ull) >> 20); }
    int* find(uint64_t k) {
        const size_t mask = keys.size() - 1;
        for (size_t i = hash(k) & mask;; i = (i + 1) & mask) {
            if (keys[i] == k) return &vals[i];
            if (keys[i] == 0) return nullptr;
        }
    }
    void put(uint64_t k, int v) {
        if (2 * (used + 1) > keys.size()) {  // grow at half full
            SetMap bigger(keys.size() * 2);
            for (size_t i = 0; i < keys.size(); ++i)
                if (keys[i]) bigger.put(keys[i], vals[i]);
            *this = std::move(bigger);
        }
        const size_t mask = keys.size() - 1;
        size_t i = hash(k) & mask;
        while (keys[i] != 0 && keys[i] != k) i = (i + 1) & mask;
        if (keys[i] == 0) ++used;
        keys[i] = k;
        vals[i] = v;
    }
};

// Scans of one block's search (same placed gates and start), memoised by
// qubit set: the completions of different candidates revisit the same sets.
struct AbsorbCache {
    const GateView& v;  // the unplaced gates after the block's first gate
    int start, kmax;
    SetMap counts, ext_at;                   // set -> absorbed gates / index into exts
    std::deque<std::vector<uint64_t>> exts;  // stable references while it grows
    int count(uint64_t S) {
        if (const int* c = counts.find(S)) return *c;
        const int c = absorb_scan(v, start, S, nullptr, nullptr, kmax);
        counts.put(S, c);
        return c;
    }
    const std::vector<uint64_t>& ext(uint64_t S) {
        if (const int* i = ext_at.find(S)) return exts[*i];
        std::vector<uint64_t> e;
        absorb_scan(v, start, S, nullptr, &e, kmax);
        std::sort(e.begin(), e.end());
        e.erase(std::unique(e.begin(), e.end()), e.end());
        ext_at.put(S, (int)exts.size());
        exts.push_back(std::move(e));
        return exts.back();
    }
    // the extension of S with the most absorbed gates (ties: fewer added qubits), 0 if none
    uint64_t greedy_step(uint64_t S) {
        uint64_t best = 0;
        int best_count = -1, best_bits = 64;
        for (uint64_t e : ext(S)) {
            const int c = count(S | e), bits = __builtin_popcountll(e);
            if (c > best_count || (c == best_count && bits < best_bits)) {
                best = e;
                best_count = c;
                best_bits = bits;
            }
        }
        return best;
    }
    // the extension whose greedy completion absorbs the most gates, among
    // the kLook extensions that absorb the most by themselves (bounds the
    // search where many gates are reachable, e.g. commuting diagonal layers)
    static constexpr size_t kLook = 16;
    uint64_t lookahead_step(uint64_t S) {
        std::vector<std::pair<int, uint64_t>> cand;
        for (uint64_t e : ext(S)) cand.emplace_back(-count(S | e), e);
        if (cand.size() > kLook) {
            std::stable_sort(cand.begin(), cand.end(),
                             [](const std::pair<int, uint64_t>& x, const std::pair<int, uint64_t>& y) {
                                 return x.first < y.first;
                             });
            cand.resize(kLook);
        }
        uint64_t best = 0;
        int best_count = -1, best_bits = 64;
        for (const auto& ce : cand) {
            const uint64_t e = ce.second;
            uint64_t T = S | e;
            while (__builtin_popcountll(T) < kmax) {
                const uint64_t nx = greedy_step(T);
                if (!nx) break;
                T |= nx;
            }
            const int c = count(T), bits = __builtin_popcountll(e);
            if (c > best_count || (c == best_count && bits < best_bits)) {
                best = e;
                best_count = c;
                best_bits = bits;
            }
        }
        return best;
    }
};

// Best-first block: start from the first unplaced gate's qubits and grow the
// set one reachable gate at a time.  Each candidate extension is scored by
// the gates absorbed once its set has been completed (the first further
// extension chosen with a one-level lookahead, the rest greedily: the
// extension with the most absorbed gates); ties: fewer added qubits.  Same
// validity rule as the plain scan (commuting past every skipped gate); on
// grid circuits it forms about half as many 6-qubit blocks as taking gates
// first come, first served.
static std::vector<int> best_first_group(const GateView& v, std::vector<char>& placed, int start, int kmax,
                                         int effort) {
    // the unplaced gates after start (at most 2^14 of them), in flat arrays
    GateView live;
    live.allq = v.allq;
    for (int j = start + 1; j < (int)v.m.size() && (int)live.m.size() < (1 << 14); ++j) {
        if (placed[j]) continue;
        live.m.push_back(v.m[j]);
        live.diag.push_back(v.diag[j]);
        live.ok.push_back(v.ok[j]);
        live.idx.push_back(j);
    }
    AbsorbCache cache{live, start, kmax, SetMap(4096), SetMap(1024), {}};
    uint64_t S = v.m[start];
    while (__builtin_popcountll(S) < kmax) {
        const std::vector<uint64_t> ext = cache.ext(S);
        if (ext.empty()) break;
        uint64_t best = 0;
        int best_count = -1, best_bits = 64;
        for (uint64_t e : ext) {
            uint64_t T = S | e;
            bool first = true;
            while (__builtin_popcountll(T) < kmax) {
                const uint64_t nx = first && effort ? cache.lookahead_step(T) : cache.greedy_step(T);
                first = false;
                if (!nx) break;
                T |= nx;
            }
            const int c = cache.count(T), bits = __builtin_popcountll(e);
            if (c > best_count || (c == best_count && bits < best_bits)) {
                best = e;
                best_count = c;
                best_bits = bits;
            }
        }
        S |= best;
    }
    std::vector<int> taken;
    absorb_scan(live, start, S, &taken, nullptr, kmax);
    for (int t : taken) placed[t] = 1;
    return taken;
}

// by_kind = false: any gates fuse while their qubits fit k_max.  by_kind =
// true: diagonal gates only with diagonal gates, in clusters of any width
// (bounded by what one wide pass holds), the others only with each other.
// What the grouping depends on: the gates' qubits and kinds, and the search
// (compared in full on a cache hit).
static std::vector<uint64_t> grouping_key(int n, const std::vector<GateRec>& in, int k_max, bool by_kind,
                                          int effort) {
    std::vector<uint64_t> key;
    key.reserve(in.size() * 2 + 1);
    key.push_back((uint64_t)n | ((uint64_t)k_max << 8) | ((uint64_t)by_kind << 16) | ((uint64_t)effort << 24));
    for (const GateRec& g : in) {
        uint64_t q = 0;
        for (int i = 0; i < g.k; ++i) q |= (uint64_t)(g.qubits[i] & 63) << (6 * i);  // ordered qubits
        key.push_back(q | ((uint64_t)g.k << 36) | ((uint64_t)g.kind << 40));
        key.push_back(g.wide_mask);
    }
    return key;
}

static void search_groups_each(int n, const std::vector<GateRec>& in, int k_max, bool by_kind, int effort,
                               const std::function<void(std::vector<int>&&)>& emit) {
    std::vector<char> placed(in.size(), 0);
    const int nchunks = (n + 7) / 8;
    GateView view;  // by kind, the dense blocks take non-diagonal gates only
    for (const GateRec& g : in) {
        view.m.push_back(qmask(g));
        view.diag.push_back(g.kind == QS_GATE_DIAGONAL);
        view.ok.push_back(!by_kind || g.kind != QS_GATE_DIAGONAL);
        view.allq |= view.m.back();
    }
    for (int start = 0; start < (int)in.size(); ++start) {
        if (placed[start]) continue;
        const bool diag = in[start].kind == QS_GATE_DIAGONAL;
        if (in[start].k > k_max && !(by_kind && diag)) {  // wider than the bound: kept as it is
            placed[start] = 1;
            emit({-1 - start});
            continue;
        }
        if (!by_kind) {
            emit(best_first_group(view, placed, start, k_max, effort));
        } else if (diag) {
            // capacity of one wide pass: cross-chunk gates and table entries
            size_t entries = 256 * (size_t)nchunks;
            int ncross = 0;
            auto fits = [&](const GateRec& g) {
                // spans a chunk boundary of the complex (8-bit) or exponent (10-bit) tables
                bool cross = false;
                for (int i = 1; i < g.k; ++i)
                    cross = cross || (g.qubits[i] >> 3) != (g.qubits[0] >> 3) || g.qubits[i] / 10 != g.qubits[0] / 10;
                if (!cross) return true;
                if (ncross + 1 > kWideDiagCross || entries + (1u << g.k) > kWideDiagTabElems) return false;
                ++ncross;
                entries += 1u << g.k;
                return true;
            };
            fits(in[start]);
            std::function<bool(const GateRec&)> accept = [&](const GateRec& g) {
                return g.kind == QS_GATE_DIAGONAL && fits(g);
            };
            emit(scan_group(in, placed, start, 0, 64, 1 << 14, kMaxK, &accept));
        } else {
            emit(best_first_group(view, placed, start, k_max, effort));
        }
    }
}

static std::vector<std::vector<int>> search_groups(int n, const std::vector<GateRec>& in, int k_max, bool by_kind,
                                                   int effort) {
    std::vector<std::vector<int>> groups;
    search_groups_each(n, in, k_max, by_kind, effort, [&](std::vector<int>&& g) { groups.push_back(std::move(g)); });
    return groups;
}

// The fused block of one group: the gate kept as it is (group {-1 - i}), a
// wide diagonal cluster (more than kMaxK qubits: its gates kept as parts), or
// the FP64 product of the group's gates on their qubits (descending order,
// qubits[0] the most significant local bit), classified.
void block_product(int n, const std::vector<GateRec>& in, const std::vector<int>& taken, GateRec& b) {
    if (taken[0] < 0) {
        b = in[-1 - taken[0]];
        b.param = -1;
        b.paulis[0] = 0;
        return;
    }
    uint64_t support = 0;
    for (int t : taken) support |= qmask(in[t]);
    if (__builtin_popcountll(support) > kMaxK) {  // a wide diagonal cluster: keep its gates
        b.k = 0;
        b.kind = QS_GATE_DIAGONAL;
        b.wide_mask = support;
        for (int t : taken) {
            b.parts.push_back(in[t]);
            b.parts.back().param = -1;
            b.parts.back().paulis[0] = 0;
        }
        return;
    }
    b.k = __builtin_popcountll(support);
    int bq[kMaxK];
    int j = 0;
    for (int q = n - 1; q >= 0; --q)
        if ((support >> q) & 1) bq[j++] = q;  // descending: qubits[0] most significant
    for (int i = 0; i < b.k; ++i) b.qubits[i] = bq[i];
    const int D = 1 << b.k;
    std::vector<double> accr((size_t)D * D, 0.0), acci((size_t)D * D, 0.0);
    for (int i = 0; i < D; ++i) accr[(size_t)i * D + i] = 1.0;
    // one-qubit gates that follow each other on a qubit (no member in between
    // touches it) are multiplied as 2 x 2 matrices first, then applied once
    GateRec one;  // the pending one-qubit product
    bool have = false;
    auto flush_one = [&]() {
        if (have) apply_into_block(one, b.k, bq, accr.data(), acci.data());
        have = false;
    };
    for (int t : taken) {
        const GateRec& g = in[t];
        if (g.k == 1 && have && g.qubits[0] == one.qubits[0]) {  // one <- g * one
            const double* x = g.m.data();
            double y[8];
            for (int r = 0; r < 2; ++r)
                for (int c2 = 0; c2 < 2; ++c2) {
                    const double ar = x[2 * (2 * r)], ai = x[2 * (2 * r) + 1], br = x[2 * (2 * r + 1)],
                                 bi = x[2 * (2 * r + 1) + 1];
                    const double pr = one.m[2 * c2], pi = one.m[2 * c2 + 1], qr = one.m[2 * (2 + c2)],
                                 qi = one.m[2 * (2 + c2) + 1];
                    y[2 * (2 * r + c2)] = (ar * pr - ai * pi) + (br * qr - bi * qi);
                    y[2 * (2 * r + c2) + 1] = (ar * pi + ai * pr) + (br * qi + bi * qr);
                }
            std::copy(y, y + 8, one.m.begin());
            one.kind = QS_GATE_DENSE;
            continue;
        }
        flush_one();
        if (g.k == 1) {
            one.k = 1;
            one.qubits[0] = g.qubits[0];
            one.m.assign(g.m.begin(), g.m.begin() + 8);
            one.kind = g.kind;
            have = true;
            continue;
        }
        apply_into_block(g, b.k, bq, accr.data(), acci.data());
    }
    flush_one();
    b.m.resize(2 * D * D);
    for (int i = 0; i < D * D; ++i) {
        b.m[2 * i] = accr[i];
        b.m[2 * i + 1] = acci[i];
    }
    b.kind = classify_matrix(b.k, b.m.data());
}

static qs_status fuse_impl(int n, const std::vector<GateRec>& in, int k_max, bool by_kind, std::vector<GateRec>& out,
                           int effort, FuseCache* cache) {
    if (k_max < 1 || k_max > kMaxK) return fail(QS_ERR_ARG, "k_max must be in 1..6");
    out.clear();
    // 1. the grouping: searched, or reused while qubits and kinds are unchanged
    std::vector<std::vector<int>> groups;
    bool hit = false;
    std::vector<uint64_t> key;
    if (cache) key = grouping_key(n, in, k_max, by_kind, effort);
    if (cache) {
        std::lock_guard<std::mutex> lk(cache->mu);
        if (cache->valid && cache->key == key) {
            groups = cache->groups;
            hit = true;
        }
    }
    if (!hit) {
        groups = search_groups(n, in, k_max, by_kind, effort);
        if (cache) {
            std::lock_guard<std::mutex> lk(cache->mu);
            cache->key = key;
            cache->groups = groups;
            cache->valid = true;
        }
    }
    // 2. the FP64 block products, independent per group: spread over host threads
    out.resize(groups.size());
    auto build = [&](size_t gi) { block_product(n, in, groups[gi], out[gi]); };
    size_t work = 0;
    for (const auto& g : groups) work += g.size();
    const unsigned nthreads = (unsigned)std::min<size_t>({(size_t)host_threads(16), groups.size(), work / 64 + 1});
    if (nthreads <= 1) {
        for (size_t gi = 0; gi < groups.size(); ++gi) build(gi);
    } else {
        std::atomic<size_t> next(0);
        std::vector<std::thread> pool;
        for (unsigned t = 0; t < nthreads; ++t)
            pool.emplace_back([&]() {
                for (size_t gi = next++; gi < groups.size(); gi = next++) build(gi);
            });
        for (auto& th : pool) th.join();
    }
    return QS_OK;
}

// fuse_gates in stream form: each group is handed to `emit` as soon as the
// block search finds it (or, on a grouping-cache hit, all at once).
qs_status fuse_each(int n, const std::vector<GateRec>& in, int k_max, int effort, FuseCache* cache,
                    const std::function<void(std::vector<int>&&)>& emit) {
    if (k_max < 1 || k_max > kMaxK) return fail(QS_ERR_ARG, "k_max must be in 1..6");
    std::vector<uint64_t> key;
    if (cache) key = grouping_key(n, in, k_max, false, effort);
    std::vector<std::vector<int>> groups;
    bool hit = false;
    if (cache) {
        std::lock_guard<std::mutex> lk(cache->mu);
        if (cache->valid && cache->key == key) {
            groups = cache->groups;
            hit = true;
        }
    }
    if (hit) {
        for (auto& g : groups) emit(std::move(g));
        return QS_OK;
    }
    search_groups_each(n, in, k_max, false, effort, [&](std::vector<int>&& g) {
        groups.push_back(g);
        emit(std::move(g));
    });
    if (cache) {
        std::lock_guard<std::mutex> lk(cache->mu);
        cache->key = std::move(key);
        cache->groups = std::move(groups);
        cache->valid = true;
    }
    return QS_OK;
}

qs_status fuse_gates(int n, const std::vector<GateRec>& in, int k_max, std::vector<GateRec>& out, int effort,
                     FuseCache* cache) {
    return fuse_impl(n, in, k_max, false, out, effort, cache);
}

qs_status fuse_by_kind(int n, const std::vector<GateRec>& in, int k_max, std::vector<GateRec>& out, int effort,
                       FuseCache* cache) {
    return fuse_impl(n, in, k_max, true, out, effort, cache);
}

// The phase tables of a wide diagonal cluster (FP64 on the host).
static void build_wide_diag(int n, const GateRec& w, Pass& p) {
    WideDiag& wd = p.wide;
    // exponent m with entry = exp(i pi m / 4), or -1
    auto root8 = [](double re, double im) {
        for (int m = 0; m < 8; ++m) {
            const double a = m * 0.78539816339744830962;
            if (fabs(re - cos(a)) < 1e-14 && fabs(im - sin(a)) < 1e-14) return m;
        }
        return -1;
    };
    bool r8 = true;
    for (const GateRec& g : w.parts) {
        const int d = 1 << g.k;
        for (int l = 0; l < d && r8; ++l) r8 = root8(g.m[2 * (l * d + l)], g.m[2 * (l * d + l) + 1]) >= 0;
    }
    wd.root8 = r8;
    const int cb = r8 ? 10 : 8, csz = 1 << cb;
    wd.chunk_bits = cb;
    const int nchunks = (n + cb - 1) / cb;
    wd.nchunks = nchunks;
    std::vector<cd> tab(csz * (size_t)nchunks, r8 ? cd(0.0) : cd(1.0)), cross;
    for (const GateRec& g : w.parts) {
        const int k = g.k, d = 1 << k;
        const int c0 = g.qubits[0] / cb;
        bool one = true;
        for (int i = 1; i < k; ++i) one = one && g.qubits[i] / cb == c0;
        auto entry = [&](int l) {
            const double re = g.m[2 * (l * d + l)], im = g.m[2 * (l * d + l) + 1];
            return r8 ? cd((double)root8(re, im), 0.0) : cd(re, im);
        };
        if (one) {
            for (int jj = 0; jj < csz; ++jj) {
                int l = 0;
                for (int i = 0; i < k; ++i) l = (l << 1) | ((jj >> (g.qubits[i] - cb * c0)) & 1);
                cd& t = tab[(size_t)csz * c0 + jj];
                if (r8) t = cd(fmod(t.real() + entry(l).real(), 8.0), 0.0);
                else t *= entry(l);
            }
        } else {
            DiagCross x{};
            x.k = (uint8_t)k;
            for (int i = 0; i < k; ++i) x.q[i] = (uint8_t)g.qubits[i];
            x.tab = (uint32_t)((size_t)csz * nchunks + cross.size());
            for (int l = 0; l < d; ++l) cross.push_back(entry(l));
            wd.cross.push_back(x);
        }
    }
    tab.insert(tab.end(), cross.begin(), cross.end());
    wd.tab_elems = (uint32_t)tab.size();
    p.mats.clear();
    for (const cd& z : tab) {
        p.mats.push_back(z.real());
        p.mats.push_back(z.imag());
    }
    p.k = __builtin_popcountll(w.wide_mask);
    p.members = (int)w.parts.size();
}

void factor_tile_scalars(Pass& p) {
    if (p.kind != PASS_TILE) return;
    cd total = 1.0;
    bool any = false;
    for (TileGate& tg : p.tgates) {
        if (tg.k != 1 || tg.kind == QS_GATE_DIAGONAL) continue;
        const double* m = p.mats.data() + 2 * (size_t)tg.mat;
        cd e[4], c = 0.0;
        for (int i = 0; i < 4; ++i) {
            e[i] = cd(m[2 * i], m[2 * i + 1]);
            if (c == 0.0 && std::abs(e[i]) > 0) c = e[i];
        }
        bool ok = true;
        cd u[4];
        for (int i = 0; i < 4 && ok; ++i) {
            u[i] = e[i] / c;
            const cd cand[5] = {0.0, 1.0, cd(0, 1), -1.0, cd(0, -1)};
            bool hit = false;
            for (const cd& z : cand)
                if (std::abs(u[i] - z) < 1e-14) {
                    u[i] = z;
                    hit = true;
                }
            ok = hit;
        }
        if (!ok) continue;
        double* w = p.mats.data() + 2 * (size_t)tg.mat;
        for (int i = 0; i < 4; ++i) {
            w[2 * i] = u[i].real();
            w[2 * i + 1] = u[i].imag();
        }
        tg.kind = kTileMulfree;
        total *= c;
        any = true;
    }
    if (!any) return;
    const double mag = std::abs(total);
    const cd ph = total / mag;
    for (int s = 0; s < 8; ++s) {
        const double a = s * 0.78539816339744830962;
        if (std::abs(ph - cd(cos(a), sin(a))) < 1e-13) {
            p.scale_mode = 1;
            p.scale_s = s;
            p.scale_mag = mag;
            return;
        }
    }
    p.scale_mode = 2;
    p.scale_c[0] = total.real();
    p.scale_c[1] = total.imag();
}

// Widen a 5-qubit dense pass to 6 qubits: an identity on the highest unused
// qubit, placed first (most significant), so the matrix is kron(I2, M).
static void pad_to_six(int n, Pass& p) {
    uint64_t used = 0;
    for (int i = 0; i < p.k; ++i) used |= 1ull << p.qubits[i];
    // the highest unused qubit: it leaves the low, contiguous index bits to
    // the sets (and qubit 0 out of the targets when the block leaves it out)
    int extra = n - 1;
    while (extra > 0 && ((used >> extra) & 1)) --extra;
    const int d = 1 << p.k, D = 2 * d;
    std::vector<double> m(2 * D * D, 0.0);
    for (int b = 0; b < 2; ++b)
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) {
                m[2 * ((b * d + r) * D + b * d + c)] = p.mats[2 * (r * d + c)];
                m[2 * ((b * d + r) * D + b * d + c) + 1] = p.mats[2 * (r * d + c) + 1];
            }
    for (int i = p.k; i > 0; --i) p.qubits[i] = p.qubits[i - 1];
    p.qubits[0] = extra;
    p.k += 1;
    p.mats.swap(m);
}

// Reorder a pass's qubit list to descending order (local bit b = b-th lowest
// qubit), permuting the matrix's rows and columns to match.
static void sort_qubits_descending(Pass& p) {
    const int k = p.k, d = 1 << k;
    int order[kMaxK];  // new position i takes old position order[i]
    for (int i = 0; i < k; ++i) order[i] = i;
    std::sort(order, order + k, [&](int x, int y) { return p.qubits[x] > p.qubits[y]; });
    int old_index[1 << kMaxK];  // new local index -> old
    for (int ln = 0; ln < d; ++ln) {
        int lo = 0;
        for (int i = 0; i < k; ++i)
            if ((ln >> (k - 1 - i)) & 1) lo |= 1 << (k - 1 - order[i]);
        old_index[ln] = lo;
    }
    std::vector<double> m(p.mats.size());
    for (int r = 0; r < d; ++r) {
        const double* src = p.mats.data() + 2 * (size_t)old_index[r] * d;
        double* dst = m.data() + 2 * (size_t)r * d;
        for (int c = 0; c < d; ++c) {
            dst[2 * c] = src[2 * old_index[c]];
            dst[2 * c + 1] = src[2 * old_index[c] + 1];
        }
    }
    int q[kMaxK];
    for (int i = 0; i < k; ++i) q[i] = p.qubits[order[i]];
    for (int i = 0; i < k; ++i) p.qubits[i] = q[i];
    p.mats.swap(m);
}

int auto_tile_qubits(int n, qs_dtype dt) {
    const int L = dt == QS_C64 ? 12 : 11;
    return std::min(L, n);
}

std::vector<std::vector<int>> group_for_tiles(const std::vector<GateRec>& units, int L, int low_bits_in_tile,
                                              size_t mat_budget) {
    const uint64_t lowmask = (1ull << low_bits_in_tile) - 1;
    std::vector<std::vector<int>> groups;
    std::vector<char> placed(units.size(), 0);
    for (int start = 0; start < (int)units.size(); ++start) {
        if (placed[start]) continue;
        std::vector<char> trial = placed;
        std::vector<int> taken = scan_group(units, trial, start, lowmask, L, 1 << 14, 4);
        size_t elems = 0, keep = 0;
        for (; keep < taken.size() && (int)keep < kMaxTileGates; ++keep) {
            const size_t d = 1u << units[taken[keep]].k;
            if (elems + d * d > mat_budget) break;
            elems += d * d;
        }
        taken.resize(std::max<size_t>(keep, 1));
        for (int t : taken) placed[t] = 1;
        groups.push_back(taken);
    }
    return groups;
}

static int low_bits(qs_dtype dt) { return dt == QS_C64 ? 5 : 4; }

// largest non-diagonal gate the tile kernel applies (register path), and
// the complex matrix entries one tile pass may stage in shared memory
constexpr int kTileDenseK = 4;
constexpr size_t kTileMatElems = 3072;

void single_block_pass(int n, qs_dtype dt, const qs_options& opt, const GateRec& g, Pass& p) {
    const bool tensor = dt == QS_C64 && opt.precision != QS_PREC_FP32 && gemm_supported(n, 6);
    if (g.k == 0) {
        p.kind = PASS_DIAG_WIDE;
        build_wide_diag(n, g, p);
        return;
    }
    p.k = g.k;
    for (int i = 0; i < g.k; ++i) p.qubits[i] = g.qubits[i];
    p.gate_kind = g.kind;
    p.mats = g.m;
    if (g.kind == QS_GATE_DIAGONAL) p.kind = PASS_DIAG;
    else if (g.kind == QS_GATE_MONOMIAL) p.kind = PASS_MONO;
    else if (g.k <= 3 || (g.k == 4 && !tensor)) p.kind = PASS_DENSE;
    else if (tensor) {
        // the tensor-core pass is 6-qubit only; a 4-qubit block is also
        // cheaper there than on the FP32 CUDA cores (64 FMA per amplitude)
        p.kind = PASS_GEMM;
        while (p.k < 6) pad_to_six(n, p);
        sort_qubits_descending(p);
    } else p.kind = PASS_DENSE_SMEM;
}

// Qubits a pass reads or writes (a superset for wide diagonal passes).
static uint64_t pass_support(int n, const Pass& p) {
    uint64_t m = 0;
    switch (p.kind) {
        case PASS_TILE:
            for (const TileGate& g : p.tgates)
                for (int i = 0; i < g.k; ++i) m |= 1ull << p.pos[g.q[i]];
            return m;
        case PASS_DIAG_WIDE: return n >= 64 ? ~0ull : (1ull << n) - 1;
        case PASS_TTILE:
            for (int i = 0; i < 12; ++i) m |= 1ull << p.tt.s[i];
            return m;
        default:
            for (int i = 0; i < p.k; ++i) m |= 1ull << p.qubits[i];
            return m;
    }
}

static int gf2_rank3(const uint8_t* v, int cnt) {  // rank of cnt vectors in GF(2)^3
    uint8_t basis[3] = {0, 0, 0};
    int rank = 0;
    for (int i = 0; i < cnt; ++i) {
        uint8_t x = v[i];
        for (int b = 2; b >= 0; --b) {
            if (!((x >> b) & 1)) continue;
            if (basis[b]) x ^= basis[b];
            else {
                basis[b] = x;
                ++rank;
                break;
            }
        }
    }
    return rank;
}

// Shared-memory positions of the 12 tile bits for a tensor tile pass (see
// the kernel): bit 0 keeps position bit 0; position bits 1-3 (the bank
// group of an 8-byte access, with bit 0) are a linear map col3 of tile bits
// 1..11, searched so that for every block the 4 lowest row bits R_b land in
// distinct bank groups (rank 3 on R_b \ {0}; rank 3 on R_b when the block
// targets bit 0, whose rows then share bank groups in pairs); the remaining
// 8 tile bits also get position bits 4-11 in order, which makes the map
// bijective.
static void choose_tile_positions(TTileDesc& d) {
    int R[kTTileMaxBlocks][4];
    bool has0[kTTileMaxBlocks];
    for (int b = 0; b < d.nb; ++b) {
        uint32_t used = 0;
        for (int i = 0; i < 6; ++i) used |= 1u << d.kbit[b][i];
        int c = 0;
        for (int t = 0; t < 12 && c < 4; ++t)
            if (!((used >> t) & 1)) R[b][c++] = t;
        has0[b] = !(used & 1u);
    }
    auto score = [&](const uint8_t* col3) {
        int ok = 0;
        for (int b = 0; b < d.nb; ++b) {
            uint8_t v[4];
            int cnt = 0;
            for (int i = 0; i < 4; ++i)
                if (R[b][i] != 0) v[cnt++] = col3[R[b][i]];
            ok += gf2_rank3(v, cnt) == 3;
        }
        return ok;
    };
    uint8_t best[12] = {0}, cur[12] = {0};
    int best_score = -1;
    uint64_t x = 0x9E3779B97F4A7C15ull;  // fixed-seed generator: the same plan every time
    for (int trial = 0; trial < 4096 && best_score < d.nb; ++trial) {
        for (int t = 1; t < 12; ++t) {
            x ^= x << 13;
            x ^= x >> 7;
            x ^= x << 17;
            cur[t] = (uint8_t)(x & 7);
        }
        if (trial == 0)  // first try: the plain identity on tile bits 1..3
            for (int t = 1; t < 12; ++t) cur[t] = t <= 3 ? (uint8_t)(1 << (t - 1)) : 0;
        const int sc = score(cur);
        if (sc > best_score) {
            best_score = sc;
            std::copy(cur, cur + 12, best);
        }
    }
    // three tile bits (not 0) whose col3 values are independent
    int P[3] = {-1, -1, -1};
    for (int a1 = 1; a1 < 12 && P[0] < 0; ++a1)
        for (int a2 = a1 + 1; a2 < 12 && P[0] < 0; ++a2)
            for (int a3 = a2 + 1; a3 < 12 && P[0] < 0; ++a3) {
                const uint8_t v[3] = {best[a1], best[a2], best[a3]};
                if (gf2_rank3(v, 3) == 3) {
                    P[0] = a1;
                    P[1] = a2;
                    P[2] = a3;
                }
            }
    if (P[0] < 0) {  // no independent triple: fall back to the identity on bits 1..3
        for (int t = 1; t < 12; ++t) best[t] = t <= 3 ? (uint8_t)(1 << (t - 1)) : 0;
        P[0] = 1;
        P[1] = 2;
        P[2] = 3;
    }
    d.poscol[0] = 1;
    int rank = 0;
    for (int t = 1; t < 12; ++t) {
        const bool inP = t == P[0] || t == P[1] || t == P[2];
        d.poscol[t] = (uint16_t)((best[t] << 1) | (inP ? 0 : (1u << (4 + rank++))));
    }
}

// Group 6-qubit tensor-core passes into tensor tile passes: a pass joins the
// group when it commutes with every pass it moves ahead of (disjoint
// qubits) and the group's qubits together with bits 0 and 1 stay within 12;
// among the candidates the one adding the fewest qubits is taken, up to
// kTTileMaxBlocks blocks.  Members keep their circuit order.
static void group_tensor_tiles(int n, std::vector<Pass>& passes) {
    const int P = (int)passes.size();
    std::vector<uint64_t> supp(P);
    for (int i = 0; i < P; ++i) supp[i] = pass_support(n, passes[i]);
    std::vector<char> placed(P, 0);
    std::vector<Pass> out;
    for (int a = 0; a < P; ++a) {
        if (placed[a]) continue;
        placed[a] = 1;
        if (passes[a].kind != PASS_GEMM) {
            out.push_back(std::move(passes[a]));
            continue;
        }
        std::vector<int> members{a};
        uint64_t cur = supp[a] | 3ull;
        while ((int)members.size() < kTTileMaxBlocks) {
            int best = -1, best_size = 13;
            // every unplaced pass between the group's start and a candidate
            // stays after the group, so the candidate must commute with it
            uint64_t blocked = 0;
            for (int b = a + 1; b < P; ++b) {
                if (placed[b]) continue;
                if (b > members.back() && passes[b].kind == PASS_GEMM && !(supp[b] & blocked)) {
                    const int sz = __builtin_popcountll(cur | supp[b]);
                    if (sz <= 12 && sz < best_size) {
                        best = b;
                        best_size = sz;
                    }
                }
                blocked |= supp[b];
            }
            if (best < 0) break;
            members.push_back(best);
            placed[best] = 1;
            cur |= supp[best];
        }
        if (members.size() == 1) {
            out.push_back(std::move(passes[a]));
            continue;
        }
        Pass t;
        t.kind = PASS_TTILE;
        uint64_t S = cur;
        for (int q = 0; q < n && __builtin_popcountll(S) < 12; ++q) S |= 1ull << q;
        int tile_of[kMaxQubits];
        int j = 0;
        for (int q = 0; q < n; ++q)
            if ((S >> q) & 1) {
                tile_of[q] = j;
                t.tt.s[j++] = q;
            }
        t.tt.nb = (int)members.size();
        t.members = 0;
        for (int b = 0; b < t.tt.nb; ++b) {
            const Pass& m = passes[members[b]];
            for (int i = 0; i < 6; ++i) t.tt.kbit[b][5 - i] = tile_of[m.qubits[i]];
            t.mats.insert(t.mats.end(), m.mats.begin(), m.mats.end());
            t.members += m.members;
        }
        choose_tile_positions(t.tt);
        out.push_back(std::move(t));
    }
    passes.swap(out);
}

// Register tile program of a tile pass (see the kernel): lanes hold tile
// bits 0..4 when the tile is loaded and stored; a gate whose qubits are not
// where its op needs them gets a new layout first (its qubits on register
// bits 0..k-1, the other register bits filled with the tile bits used
// soonest by later gates).  The shared-memory positions of the transposes
// are a linear map of the tile bits whose bank-group part is searched so that
// every layout's lane bits hit all bank groups.
bool build_rtile_program(qs_dtype dt, const Pass& p, RTProgram& prog) {
    const int L = rtile_bits(dt), RB = L - 8;
    if (p.kind != PASS_TILE || p.L != L) return false;
    for (const TileGate& g : p.tgates)
        if (g.kind != QS_GATE_DIAGONAL && g.k > RB) return false;
    prog = RTProgram{};
    const int G = (int)p.tgates.size();
    auto next_use = [&](int from, int bit) {
        for (int i = from; i < G; ++i) {
            const TileGate& g = p.tgates[i];
            if (g.kind == QS_GATE_DIAGONAL) continue;
            for (int j = 0; j < g.k; ++j)
                if (g.q[j] == bit) return i;
        }
        return G + 1;
    };
    struct Lay {
        int lane[5], reg[4], warp[3];
    };
    std::vector<Lay> lays;
    auto finish = [&](Lay& l) {  // warps: the tile bits on neither lanes nor registers
        uint32_t used = 0;
        for (int i = 0; i < 5; ++i) used |= 1u << l.lane[i];
        for (int i = 0; i < RB; ++i) used |= 1u << l.reg[i];
        int w = 0;
        for (int b = 0; b < L; ++b)
            if (!((used >> b) & 1)) {
                if (w >= 3) return false;
                l.warp[w++] = b;
            }
        for (int i = RB; i < 4; ++i) l.reg[i] = 0;
        return w == 3;
    };
    auto index_of = [&](const Lay& l) {
        for (size_t i = 0; i < lays.size(); ++i) {
            bool eq = true;
            for (int j = 0; j < 5; ++j) eq &= lays[i].lane[j] == l.lane[j];
            for (int j = 0; j < RB; ++j) eq &= lays[i].reg[j] == l.reg[j];
            if (eq) return (int)i;
        }
        if ((int)lays.size() >= kRTMaxLayouts) return -1;
        lays.push_back(l);
        return (int)lays.size() - 1;
    };
    auto find = [](const int* arr, int cnt, int v) {
        for (int i = 0; i < cnt; ++i)
            if (arr[i] == v) return i;
        return -1;
    };
    std::vector<RTOp> ops;
    // initial layout: lanes 0..4, registers the RB high bits used soonest
    Lay cur{};
    for (int i = 0; i < 5; ++i) cur.lane[i] = i;
    {
        std::vector<int> high;
        for (int b = 5; b < L; ++b) high.push_back(b);
        std::stable_sort(high.begin(), high.end(), [&](int x, int y) { return next_use(0, x) < next_use(0, y); });
        for (int i = 0; i < RB; ++i) cur.reg[i] = high[i];
        if (!finish(cur)) return false;
    }
    int curi = index_of(cur);
    prog.load_lay = curi;
    auto move_to = [&](Lay& nl) {
        if (!finish(nl)) return false;
        const int idx = index_of(nl);
        if (idx < 0) return false;
        RTOp op{};
        op.type = RT_LAYOUT;
        op.arg = (uint8_t)idx;
        ops.push_back(op);
        cur = nl;
        curi = idx;
        return true;
    };
    for (int gi = 0; gi < G; ++gi) {
        const TileGate& g = p.tgates[gi];
        RTOp op{};
        op.k = g.k;
        op.mat = g.mat;
        for (int i = 0; i < g.k; ++i) op.q[i] = g.q[i];
        op.mulfree = g.kind == kTileMulfree ? 1 : 0;
        if (g.kind == QS_GATE_DIAGONAL) {
            op.type = RT_DIAG;
            ops.push_back(op);
            continue;
        }
        if (g.k == 1) {
            const int q = g.q[0];
            int r = find(cur.reg, RB, q);
            if (r >= 0) {
                op.type = RT_GATE1;
                op.arg = (uint8_t)r;
                ops.push_back(op);
                continue;
            }
            const int ln = find(cur.lane, 5, q);
            if (ln >= 0) {
                op.type = RT_LANE1;
                op.arg = (uint8_t)ln;
                ops.push_back(op);
                continue;
            }
            // a warp bit: it replaces the register bit used latest
            int worst = 0;
            for (int i = 1; i < RB; ++i)
                if (next_use(gi + 1, cur.reg[i]) > next_use(gi + 1, cur.reg[worst])) worst = i;
            Lay nl = cur;
            nl.reg[worst] = q;
            if (!move_to(nl)) return false;
            op.type = RT_GATE1;
            op.arg = (uint8_t)worst;
            ops.push_back(op);
            continue;
        }
        bool in_place = true;  // local bit i = q[k-1-i] on register bit i
        for (int i = 0; i < g.k; ++i) in_place &= cur.reg[i] == g.q[g.k - 1 - i];
        if (!in_place) {
            Lay nl{};
            uint32_t taken = 0;
            for (int i = 0; i < g.k; ++i) {
                nl.reg[i] = g.q[g.k - 1 - i];
                taken |= 1u << nl.reg[i];
            }
            // fill the other register bits: current registers, then warps, used soonest first
            std::vector<int> cand;
            for (int i = 0; i < RB; ++i)
                if (!((taken >> cur.reg[i]) & 1)) cand.push_back(cur.reg[i]);
            std::stable_sort(cand.begin(), cand.end(), [&](int x, int y) { return next_use(gi + 1, x) < next_use(gi + 1, y); });
            std::vector<int> cw;
            for (int i = 0; i < 3; ++i)
                if (!((taken >> cur.warp[i]) & 1)) cw.push_back(cur.warp[i]);
            std::stable_sort(cw.begin(), cw.end(), [&](int x, int y) { return next_use(gi + 1, x) < next_use(gi + 1, y); });
            cand.insert(cand.end(), cw.begin(), cw.end());
            int fill = g.k;
            for (int b : cand)
                if (fill < RB) {
                    nl.reg[fill++] = b;
                    taken |= 1u << b;
                }
            if (fill < RB) return false;
            // lanes: the current lanes, a lane bit now in the registers replaced
            // by the lowest tile bit that is free
            for (int i = 0; i < 5; ++i) {
                int b = cur.lane[i];
                if ((taken >> b) & 1) {
                    b = -1;
                    for (int c = 0; c < L && b < 0; ++c) {
                        bool on_lane = false;
                        for (int j = 0; j < 5; ++j) on_lane |= (j < i ? nl.lane[j] : cur.lane[j]) == c;
                        if (!((taken >> c) & 1) && !on_lane) b = c;
                    }
                    if (b < 0) return false;
                }
                nl.lane[i] = b;
                taken |= 1u << b;
            }
            if (!move_to(nl)) return false;
        }
        op.type = RT_GATE;
        ops.push_back(op);
    }
    // the store layout: lanes back on tile bits 0..4
    bool natural = true;
    for (int i = 0; i < 5; ++i) natural &= cur.lane[i] == i;
    if (!natural) {
        Lay nl{};
        uint32_t taken = 0x1Fu;
        for (int i = 0; i < 5; ++i) nl.lane[i] = i;
        int fill = 0;
        for (int i = 0; i < RB; ++i)
            if (cur.reg[i] >= 5) {
                nl.reg[fill++] = cur.reg[i];
                taken |= 1u << cur.reg[i];
            }
        for (int b = 5; b < L && fill < RB; ++b)
            if (!((taken >> b) & 1)) {
                nl.reg[fill++] = b;
                taken |= 1u << b;
            }
        if (!move_to(nl)) return false;
    }
    prog.store_lay = curi;
    if ((int)ops.size() > kRTMaxOps) return false;
    prog.nops = (int)ops.size();
    for (int i = 0; i < prog.nops; ++i) prog.ops[i] = ops[i];
    prog.nlay = (int)lays.size();
    for (int i = 0; i < prog.nlay; ++i) {
        for (int j = 0; j < 5; ++j) prog.lay[i].lane[j] = (uint8_t)lays[i].lane[j];
        for (int j = 0; j < 4; ++j) prog.lay[i].reg[j] = (uint8_t)lays[i].reg[j];
        for (int j = 0; j < 3; ++j) prog.lay[i].warp[j] = (uint8_t)lays[i].warp[j];
    }
    // positions: bank-group bits (nb = 4 for 8-byte, 3 for 16-byte elements)
    // a linear map of the tile bits with full rank on every layout's lanes
    const int nb = dt == QS_C64 ? 4 : 3;
    auto rank_of = [&](const uint8_t* col, const int* bits, int cnt) {
        uint8_t basis[4] = {0, 0, 0, 0};
        int rank = 0;
        for (int i = 0; i < cnt; ++i) {
            uint8_t x = col[bits[i]];
            for (int b = nb - 1; b >= 0 && x; --b) {
                if (!((x >> b) & 1)) continue;
                if (basis[b]) x ^= basis[b];
                else {
                    basis[b] = x;
                    ++rank;
                    x = 0;
                }
            }
        }
        return rank;
    };
    uint8_t best[12] = {0}, col[12] = {0};
    int best_ok = -1;
    uint64_t x = 0x2545F4914F6CDD1Dull;  // fixed-seed generator: the same plan every time
    for (int trial = 0; trial < 4096 && best_ok < (int)lays.size(); ++trial) {
        for (int b = 0; b < L; ++b) {
            if (trial == 0) col[b] = b < nb ? (uint8_t)(1u << b) : 0;   // first try: the identity on bits 0..nb-1
            else {
                x ^= x << 13;
                x ^= x >> 7;
                x ^= x << 17;
                col[b] = (uint8_t)(x & ((1u << nb) - 1));
            }
        }
        int ok = 0;
        for (const Lay& l : lays) ok += rank_of(col, l.lane, 5) == nb;
        if (ok > best_ok) {
            best_ok = ok;
            std::copy(col, col + L, best);
        }
    }
    int P[4] = {-1, -1, -1, -1};  // nb tile bits on which the map is invertible
    {
        std::vector<int> chosen;
        for (int b = 0; b < L && (int)chosen.size() < nb; ++b) {
            chosen.push_back(b);
            if (rank_of(best, chosen.data(), (int)chosen.size()) < (int)chosen.size()) chosen.pop_back();
        }
        if ((int)chosen.size() < nb) {  // no full rank: the identity on bits 0..nb-1
            for (int b = 0; b < L; ++b) best[b] = b < nb ? (uint8_t)(1u << b) : 0;
            chosen.clear();
            for (int b = 0; b < nb; ++b) chosen.push_back(b);
        }
        for (int i = 0; i < nb; ++i) P[i] = chosen[i];
    }
    int hi = 0;
    for (int b = 0; b < L; ++b) {
        const bool inP = find(P, nb, b) >= 0;
        prog.poscol[b] = (uint16_t)(best[b] | (inP ? 0u : 1u << (nb + hi++)));
    }
    return true;
}

// The dynamic program of the bit-0 placement over a run of 6-qubit passes
// (described below), from state s0 (-1 standard order, else the bit that
// qubit 0's index bit is exchanged with); end_free: the run may end in any
// state.  choice[k]: -2 keep, -1 restore, else the new exchange bit.
// Returns the number of passes left with bit 0 a target, or -1 if the run
// cannot end in standard order.
int bit0_plan(int n, const std::vector<const Pass*>& run, int s0, bool end_free, std::vector<int>& choice) {
    const int K = (int)run.size(), S = n + 1;   // state index s + 1; s = -1: standard order
    auto phys = [](int s, int x) { return s < 0 ? x : x == 0 ? s : x == s ? 0 : x; };
    std::vector<uint64_t> T(K, 0);
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < run[k]->k; ++i) T[k] |= 1ull << run[k]->qubits[i];
    auto ptargets = [&](int k, int s) {
        uint64_t m = 0;
        for (int x = 0; x < n; ++x)
            if ((T[k] >> x) & 1) m |= 1ull << phys(s, x);
        return m;
    };
    auto candidates = [&](uint64_t pt, int* c) {  // non-target bits of rank 1..3
        int rank = 0, cnt = 0;
        for (int b = 0; b < n && rank <= 3; ++b) {
            if ((pt >> b) & 1) continue;
            if (rank >= 1) c[cnt++] = b;
            ++rank;
        }
        return cnt;
    };
    const int INF = 1 << 28;
    std::vector<int> cost((size_t)(K + 1) * S, INF), ch((size_t)K * S, -2);  // -2 keep, -1 back, else new a
    for (int idx = 0; idx < S; ++idx)
        if (end_free || idx == 0) cost[(size_t)K * S + idx] = 0;
    for (int k = K - 1; k >= 0; --k)
        for (int idx = 0; idx < S; ++idx) {
            const int s = idx - 1;
            if (s == 0) continue;
            const uint64_t pt = ptargets(k, s);
            const int q0t = (int)(pt & 1);
            int best = std::min(INF, q0t + cost[(size_t)(k + 1) * S + idx]), bc = -2;
            if (!q0t) {
                int c[3];
                const int cnt = candidates(pt, c);
                for (int i = 0; i < cnt; ++i) {
                    if (s < 0) {
                        const int v = cost[(size_t)(k + 1) * S + c[i] + 1];
                        if (v < best) {
                            best = v;
                            bc = c[i];
                        }
                    } else if (c[i] == s) {
                        const int v = cost[(size_t)(k + 1) * S];
                        if (v < best) {
                            best = v;
                            bc = -1;
                        }
                    }
                }
            }
            cost[(size_t)k * S + idx] = best;
            ch[(size_t)k * S + idx] = bc;
        }
    const int total = cost[(size_t)s0 + 1];
    choice.assign(K, -2);
    int s = s0;
    for (int k = 0; k < K && total < INF; ++k) {
        const int bc = ch[(size_t)k * S + s + 1];
        choice[k] = bc;
        s = bc == -2 ? s : bc == -1 ? -1 : bc;
    }
    return total < INF ? total : -1;
}

int bit0_apply(Pass& p, int s, int bc) {
    auto phys = [](int s, int x) { return s < 0 ? x : x == 0 ? s : x == s ? 0 : x; };
    for (int i = 0; i < p.k; ++i) p.qubits[i] = phys(s, p.qubits[i]);
    sort_qubits_descending(p);
    if (bc == -2) {
        p.swap_p = -1;
        return s;
    }
    if (bc == -1) {
        p.swap_p = s;
        return -1;
    }
    p.swap_p = bc;
    return bc;
}

// Qubit 0 out of the targets of 6-qubit tensor-core passes: a reordering of
// index bits, the GPU form of the paper's bit-permuting recursive transform
// (Section 5.1), folded into passes that run anyway.  A pass whose targets
// leave bit 0 free may write its tile with bit 0 exchanged with one of its
// next three lowest non-target bits (the tile maps onto itself and the
// stores stay coalesced), so the state is then stored with two qubits'
// index bits exchanged.  Over each run of consecutive 6-qubit passes a
// dynamic program over the states {standard order} and {qubits 0 and a
// exchanged} (bit0_plan) picks the exchanges that leave the fewest passes
// with bit 0 among their physical targets (those passes gather 16-byte
// pairs along bit 0, the slower form), starting and ending the run in
// standard order.  Each pass's qubits become physical bits (its matrix
// reordered to match).
static void place_bit0_run(int n, std::vector<Pass>& passes, size_t i0, size_t i1) {
    std::vector<const Pass*> run;
    for (size_t i = i0; i < i1; ++i) run.push_back(&passes[i]);
    std::vector<int> choice;
    if (bit0_plan(n, run, -1, false, choice) < 0) return;   // cannot happen: keeping standard order is feasible
    int s = -1;
    for (size_t i = i0; i < i1; ++i) s = bit0_apply(passes[i], s, choice[i - i0]);
}

static void place_bit0(int n, std::vector<Pass>& passes) {
    size_t i = 0;
    while (i < passes.size()) {
        if (passes[i].kind != PASS_GEMM) {
            ++i;
            continue;
        }
        size_t j = i;
        while (j < passes.size() && passes[j].kind == PASS_GEMM) ++j;
        if (j - i >= 2) place_bit0_run(n, passes, i, j);
        i = j;
    }
}

qs_status build_passes(int n, qs_dtype dt, const std::vector<GateRec>& blocks,
                       const qs_options& opt, std::vector<Pass>& passes) {
    passes.clear();
    const int L = opt.tile_qubits > 0 ? std::min(opt.tile_qubits, n) : auto_tile_qubits(n, dt);
    const int b = std::min(low_bits(dt), L);
    const uint64_t lowmask = (b >= 64) ? ~0ull : ((1ull << b) - 1);
    std::vector<char> placed(blocks.size(), 0);
    for (int start = 0; start < (int)blocks.size(); ++start) {
        if (placed[start]) continue;
        std::vector<int> taken;
        const bool start_ok = blocks[start].k > 0 &&
                              (blocks[start].kind == QS_GATE_DIAGONAL || blocks[start].k <= kTileDenseK);
        if (opt.use_tile && start_ok && blocks[start].k <= L && (int)blocks.size() > 1) {
            std::vector<char> trial = placed;
            std::function<bool(const GateRec&)> not_wide = [](const GateRec& g) { return g.k > 0; };
            taken = scan_group(blocks, trial, start, lowmask, L, 1 << 14, kTileDenseK, &not_wide);
            // keep a prefix within the gate-count and shared-matrix budgets
            // (members are in circuit order, so any prefix is a valid group)
            size_t elems = 0, keep = 0;
            for (; keep < taken.size() && (int)keep < kMaxTileGates; ++keep) {
                const size_t d = 1u << blocks[taken[keep]].k;
                if (elems + d * d > kTileMatElems) break;
                elems += d * d;
            }
            taken.resize(std::max<size_t>(keep, 1));
            for (int t : taken) placed[t] = 1;
        } else {
            taken.push_back(start);
            placed[start] = 1;
        }
        Pass p;
        if (taken.size() == 1) {
            single_block_pass(n, dt, opt, blocks[taken[0]], p);
        } else {
            p.kind = PASS_TILE;
            uint64_t S = lowmask;
            for (int t : taken)
                for (int i = 0; i < blocks[t].k; ++i) S |= 1ull << blocks[t].qubits[i];
            // fill the tile up to L qubits with the lowest unused bits so
            // the rows stay long (coalesced) -- extra bits cost nothing
            for (int q = 0; q < n && __builtin_popcountll(S) < L; ++q) S |= 1ull << q;
            int local_of[kMaxQubits];
            int j = 0;
            for (int q = 0; q < n; ++q)
                if ((S >> q) & 1) {
                    local_of[q] = j;
                    p.pos[j++] = q;
                }
            p.L = j;
            for (int t : taken) {
                const GateRec& g = blocks[t];
                TileGate tg{};
                tg.k = (uint8_t)g.k;
                tg.kind = (uint8_t)g.kind;
                for (int i = 0; i < g.k; ++i) tg.q[i] = (uint8_t)local_of[g.qubits[i]];
                tg.mat = (uint32_t)(p.mats.size() / 2);
                p.mats.insert(p.mats.end(), g.m.begin(), g.m.end());
                p.tgates.push_back(tg);
            }
        }
        passes.push_back(std::move(p));
    }
    // 3xFP16 on the tensor cores: several 6-qubit blocks per HBM round trip
    if (opt.tensor_tiles && dt == QS_C64 && opt.precision == QS_PREC_3XFP16 && ttile_supported(n))
        group_tensor_tiles(n, passes);
    place_bit0(n, passes);
    return QS_OK;
}

}  // namespace qsgb
