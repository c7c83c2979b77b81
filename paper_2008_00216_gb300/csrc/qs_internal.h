// Internal declarations of the GB300 state-vector library (not part of the
// C ABI).  Host objects, plan passes and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qsgb.h"

namespace qsgb {

constexpr int kMaxQubits = 36;
constexpr int kMaxK = 6;            // largest gate / fused block
constexpr int kMaxTileGates = 96;   // gates per shared-memory tile pass

// ----------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
qs_status fail(qs_status st, const char* fmt, ...);
qs_status cuda_fail(cudaError_t e, const char* what);
#define QS_CUDA(call)                                                          \
    do {                                                                       \
        cudaError_t _e = (call);                                               \
        if (_e != cudaSuccess) return ::qsgb::cuda_fail(_e, #call);            \
    } while (0)

// ----------------------------------------------------------------- gates
struct GateRec {
    int k = 0;
    int qubits[kMaxK] = {0};
    std::vector<double> m;          // 2 * 4^k doubles, interleaved, Kronecker order
    int kind = QS_GATE_DENSE;
    int param = -1;                 // >= 0: exp(-i theta P / 2)
    char paulis[kMaxK + 1] = {0};   // generator P (one letter per qubit)
    // a cluster of diagonal gates of any width (k = 0, kind = diagonal): its
    // member gates and the union of their qubits
    std::vector<GateRec> parts;
    uint64_t wide_mask = 0;
};

// Exact structural class of a 2^k x 2^k FP64 matrix.
int classify_matrix(int k, const double* m);
// m = exp(-i theta P / 2) for the Pauli string (Kronecker order).
void rotation_matrix(int k, const char* paulis, double theta, double* m);
// The Pauli string's 2^k x 2^k matrix.
void pauli_matrix(int k, const char* paulis, double* m);

}  // namespace qsgb

namespace qsgb {
// The grouping found by the block search for one circuit, reused while the
// gates' qubits and structural kinds are unchanged (new angles only change
// the FP64 block products).
struct FuseCache {
    std::mutex mu;
    std::vector<uint64_t> key;   // the search's settings and every gate's qubits and kind
    bool valid = false;
    std::vector<std::vector<int>> groups;
};
}  // namespace qsgb

struct qs_circuit {
    int n = 0;
    int num_params = 0;
    std::vector<qsgb::GateRec> gates;
    std::shared_ptr<qsgb::FuseCache> fuse_cache = std::make_shared<qsgb::FuseCache>();
};

struct qs_pauli_sum {
    int n = 0;
    struct Term {
        double coeff;
        uint64_t xmask;   // X or Y positions (bit flips)
        uint64_t zmask;   // Z or Y positions (sign from the input bit)
        int ny;           // number of Y factors (phase i^ny)
    };
    std::vector<Term> terms;
};

struct qs_state {
    int n = 0;
    qs_dtype dt = QS_C64;
    void* data = nullptr;
    bool owned = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    // device scratch for reductions (partials), allocated at create/wrap
    double* scratch = nullptr;
    size_t scratch_doubles = 0;
    double* host_pinned = nullptr;  // small pinned buffer for results
    int* errflag = nullptr;         // device int in scratch: set by timed-out device waits
    uint64_t size() const { return 1ull << n; }
    size_t amp_bytes() const { return dt == QS_C64 ? 8 : 16; }
};

namespace qsgb {

// ----------------------------------------------------------------- passes
enum PassKind {
    PASS_TILE = 0,       // several gates on a shared-memory tile
    PASS_DENSE = 1,      // one dense gate, k <= 4, strided register kernel
    PASS_DIAG = 2,       // one diagonal gate (phase table), streaming
    PASS_MONO = 3,       // one permutation-with-phase gate
    PASS_GEMM = 4,       // one dense k in {5,6} gate on tensor cores
    PASS_DENSE_SMEM = 5, // one dense gate via a shared-memory block GEMM (SIMT)
    PASS_DIAG_WIDE = 6,  // a cluster of diagonal gates of any width: per-chunk phase tables
    PASS_TTILE = 7       // up to two dense 6-qubit blocks per round trip on tensor cores (3xFP16)
};

struct DiagCross {
    uint8_t k;
    uint8_t q[kMaxK];      // global qubits, q[0] the most significant local bit
    uint32_t tab;          // offset of its 2^k diagonal entries in the tables
};

// A wide diagonal pass: phase(x) = prod_c T_c[chunk c of x] * prod_cross d_g(bits of g),
// chunks of 8 index bits.  root8: every entry is exp(i pi m / 4); the
// tables then hold the integers m (real parts), chunks are 10 bits wide, and
// the kernel adds exponents mod 8.
struct WideDiag {
    int nchunks = 0;
    int chunk_bits = 8;             // 10 when root8
    bool root8 = false;
    std::vector<DiagCross> cross;   // gates spanning chunks; tab = element offset after the chunk tables
    uint32_t tab_elems = 0;
};
constexpr uint32_t kWideDiagTabElems = 3072;       // complex tables (shared memory)
constexpr uint32_t kWideDiagRoot8Elems = 8192;     // exponent tables (one byte each in shared memory)
constexpr int kWideDiagCross = 48;

struct TileGate {
    uint8_t k;
    uint8_t kind;         // QS_GATE_*, or kTileMulfree
    uint8_t q[kMaxK];     // tile-local bit positions (Kronecker order)
    uint32_t mat;         // element offset of the matrix in the pass buffer
};
// tile gate kind: a one-qubit matrix with entries in {0, +-1, +-i} (its
// scalar factor moved to the pass's scale), applied without multiplies
constexpr uint8_t kTileMulfree = 8;

// Register tile program of a tile pass (k_rtile): the tile's amplitudes live
// in registers, 2^RB per thread of a 256-thread block (L = RB + 8 tile bits:
// 5 on the lanes, RB on a thread's registers, 3 on the warps).  A layout
// says which tile bit each lane, register and warp bit holds; ops run in
// the current layout and LAYOUT ops move the tile between layouts through a
// swizzled shared-memory transpose.
constexpr int kRTMaxLayouts = 48, kRTMaxOps = 160;
enum RTOpType : uint8_t {
    RT_GATE = 0,    // k-qubit gate on register bits 0..k-1 (local bit i = register bit i)
    RT_GATE1 = 1,   // one-qubit gate on register bit `arg`
    RT_LANE1 = 2,   // one-qubit gate on lane bit `arg` (warp shuffles)
    RT_DIAG = 3,    // diagonal gate on tile bits q[] (Kronecker order), any layout
    RT_LAYOUT = 4   // move to layout `arg`
};
struct RTLayout {
    uint8_t lane[5];
    uint8_t reg[4];
    uint8_t warp[3];
};
struct RTOp {
    uint8_t type, k, arg, mulfree;
    uint8_t q[6];
    uint32_t mat;   // element offset of the gate's matrix in the pass buffer
};
struct RTProgram {
    int nops = 0, nlay = 0;
    int load_lay = 0, store_lay = 0;
    RTLayout lay[kRTMaxLayouts];
    RTOp ops[kRTMaxOps];
    uint16_t poscol[12] = {0};   // shared-memory position of tile bit i (linear, bijective)
};
// The register tile size of a dtype: 12 tile bits for complex64, 11 for complex128.
int rtile_bits(qs_dtype dt);

// A tensor tile pass (PASS_TTILE): up to kTTileMaxBlocks dense 6-qubit
// blocks applied to 12-qubit tiles held in shared memory.
constexpr int kTTileMaxBlocks = 2;
struct TTileDesc {
    int nb = 0;                        // blocks, applied in order
    int s[12] = {0};                   // tile qubits: physical bits ascending, s[0] = 0, s[1] = 1
    int kbit[kTTileMaxBlocks][6] = {};  // block b: tile bit of local-index bit i (LSB first)
    uint16_t poscol[12] = {0};         // shared-memory position of tile bit i (linear, bijective)
};

struct Pass {
    int kind = PASS_DENSE;
    TTileDesc tt;                      // PASS_TTILE
    // single-gate passes
    int k = 0;
    int qubits[kMaxK] = {0};
    int gate_kind = QS_GATE_DENSE;
    // tile passes: local bit i -> global bit pos[i]; pos[0..L-1]
    int L = 0;
    int pos[16] = {0};
    std::vector<TileGate> tgates;
    WideDiag wide;                  // PASS_DIAG_WIDE
    int members = 1;                // gates applied by a single-block pass
    // PASS_GEMM: physical bit exchanged with bit 0 in the pass's writes (-1:
    // none); the state after the pass is stored with those two bits swapped
    int swap_p = -1;
    RTProgram rt;                   // PASS_TILE: register tile program (rt.nops > 0: k_rtile)
    // tile passes: product of the scalars factored out of kTileMulfree gates,
    // applied at write-back.  mode 1: mag * exp(i pi s / 4); mode 2: scale_c
    int scale_mode = 0;
    int scale_s = 0;
    double scale_mag = 1.0;
    double scale_c[2] = {1.0, 0.0};
    // matrices (FP64 host copies; converted on upload)
    std::vector<double> mats;       // concatenated interleaved matrices
    size_t dev_offset = 0;          // element offset in the plan's device buffer
};

// Compile a tile pass into a register tile program (false: the pass keeps
// the shared-memory tile kernel).
bool build_rtile_program(qs_dtype dt, const Pass& p, RTProgram& prog);
cudaError_t launch_rtile(void* psi, int n, qs_dtype dt, const Pass& ps, const void* dmats, cudaStream_t st);

}  // namespace qsgb

struct qs_plan {
    int n = 0;
    qs_dtype dt = QS_C64;
    qs_options opt{};
    std::vector<qsgb::Pass> passes;
    void* dev_mats = nullptr;       // float2 or double2 matrices of all passes
    size_t dev_elems = 0;
    int device = 0;
    cudaStream_t stream = nullptr;  // set: matrices allocated and freed in this stream's order
};

namespace qsgb {

// ----------------------------------------------------------------- planner
// qs_plan_create with the matrices uploaded and (at destruction) freed in the
// order of `stream` (no device-wide synchronisation); nullptr = qs_plan_create.
qs_status plan_create_on(const qs_circuit* c, qs_dtype dt, const qs_options* opt, cudaStream_t stream, qs_plan** out);
// Pinned host staging for uploads that must not wait for the stream: a copy
// from pageable memory may wait for the stream's earlier work before it is
// staged.  A buffer is reused once the stream has consumed its last copies
// (`done`, recorded by the user after them).
struct PinnedStage {
    char* p = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;  // recorded after the last copy out of the buffer
    int dev = -1;
    ~PinnedStage() {
        if (done) cudaEventSynchronize(done);
        if (p) cudaFreeHost(p);
        if (done) cudaEventDestroy(done);
    }
    cudaError_t reserve(size_t bytes, int device) {
        if (done) {
            cudaError_t e = cudaEventSynchronize(done);
            if (e != cudaSuccess) return e;
        }
        if (dev != device && done) {
            cudaEventDestroy(done);
            done = nullptr;
        }
        if (!done) {
            cudaError_t e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
            dev = device;
        }
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&p), bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) cap = bytes;
        return e;
    }
};
// stream-ordered allocation from the library's memory pool on the current
// device (keeps its reservations between calls; free with cudaFreeAsync)
cudaError_t lib_malloc_async(void** ptr, size_t bytes, cudaStream_t st);
// A plan of ready passes (matrices uploaded and converted, in `stream` order when given).
qs_status plan_from_passes(int n, qs_dtype dt, const qs_options& opt, std::vector<Pass>&& passes, cudaStream_t stream,
                           qs_plan** out);
// effort 1: each candidate block scored with a one-level lookahead; 0: greedy
qs_status fuse_gates(int n, const std::vector<GateRec>& in, int k_max, std::vector<GateRec>& out, int effort = 1,
                     FuseCache* cache = nullptr);
// Clustering by kind (Sections 4.2, 4.5): diagonal gates join diagonal
// clusters of any width (one wide pass each), the others fuse among
// themselves up to k_max qubits.  Clusters on <= 6 qubits come back as
// ordinary diagonal blocks.
qs_status fuse_by_kind(int n, const std::vector<GateRec>& in, int k_max, std::vector<GateRec>& out, int effort = 1,
                       FuseCache* cache = nullptr);
qs_status build_passes(int n, qs_dtype dt, const std::vector<GateRec>& blocks,
                       const qs_options& opt, std::vector<Pass>& passes);
// The pass of one fused block on its own (no tile grouping).
void single_block_pass(int n, qs_dtype dt, const qs_options& opt, const GateRec& g, Pass& p);
// Fuse and run together on the tensor cores: each block's pass is launched
// as soon as it is found and multiplied (qs_host.cpp)
// blocks_out (optional): the block products of the circuit's fusion groups,
// in group order (filled when the call succeeds)
qs_status apply_streamed(qs_state* s, const qs_circuit* c, const qs_options& opt,
                         std::vector<GateRec>* blocks_out = nullptr);
// bit-0 placement over 6-qubit passes (qs_plan.cpp)
int bit0_plan(int n, const std::vector<const Pass*>& run, int s0, bool end_free, std::vector<int>& choice);
int bit0_apply(Pass& p, int s, int bc);
// One group's fused block (see fuse_gates): the FP64 product of in[taken].
void block_product(int n, const std::vector<GateRec>& in, const std::vector<int>& taken, GateRec& b);
// fuse_gates in stream form: each group of gate indices goes to `emit` as soon
// as the block search finds it (group {-1 - i}: gate i kept as it is).
qs_status fuse_each(int n, const std::vector<GateRec>& in, int k_max, int effort, FuseCache* cache,
                    const std::function<void(std::vector<int>&&)>& emit);
int auto_tile_qubits(int n, qs_dtype dt);
// Section 4.1: one-qubit tile gates that are a scalar times a matrix with
// entries in {0, +-1, +-i} (H, sqrt X, sqrt Y, X, Y, ...) become kTileMulfree
// gates; the pass keeps the product of their scalars.
void factor_tile_scalars(Pass& p);
// Greedy commuting-reorder grouping of `units` (in order) into tiles of L
// qubits that always contain the lowest `low_bits_in_tile` qubits; dense
// members have k <= 4; each group's matrices fit `mat_budget` entries.
std::vector<std::vector<int>> group_for_tiles(const std::vector<GateRec>& units, int L, int low_bits_in_tile,
                                              size_t mat_budget);

// ----------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return the launch error (cudaSuccess).
// `dmats` points at the pass's matrices already converted to the state's
// precision (complex float or double, interleaved).
cudaError_t launch_dense(void* psi, int n, qs_dtype dt, int k, const int* qubits,
                         const double* m_host, cudaStream_t st);
cudaError_t launch_diag(void* psi, int n, qs_dtype dt, int k, const int* qubits,
                        const double* m_host, cudaStream_t st);
cudaError_t launch_mono(void* psi, int n, qs_dtype dt, int k, const int* qubits,
                        const double* m_host, cudaStream_t st);
cudaError_t launch_dense_smem(void* psi, int n, qs_dtype dt, int k, const int* qubits,
                              const void* dmat, cudaStream_t st);
cudaError_t launch_tile(void* psi, int n, qs_dtype dt, const Pass& p, const void* dmats,
                        cudaStream_t st);
cudaError_t launch_diag_wide(void* psi, int n, qs_dtype dt, const WideDiag& w, const void* dtables,
                             cudaStream_t st);
// Tensor-core pass for a dense 6-qubit gate on a complex64 state (n >= 11);
// `err` (device int) is set to 1 if a bounded device wait timed out.
bool gemm_supported(int n, int k);
// Gram matrices of the block adjoint sweep (qs_gram.cu).  A gate of a fused
// block in the block's local coordinates (its six Gram targets, local bit b
// = the b-th lowest target), for the gradient recursion.
struct BlockGradGate {
    int k;                   // gate qubits
    int lb[6];               // local bit of the gate's qubit t (t = 0: most significant in its matrix)
    int param;               // parameter index, or -1
    int xmask, zmask, ny;    // generator in local bits: X or Y bits, Y or Z bits, number of Y
    int diag;                // the matrix is diagonal
    int flags;               // kGradNoUpdate: gradient only; kGradCompactDiag: the 2^k diagonal entries alone
    uint32_t moff;           // offset of its 2^k x 2^k complex64 matrix in the gate-matrix array
};
constexpr int kGradNoUpdate = 1, kGradCompactDiag = 2;
bool gram_supported(int n);
size_t gram_workspace_elems(int n);   // doubles of one n-qubit Gram matrix's per-CTA parts
// The per-CTA parts (into ws, gram_workspace_elems(n) doubles) of
// M = sum over the sets of psi_s lambda_s^dagger over the six `targets`
// (descending); M is 2 x 64 x 64 FP64, Re rows then Im rows.
cudaError_t launch_gram(const void* psi, const void* lam, int n, const int* targets, double* ws, int* err,
                        cudaStream_t st);
// M of nslots Gram matrices (Mall, 8192 doubles each) from their parts
// (ws, gram_workspace_elems(n) doubles each), FP64 in a fixed order.
cudaError_t launch_gram_reduce(const double* ws, int n, int nslots, double* Mall, cudaStream_t st);
// One CTA per block: gates[gate0[b] .. gate0[b+1]) from the block's last
// gate to its first; gradient of parameter p into sums[2p + 1].
cudaError_t launch_block_grads(const double* Mall, int nslots, const BlockGradGate* gates, const int* gate0,
                               const void* mats, double* sums, cudaStream_t st);
// A tensor tile pass on a complex64 state (3xFP16): dmat holds d.nb 64 x 64
// float2 matrices, each in the one-block pass's local-index order.
cudaError_t launch_ttile(void* psi, int n, const TTileDesc& d, const void* dmat, int* err, cudaStream_t st);
bool ttile_supported(int n);

// inject = 1 (testing only): in block 0 one producer warp withholds its
// first "operand ready" arrival, so the MMA issuer's bounded wait runs out
// swap_p >= 0: the pass writes each amplitude with index bits 0 and swap_p
// exchanged (both must be among the pass's four lowest non-target bits)
cudaError_t launch_gemm(void* psi, int n, int k, const int* qubits, const void* dmat_f32,
                        int precision, int* err, cudaStream_t st, int inject = 0, int swap_p = -1);

cudaError_t launch_init_basis(void* psi, int n, qs_dtype dt, uint64_t index, cudaStream_t st);
cudaError_t launch_init_uniform(void* psi, int n, qs_dtype dt, cudaStream_t st);

// Reductions write `nparts` FP64 partial sums to scratch, then one block
// sums them in a fixed order into result[0..count).
int reduce_blocks();
cudaError_t launch_norm(const void* psi, int n, qs_dtype dt, double* scratch, double* result,
                        cudaStream_t st);
// out = H psi (distinct memory) and result[0] = <psi|H|psi>, in tile passes
// that each read psi once (qs_pauli.cu); scratch holds reduce_blocks()
// partial sums.
cudaError_t launch_apply_pauli_sum(const void* psi, void* out, int n, qs_dtype dt,
                                   const qs_pauli_sum& h, cudaStream_t st);
cudaError_t launch_expectation(const void* psi, int n, qs_dtype dt, const qs_pauli_sum& h, double* scratch,
                               double* result, cudaStream_t st);
// result[0] = (set) or += the fixed-order sum of `cols` partials.
cudaError_t launch_accumulate(const double* partials, int cols, double* result, bool set, cudaStream_t st);
// <a|b> partial sums (complex, FP64) into result[0..1].
cudaError_t launch_inner(const void* a, const void* b, int n, qs_dtype dt, double* scratch,
                         double* result, cudaStream_t st);

cudaError_t launch_sum_partials(const double* partials, int rows, int cols, double* out,
                                cudaStream_t st);

// Reverse-sweep tile pass over psi and lambda together: for each member in
// order, optionally accumulate <lambda|P|psi> on the tile (parameter slot),
// then apply the member's matrix (U^dagger) to both tiles.
struct AdjTileGate {
    TileGate g;            // U^dagger on local qubits
    int slot;              // parameter, or -1
    uint32_t px, pz;       // Pauli generator on local bits: flip mask, sign mask
    uint8_t ny;            // number of Y factors
    uint8_t mulfree;       // diagonal with every phase in {+-1, +-i}
    uint8_t form;          // single-qubit U^dagger: 0 complex, 1 diagonal, 2 real
    uint8_t pad;
};
cudaError_t launch_adjoint_tile(void* psi, void* lam, int n, qs_dtype dt, int L, const int* pos,
                                const std::vector<AdjTileGate>& gates, const void* dmats, size_t mat_elems,
                                double* partials, int nblocks, cudaStream_t st);

// Stage steps of the adjoint reverse sweep (a run of pairwise-commuting
// gates: all gradients from one (psi, lambda), then the run's inverse).
constexpr int kStageGradGens = 16;    // generators per k_grad_pairs launch
constexpr int kStageDiagGens = 32;    // one-qubit Z generators per k_diag_stage launch
constexpr int kStageDiagMulti = 8;    // multi-qubit Z generators per k_diag_stage launch
constexpr int kStageDiagCross = 32;   // gates spanning two 8-qubit chunks
constexpr uint32_t kStageDiagTabElems = 3072;
struct StageGen {
    uint32_t px, pz;       // generator on the tile's local bits: flip mask, sign mask
    int ny;                // number of Y factors
    int slot;              // parameter
};
// <lambda|P_g|psi> partial sums for each generator (tile over pos[0..L-1]).
cudaError_t launch_grad_pairs(const void* psi, const void* lam, int n, qs_dtype dt, int L, const int* pos,
                              const std::vector<StageGen>& gens, double* partials, int nblocks, cudaStream_t st);
// Z-generator gradients of a diagonal run, and (apply) its inverse on psi and
// lambda: tables = nchunks x 256 chunk phases, then the cross gates' entries.
cudaError_t launch_diag_stage(void* psi, void* lam, int n, qs_dtype dt, int nchunks, const std::vector<DiagCross>& cross,
                              const void* dtables, uint32_t tab_elems, const std::vector<uint64_t>& zmasks,
                              const std::vector<int>& slots, bool apply, double* partials, int nblocks,
                              cudaStream_t st);

// Fused reverse-sweep pass: consecutive stages whose non-diagonal gates act on
// one qubit, in one read/write pass over psi and lambda.  A tile of 2^L
// amplitudes (qubits pos[0..L-1], ascending; pos[i] = i for the low rows)
// stays in registers: a thread holds 2^(L-8) amplitudes of each state, the
// register index j covering the tile bits a..a+L-9 of the current layout
// (lay_a[layout]); layout 0 (a = L - 8) is the one loaded and stored.
constexpr int kSweepTileC64 = 12;     // L for complex64
constexpr int kSweepTileC128 = 11;    // L for complex128
constexpr int kSweepMaxOps = 256;
constexpr int kSweepMaxGrads = 128;
constexpr int kSweepMaxDiags = 4;
constexpr int kSweepMaxCross = 64;
constexpr int kSweepMaxGens = 96;
constexpr int kSweepMaxLayouts = 4;
constexpr int kSweepDiagGens = 40;    // Z generators of one diagonal op
constexpr int kSweepDiagCross = 32;
inline uint32_t sweep_tab_budget(qs_dtype dt) { return dt == QS_C64 ? 3072u : 1536u; }
// SWEEP_G1ALL: one-qubit gates of one form (G1_RSHEAR, G1_RSHEAR_Y or
// G1_CSHEAR_X) and generator on every register bit, in bit order, with
// consecutive coefficient sets from idx
enum SweepOpType { SWEEP_LAYOUT = 0, SWEEP_G1 = 1, SWEEP_DIAG = 2, SWEEP_G1ALL = 3 };
// One-qubit op forms.  U^dagger, times a phase common to psi and lambda (it
// cancels in Im <lambda|P|psi>), is M = [[a, -conj(b)], [b, conj(a)]] with
// Re a >= 0, applied as three in-place shears p0 += z p1, p1 += y p0,
// p0 += x p1 (y = b, x = (a - 1) / b, z = (conj(a) - 1) / b), or directly.
enum SweepG1Form {
    G1_DIRECT = 0,         // the four entries, any generator
    G1_RSHEAR = 1,         // real shears, no gradient
    G1_RSHEAR_Y = 2,       // real shears, generator Y
    G1_RSHEAR_NEG = 3,     // p1 negated, then real shears (a reflection), no gradient
    G1_CSHEAR = 4,         // complex shears, no gradient
    G1_CSHEAR_X = 5,       // complex shears, generator X
    G1_FF_CPLX = 6,        // complex128 in float-float: U^dagger's four entries
    G1_FF_REAL = 7,        // the same, all four real
    G1_FORMS = 8
};
struct SweepOpRec {
    uint8_t type;          // SweepOpType
    uint8_t arg;           // LAYOUT: the new layout; G1: register bit
    uint8_t form;          // G1: SweepG1Form
    uint8_t gen;           // G1: generator 0 none, 1 X, 2 Y, 3 Z
    uint32_t idx;          // G1: coefficients (4 elements: the entries, or z, y, x); DIAG: diagonal record
};
struct SweepDiagRec {
    uint8_t nchunks;       // chunk c = qubits 8c .. 8c+7; chunk 0 (with the register qubits) is looked up per amplitude
    uint8_t pad0;
    uint8_t ncross, nct;   // cross gates; the first nct hold a register qubit
    uint16_t cross0, gen0; // first cross gate / Z generator in the pass's lists
    uint8_t ngen, nstaged; // Z generators; the first nstaged are summed per thread
    uint32_t tab;          // element offset of the chunk tables in the pass's table block
};
// Z-generator gradient of a diagonal op (run in the low layout: register bit
// k = qubit k), sum_x (-1)^popc(x & zmask) Im(conj(l_x) p_x), with t_x the
// summand and S its sum over a tile.
//   block (src != kZStaged): at most one tile bit in the mask; the gradient
//     is (-1)^popc(tile base & mthr) (S - 2 X), X = 0 (src 0), the sum over
//     register bit src-1 set (src 1..RB), or over thread bit src-RB-1 set
//   staged: the sign from the thread's fixed bits (mthr) times a register
//     sum: kind 0 all, 1..RB register bit kind-1 negated, RB+1 jmask bit j
//     negated; one value per thread, summed with the G1 gradients
constexpr uint8_t kZStaged = 255;
struct SweepZGen {
    uint64_t mthr;
    uint16_t jmask;
    uint16_t local;        // block: its gradient slot in the pass
    uint8_t kind;
    uint8_t src;
    uint8_t pad[2];
};
struct SweepPassDesc {
    int L = 0;
    int pos[16] = {0};
    int nlay = 0;
    int lay_a[kSweepMaxLayouts] = {0};
    int load_lay = 0, store_lay = 0;  // the tile's load and store layouts: 0 or 1 (both coalesced)
    std::vector<SweepOpRec> ops;
    std::vector<SweepDiagRec> diags;
    std::vector<DiagCross> cross;      // tab: element offset in the pass's table block
    std::vector<SweepZGen> gens;
    std::vector<int> slots;            // gradient order -> parameter
    std::vector<double> mats, tabs;    // FP64 interleaved complex
    size_t mat0 = 0, tab0 = 0;         // element offsets in the sweep's device buffers
};
// Register-layout starts for a dtype: tile bit i is held in registers by the
// first layout l with lay_a[l] <= i < lay_a[l] + L - 8.
int sweep_layouts(qs_dtype dt, int* lay_a);
cudaError_t launch_sweep_pass(void* psi, void* lam, int n, qs_dtype dt, const SweepPassDesc& p, const void* dmats,
                              const void* dtabs, double* partials, int nblocks, cudaStream_t st);

int num_sms();

// State helpers shared by the C ABI files: argument check of a state, its
// result slots (device doubles after the partials), and the report of a
// timed-out bounded device wait (QS_ERR_TIMEOUT; the flag is cleared).
qs_status check_state(const qs_state* s);
double* result_area(const qs_state* s);
qs_status check_device_flag(const qs_state* s);

// Host threads a planning step may use (fusion products, stage plans): the
// hardware's, at most `cap`; workers that already run in parallel (batched
// gradients) set the calling thread's cap to 1.
unsigned host_threads(unsigned cap);
unsigned set_host_thread_cap(unsigned cap);   // returns the previous cap

}  // namespace qsgb
