// C ABI entry points: argument checks, object management and the host side
// of every operation.  Device work goes through the launchers in the .cu
// files; nothing here computes on amplitudes.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <deque>
#include <string>
#include <thread>
#include <map>
#include <mutex>
#include <set>
#include <memory>
#include <new>

#include "qs_internal.h"

namespace qsgb {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

qs_status fail(qs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

qs_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return QS_ERR_OOM;
    return QS_ERR_CUDA;
}

// kernels whose dynamic shared-memory limit is already raised, per device
static std::mutex g_attr_mu;
static std::set<std::pair<const void*, int>> g_attr_done;

bool smem_attr_done(const void* kernel, int device) {
    std::lock_guard<std::mutex> lock(g_attr_mu);
    return g_attr_done.count({kernel, device}) != 0;
}

void smem_attr_mark(const void* kernel, int device) {
    std::lock_guard<std::mutex> lock(g_attr_mu);
    g_attr_done.insert({kernel, device});
}

static thread_local unsigned g_thread_cap = 0;  // 0: none

unsigned host_threads(unsigned cap) {
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    if (g_thread_cap) hw = std::min(hw, g_thread_cap);
    return std::min(hw, cap);
}

unsigned set_host_thread_cap(unsigned cap) {
    const unsigned prev = g_thread_cap;
    g_thread_cap = cap;
    return prev;
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 148;
        cached[dev] = v;
    }
    return cached[dev];
}

static qs_status check_gate_args(int n, const int* qubits, int k, const double* m) {
    if (!qubits || !m) return fail(QS_ERR_ARG, "null qubits or matrix");
    if (k < 1 || k > kMaxK) return fail(QS_ERR_ARG, "gate size k=%d outside 1..6", k);
    if (k > n) return fail(QS_ERR_ARG, "gate on %d qubits in a %d-qubit state", k, n);
    uint64_t seen = 0;
    for (int i = 0; i < k; ++i) {
        if (qubits[i] < 0 || qubits[i] >= n)
            return fail(QS_ERR_ARG, "qubit %d out of range 0..%d", qubits[i], n - 1);
        if ((seen >> qubits[i]) & 1) return fail(QS_ERR_ARG, "duplicate qubit %d", qubits[i]);
        seen |= 1ull << qubits[i];
    }
    const int d = 1 << k;
    for (int i = 0; i < 2 * d * d; ++i)
        if (!std::isfinite(m[i])) return fail(QS_ERR_ARG, "matrix entry %d is not finite", i);
    return QS_OK;
}

qs_status check_state(const qs_state* s) {
    if (!s) return fail(QS_ERR_ARG, "null state");
    int dev = -1;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev != s->device)
        return fail(QS_ERR_ARG, "state lives on device %d but device %d is current", s->device, dev);
    return QS_OK;
}

static qs_status state_setup(qs_state* s) {
    // reduction partials (two per block, plus a result area) and a small
    // pinned buffer for results
    s->scratch_doubles = (size_t)reduce_blocks() * 2 + 64;
    QS_CUDA(cudaMalloc(&s->scratch, s->scratch_doubles * sizeof(double)));
    QS_CUDA(cudaMallocHost(&s->host_pinned, 64 * sizeof(double)));
    s->errflag = reinterpret_cast<int*>(s->scratch + s->scratch_doubles - 1);
    QS_CUDA(cudaMemset(s->errflag, 0, sizeof(int)));
    return QS_OK;
}

double* result_area(const qs_state* s) {
    return s->scratch + s->scratch_doubles - 64;
}

// After a stream synchronisation: report (and clear) a device-side wait that
// gave up since the last check.
qs_status check_device_flag(const qs_state* s) {
    int flag = 0;
    QS_CUDA(cudaMemcpy(&flag, s->errflag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        QS_CUDA(cudaMemset(s->errflag, 0, sizeof(int)));
        return fail(QS_ERR_TIMEOUT, "a bounded device-side wait timed out; results of that pass are invalid");
    }
    return QS_OK;
}

}  // namespace qsgb

using namespace qsgb;

extern "C" {

const char* qs_version(void) { return "qsgb 0.1 (sm_103a)"; }

const char* qs_status_string(qs_status s) {
    switch (s) {
        case QS_OK: return "ok";
        case QS_ERR_ARG: return "invalid argument";
        case QS_ERR_OOM: return "out of memory";
        case QS_ERR_CUDA: return "CUDA error";
        case QS_ERR_UNSUPPORTED: return "unsupported";
        case QS_ERR_TIMEOUT: return "device wait timed out";
        case QS_ERR_STATE: return "object in wrong state";
    }
    return "unknown status";
}

const char* qs_last_error(void) { return g_last_error.c_str(); }

qs_status qs_options_default(qs_options* opt) {
    if (!opt) return fail(QS_ERR_ARG, "null options");
    memset(opt, 0, sizeof(*opt));
    opt->k_max = 4;
    opt->tile_qubits = 0;
    opt->use_tile = 1;
    opt->precision = QS_PREC_FP32;
    opt->fuse = 1;
    opt->fusion_effort = 1;
    return QS_OK;
}

// ------------------------------------------------------------------ state

qs_status qs_state_create(int n, qs_dtype dt, void* stream, qs_state** out) {
    if (!out) return fail(QS_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (n < 1 || n > kMaxQubits) return fail(QS_ERR_ARG, "n=%d outside 1..%d", n, kMaxQubits);
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_ERR_ARG, "bad dtype");
    const size_t bytes = (size_t(1) << n) * (dt == QS_C64 ? 8 : 16);
    size_t free_b = 0, total_b = 0;
    QS_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (bytes + (64u << 20) > free_b)
        return fail(QS_ERR_OOM, "state needs %zu bytes, %zu free", bytes, free_b);
    std::unique_ptr<qs_state> s(new (std::nothrow) qs_state);
    if (!s) return fail(QS_ERR_OOM, "host allocation failed");
    s->n = n;
    s->dt = dt;
    s->stream = (cudaStream_t)stream;
    QS_CUDA(cudaGetDevice(&s->device));
    cudaError_t e = cudaMallocAsync(&s->data, bytes, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(state)");
    s->owned = true;
    qs_status st = state_setup(s.get());
    if (st != QS_OK) {
        cudaFreeAsync(s->data, s->stream);
        return st;
    }
    e = launch_init_basis(s->data, n, dt, 0, s->stream);
    if (e != cudaSuccess) {
        qs_state_destroy(s.release());
        return cuda_fail(e, "init |0>");
    }
    *out = s.release();
    return QS_OK;
}

qs_status qs_state_wrap(void* device_ptr, int n, qs_dtype dt, void* stream, qs_state** out) {
    if (!out) return fail(QS_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!device_ptr) return fail(QS_ERR_ARG, "null device pointer");
    if (((uintptr_t)device_ptr) & 15) return fail(QS_ERR_ARG, "device pointer not 16-byte aligned");
    if (n < 1 || n > kMaxQubits) return fail(QS_ERR_ARG, "n=%d outside 1..%d", n, kMaxQubits);
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_ERR_ARG, "bad dtype");
    cudaPointerAttributes attr;
    QS_CUDA(cudaPointerGetAttributes(&attr, device_ptr));
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(QS_ERR_ARG, "pointer is not device memory");
    std::unique_ptr<qs_state> s(new (std::nothrow) qs_state);
    if (!s) return fail(QS_ERR_OOM, "host allocation failed");
    s->n = n;
    s->dt = dt;
    s->data = device_ptr;
    s->owned = false;
    s->stream = (cudaStream_t)stream;
    QS_CUDA(cudaGetDevice(&s->device));
    if (attr.device != s->device)
        return fail(QS_ERR_ARG, "pointer on device %d, current device %d", attr.device, s->device);
    qs_status st = state_setup(s.get());
    if (st != QS_OK) return st;
    *out = s.release();
    return QS_OK;
}

qs_status qs_state_destroy(qs_state* s) {
    if (!s) return QS_OK;
    if (s->owned && s->data) cudaFreeAsync(s->data, s->stream);
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    if (s->scratch) cudaFree(s->scratch);
    if (s->host_pinned) cudaFreeHost(s->host_pinned);
    delete s;
    return QS_OK;
}

qs_status qs_state_set_stream(qs_state* s, void* stream) {
    if (!s) return fail(QS_ERR_ARG, "null state");
    s->stream = (cudaStream_t)stream;
    return QS_OK;
}

qs_status qs_state_info(const qs_state* s, int* n, qs_dtype* dt, void** device_ptr) {
    if (!s) return fail(QS_ERR_ARG, "null state");
    if (n) *n = s->n;
    if (dt) *dt = s->dt;
    if (device_ptr) *device_ptr = s->data;
    return QS_OK;
}

qs_status qs_state_init_basis(qs_state* s, uint64_t index) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (index >= s->size()) return fail(QS_ERR_ARG, "basis index out of range");
    QS_CUDA(launch_init_basis(s->data, s->n, s->dt, index, s->stream));
    return QS_OK;
}

qs_status qs_state_init_uniform(qs_state* s) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    QS_CUDA(launch_init_uniform(s->data, s->n, s->dt, s->stream));
    return QS_OK;
}

qs_status qs_state_copy(qs_state* dst, const qs_state* src) {
    qs_status st = check_state(dst);
    if (st != QS_OK) return st;
    st = check_state(src);
    if (st != QS_OK) return st;
    if (dst->n != src->n || dst->dt != src->dt) return fail(QS_ERR_ARG, "state shapes differ");
    if (dst->data == src->data) return QS_OK;
    QS_CUDA(cudaMemcpyAsync(dst->data, src->data, src->size() * src->amp_bytes(),
                            cudaMemcpyDeviceToDevice, dst->stream));
    return QS_OK;
}

// ------------------------------------------------------------------ gates

static qs_status apply_one(qs_state* s, const GateRec& g) {
    cudaError_t e;
    if (g.kind == QS_GATE_DIAGONAL) {
        e = launch_diag(s->data, s->n, s->dt, g.k, g.qubits, g.m.data(), s->stream);
    } else if (g.kind == QS_GATE_MONOMIAL) {
        e = launch_mono(s->data, s->n, s->dt, g.k, g.qubits, g.m.data(), s->stream);
    } else if (g.k <= 4) {
        e = launch_dense(s->data, s->n, s->dt, g.k, g.qubits, g.m.data(), s->stream);
    } else {
        // large dense gate: stage the converted matrix in device scratch
        const int d = 1 << g.k;
        const size_t elems = (size_t)d * d;
        void* dm = nullptr;
        const size_t bytes = elems * (s->dt == QS_C64 ? 8 : 16);
        QS_CUDA(cudaMallocAsync(&dm, bytes, s->stream));
        std::vector<float> f;
        const void* src = g.m.data();
        if (s->dt == QS_C64) {
            f.resize(2 * elems);
            for (size_t i = 0; i < 2 * elems; ++i) f[i] = (float)g.m[i];
            src = f.data();
        }
        e = cudaMemcpyAsync(dm, src, bytes, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // host copy stays valid
        if (e == cudaSuccess) e = launch_dense_smem(s->data, s->n, s->dt, g.k, g.qubits, dm, s->stream);
        cudaFreeAsync(dm, s->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gate launch");
    return QS_OK;
}

qs_status qs_apply_gate(qs_state* s, const int* qubits, int k, const double* m) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    st = check_gate_args(s->n, qubits, k, m);
    if (st != QS_OK) return st;
    GateRec g;
    g.k = k;
    for (int i = 0; i < k; ++i) g.qubits[i] = qubits[i];
    g.m.assign(m, m + 2 * (1 << k) * (1 << k));
    g.kind = classify_matrix(k, m);
    return apply_one(s, g);
}

// --------------------------------------------------------------- circuits

qs_status qs_circuit_create(int n, qs_circuit** out) {
    if (!out) return fail(QS_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (n < 1 || n > kMaxQubits) return fail(QS_ERR_ARG, "n=%d outside 1..%d", n, kMaxQubits);
    qs_circuit* c = new (std::nothrow) qs_circuit;
    if (!c) return fail(QS_ERR_OOM, "host allocation failed");
    c->n = n;
    *out = c;
    return QS_OK;
}

qs_status qs_circuit_destroy(qs_circuit* c) {
    delete c;
    return QS_OK;
}

qs_status qs_circuit_add(qs_circuit* c, const int* qubits, int k, const double* m) {
    if (!c) return fail(QS_ERR_ARG, "null circuit");
    qs_status st = check_gate_args(c->n, qubits, k, m);
    if (st != QS_OK) return st;
    GateRec g;
    g.k = k;
    for (int i = 0; i < k; ++i) g.qubits[i] = qubits[i];
    g.m.assign(m, m + 2 * (1 << k) * (1 << k));
    g.kind = classify_matrix(k, m);
    c->gates.push_back(std::move(g));
    return QS_OK;
}

qs_status qs_circuit_add_gates(qs_circuit* c, int count, const int* ks, const int* qubits, const double* mats) {
    if (!c) return fail(QS_ERR_ARG, "null circuit");
    if (count < 0) return fail(QS_ERR_ARG, "negative gate count");
    if (count > 0 && (!ks || !qubits || !mats)) return fail(QS_ERR_ARG, "null argument");
    size_t qo = 0, mo = 0;
    for (int i = 0; i < count; ++i) {  // every gate checked before any is appended
        const int k = ks[i];
        if (k < 1 || k > kMaxK) return fail(QS_ERR_ARG, "gate %d: bad size %d", i, k);
        qs_status st = check_gate_args(c->n, qubits + qo, k, mats + mo);
        if (st != QS_OK) {
            const std::string why = qs_last_error();
            return fail(st, "gate %d: %s", i, why.c_str());
        }
        qo += (size_t)k;
        mo += 2 * ((size_t)1 << (2 * k));
    }
    c->gates.reserve(c->gates.size() + (size_t)count);
    qo = mo = 0;
    for (int i = 0; i < count; ++i) {
        const int k = ks[i];
        const size_t len = 2 * ((size_t)1 << (2 * k));
        GateRec g;
        g.k = k;
        for (int j = 0; j < k; ++j) g.qubits[j] = qubits[qo + j];
        g.m.assign(mats + mo, mats + mo + len);
        g.kind = classify_matrix(k, g.m.data());
        c->gates.push_back(std::move(g));
        qo += (size_t)k;
        mo += len;
    }
    return QS_OK;
}

qs_status qs_circuit_add_rotation(qs_circuit* c, const int* qubits, int k, const char* paulis,
                                  int param, double theta) {
    if (!c || !qubits || !paulis) return fail(QS_ERR_ARG, "null argument");
    if (k < 1 || k > kMaxK || k > c->n) return fail(QS_ERR_ARG, "bad rotation size %d", k);
    if (param < 0) return fail(QS_ERR_ARG, "parameter index must be >= 0");
    if ((int)strnlen(paulis, kMaxK + 1) != k) return fail(QS_ERR_ARG, "Pauli string length != k");
    for (int i = 0; i < k; ++i)
        if (!strchr("IXYZ", paulis[i])) return fail(QS_ERR_ARG, "bad Pauli letter '%c'", paulis[i]);
    GateRec g;
    g.k = k;
    for (int i = 0; i < k; ++i) g.qubits[i] = qubits[i];
    g.m.resize(2 * (1 << k) * (1 << k));
    rotation_matrix(k, paulis, theta, g.m.data());
    qs_status st = check_gate_args(c->n, qubits, k, g.m.data());
    if (st != QS_OK) return st;
    g.kind = classify_matrix(k, g.m.data());
    g.param = param;
    memcpy(g.paulis, paulis, k);
    g.paulis[k] = 0;
    c->gates.push_back(std::move(g));
    c->num_params = std::max(c->num_params, param + 1);
    return QS_OK;
}

qs_status qs_circuit_set_params(qs_circuit* c, const double* theta, int num) {
    if (!c || (!theta && num > 0)) return fail(QS_ERR_ARG, "null argument");
    if (num < c->num_params) return fail(QS_ERR_ARG, "need %d parameters, got %d", c->num_params, num);
    for (GateRec& g : c->gates) {
        if (g.param < 0) continue;
        rotation_matrix(g.k, g.paulis, theta[g.param], g.m.data());
        g.kind = classify_matrix(g.k, g.m.data());
    }
    return QS_OK;
}

qs_status qs_circuit_size(const qs_circuit* c, int* n, int* num_gates, int* num_params) {
    if (!c) return fail(QS_ERR_ARG, "null circuit");
    if (n) *n = c->n;
    if (num_gates) *num_gates = (int)c->gates.size();
    if (num_params) *num_params = c->num_params;
    return QS_OK;
}

qs_status qs_circuit_gate(const qs_circuit* c, int index, int* k, int* qubits, double* m, int* kind) {
    if (!c) return fail(QS_ERR_ARG, "null circuit");
    if (index < 0 || index >= (int)c->gates.size()) return fail(QS_ERR_ARG, "gate index out of range");
    const GateRec& g = c->gates[index];
    if (k) *k = g.k;
    if (qubits) memcpy(qubits, g.qubits, sizeof(int) * g.k);
    if (m) memcpy(m, g.m.data(), sizeof(double) * g.m.size());
    if (kind) *kind = g.kind;
    return QS_OK;
}

qs_status qs_fuse(const qs_circuit* in, int k_max, qs_circuit** out) {
    if (!in || !out) return fail(QS_ERR_ARG, "null argument");
    *out = nullptr;
    std::unique_ptr<qs_circuit> c(new (std::nothrow) qs_circuit);
    if (!c) return fail(QS_ERR_OOM, "host allocation failed");
    c->n = in->n;
    qs_status st = fuse_gates(in->n, in->gates, k_max, c->gates);
    if (st != QS_OK) return st;
    *out = c.release();
    return QS_OK;
}

// ------------------------------------------------------------------ plans

qs_status qs_plan_create(const qs_circuit* c, qs_dtype dt, const qs_options* opt_in, qs_plan** out) {
    return plan_create_on(c, dt, opt_in, nullptr, out);
}

}  // extern "C"

qs_status qsgb::plan_create_on(const qs_circuit* c, qs_dtype dt, const qs_options* opt_in, cudaStream_t stream,
                               qs_plan** out) {
    if (!c || !out) return fail(QS_ERR_ARG, "null argument");
    *out = nullptr;
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_ERR_ARG, "bad dtype");
    qs_options opt;
    if (opt_in) {
        opt = *opt_in;
    } else {
        qs_options_default(&opt);
        if (dt == QS_C128) opt.k_max = 3;  // blocks the float-float register tile applies
    }
    if (opt.k_max < 1 || opt.k_max > kMaxK) return fail(QS_ERR_ARG, "k_max outside 1..6");
    if (opt.fusion_effort < 0 || opt.fusion_effort > 1) return fail(QS_ERR_ARG, "fusion_effort must be 0 or 1");
    const int maxL = dt == QS_C64 ? 13 : 12;
    if (opt.tile_qubits != 0 && (opt.tile_qubits < 6 || opt.tile_qubits > maxL))
        return fail(QS_ERR_ARG, "tile_qubits outside 6..%d", maxL);
    if (opt.precision < QS_PREC_FP32 || opt.precision > QS_PREC_3XFP16)
        return fail(QS_ERR_ARG, "bad precision");
    std::vector<GateRec> blocks;
    qs_status st;
    if (opt.fuse) {
        FuseCache* fc = c->fuse_cache.get();
        st = opt.diag_clusters ? fuse_by_kind(c->n, c->gates, opt.k_max, blocks, opt.fusion_effort, fc)
                               : fuse_gates(c->n, c->gates, opt.k_max, blocks, opt.fusion_effort, fc);
        if (st != QS_OK) return st;
    } else {
        blocks = c->gates;
    }
    std::vector<Pass> passes;
    st = build_passes(c->n, dt, blocks, opt, passes);
    if (st != QS_OK) return st;
    for (Pass& ps : passes) {
        factor_tile_scalars(ps);
        if (ps.kind == PASS_TILE && !build_rtile_program(dt, ps, ps.rt)) ps.rt.nops = 0;
    }
    return plan_from_passes(c->n, dt, opt, std::move(passes), stream, out);
}

// A plan of ready passes: their matrices are uploaded, converted to the
// state's precision (in `stream` order when one is given).
qs_status qsgb::plan_from_passes(int n, qs_dtype dt, const qs_options& opt, std::vector<Pass>&& passes,
                                 cudaStream_t stream, qs_plan** out) {
    *out = nullptr;
    std::unique_ptr<qs_plan> p(new (std::nothrow) qs_plan);
    if (!p) return fail(QS_ERR_OOM, "host allocation failed");
    p->n = n;
    p->dt = dt;
    p->opt = opt;
    QS_CUDA(cudaGetDevice(&p->device));
    p->passes = std::move(passes);
    // upload every pass's matrices, converted to the state's precision
    size_t total = 0;
    for (Pass& ps : p->passes) {
        ps.dev_offset = total;
        total += ps.mats.size() / 2;
    }
    p->dev_elems = total;
    if (total) {
        const size_t esz = dt == QS_C64 ? 8 : 16;
        std::vector<char> host(total * esz);
        size_t at = 0;
        for (const Pass& ps : p->passes) {
            for (size_t i = 0; i < ps.mats.size(); ++i) {
                if (dt == QS_C64) ((float*)host.data())[2 * at + i] = (float)ps.mats[i];
                else ((double*)host.data())[2 * at + i] = ps.mats[i];
            }
            at += ps.mats.size() / 2;
        }
        if (stream) {
            // a pageable source is staged before the call returns, so `host` may go
            p->stream = stream;
            QS_CUDA(cudaMallocAsync(&p->dev_mats, total * esz, stream));
            cudaError_t e = cudaMemcpyAsync(p->dev_mats, host.data(), total * esz, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) {
                cudaFreeAsync(p->dev_mats, stream);
                return cuda_fail(e, "plan matrix upload");
            }
        } else {
            QS_CUDA(cudaMalloc(&p->dev_mats, total * esz));
            cudaError_t e = cudaMemcpy(p->dev_mats, host.data(), total * esz, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(p->dev_mats);
                return cuda_fail(e, "plan matrix upload");
            }
        }
    }
    *out = p.release();
    return QS_OK;
}

extern "C" {

qs_status qs_plan_destroy(qs_plan* p) {
    if (!p) return QS_OK;
    if (p->dev_mats) {
        if (p->stream) cudaFreeAsync(p->dev_mats, p->stream);
        else cudaFree(p->dev_mats);
    }
    delete p;
    return QS_OK;
}

qs_status qs_plan_info(const qs_plan* p, int* num_passes, int* num_launches, int* per_kind) {
    if (!p) return fail(QS_ERR_ARG, "null plan");
    if (num_passes) *num_passes = (int)p->passes.size();
    if (num_launches) *num_launches = (int)p->passes.size();
    if (per_kind) {
        for (int i = 0; i < 8; ++i) per_kind[i] = 0;
        for (const Pass& ps : p->passes) per_kind[ps.kind]++;
    }
    return QS_OK;
}

qs_status qs_plan_execute(qs_state* s, const qs_plan* p) { return qs_plan_execute_range(s, p, 0, -1); }

qs_status qs_plan_pass(const qs_plan* p, int i, int* kind, int* width, int* num_gates) {
    if (!p) return fail(QS_ERR_ARG, "null plan");
    if (i < 0 || i >= (int)p->passes.size()) return fail(QS_ERR_ARG, "pass index out of range");
    const Pass& ps = p->passes[i];
    if (kind) *kind = ps.kind;
    if (width) *width = ps.kind == PASS_TILE ? ps.L : ps.kind == PASS_TTILE ? 12 : ps.k;
    if (num_gates) *num_gates = ps.kind == PASS_TILE ? (int)ps.tgates.size() : ps.members;
    return QS_OK;
}

}  // extern "C"

// One pass on the state's stream; `dm` holds its matrices in the state's
// precision (the passes that take their matrix as a kernel argument ignore it).
static cudaError_t launch_pass(qs_state* s, const Pass& ps, const void* dm, int precision, int inject = 0) {
    switch (ps.kind) {
        case PASS_TILE:
            return ps.rt.nops > 0 ? launch_rtile(s->data, s->n, s->dt, ps, dm, s->stream)
                                  : launch_tile(s->data, s->n, s->dt, ps, dm, s->stream);
        case PASS_DENSE: return launch_dense(s->data, s->n, s->dt, ps.k, ps.qubits, ps.mats.data(), s->stream);
        case PASS_DIAG: return launch_diag(s->data, s->n, s->dt, ps.k, ps.qubits, ps.mats.data(), s->stream);
        case PASS_MONO: return launch_mono(s->data, s->n, s->dt, ps.k, ps.qubits, ps.mats.data(), s->stream);
        case PASS_GEMM:
            return launch_gemm(s->data, s->n, ps.k, ps.qubits, dm, precision, s->errflag, s->stream, inject, ps.swap_p);
        case PASS_DIAG_WIDE: return launch_diag_wide(s->data, s->n, s->dt, ps.wide, dm, s->stream);
        case PASS_TTILE: return launch_ttile(s->data, s->n, ps.tt, dm, s->errflag, s->stream);
        case PASS_DENSE_SMEM: return launch_dense_smem(s->data, s->n, s->dt, ps.k, ps.qubits, dm, s->stream);
    }
    return cudaErrorInvalidValue;
}

// one pinned staging buffer per host thread for the streamed path's matrix
// uploads (PinnedStage: a copy from pageable memory may wait for the
// stream's earlier work before it is staged)
namespace {
thread_local PinnedStage t_stage;
// a copy stream per host thread (and device) for those uploads, so that a
// pass's matrix copy does not sit between two kernels of the state's stream
struct CopyLane {
    int dev = -1;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    ~CopyLane() {
        if (ev) cudaEventDestroy(ev);
        if (cs) cudaStreamDestroy(cs);
    }
    cudaError_t get(int device) {
        if (dev == device && cs) return cudaSuccess;
        if (ev) cudaEventDestroy(ev);
        if (cs) cudaStreamDestroy(cs);
        ev = nullptr;
        cs = nullptr;
        dev = device;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        return e;
    }
};
thread_local CopyLane t_copy;
}  // namespace

// The library's stream-ordered memory pool on the current device: it keeps
// what it has reserved between calls (the adjoint sweep's scratch, tens to
// hundreds of MB, is then not mapped again on every call); the memory is
// held until the process exits.
cudaError_t qsgb::lib_malloc_async(void** ptr, size_t bytes, cudaStream_t st) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&pools[dev], &props);
            if (e != cudaSuccess) {
                pools[dev] = nullptr;
                return e;
            }
            uint64_t keep = ~0ull;
            e = cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) return e;
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}


// Fuse and run together (qs_apply_circuit and the adjoint gradient's forward
// on the tensor cores): a host thread runs the block search and hands over
// each group as soon as it is found (all at once when the circuit's grouping
// is cached); worker threads form the groups' blocks (FP64 products) and
// passes in parallel; this thread uploads each pass's matrix through pinned
// staging and launches the passes in order, so the GPU runs pass i while
// later blocks are being found and multiplied.  Passes wait in a look-ahead
// window so that the bit-0 placement of the planned path (bit0_plan) can
// keep qubit 0 out of the 6-qubit passes' targets here too: the window's
// leading run of 6-qubit passes is planned from the current exchange state,
// the first pass is committed and launched.  The window grows with the
// passes already queued (so the GPU starts at once, also when the grouping
// comes from the cache all at once) up to 3 passes while the search runs and
// 8 once it is done.
qs_status qsgb::apply_streamed(qs_state* s, const qs_circuit* c, const qs_options& opt,
                               std::vector<GateRec>* blocks_out) {
    constexpr size_t kWindow = 3, kWindowDone = 8;
    const int n = c->n;
    const size_t esz = s->amp_bytes();
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::vector<int>> groups;           // in search order
    std::vector<std::unique_ptr<Pass>> formed;      // formed[i]: the pass of group i, once ready
    std::deque<GateRec> kept;                       // kept[i]: group i's block (blocks_out only)
    size_t next_group = 0;                          // the next group a worker takes
    bool done = false, stop = false;
    qs_status fst = QS_OK;
    std::string fmsg;
    std::thread search([&]() {
        const qs_status st = fuse_each(n, c->gates, opt.k_max, opt.fusion_effort, c->fuse_cache.get(),
                                       [&](std::vector<int>&& g) {
                                           std::lock_guard<std::mutex> lk(mu);
                                           groups.push_back(std::move(g));
                                           formed.emplace_back();
                                           if (blocks_out) kept.emplace_back();
                                           cv.notify_all();
                                       });
        std::lock_guard<std::mutex> lk(mu);
        fst = st;
        if (st != QS_OK) fmsg = qs_last_error();
        done = true;
        cv.notify_all();
    });
    auto form = [&](size_t i, const std::vector<int>& g) {  // group i's block and pass
        GateRec b;
        block_product(n, c->gates, g, b);
        std::unique_ptr<Pass> p(new Pass);
        single_block_pass(n, s->dt, opt, b, *p);
        factor_tile_scalars(*p);
        std::lock_guard<std::mutex> lk(mu);
        formed[i] = std::move(p);
        if (blocks_out) kept[i] = std::move(b);
        cv.notify_all();
    };
    auto worker = [&]() {
        for (;;) {
            std::vector<int> g;
            size_t i;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&]() { return stop || next_group < groups.size() || done; });
                if (stop || next_group >= groups.size()) {
                    if (stop || done) return;
                    continue;
                }
                i = next_group++;
                g = groups[i];
            }
            form(i, g);
        }
    };
    // the workers start once the first pass is launched: the first block is
    // formed on this thread, so the GPU does not wait for threads to start
    std::vector<std::thread> workers;
    const unsigned nw = std::max(1u, std::min(4u, host_threads(4)));
    auto start_workers = [&]() {
        if (workers.empty())
            for (unsigned w = 0; w < nw; ++w) workers.emplace_back(worker);
    };

    qs_status st = QS_OK;
    int dev = 0;
    cudaError_t ge = cudaGetDevice(&dev);
    if (ge == cudaSuccess) ge = t_stage.reserve(2u << 20, dev);  // 64 complex64 6-qubit matrices
    if (ge == cudaSuccess) ge = t_copy.get(dev);
    // the device copies of the staged matrices: one buffer for the call,
    // filled on the copy stream once its allocation is ordered there
    char* dbuf = nullptr;
    if (ge == cudaSuccess) ge = cudaMallocAsync(reinterpret_cast<void**>(&dbuf), t_stage.cap, s->stream);
    if (ge == cudaSuccess) ge = cudaEventRecord(t_copy.ev, s->stream);
    if (ge == cudaSuccess) ge = cudaStreamWaitEvent(t_copy.cs, t_copy.ev, 0);
    if (ge != cudaSuccess) st = cuda_fail(ge, "pinned staging");
    size_t stage_at = 0;  // bytes of the staging buffer used by this call
    auto launch_one = [&](Pass& p) {
        void* dm = nullptr;    // a matrix allocated for this pass alone
        void* mine = nullptr;  // where the pass reads its matrix
        const size_t elems = p.mats.size() / 2;
        cudaError_t e = cudaSuccess;
        if (elems && p.kind != PASS_DENSE && p.kind != PASS_DIAG && p.kind != PASS_MONO) {
            const size_t bytes = elems * esz;
            std::vector<char> host;
            if (dbuf && stage_at + bytes <= t_stage.cap) {  // pinned, on the copy stream
                char* src = t_stage.p + stage_at;
                for (size_t i = 0; i < p.mats.size(); ++i) {
                    if (s->dt == QS_C64) ((float*)src)[i] = (float)p.mats[i];
                    else ((double*)src)[i] = p.mats[i];
                }
                mine = dbuf + stage_at;
                stage_at += (bytes + 255) & ~(size_t)255;
                e = cudaMemcpyAsync(mine, src, bytes, cudaMemcpyHostToDevice, t_copy.cs);
                if (e == cudaSuccess) e = cudaEventRecord(t_copy.ev, t_copy.cs);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, t_copy.ev, 0);
            } else {  // beyond the staging buffer: a pageable source, staged by the driver
                host.resize(bytes);
                for (size_t i = 0; i < p.mats.size(); ++i) {
                    if (s->dt == QS_C64) ((float*)host.data())[i] = (float)p.mats[i];
                    else ((double*)host.data())[i] = p.mats[i];
                }
                e = cudaMallocAsync(&dm, bytes, s->stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(dm, host.data(), bytes, cudaMemcpyHostToDevice, s->stream);
                mine = dm;
            }
        }
        if (e == cudaSuccess) e = launch_pass(s, p, mine, opt.precision);
        if (dm) cudaFreeAsync(dm, s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "streamed pass");
    };
    int xs = -1;  // exchange state: -1 standard order, else the bit exchanged with bit 0
    auto restore = [&]() {  // back to standard order with a permutation pass
        GateRec g;
        g.k = 2;
        g.qubits[0] = xs;
        g.qubits[1] = 0;
        g.m.assign(32, 0.0);
        const int perm[4] = {0, 2, 1, 3};
        for (int r = 0; r < 4; ++r) g.m[2 * (r * 4 + perm[r])] = 1.0;
        g.kind = QS_GATE_MONOMIAL;
        Pass p;
        single_block_pass(n, s->dt, opt, g, p);
        launch_one(p);
        xs = -1;
    };
    std::deque<Pass> pending;
    size_t launched = 0;
    auto drain = [&](bool final, bool search_done) {
        const size_t win = std::min(search_done ? kWindowDone : kWindow, launched);
        while (st == QS_OK && !pending.empty() && (final || pending.size() > win)) {
            Pass& p0 = pending.front();
            if (p0.kind == PASS_GEMM) {
                std::vector<const Pass*> run;
                size_t k = 0;
                while (k < pending.size() && pending[k].kind == PASS_GEMM) run.push_back(&pending[k++]);
                const bool end_free = !final && k == pending.size();  // the run may go on past the window
                std::vector<int> choice;
                const int bc = bit0_plan(n, run, xs, end_free, choice) >= 0 ? choice[0] : -2;
                xs = bit0_apply(p0, xs, bc);
            } else if (xs >= 0) {
                if (p0.kind == PASS_DENSE || p0.kind == PASS_DIAG || p0.kind == PASS_MONO) {
                    for (int i = 0; i < p0.k; ++i)  // any qubit order: relabel in place
                        p0.qubits[i] = p0.qubits[i] == 0 ? xs : p0.qubits[i] == xs ? 0 : p0.qubits[i];
                } else {
                    restore();
                }
            }
            launch_one(p0);
            pending.pop_front();
            ++launched;
        }
        if (final && st == QS_OK && xs >= 0) restore();
    };
    {
        std::vector<int> g0;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&]() { return !groups.empty() || done; });
            if (!groups.empty() && next_group == 0) {
                next_group = 1;
                g0 = groups[0];
            }
        }
        if (!g0.empty()) form(0, g0);
    }
    for (size_t i = 0;; ++i) {
        std::unique_ptr<Pass> p;
        bool search_done;
        if (i == 1) start_workers();
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&]() { return (i < formed.size() && formed[i]) || (done && i >= groups.size()); });
            if (i >= groups.size()) break;
            p = std::move(formed[i]);
            search_done = done;
        }
        if (st != QS_OK) continue;  // drain the search and workers after a failure
        pending.push_back(std::move(*p));
        drain(false, search_done);
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
        cv.notify_all();
    }
    for (auto& w : workers) w.join();
    search.join();
    if (fst != QS_OK) {
        if (dbuf) cudaFreeAsync(dbuf, s->stream);
        if (t_stage.done) cudaEventRecord(t_stage.done, s->stream);
        return fail(fst, "%s", fmsg.c_str());
    }
    drain(true, true);
    if (dbuf) cudaFreeAsync(dbuf, s->stream);  // after the passes, which waited for every copy
    if (t_stage.done) cudaEventRecord(t_stage.done, s->stream);  // the staging buffer is free once this passes
    if (blocks_out && st == QS_OK) blocks_out->assign(std::make_move_iterator(kept.begin()), std::make_move_iterator(kept.end()));
    return st;
}

extern "C" {

qs_status qs_plan_execute_range(qs_state* s, const qs_plan* p, int first, int count) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (!p) return fail(QS_ERR_ARG, "null plan");
    const int np = (int)p->passes.size();
    if (first < 0 || first > np) return fail(QS_ERR_ARG, "first pass out of range");
    const int last = count < 0 ? np : std::min(np, first + count);
    if (p->n != s->n || p->dt != s->dt) return fail(QS_ERR_ARG, "plan built for another n/dtype");
    if (p->device != s->device) return fail(QS_ERR_ARG, "plan built on another device");
    const size_t esz = s->dt == QS_C64 ? 8 : 16;
    for (int pi = first; pi < last; ++pi) {
        const Pass& ps = p->passes[pi];
        const char* dm = (const char*)p->dev_mats + ps.dev_offset * esz;
        cudaError_t e = launch_pass(s, ps, dm, p->opt.precision, p->opt.inject_mma_timeout);
        if (e != cudaSuccess) return cuda_fail(e, "pass launch");
    }
    return QS_OK;
}

qs_status qs_apply_circuit(qs_state* s, const qs_circuit* c, qs_precision prec) {
    if (!s || !c) return fail(QS_ERR_ARG, "null argument");
    if (c->n != s->n) return fail(QS_ERR_ARG, "circuit and state qubit counts differ");
    qs_options opt;
    qs_options_default(&opt);
    opt.precision = prec;
    if (prec != QS_PREC_FP32 && s->dt == QS_C64) opt.k_max = 6;  // 6-qubit blocks on the tensor cores
    if (s->dt == QS_C128) opt.k_max = 3;  // blocks the float-float register tile applies
    if (opt.precision < QS_PREC_FP32 || opt.precision > QS_PREC_3XFP16) return fail(QS_ERR_ARG, "bad precision");
    if (s->dt == QS_C64 && prec != QS_PREC_FP32 && gemm_supported(s->n, 6)) {
        qs_status st = check_state(s);
        if (st != QS_OK) return st;
        return apply_streamed(s, c, opt);
    }
    qs_plan* p = nullptr;
    // matrices allocated and freed in the state's stream order: no synchronisation
    qs_status st = plan_create_on(c, s->dt, &opt, s->stream, &p);
    if (st != QS_OK) return st;
    st = qs_plan_execute(s, p);
    qs_plan_destroy(p);
    return st;
}

// ------------------------------------------------------------- read back

qs_status qs_amplitudes(const qs_state* s, uint64_t first, uint64_t count, double* out) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (!out && count) return fail(QS_ERR_ARG, "null output");
    if (first > s->size() || count > s->size() - first) return fail(QS_ERR_ARG, "range out of bounds");
    if (!count) return QS_OK;
    const size_t esz = s->amp_bytes();
    const char* src = (const char*)s->data + first * esz;
    if (s->dt == QS_C128) {
        QS_CUDA(cudaMemcpyAsync(out, src, count * esz, cudaMemcpyDeviceToHost, s->stream));
        QS_CUDA(cudaStreamSynchronize(s->stream));
        return check_device_flag(s);
    }
    // complex64: copy in chunks through a host buffer, widen to FP64
    const uint64_t chunk = 1ull << 22;
    std::vector<float> buf((size_t)std::min(count, chunk) * 2);
    for (uint64_t at = 0; at < count; at += chunk) {
        const uint64_t c = std::min(chunk, count - at);
        QS_CUDA(cudaMemcpyAsync(buf.data(), src + at * esz, c * esz, cudaMemcpyDeviceToHost, s->stream));
        QS_CUDA(cudaStreamSynchronize(s->stream));
        for (uint64_t i = 0; i < 2 * c; ++i) out[2 * at + i] = (double)buf[i];
    }
    return check_device_flag(s);
}

qs_status qs_norm(const qs_state* s, double* out) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (!out) return fail(QS_ERR_ARG, "null output");
    double* res = result_area(s);
    QS_CUDA(launch_norm(s->data, s->n, s->dt, s->scratch, res, s->stream));
    QS_CUDA(cudaMemcpyAsync(s->host_pinned, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA(cudaStreamSynchronize(s->stream));
    *out = s->host_pinned[0];
    return check_device_flag(s);
}

qs_status qs_state_sync(qs_state* s) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    QS_CUDA(cudaStreamSynchronize(s->stream));
    return check_device_flag(s);
}

// ------------------------------------------------------------ observables

qs_status qs_pauli_sum_create(int n, qs_pauli_sum** out) {
    if (!out) return fail(QS_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (n < 1 || n > kMaxQubits) return fail(QS_ERR_ARG, "n=%d outside 1..%d", n, kMaxQubits);
    qs_pauli_sum* h = new (std::nothrow) qs_pauli_sum;
    if (!h) return fail(QS_ERR_OOM, "host allocation failed");
    h->n = n;
    *out = h;
    return QS_OK;
}

qs_status qs_pauli_sum_destroy(qs_pauli_sum* h) {
    delete h;
    return QS_OK;
}

qs_status qs_pauli_sum_add(qs_pauli_sum* h, double coeff, const int* qubits, const char* paulis, int len) {
    if (!h || (len > 0 && (!qubits || !paulis))) return fail(QS_ERR_ARG, "null argument");
    if (len < 0 || len > h->n) return fail(QS_ERR_ARG, "bad term length %d", len);
    if (!(coeff == coeff)) return fail(QS_ERR_ARG, "coefficient is NaN");
    qs_pauli_sum::Term t{coeff, 0, 0, 0};
    uint64_t seen = 0;
    for (int i = 0; i < len; ++i) {
        const int q = qubits[i];
        if (q < 0 || q >= h->n) return fail(QS_ERR_ARG, "qubit %d out of range", q);
        if ((seen >> q) & 1) return fail(QS_ERR_ARG, "duplicate qubit %d in term", q);
        seen |= 1ull << q;
        switch (paulis[i]) {
            case 'I': break;
            case 'X': t.xmask |= 1ull << q; break;
            case 'Y': t.xmask |= 1ull << q; t.zmask |= 1ull << q; t.ny++; break;
            case 'Z': t.zmask |= 1ull << q; break;
            default: return fail(QS_ERR_ARG, "bad Pauli letter '%c'", paulis[i]);
        }
    }
    h->terms.push_back(t);
    return QS_OK;
}

qs_status qs_expectation(const qs_state* s, const qs_pauli_sum* h, double* out) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (!h || !out) return fail(QS_ERR_ARG, "null argument");
    if (h->n != s->n) return fail(QS_ERR_ARG, "Hamiltonian and state qubit counts differ");
    double* res = result_area(s);
    QS_CUDA(launch_expectation(s->data, s->n, s->dt, *h, s->scratch, res, s->stream));
    QS_CUDA(cudaMemcpyAsync(s->host_pinned, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA(cudaStreamSynchronize(s->stream));
    *out = s->host_pinned[0];
    return QS_OK;
}

qs_status qs_apply_pauli_sum(const qs_state* psi, const qs_pauli_sum* h, qs_state* out) {
    qs_status st = check_state(psi);
    if (st != QS_OK) return st;
    st = check_state(out);
    if (st != QS_OK) return st;
    if (!h) return fail(QS_ERR_ARG, "null Hamiltonian");
    if (h->n != psi->n || out->n != psi->n || out->dt != psi->dt)
        return fail(QS_ERR_ARG, "shapes differ");
    if (out->data == psi->data) return fail(QS_ERR_ARG, "output must not alias the input");
    QS_CUDA(launch_apply_pauli_sum(psi->data, out->data, psi->n, psi->dt, *h, out->stream));
    return QS_OK;
}

}  // extern "C"
