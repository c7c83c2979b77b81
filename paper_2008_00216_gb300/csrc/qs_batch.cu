// Batched execution: many circuits of uneven width in one persistent launch.
//
// Circuits with n <= L (the tile width) run entirely inside one CTA: the
// state starts as |0...0> in shared memory, every fused block is applied
// there and the result is written once.  Wider circuits are split into
// shared-memory tile passes (the same grouping as the single-circuit plan,
// every group a tile); each pass is cut into work items of a few tiles.
// Items are queued pass-major across circuits and claimed through an atomic
// ticket.  An item of pass p waits, with a bounded spin, until the
// circuit's items of earlier passes are finished -- those were claimed
// earlier by CTAs that are already running, so the wait always ends unless
// something has gone wrong, in which case the error flag is raised and the
// CTA stops.  The first pass of a circuit synthesises |0...0> in shared
// memory instead of reading it.  State traffic of the wide circuits (up to
// 2^22 amplitudes, 32 MB in complex64) mostly stays in the 129 MB L2.
#include <algorithm>
#include <map>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include "qs_device.cuh"
#include "qs_internal.h"
#include "qs_tile.cuh"

namespace qsgb {
namespace batch {

struct Circ {
    uint64_t off;      // amplitude offset of the state in the caller's buffer
    int n;
    int pass0;         // first pass in the pass array
    int npass;
    int pad;
};
struct PassD {
    int L, b, ngates, gate0;
    int pos[16];
    uint32_t items_before;   // items of this circuit in earlier passes
    uint32_t pad;
};
struct Item {
    int circ, pass;
    uint32_t t0, t1;   // tiles [t0, t1) of the pass
};

constexpr long long kTimeout = 4ll << 30;   // ~2 s of clock64

template <typename R>
__global__ void __launch_bounds__(256) k_batch(typename C2<R>::T* __restrict__ states, const Circ* __restrict__ circs,
                                               const PassD* __restrict__ passes, const TileGate* __restrict__ gates,
                                               const typename C2<R>::T* __restrict__ mats, const Item* __restrict__ items,
                                               int nitems, int Lmax, unsigned* counters, int* err) {
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    T* mbuf = tile + (1u << Lmax);                                   // one gate matrix (<= 16 x 16)
    uint64_t* rowoff = reinterpret_cast<uint64_t*>(mbuf + 256);
    __shared__ int s_item, s_fail;
    unsigned* ticket = counters;
    unsigned* finished = counters + 1;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = (int)atomicAdd(ticket, 1u);
            s_fail = 0;
        }
        __syncthreads();
        const int id = s_item;
        if (id >= nitems) break;
        const Item it = items[id];
        const Circ c = circs[it.circ];
        const PassD& p = passes[c.pass0 + it.pass];
        if (threadIdx.x == 0 && p.items_before > 0) {
            // wait for this circuit's earlier passes (claimed earlier, running)
            const long long t0 = clock64();
            while (atomicAdd(&finished[it.circ], 0u) < p.items_before) {
                if (*(volatile int*)err || clock64() - t0 > kTimeout) {
                    atomicExch(err, 1);
                    s_fail = 1;
                    break;
                }
            }
            __threadfence();
        }
        __syncthreads();
        if (s_fail) break;
        const int L = p.L, b = p.b;
        const uint32_t rowlen = 1u << b;
        for (uint32_t h = threadIdx.x; h < (1u << (L - b)); h += blockDim.x) {
            uint64_t o = 0;
            for (int i = b; i < L; ++i)
                if ((h >> (i - b)) & 1) o |= 1ull << p.pos[i];
            rowoff[h] = o;
        }
        __syncthreads();
        T* psi = states + c.off;
        for (uint32_t t = it.t0; t < it.t1; ++t) {
            uint64_t base = t;
            for (int i = 0; i < L; ++i) base = insert_zero(base, p.pos[i]);
            if (it.pass == 0) {  // |0...0>: amplitude 1 at global index 0 only
                for (uint32_t e = threadIdx.x; e < (1u << L); e += blockDim.x) {
                    T v;
                    v.x = (base == 0 && e == 0) ? (R)1 : (R)0;
                    v.y = 0;
                    tile[e] = v;
                }
            } else {
                tile_gather<T, true>(tile, psi, base, rowoff, b, L);
            }
            __syncthreads();
            for (int gi = 0; gi < p.ngates; ++gi) {
                const TileGate g = gates[p.gate0 + gi];
                const int D = 1 << g.k;
                for (int i = threadIdx.x; i < D * D; i += blockDim.x) mbuf[i] = mats[g.mat + i];
                __syncthreads();
                if (g.kind == QS_GATE_DIAGONAL) {
                    tile_diag(tile, L, g, mbuf);
                } else {
                    switch (g.k) {
                        case 1: tile_dense<T, 1>(tile, L, g, mbuf); break;
                        case 2: tile_dense<T, 2>(tile, L, g, mbuf); break;
                        case 3: tile_dense<T, 3>(tile, L, g, mbuf); break;
                        case 4: tile_dense<T, 4>(tile, L, g, mbuf); break;
                        default: break;  // excluded by the planner
                    }
                }
                __syncthreads();
            }
            for (uint32_t e = threadIdx.x; e < (1u << L); e += blockDim.x)
                __stcg(psi + base + rowoff[e >> b] + (e & (rowlen - 1)), tile[e]);
            __syncthreads();
        }
        // publish: every thread's stores are ordered before the count
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&finished[it.circ], 1u);
    }
}

}  // namespace batch
}  // namespace qsgb

struct qs_batch {
    int count = 0;
    qs_dtype dt = QS_C64;
    qs_options opt{};
    int device = 0;
    int Lmax = 0;
    std::vector<uint64_t> offsets;   // count + 1
    int nitems = 0, npasses = 0, ngates = 0;
    void* d_circ = nullptr;
    void* d_pass = nullptr;
    void* d_gates = nullptr;
    void* d_mats = nullptr;
    void* d_items = nullptr;
    unsigned* d_counters = nullptr;
    int* d_err = nullptr;
    int grid = 0;
    size_t smem = 0;
    // captured launch (reset counters + kernel) for one state buffer
    cudaGraphExec_t exec = nullptr;
    void* exec_states = nullptr;
    cudaStream_t last_stream = nullptr;
};

namespace qsgb {

static void free_batch_device(qs_batch* b) {
    cudaFree(b->d_circ);
    cudaFree(b->d_pass);
    cudaFree(b->d_gates);
    cudaFree(b->d_mats);
    cudaFree(b->d_items);
    cudaFree(b->d_counters);
    if (b->exec) cudaGraphExecDestroy(b->exec);
}

template <typename V>
static cudaError_t upload(void** dst, const std::vector<V>& v) {
    const size_t bytes = std::max<size_t>(1, v.size()) * sizeof(V);
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice);
    return e;
}

// Every group of fused blocks becomes a tile pass over local bits `pos`.
static void tile_passes(int n, qs_dtype dt, const std::vector<GateRec>& blocks, int L, std::vector<Pass>& out) {
    qs_options o;
    qs_options_default(&o);
    o.use_tile = 1;
    o.tile_qubits = L;
    std::vector<Pass> ps;
    build_passes(n, dt, blocks, o, ps);
    out.clear();
    for (Pass& p : ps) {
        if (p.kind == PASS_TILE) {
            out.push_back(std::move(p));
            continue;
        }
        // a single-block pass: a tile whose bits are the low bits plus the block's qubits
        Pass t;
        t.kind = PASS_TILE;
        uint64_t S = 0;
        for (int i = 0; i < p.k; ++i) S |= 1ull << p.qubits[i];
        for (int q = 0; q < n && __builtin_popcountll(S) < L; ++q) S |= 1ull << q;
        int local_of[kMaxQubits];
        int j = 0;
        for (int q = 0; q < n; ++q)
            if ((S >> q) & 1) {
                local_of[q] = j;
                t.pos[j++] = q;
            }
        t.L = j;
        TileGate tg{};
        tg.k = (uint8_t)p.k;
        tg.kind = (uint8_t)p.gate_kind;
        for (int i = 0; i < p.k; ++i) tg.q[i] = (uint8_t)local_of[p.qubits[i]];
        tg.mat = 0;
        t.tgates.push_back(tg);
        t.mats = p.mats;
        out.push_back(std::move(t));
    }
}

}  // namespace qsgb

using namespace qsgb;

extern "C" {

qs_status qs_batch_create(const qs_circuit* const* circuits, int count, qs_dtype dt, const qs_options* opt_in,
                          qs_batch** out) {
    if (!out || !circuits) return fail(QS_ERR_ARG, "null argument");
    *out = nullptr;
    if (count < 1) return fail(QS_ERR_ARG, "empty batch");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_ERR_ARG, "bad dtype");
    qs_options opt;
    if (opt_in) opt = *opt_in;
    else {
        qs_options_default(&opt);
        opt.k_max = 3;
    }
    if (opt.k_max < 1 || opt.k_max > 4) return fail(QS_ERR_ARG, "batched k_max must be 1..4");
    const int Lmax = opt.tile_qubits ? opt.tile_qubits : (dt == QS_C64 ? 13 : 12);
    if (Lmax < 6 || Lmax > (dt == QS_C64 ? 13 : 12)) return fail(QS_ERR_ARG, "batched tile_qubits out of range");
    std::unique_ptr<qs_batch> b(new (std::nothrow) qs_batch);
    if (!b) return fail(QS_ERR_OOM, "host allocation failed");
    b->count = count;
    b->dt = dt;
    b->opt = opt;
    b->Lmax = Lmax;
    QS_CUDA(cudaGetDevice(&b->device));

    std::vector<batch::Circ> circs(count);
    std::vector<batch::PassD> passes;
    std::vector<TileGate> gates;
    std::vector<double> mats;   // interleaved complex, converted on upload
    std::vector<std::vector<batch::Item>> per_pass_items;  // large circuits, indexed by pass
    std::vector<batch::Item> small_items;
    std::vector<std::pair<double, int>> small_cost;
    b->offsets.assign(count + 1, 0);
    for (int c = 0; c < count; ++c) {
        const qs_circuit* qc = circuits[c];
        if (!qc) return fail(QS_ERR_ARG, "null circuit %d", c);
        if (qc->n > 30) return fail(QS_ERR_UNSUPPORTED, "batched circuits are limited to 30 qubits");
        b->offsets[c + 1] = b->offsets[c] + (1ull << qc->n);
        std::vector<GateRec> blocks;
        qs_status st = fuse_gates(qc->n, qc->gates, opt.k_max, blocks);
        if (st != QS_OK) return st;
        for (const GateRec& g : blocks)
            if (g.kind != QS_GATE_DIAGONAL && g.k > 4)
                return fail(QS_ERR_UNSUPPORTED, "circuit %d has a dense gate on more than 4 qubits", c);
        circs[c].off = b->offsets[c];
        circs[c].n = qc->n;
        circs[c].pass0 = (int)passes.size();
        const int n = qc->n;
        if (n <= Lmax) {
            // the whole circuit in one CTA: one pass over all n bits
            batch::PassD p{};
            p.L = n;
            p.b = n;
            p.gate0 = (int)gates.size();
            for (int i = 0; i < n; ++i) p.pos[i] = i;
            double cost = 0;
            for (const GateRec& g : blocks) {
                TileGate tg{};
                tg.k = (uint8_t)g.k;
                tg.kind = (uint8_t)g.kind;
                for (int i = 0; i < g.k; ++i) tg.q[i] = (uint8_t)g.qubits[i];
                tg.mat = (uint32_t)(mats.size() / 2);
                mats.insert(mats.end(), g.m.begin(), g.m.end());
                gates.push_back(tg);
                cost += (double)(1 << g.k);
            }
            p.ngates = (int)(gates.size() - p.gate0);
            p.items_before = 0;
            passes.push_back(p);
            circs[c].npass = 1;
            small_items.push_back({c, 0, 0, 1});
            small_cost.push_back({cost * (double)(1ull << n), (int)small_items.size() - 1});
            continue;
        }
        std::vector<Pass> tp;
        tile_passes(n, dt, blocks, Lmax, tp);
        uint32_t before = 0;
        for (size_t pi = 0; pi < tp.size(); ++pi) {
            const Pass& ps = tp[pi];
            batch::PassD p{};
            p.L = ps.L;
            int bb = 0;
            while (bb < ps.L && ps.pos[bb] == bb) ++bb;
            p.b = bb;
            if (ps.L > Lmax || ps.L - bb > Lmax - 4)
                return fail(QS_ERR_STATE, "internal: tile pass wider than the batched kernel's buffers");
            for (int i = 0; i < ps.L; ++i) p.pos[i] = ps.pos[i];
            p.gate0 = (int)gates.size();
            const uint32_t mat0 = (uint32_t)(mats.size() / 2);
            for (const TileGate& g0 : ps.tgates) {
                TileGate g = g0;
                g.mat += mat0;
                gates.push_back(g);
            }
            mats.insert(mats.end(), ps.mats.begin(), ps.mats.end());
            p.ngates = (int)ps.tgates.size();
            p.items_before = before;
            passes.push_back(p);
            const uint32_t ntiles = 1u << (n - ps.L);
            const uint32_t chunk = std::max<uint32_t>(1, std::min<uint32_t>(8, ntiles / 16));
            if (per_pass_items.size() <= pi) per_pass_items.resize(pi + 1);
            for (uint32_t t0 = 0; t0 < ntiles; t0 += chunk) {
                per_pass_items[pi].push_back({c, (int)pi, t0, std::min(ntiles, t0 + chunk)});
                ++before;
            }
        }
        circs[c].npass = (int)tp.size();
    }
    if (opt.inject_wait_timeout) {
        // testing: the last pass of the last wide circuit waits for a count
        // that is never reached, so its bounded wait runs out
        for (int c = count - 1; c >= 0; --c)
            if (circs[c].npass > 1) {
                passes[circs[c].pass0 + circs[c].npass - 1].items_before = 0xFFFFFFFFu;
                break;
            }
    }
    // queue: the whole-in-one-CTA circuits, most expensive first, then the
    // wide circuits' items pass-major across circuits
    std::sort(small_cost.begin(), small_cost.end(), [](auto& x, auto& y) { return x.first > y.first; });
    std::vector<batch::Item> items;
    for (auto& sc : small_cost) items.push_back(small_items[sc.second]);
    for (auto& v : per_pass_items) items.insert(items.end(), v.begin(), v.end());
    b->nitems = (int)items.size();
    b->npasses = (int)passes.size();
    b->ngates = (int)gates.size();

    cudaError_t e = upload(&b->d_circ, circs);
    if (e == cudaSuccess) e = upload(&b->d_pass, passes);
    if (e == cudaSuccess) e = upload(&b->d_gates, gates);
    if (e == cudaSuccess) e = upload(&b->d_items, items);
    if (e == cudaSuccess) {
        if (dt == QS_C64) {
            std::vector<float> f(mats.begin(), mats.end());
            e = upload(&b->d_mats, f);
        } else {
            e = upload(&b->d_mats, mats);
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(unsigned) * (count + 1) + sizeof(int));
    if (e != cudaSuccess) {
        free_batch_device(b.get());
        return cuda_fail(e, "batch upload");
    }
    b->d_err = reinterpret_cast<int*>(b->d_counters + count + 1);
    QS_CUDA(cudaMemset(b->d_err, 0, sizeof(int)));
    const size_t esz = dt == QS_C64 ? 8 : 16;
    // tile + one gate matrix + row offsets (tiles keep >= 4 low bits per row)
    b->smem = esz * ((1u << Lmax) + 256) + sizeof(uint64_t) * (1u << (Lmax - 4));
    int per_sm = 0;
    if (dt == QS_C64) {
        QS_CUDA(allow_max_dynamic_smem(batch::k_batch<float>));
        QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch::k_batch<float>, 256, b->smem));
    } else {
        QS_CUDA(allow_max_dynamic_smem(batch::k_batch<double>));
        QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch::k_batch<double>, 256, b->smem));
    }
    b->grid = std::max(1, std::min(b->nitems, num_sms() * std::max(1, per_sm)));
    *out = b.release();
    return QS_OK;
}

qs_status qs_batch_layout(const qs_batch* b, uint64_t* offsets) {
    if (!b || !offsets) return fail(QS_ERR_ARG, "null argument");
    for (int i = 0; i <= b->count; ++i) offsets[i] = b->offsets[i];
    return QS_OK;
}

qs_status qs_batch_info(const qs_batch* b, int* items, int* passes, int* gates, int* grid) {
    if (!b) return fail(QS_ERR_ARG, "null batch");
    if (items) *items = b->nitems;
    if (passes) *passes = b->npasses;
    if (gates) *gates = b->ngates;
    if (grid) *grid = b->grid;
    return QS_OK;
}

static cudaError_t batch_enqueue(qs_batch* b, void* states, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned) * (b->count + 1), st);
    if (e != cudaSuccess) return e;
    if (b->dt == QS_C64)
        batch::k_batch<float><<<b->grid, 256, b->smem, st>>>(
            (float2*)states, (const batch::Circ*)b->d_circ, (const batch::PassD*)b->d_pass, (const TileGate*)b->d_gates,
            (const float2*)b->d_mats, (const batch::Item*)b->d_items, b->nitems, b->Lmax, b->d_counters, b->d_err);
    else
        batch::k_batch<double><<<b->grid, 256, b->smem, st>>>(
            (double2*)states, (const batch::Circ*)b->d_circ, (const batch::PassD*)b->d_pass,
            (const TileGate*)b->d_gates, (const double2*)b->d_mats, (const batch::Item*)b->d_items, b->nitems, b->Lmax,
            b->d_counters, b->d_err);
    return cudaGetLastError();
}

qs_status qs_batch_run(qs_batch* b, void* device_states, void* stream) {
    if (!b || !device_states) return fail(QS_ERR_ARG, "null argument");
    if (((uintptr_t)device_states) & 15) return fail(QS_ERR_ARG, "state buffer not 16-byte aligned");
    int dev = -1;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) return fail(QS_ERR_ARG, "batch built on device %d, device %d current", b->device, dev);
    cudaStream_t st = (cudaStream_t)stream;
    b->last_stream = st;
    if (!b->exec || b->exec_states != device_states) {
        // capture "reset counters + persistent kernel" once per state buffer
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaStream_t cap;
        QS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = batch_enqueue(b, device_states, cap);
            e = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
        b->exec_states = device_states;
    }
    QS_CUDA(cudaGraphLaunch(b->exec, st));
    return QS_OK;
}

qs_status qs_batch_sync(qs_batch* b) {
    if (!b) return fail(QS_ERR_ARG, "null batch");
    QS_CUDA(cudaStreamSynchronize(b->last_stream));
    int flag = 0;
    QS_CUDA(cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        QS_CUDA(cudaMemset(b->d_err, 0, sizeof(int)));
        return fail(QS_ERR_TIMEOUT, "a batched work item waited too long for its circuit's earlier passes");
    }
    return QS_OK;
}

qs_status qs_batch_destroy(qs_batch* b) {
    if (!b) return QS_OK;
    cudaDeviceSynchronize();
    free_batch_device(b);
    delete b;
    return QS_OK;
}

qs_status qs_batch_autotune(const qs_circuit* const* circuits, int count, qs_dtype dt, void* device_states, void* stream,
                            qs_options* best) {
    if (!best) return fail(QS_ERR_ARG, "null output");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    QS_CUDA(cudaEventCreate(&e0));
    QS_CUDA(cudaEventCreate(&e1));
    float best_ms = -1.f;
    const int Ls[2] = {dt == QS_C64 ? 13 : 12, dt == QS_C64 ? 12 : 11};
    for (int k = 2; k <= 4; ++k)
        for (int L : Ls) {
            qs_options o;
            qs_options_default(&o);
            o.k_max = k;
            o.tile_qubits = L;
            qs_batch* b = nullptr;
            qs_status s = qs_batch_create(circuits, count, dt, &o, &b);
            if (s != QS_OK) continue;
            float ms = 0.f;
            s = qs_batch_run(b, device_states, stream);  // warm-up (and capture)
            if (s == QS_OK) s = qs_batch_sync(b);
            if (s == QS_OK) {
                cudaEventRecord(e0, st);
                s = qs_batch_run(b, device_states, stream);
                cudaEventRecord(e1, st);
                if (s == QS_OK) s = qs_batch_sync(b);
                cudaEventElapsedTime(&ms, e0, e1);
            }
            qs_batch_destroy(b);
            if (s != QS_OK) continue;
            if (best_ms < 0.f || ms < best_ms) {
                best_ms = ms;
                *best = o;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms < 0.f) return fail(QS_ERR_CUDA, "no batched configuration ran");
    return QS_OK;
}

}  // extern "C"
