// C ABI of libsv: argument checking, plan and observable caches, per-stream
// scratch, and the launch sequences of every entry point in sv.h.
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <memory>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "hbm.h"
#include "sample.h"
#include "kernels.h"
#include "planner.h"
#include "sv.h"

using namespace svk;

namespace svk {
void noalloc_forget();  // noalloc.cu: drops the cached array addresses
}  // namespace svk

namespace {

thread_local std::string g_last_error;

sv_status fail(sv_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

sv_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define SV_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

struct DeviceBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    DeviceBuf() = default;
    DeviceBuf(const DeviceBuf &) = delete;
    DeviceBuf &operator=(const DeviceBuf &) = delete;
    ~DeviceBuf() {
        if (ptr) cudaFree(ptr);
    }
};

// Packs host arrays into one device allocation at 256-byte aligned offsets.
struct Packer {
    std::vector<unsigned char> bytes;
    size_t add(const void *src, size_t n) {
        size_t off = (bytes.size() + 255) & ~size_t(255);
        bytes.resize(off + n);
        if (n) std::memcpy(bytes.data() + off, src, n);
        return off;
    }
};

struct PlanEntry {
    std::vector<sv_gate> gates;  // exact key check against hash collisions
    int n = 0, n_params = 0, input_dim = 0;
    HostProgram host;
    std::vector<TilePass> tiles;  // tile plans: one kernel descriptor per pass
    DeviceBuf buf;
    Program dev{};
};

// Tile passes of lambda = H psi for one tile size, uploaded.
struct HPlanEntry {
    HostHPlan host;
    DeviceBuf buf;
    std::vector<HPass> passes;  // with device pointers
};

struct ObsEntry {
    std::vector<uint64_t> xm, zm;
    std::vector<double> c;
    HostObservable host;
    DeviceBuf buf;
    Observable dev{};
    DeviceBuf dtab;  // diagonal tables D_g(j) for on-chip sizes, or empty
    // by tile bits and the qubits' bit layout of the states they run on
    std::map<std::pair<int, std::vector<int>>, std::unique_ptr<HPlanEntry>> hplans;
};

struct ArrayEntry {
    std::vector<unsigned char> bytes;
    DeviceBuf buf;
};

// Launch shape chosen by sv_autotune for one problem structure and kernel.
struct Tuned {
    int R = 0, tpb = 0, epi = 0;
    int tc = 0;  // tile passes: forward stages as tensor-core blocks
    float us = 0.f;
};

struct DeviceCtx {
    std::mutex mu;
    int sms = 152;
    std::unordered_map<uint64_t, Tuned> tuned;
    std::unordered_map<uint64_t, std::unique_ptr<PlanEntry>> plans;
    std::unordered_map<uint64_t, std::unique_ptr<ObsEntry>> obs;
    std::unordered_map<uint64_t, std::unique_ptr<ArrayEntry>> arrays;
    std::unordered_map<cudaStream_t, std::unique_ptr<DeviceBuf>> scratch;
    std::unordered_map<cudaStream_t, std::unique_ptr<DeviceBuf>> scratch_big;  // device-memory states
    // Phase timing of tile adjoints: per chunk, events before the forward,
    // H and reverse phases and after the reverse.
    bool timing = false;
    std::vector<cudaEvent_t> phase_ev;
    int phase_used = 0;
    // The last adjoint of states in device memory: its checkpoint interval and
    // the algorithmic bytes of its reverse tile passes.
    int last_every = 0;
    int64_t last_rev_bytes = 0;
    // Uneven batches: one instantiated graph per configuration, and the
    // stream the captures run on.
    std::unordered_map<uint64_t, std::unique_ptr<struct MultiGraph>> graphs;
    cudaStream_t capture_stream = nullptr;
    // Target distributions rewritten for relabeled states, per stream.
    std::unordered_map<cudaStream_t, std::unique_ptr<DeviceBuf>> relayout;
    // Host-buffer entry points: pinned host and device staging per stream.
    std::unordered_map<cudaStream_t, std::unique_ptr<struct HostIO>> hostio;
    // Device error word of the kernels with bounded waits (0 = none gave up).
    DeviceBuf err;
    // Host-buffer parameter-shift calls captured as graphs (theta in, the
    // energy launch and its dependent assembly, results out), by launch key.
    std::unordered_map<uint64_t, std::unique_ptr<struct HostGraph>> host_graphs;
};

struct HostGraph {
    cudaGraphExec_t exec = nullptr;
    bool failed = false;  // capture or instantiation refused: run eagerly
    ~HostGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

struct HostIO {
    void *host = nullptr;  // pinned
    void *dev = nullptr;
    size_t bytes = 0;
    ~HostIO() {
        if (host) cudaFreeHost(host);
        if (dev) cudaFree(dev);
    }
};

struct MultiGraph {
    cudaGraphExec_t exec = nullptr;
    DeviceBuf buf;  // descriptors, item tables and every problem's states and sums
    ~MultiGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

// Records phase event `i` of the current timed call (creating it on first use).
void phase_mark(DeviceCtx *ctx, cudaStream_t st) {
    if (!ctx->timing) return;
    if (ctx->phase_used == (int)ctx->phase_ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        ctx->phase_ev.push_back(e);
    }
    cudaEventRecord(ctx->phase_ev[ctx->phase_used++], st);
}

std::mutex g_mu;
std::unordered_map<int, std::unique_ptr<DeviceCtx>> g_ctx;

DeviceCtx *context(int *dev_out = nullptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (dev_out) *dev_out = dev;
    std::lock_guard<std::mutex> lk(g_mu);
    auto &p = g_ctx[dev];
    if (!p) {
        p.reset(new DeviceCtx());
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            p->sms = sms;
    }
    return p.get();
}

uint64_t mix64(uint64_t h, uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h * 0xff51afd7ed558ccdull;
}

uint64_t hash_bytes(const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    uint64_t h = 0xcbf29ce484222325ull ^ n;
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 0x100000001b3ull;
    return h;
}

int swz_bits(sv_dtype d) { return d == SV_C128 ? 3 : 4; }

// Compiled program of a circuit for (reg_bits, fusion, dtype), cached.
// tile_bits > 0: the circuit cut into tile passes of 2^tile_bits amplitudes
// (states in device memory) instead of one on-chip program.
sv_status get_plan(DeviceCtx *ctx, const sv_circuit &c, int R, bool fuse, sv_dtype dt,
                   PlanEntry **out, int tile_bits = 0, int coalesce = 0, bool relabel = false) {
    if (coalesce <= 0) coalesce = dt == SV_C128 ? 3 : 4;
    if (tile_bits <= 0) relabel = false;
    uint64_t key = hash_circuit(c);
    key = mix64(key, (uint64_t)R);
    key = mix64(key, fuse ? 1 : 0);
    key = mix64(key, (uint64_t)swz_bits(dt));
    key = mix64(key, (uint64_t)(1000 + tile_bits));
    key = mix64(key, (uint64_t)(2000 + coalesce));
    key = mix64(key, relabel ? 0x7e1abe1ull : 0ull);
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        PlanEntry *e = it->second.get();
        if (e->n == c.n_qubits && e->n_params == c.n_params && e->input_dim == c.input_dim &&
            e->gates.size() == (size_t)c.n_gates &&
            (c.n_gates == 0 || std::memcmp(e->gates.data(), c.gates, sizeof(sv_gate) * c.n_gates) == 0)) {
            *out = e;
            return SV_OK;
        }
    }
    std::unique_ptr<PlanEntry> e(new PlanEntry());
    std::string err;
    if (tile_bits > 0) {
        err = plan_passes(c, tile_bits, coalesce, R, fuse, swz_bits(dt), &e->host, relabel);
        if (err.empty()) err = build_tile_passes(e->host, dt == SV_C128 ? 16 : 8, &e->tiles);
    } else {
        err = plan_circuit(c, R, fuse, swz_bits(dt), &e->host);
    }
    if (!err.empty()) return fail(SV_ERR_ARG, "circuit: " + err);
    e->gates.assign(c.gates, c.gates + c.n_gates);
    e->n = c.n_qubits;
    e->n_params = c.n_params;
    e->input_dim = c.input_dim;
    const HostProgram &h = e->host;
    Packer pk;
    size_t o_st = pk.add(h.stages.data(), h.stages.size() * sizeof(Stage));
    size_t o_op = pk.add(h.ops.data(), h.ops.size() * sizeof(Op));
    size_t o_gr = pk.add(h.groups.data(), h.groups.size() * sizeof(Group));
    size_t o_me = pk.add(h.members.data(), h.members.size() * sizeof(Member));
    size_t o_tb = pk.add(h.tbase.data(), h.tbase.size() * sizeof(ThreadBase));
    pk.bytes.resize((pk.bytes.size() + 255) & ~size_t(255));  // whole 16-byte units for staging
    e->buf.bytes = pk.bytes.size() ? pk.bytes.size() : 256;
    SV_CUDA(cudaMalloc(&e->buf.ptr, e->buf.bytes));
    if (!pk.bytes.empty())
        SV_CUDA(cudaMemcpy(e->buf.ptr, pk.bytes.data(), pk.bytes.size(), cudaMemcpyHostToDevice));
    unsigned char *base = (unsigned char *)e->buf.ptr;
    Program &p = e->dev;
    p.n = h.n;
    p.R = h.R;
    p.n_stages = (int)h.stages.size();
    p.n_groups = (int)h.groups.size();
    p.n_params = h.n_params;
    p.input_dim = h.input_dim;
    p.swz_bits = h.swz_bits;
    p.stages = (const Stage *)(base + o_st);
    p.ops = (const Op *)(base + o_op);
    p.groups = (const Group *)(base + o_gr);
    p.members = (const Member *)(base + o_me);
    p.tbase = h.tbase.empty() ? nullptr : (const ThreadBase *)(base + o_tb);
    *out = e.get();
    ctx->plans[key] = std::move(e);
    return SV_OK;
}

// Tables of the diagonals D_g(j) are built for states that fit on chip and
// tables of at most 2^20 entries.
constexpr int kDtabMaxQubits = 13;
constexpr int64_t kDtabMaxEntries = int64_t(1) << 20;

sv_status get_obs(DeviceCtx *ctx, const sv_pauli_sum &h, int n, sv_dtype dt, ObsEntry **out,
                  cudaStream_t st) {
    if (h.n_terms < 0 || (h.n_terms > 0 && (!h.x_mask || !h.z_mask || !h.coeff)))
        return fail(SV_ERR_ARG, "observable: missing arrays");
    uint64_t key = mix64(hash_observable(h), (uint64_t)swz_bits(dt));
    key = mix64(key, (uint64_t)n);
    auto it = ctx->obs.find(key);
    if (it != ctx->obs.end()) {
        ObsEntry *e = it->second.get();
        if (e->xm.size() == (size_t)h.n_terms &&
            std::memcmp(e->xm.data(), h.x_mask, 8 * h.n_terms) == 0 &&
            std::memcmp(e->zm.data(), h.z_mask, 8 * h.n_terms) == 0 &&
            std::memcmp(e->c.data(), h.coeff, 8 * h.n_terms) == 0 && e->host.n == n) {
            *out = e;
            return SV_OK;
        }
    }
    std::unique_ptr<ObsEntry> e(new ObsEntry());
    std::string err = plan_observable(h, n, swz_bits(dt), &e->host);
    if (!err.empty()) return fail(SV_ERR_ARG, "observable: " + err);
    e->xm.assign(h.x_mask, h.x_mask + h.n_terms);
    e->zm.assign(h.z_mask, h.z_mask + h.n_terms);
    e->c.assign(h.coeff, h.coeff + h.n_terms);
    Packer pk;
    size_t o_g = pk.add(e->host.tgroups.data(), e->host.tgroups.size() * sizeof(TermGroup));
    size_t o_t = pk.add(e->host.terms.data(), e->host.terms.size() * sizeof(Term));
    pk.bytes.resize((pk.bytes.size() + 255) & ~size_t(255));
    e->buf.bytes = pk.bytes.size() ? pk.bytes.size() : 256;
    SV_CUDA(cudaMalloc(&e->buf.ptr, e->buf.bytes));
    if (!pk.bytes.empty())
        SV_CUDA(cudaMemcpy(e->buf.ptr, pk.bytes.data(), pk.bytes.size(), cudaMemcpyHostToDevice));
    unsigned char *base = (unsigned char *)e->buf.ptr;
    e->dev.n_tgroups = (int)e->host.tgroups.size();
    e->dev.n_terms = (int)e->host.terms.size();
    e->dev.real = 1;
    for (const Term &tm : e->host.terms) e->dev.real &= (tm.phase & 1) == 0;
    e->dev.tgroups = (const TermGroup *)(base + o_g);
    e->dev.terms = (const Term *)(base + o_t);
    const int64_t entries = (int64_t(1) << n) * e->dev.n_tgroups;
    if (n <= kDtabMaxQubits && entries > 0 && entries <= kDtabMaxEntries) {
        e->dtab.bytes = (size_t)entries * (dt == SV_C128 ? 16 : 8);
        SV_CUDA(cudaMalloc(&e->dtab.ptr, e->dtab.bytes));
        SV_CUDA(launch_build_dtable(dt == SV_C128, e->dev, n, e->dtab.ptr, st));
        SV_CUDA(cudaStreamSynchronize(st));  // usable from any stream afterwards
    }
    *out = e.get();
    ctx->obs[key] = std::move(e);
    return SV_OK;
}

// Small host arrays (references, slot lists) uploaded once and cached by content.
sv_status get_array(DeviceCtx *ctx, const void *host, size_t bytes, const void **dev) {
    const uint64_t key = hash_bytes(host, bytes);
    auto it = ctx->arrays.find(key);
    if (it != ctx->arrays.end() && it->second->bytes.size() == bytes &&
        std::memcmp(it->second->bytes.data(), host, bytes) == 0) {
        *dev = it->second->buf.ptr;
        return SV_OK;
    }
    std::unique_ptr<ArrayEntry> e(new ArrayEntry());
    e->bytes.assign((const unsigned char *)host, (const unsigned char *)host + bytes);
    e->buf.bytes = bytes ? bytes : 16;
    SV_CUDA(cudaMalloc(&e->buf.ptr, e->buf.bytes));
    if (bytes) SV_CUDA(cudaMemcpy(e->buf.ptr, host, bytes, cudaMemcpyHostToDevice));
    *dev = e->buf.ptr;
    ctx->arrays[key] = std::move(e);
    return SV_OK;
}

// Library scratch for one stream, grown on demand (growth synchronizes the stream).
sv_status get_scratch(DeviceCtx *ctx, cudaStream_t st, size_t bytes, void **out) {
    auto &s = ctx->scratch[st];
    if (!s) s.reset(new DeviceBuf());
    if (s->bytes < bytes) {
        if (s->ptr) {
            SV_CUDA(cudaStreamSynchronize(st));
            cudaFree(s->ptr);
            s->ptr = nullptr;
            s->bytes = 0;
        }
        size_t want = bytes < 4096 ? 4096 : bytes;
        SV_CUDA(cudaMalloc(&s->ptr, want));
        s->bytes = want;
    }
    *out = s->ptr;
    return SV_OK;
}

// Pinned host + device staging of `bytes` for one stream, grown on demand
// (growth synchronizes the stream).
sv_status get_hostio(DeviceCtx *ctx, cudaStream_t st, size_t bytes, HostIO **out) {
    auto &h = ctx->hostio[st];
    if (!h) h.reset(new HostIO());
    if (h->bytes < bytes) {
        SV_CUDA(cudaStreamSynchronize(st));
        if (h->host) cudaFreeHost(h->host);
        if (h->dev) cudaFree(h->dev);
        h->host = h->dev = nullptr;
        h->bytes = 0;
        const size_t want = bytes < 4096 ? 4096 : bytes;
        SV_CUDA(cudaMallocHost(&h->host, want));
        SV_CUDA(cudaMalloc(&h->dev, want));
        h->bytes = want;
    }
    *out = h.get();
    return SV_OK;
}

sv_status check_circuit(const sv_circuit *c, int n_limit) {
    if (!c) return fail(SV_ERR_ARG, "circuit is NULL");
    if (c->n_qubits < 1 || c->n_qubits > n_limit)
        return fail(SV_ERR_ARG, "circuit n_qubits out of range");
    if (c->n_gates < 0 || (c->n_gates > 0 && !c->gates))
        return fail(SV_ERR_ARG, "circuit gates missing");
    if (c->n_params < 0 || c->input_dim < 0) return fail(SV_ERR_ARG, "negative sizes");
    return SV_OK;
}

int default_regbits(const sv_plan_opts *o) { return (o && o->reg_bits > 0) ? o->reg_bits : 0; }
int default_tpb(const sv_plan_opts *o) { return (o && o->threads_per_block > 0) ? o->threads_per_block : 0; }
bool use_fusion(const sv_plan_opts *o) { return !(o && o->no_fusion); }
bool use_relabel(const sv_plan_opts *o) { return !(o && o->no_relabel); }

// Planner register bits for a kernel kind: the launch shape decides R first.
sv_status shape_for(int kind, const sv_circuit &c, int n_groups_hint, sv_dtype dt, int n_slots,
                    const sv_plan_opts *opts, OnchipShape *sh, int sms, uint32_t const_bytes = 0) {
    const char *err = onchip_shape(kind, c.n_qubits, n_groups_hint, c.n_params, dt == SV_C128,
                                   n_slots, default_regbits(opts), default_tpb(opts), sh, sms,
                                   const_bytes);
    if (err) return fail(SV_ERR_UNSUPPORTED, err);
    return SV_OK;
}

// The arrays a block copies into shared memory before it starts.
BlockConst make_block_const(const PlanEntry *plan, const ObsEntry *obs, const void *dtab,
                            bool with_tbase) {
    BlockConst b{};
    uint32_t off = 0;
    auto add = [&](int k, const void *src, size_t bytes) {
        if (!src || !bytes) return;
        const uint32_t n16 = (uint32_t)((bytes + 15) / 16);
        b.src[k] = (const uint4 *)src;
        b.n16[k] = n16;
        b.off[k] = off;
        off += n16 * 16;
    };
    const HostProgram &h = plan->host;
    add(0, plan->dev.stages, h.stages.size() * sizeof(Stage));
    add(1, plan->dev.ops, h.ops.size() * sizeof(Op));
    add(2, plan->dev.groups, h.groups.size() * sizeof(Group));
    add(3, plan->dev.members, h.members.size() * sizeof(Member));
    if (with_tbase) add(7, plan->dev.tbase, h.tbase.size() * sizeof(ThreadBase));
    if (obs) {
        add(4, obs->dev.tgroups, obs->host.tgroups.size() * sizeof(TermGroup));
        add(5, obs->dev.terms, obs->host.terms.size() * sizeof(Term));
        if (dtab) add(6, dtab, obs->dtab.bytes);
    }
    b.bytes = off;
    return b;
}

// Plan + final launch shape (the shape needs the group count of the plan and
// the size of the block-constant arrays when `bc` is requested).
sv_status plan_and_shape(DeviceCtx *ctx, int kind, const sv_circuit &c, sv_dtype dt, int n_slots,
                         const sv_plan_opts *opts, PlanEntry **plan, OnchipShape *sh,
                         const Tuned *tuned = nullptr, const ObsEntry *obs = nullptr,
                         const void *dtab = nullptr, BlockConst *bc = nullptr) {
    sv_plan_opts o2{};
    if (tuned && !(opts && (opts->reg_bits > 0 || opts->threads_per_block > 0))) {
        if (opts) o2 = *opts;
        o2.reg_bits = tuned->R;
        o2.threads_per_block = tuned->tpb;
        opts = &o2;
    }
    OnchipShape pre{};
    sv_status s = shape_for(kind, c, 0, dt, n_slots, opts, &pre, ctx->sms);
    if (s != SV_OK) return s;
    s = get_plan(ctx, c, pre.R, use_fusion(opts), dt, plan);
    if (s != SV_OK) return s;
    if (!bc) return shape_for(kind, c, (*plan)->dev.n_groups, dt, n_slots, opts, sh, ctx->sms, 0);
    // Stage as much as fits: everything, then without the tables, then
    // without the thread bases, then only the program and terms.
    for (int variant = 0; variant < 4; ++variant) {
        *bc = make_block_const(*plan, obs, (variant & 1) ? nullptr : dtab, !(variant & 2));
        s = shape_for(kind, c, (*plan)->dev.n_groups, dt, n_slots, opts, sh, ctx->sms, bc->bytes);
        if (s != SV_OK) return s;
        if (sh->const_bytes || !bc->bytes) return SV_OK;
    }
    return SV_OK;
}

sv_status check_problem(const sv_problem *p, bool need_cost_arrays) {
    if (!p) return fail(SV_ERR_ARG, "problem is NULL");
    if (p->dtype != SV_C64 && p->dtype != SV_C128) return fail(SV_ERR_ARG, "bad dtype");
    sv_status s = check_circuit(p->circuit, p->dtype == SV_C128 ? 29 : 30);
    if (s != SV_OK) return s;
    if (!p->observable) return fail(SV_ERR_ARG, "observable is NULL");
    if (p->observable->n_qubits != p->circuit->n_qubits)
        return fail(SV_ERR_ARG, "observable and circuit qubit counts differ");
    if (p->n_instances < 1) return fail(SV_ERR_ARG, "n_instances must be >= 1");
    if (!p->refs) return fail(SV_ERR_ARG, "refs is NULL");
    const int64_t dim = int64_t(1) << p->circuit->n_qubits;
    for (int i = 0; i < p->n_instances; ++i)
        if (p->refs[i] < 0 || p->refs[i] >= dim) return fail(SV_ERR_ARG, "reference out of range");
    if (p->circuit->input_dim > 0 && (!p->inputs || p->input_stride < p->circuit->input_dim))
        return fail(SV_ERR_ARG, "circuit reads inputs but inputs/input_stride are missing");
    if (need_cost_arrays) {
        if (p->cost == SV_COST_LINEAR && !p->weights) return fail(SV_ERR_ARG, "weights are NULL");
        if (p->cost == SV_COST_MSE && !p->targets) return fail(SV_ERR_ARG, "targets are NULL");
    }
    if (p->cost != SV_COST_LINEAR && p->cost != SV_COST_MSE) return fail(SV_ERR_ARG, "bad cost");
    return SV_OK;
}

uint64_t tune_key(const sv_problem *p, int kind, int n_slots) {
    uint64_t k = mix64(hash_circuit(*p->circuit), hash_observable(*p->observable));
    k = mix64(k, (uint64_t)kind);
    k = mix64(k, (uint64_t)n_slots);
    k = mix64(k, (uint64_t)p->dtype);
    k = mix64(k, (uint64_t)use_fusion(p->opts));
    return k;
}

const Tuned *find_tuned(DeviceCtx *ctx, const sv_problem *p, int kind, int n_slots) {
    auto it = ctx->tuned.find(tune_key(p, kind, n_slots));
    return it == ctx->tuned.end() ? nullptr : &it->second;
}

// The expectation epilogue: diagonal tables when requested (or tuned, or by
// default) and available, otherwise the per-term loop.
const void *pick_dtab(const ObsEntry *obs, const sv_plan_opts *opts, const Tuned *t) {
    int epi = (opts && opts->epilogue > 0) ? opts->epilogue : (t && t->epi > 0 ? t->epi : 2);
    return epi == 2 ? obs->dtab.ptr : nullptr;
}

CostSource cost_of(const sv_problem *p, const double *ext) {
    CostSource c{};
    c.cost = p->cost;
    c.n_instances = p->n_instances;
    c.ext_weights = ext;
    c.weights = p->weights;
    c.targets = p->targets;
    return c;
}

// ------------------------------------------------ device-memory states

// Second per-stream scratch for tile-pass state buffers (grown on demand).
sv_status get_big_scratch(DeviceCtx *ctx, cudaStream_t st, size_t bytes, void **out) {
    auto &s = ctx->scratch_big[st];
    if (!s) s.reset(new DeviceBuf());
    if (s->bytes < bytes) {
        if (s->ptr) {
            SV_CUDA(cudaStreamSynchronize(st));
            cudaFree(s->ptr);
            s->ptr = nullptr;
            s->bytes = 0;
        }
        SV_CUDA(cudaMalloc(&s->ptr, bytes));
        s->bytes = bytes;
    }
    *out = s->ptr;
    return SV_OK;
}

// Bytes a tile-pass call may claim: 80 % of what is free plus what its own
// big scratch already holds.
size_t big_budget(DeviceCtx *ctx, cudaStream_t st) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    auto it = ctx->scratch_big.find(st);
    const size_t have = (it != ctx->scratch_big.end() && it->second) ? it->second->bytes : 0;
    return (size_t)(0.8 * (double)fr) + have;
}

// lambda = H psi and <H> for states in device memory: tiles of 2^12
// (complex64) / 2^11 (complex128) amplitudes, or the whole state below that.
int h_tile_bits(int n, sv_dtype dt) {
    const int t = dt == SV_C128 ? 11 : 12;
    return n < t ? n : t;
}

// layout: qubit q in bit layout[q] of the amplitude index (states left
// relabeled by tile passes), or null / empty for the identity; the terms'
// masks are moved to those bits.
sv_status get_hplan(ObsEntry *obs, int n, sv_dtype dt, HPlanEntry **out,
                    const std::vector<int> *layout = nullptr) {
    const int t = h_tile_bits(n, dt);
    std::vector<int> lay;
    if (layout)
        for (int q = 0; q < (int)layout->size(); ++q)
            if ((*layout)[q] != q) {
                lay = *layout;
                break;
            }
    std::unique_ptr<HPlanEntry> &slot = obs->hplans[{t, lay}];
    if (!slot) {
        std::unique_ptr<HPlanEntry> e(new HPlanEntry());
        const HostObservable *ho = &obs->host;
        HostObservable moved;
        if (!lay.empty()) {
            auto move = [&](uint64_t m) {
                uint64_t r = 0;
                for (int q = 0; q < n; ++q)
                    if ((m >> q) & 1ull) r |= 1ull << lay[q];
                return r;
            };
            std::vector<uint64_t> xm(obs->xm.size()), zm(obs->zm.size());
            for (size_t i = 0; i < xm.size(); ++i) {
                xm[i] = move(obs->xm[i]);
                zm[i] = move(obs->zm[i]);
            }
            sv_pauli_sum h{};
            h.n_qubits = n;
            h.n_terms = (int32_t)xm.size();
            h.x_mask = xm.data();
            h.z_mask = zm.data();
            h.coeff = obs->c.data();
            std::string err = plan_observable(h, n, swz_bits(dt), &moved);
            if (!err.empty()) return fail(SV_ERR_ARG, "observable: " + err);
            ho = &moved;
        }
        std::string err = plan_h_passes(*ho, t, dt == SV_C128 ? 3 : 4, &e->host);
        if (!err.empty()) return fail(SV_ERR_ARG, "observable: " + err);
        const HostHPlan &h = e->host;
        Packer pk;
        const size_t og = pk.add(h.groups.data(), h.groups.size() * sizeof(HGroup));
        const size_t oc = pk.add(h.classes.data(), h.classes.size() * sizeof(HClass));
        const size_t ot = pk.add(h.terms.data(), h.terms.size() * sizeof(HTerm));
        const size_t orw = pk.add(h.rows.data(), h.rows.size() * sizeof(HRow));
        e->buf.bytes = pk.bytes.size() ? pk.bytes.size() : 256;
        SV_CUDA(cudaMalloc(&e->buf.ptr, e->buf.bytes));
        if (!pk.bytes.empty())
            SV_CUDA(cudaMemcpy(e->buf.ptr, pk.bytes.data(), pk.bytes.size(), cudaMemcpyHostToDevice));
        const unsigned char *base = (const unsigned char *)e->buf.ptr;
        for (size_t i = 0; i < h.passes.size(); ++i) {
            HPass P = h.passes[i];
            P.groups = (const HGroup *)(base + og) + h.g_begin[i];
            P.classes = (const HClass *)(base + oc) + h.c_begin[i];
            P.terms = (const HTerm *)(base + ot) + h.t_begin[i];
            P.rows = (const HRow *)(base + orw) + h.r_begin[i];
            e->passes.push_back(P);
        }
        slot = std::move(e);
    }
    *out = slot.get();
    return SV_OK;
}

int64_t tile_blocks(const DeviceCtx *ctx, int64_t tiles);

// E[r] = <psi_r|H|psi_r> for n_rows states (and lam = H psi unless lam is
// null) by tile passes.
sv_status h_tiles(DeviceCtx *ctx, ObsEntry *obs, int n, sv_dtype dt, int n_rows, const void *psi,
                  void *lam, double *E, cudaStream_t st, const std::vector<int> *layout = nullptr) {
    HPlanEntry *hp = nullptr;
    sv_status s = get_hplan(obs, n, dt, &hp, layout);
    if (s != SV_OK) return s;
    SV_CUDA(cudaMemsetAsync(E, 0, sizeof(double) * (size_t)n_rows, st));
    for (const HPass &P : hp->passes) {
        const int64_t tiles = (int64_t)n_rows << P.n_tile_bits;
        cudaError_t e = launch_tile_h(dt == SV_C128, P, n, n_rows, psi, lam, E,
                                      tile_blocks(ctx, tiles), st);
        if (e != cudaSuccess) return cuda_fail(e, "H tile pass");
    }
    return SV_OK;
}

bool wants_tiles(int n, sv_dtype dt, const sv_plan_opts *o) {
    if (o && o->tile_bits > 0) return true;
    return n > (dt == SV_C128 ? 12 : 13);
}

struct TileCfg {
    int t, R, c;  // tile bits, register bits, coalesced low qubits
    bool tc;      // forward stages as tensor-core blocks
};

// The device error word (allocated and zeroed on first use).
int *device_err(DeviceCtx *ctx) {
    if (!ctx->err.ptr) {
        if (cudaMalloc(&ctx->err.ptr, 256) != cudaSuccess) {
            ctx->err.ptr = nullptr;
            return nullptr;
        }
        ctx->err.bytes = 256;
        if (cudaMemset(ctx->err.ptr, 0, 256) != cudaSuccess) return nullptr;
    }
    return (int *)ctx->err.ptr;
}

// Tuning keys of the tile tier (by instance count), beside the on-chip kinds.
constexpr int kTileEnergyKey = 10 + ONCHIP_ENERGY, kTileAdjointKey = 10 + ONCHIP_ADJOINT;

// tn: a tuned tile shape (R = register bits, tpb = 2^(t - R) threads), used
// when opts leave tile_bits and reg_bits at zero.
sv_status tile_cfg(int n, sv_dtype dt, const sv_plan_opts *o, TileCfg *cfg,
                   const Tuned *tn = nullptr) {
    if (tn && tn->R > 0 && (!o || (o->tile_bits <= 0 && o->reg_bits <= 0))) {
        sv_plan_opts t{};
        if (o) t = *o;
        t.reg_bits = tn->R;
        t.tile_bits = tn->R + __builtin_ctz((unsigned)tn->tpb);
        t.tensor_blocks = tn->tc;
        return tile_cfg(n, dt, &t, cfg, nullptr);
    }
    const int c = (o && o->coalesce_bits > 0) ? o->coalesce_bits : (dt == SV_C128 ? 3 : 4);
    const int rmax = dt == SV_C128 ? 3 : 4;
    // Default: 2^11 (complex64) / 2^10 (complex128) amplitudes per tile with
    // 4 / 2 register bits: 128 / 256 threads per block.
    int t = (o && o->tile_bits > 0) ? o->tile_bits : (dt == SV_C128 ? 10 : 11);
    if (t > n) t = n;
    if (t < c + 2 || t > 12)
        return fail(SV_ERR_UNSUPPORTED, "tile passes need 2^tile_bits amplitudes with tile_bits in "
                                        "[coalesced bits + 2, 12] and at most n_qubits");
    int R = (o && o->reg_bits > 0) ? o->reg_bits : std::min(dt == SV_C128 ? 2 : 4, t - 5);
    if (R < 2 || R > rmax) return fail(SV_ERR_ARG, "reg_bits for tile passes must be 2..4 (2..3 complex128)");
    if (t - R > 8) R = t - 8;
    if (R > rmax) return fail(SV_ERR_UNSUPPORTED, "tile too large for the register width");
    if (t - R < 5)
        return fail(SV_ERR_UNSUPPORTED, "tile passes need tile_bits - reg_bits >= 5 (a warp of threads)");
    if (c + 2 > t) return fail(SV_ERR_ARG, "coalesce_bits must be at most tile_bits - 2");
    const bool tc = o && o->tensor_blocks;
    if (tc && (dt == SV_C128 || R != 4 || (t != 11 && t != 12)))
        return fail(SV_ERR_UNSUPPORTED, "tensor_blocks: complex64 tile passes with reg_bits 4 and "
                                        "tile_bits 11 or 12 only");
    cfg->t = t;
    cfg->R = R;
    cfg->c = c;
    cfg->tc = tc;
    return SV_OK;
}

// Upper bound on the blocks of a tile-pass launch (the launcher caps it by
// the kernel's occupancy): at most one block per tile.
int64_t tile_blocks(const DeviceCtx *ctx, int64_t tiles) {
    const int64_t b = (int64_t)ctx->sms * 8;
    return b < tiles ? b : tiles;
}

// Forward tile passes of `pe` over src.n_slots states (|ref> first when init).
// After pass i with (i + 1) % every == 0 (and not the last pass) the states
// are copied to checkpoint (i + 1) / every - 1 of `ck`.
sv_status tiles_forward(DeviceCtx *ctx, const PlanEntry *pe, int R, sv_dtype dt,
                        const SlotSource &src, void *states, void *mats, bool init, void *ck,
                        int every, cudaStream_t st, bool tc = false) {
    const int c128 = dt == SV_C128, n = pe->n, G = pe->dev.n_groups;
    const size_t sbytes = ((size_t)src.n_slots << n) * (c128 ? 16 : 8);
    cudaError_t e = launch_group_mats(c128, pe->dev, src, mats, st);
    if (e != cudaSuccess) return cuda_fail(e, "group matrices");
    if (init) {
        e = launch_init_states(c128, states, n, src, st);
        if (e != cudaSuccess) return cuda_fail(e, "state init");
    }
    // A pass that ends at a stored forward state writes its output there
    // (out of place) and the next pass reads it from there: no copies.  The
    // last pass always writes `states`.
    const auto &passes = pe->tiles;
    const void *in = states;
    for (size_t i = 0; i < passes.size(); ++i) {
        const TilePass &tp = passes[i];
        const int64_t tiles = (int64_t)src.n_slots << tp.n_tile_bits;
        const uint32_t smem = tile_fwd_smem(c128, tp);
        if (smem > 220u * 1024u) return fail(SV_ERR_UNSUPPORTED, "tile pass needs too much shared memory");
        void *out = states;
        if (ck && every > 0 && (i + 1) % every == 0 && i + 1 < passes.size())
            out = (char *)ck + ((i + 1) / every - 1) * sbytes;
        if (tc && tile_fwd_tc_supported(c128, tp)) {
            int *err = device_err(ctx);
            if (!err) return fail(SV_ERR_CUDA, "device error word");
            e = launch_tile_fwd_tc(tp, n, src.n_slots, mats, G, out, tile_blocks(ctx, tiles), st,
                                   err, in);
            if (e != cudaSuccess) return cuda_fail(e, "forward tile pass (tensor cores)");
        } else {
            e = launch_tile_fwd(c128, tp, n, src.n_slots, mats, G, out, tile_blocks(ctx, tiles), st,
                                in);
            if (e != cudaSuccess) return cuda_fail(e, "forward tile pass");
        }
        in = out;
    }
    return SV_OK;
}

// Energies of n_slots slots (parameter-shift or instance slots) of states in
// device memory, in groups of slots that fit the memory budget.
sv_status tiles_energies(DeviceCtx *ctx, const sv_problem *p, const double *theta, int mode,
                         int n_slots, double *E, cudaStream_t st, int slot_begin = 0) {
    const sv_dtype dt = p->dtype;
    const int c128 = dt == SV_C128, n = p->circuit->n_qubits, I = p->n_instances;
    TileCfg cfg{};
    sv_status s = tile_cfg(n, dt, p->opts, &cfg, find_tuned(ctx, p, kTileEnergyKey, p->n_instances));
    if (s != SV_OK) return s;
    PlanEntry *pe = nullptr;
    s = get_plan(ctx, *p->circuit, cfg.R, use_fusion(p->opts), dt, &pe, cfg.t, cfg.c,
                 use_relabel(p->opts));
    if (s != SV_OK) return s;
    ObsEntry *obs = nullptr;
    s = get_obs(ctx, *p->observable, n, dt, &obs, st);
    if (s != SV_OK) return s;
    const void *drefs = nullptr;
    s = get_array(ctx, p->refs, sizeof(int64_t) * I, &drefs);
    if (s != SV_OK) return s;
    const size_t csz = c128 ? 16 : 8, sb = csz << n;
    const size_t mb = (size_t)pe->dev.n_groups * 4 * csz;
    const size_t per = sb + mb;
    int64_t chunk = (int64_t)(big_budget(ctx, st) / (per + 512));
    if (chunk < 1) return fail(SV_ERR_OOM, "one state does not fit in free device memory");
    if (chunk > n_slots) chunk = n_slots;
    if (chunk > 65535) chunk = 65535;  // one grid row per state in the expectation
    void *big = nullptr;
    const size_t mats_off = ((size_t)chunk * sb + 255) & ~size_t(255);
    s = get_big_scratch(ctx, st, mats_off + (size_t)chunk * mb + 256, &big);
    if (s != SV_OK) return s;
    for (int64_t c0 = 0; c0 < n_slots; c0 += chunk) {
        SlotSource src{};
        src.mode = mode;
        src.n_slots = (int)std::min<int64_t>(chunk, n_slots - c0);
        src.n_instances = I;
        src.refs = (const int64_t *)drefs;
        src.theta = theta;
        src.inputs = p->inputs;
        src.input_stride = p->input_stride;
        src.slot_base = slot_begin + (int)c0;
        s = tiles_forward(ctx, pe, cfg.R, dt, src, big, (char *)big + mats_off, true, nullptr, 0, st,
                          cfg.tc);
        if (s != SV_OK) return s;
        s = h_tiles(ctx, obs, n, dt, src.n_slots, big, nullptr, E + c0, st, &pe->host.layout);
        if (s != SV_OK) return s;
    }
    return SV_OK;
}

// Adjoint gradient of states in device memory: forward passes with stored
// states every `every` passes, lambda = H psi, reverse passes accumulating the
// reduced matrices, per-slot gradients, then the sum over instances.
// ddcl_target (device [2^n]) replaces lambda = H psi by the JS divergence's
// lambda (data-driven circuit learning); the slot energies are then JS.
sv_status tiles_adjoint(DeviceCtx *ctx, const sv_problem *p, const double *theta,
                        const double *weights, double *energy_out, double *loss_out,
                        double *grad_out, int every, cudaStream_t st,
                        const double *ddcl_target = nullptr, const TileCfg *forced = nullptr) {
    ctx->phase_used = 0;
    ctx->last_every = 0;
    ctx->last_rev_bytes = 0;
    const sv_dtype dt = p->dtype;
    const int c128 = dt == SV_C128, n = p->circuit->n_qubits, I = p->n_instances;
    const int P = p->circuit->n_params, Pp = P > 0 ? P : 1;
    TileCfg cfg{};
    sv_status s = forced ? SV_OK : tile_cfg(n, dt, p->opts, &cfg, find_tuned(ctx, p, kTileAdjointKey, I));
    if (s != SV_OK) return s;
    if (forced) cfg = *forced;
    PlanEntry *pe = nullptr;
    s = get_plan(ctx, *p->circuit, cfg.R, use_fusion(p->opts), dt, &pe, cfg.t, cfg.c,
                 use_relabel(p->opts));
    if (s != SV_OK) return s;
    if (ddcl_target) {
        // The passes leave qubit q in index bit layout[q]: rewrite the target
        // distribution in that bit order for the JS divergence.
        const std::vector<int> &lay = pe->host.layout;
        bool moved = false;
        for (int q = 0; q < (int)lay.size(); ++q) moved |= lay[q] != q;
        if (moved) {
            std::vector<int32_t> who(n);
            for (int q = 0; q < n; ++q) who[lay[q]] = q;
            auto &buf = ctx->relayout[st];
            if (!buf) buf.reset(new DeviceBuf());
            const size_t bytes = sizeof(double) << n;
            if (buf->bytes < bytes) {
                SV_CUDA(cudaStreamSynchronize(st));
                if (buf->ptr) cudaFree(buf->ptr);
                buf->ptr = nullptr;
                buf->bytes = 0;
                SV_CUDA(cudaMalloc(&buf->ptr, bytes));
                buf->bytes = bytes;
            }
            cudaError_t e = launch_relayout(n, who.data(), ddcl_target, (double *)buf->ptr, st);
            if (e != cudaSuccess) return cuda_fail(e, "target relayout");
            ddcl_target = (const double *)buf->ptr;
        }
    }
    ObsEntry *obs = nullptr;
    if (!ddcl_target) {
        s = get_obs(ctx, *p->observable, n, dt, &obs, st);
        if (s != SV_OK) return s;
    }
    const void *drefs = nullptr;
    s = get_array(ctx, p->refs, sizeof(int64_t) * I, &drefs);
    if (s != SV_OK) return s;
    const int G = pe->dev.n_groups;
    const int npass = (int)pe->tiles.size();
    const size_t csz = c128 ? 16 : 8, sb = csz << n;
    const size_t budget = big_budget(ctx, st);
    auto per_instance = [&](int ev) {
        const size_t ncp_ = npass > 1 ? (size_t)((npass - 1) / ev) : 0;
        return (2 + ncp_) * sb + (size_t)G * 4 * csz + (size_t)G * 64;
    };
    if (every <= 0) {
        // The most stored states that still let every instance run at once:
        // a reverse pass followed by a restart from a stored state skips
        // writing psi, and un-computation rounding spans fewer passes.
        every = 4;
        for (int ev : {1, 2})
            if (budget / (per_instance(ev) + 2048) >= (size_t)I) {
                every = ev;
                break;
            }
    }
    const int ncp = npass > 1 ? (npass - 1) / every : 0;
    ctx->last_every = every;
    const size_t per = per_instance(every);
    int64_t chunk = (int64_t)(budget / (per + 2048));
    if (chunk < 1) return fail(SV_ERR_OOM, "psi, lambda and the stored states do not fit");
    if (chunk > I) chunk = I;
    if (chunk > 65535) chunk = 65535;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t o_lam = up((size_t)chunk * sb), o_ck = o_lam + up((size_t)chunk * sb);
    const size_t o_mats = o_ck + up((size_t)ncp * chunk * sb);
    const size_t o_rho = o_mats + up((size_t)chunk * G * 4 * csz);
    const size_t total = o_rho + up((size_t)chunk * G * 64);
    void *big = nullptr;
    s = get_big_scratch(ctx, st, total, &big);
    if (s != SV_OK) return s;
    char *bb = (char *)big;
    void *scr = nullptr;
    s = get_scratch(ctx, st, sizeof(double) * ((size_t)I * Pp + I), &scr);
    if (s != SV_OK) return s;
    double *Gs = (double *)scr, *Es = Gs + (size_t)I * Pp;
    SV_CUDA(cudaMemsetAsync(Gs, 0, sizeof(double) * (size_t)I * Pp, st));
    const CostSource cs = cost_of(p, weights);
    const auto &passes = pe->tiles;
    for (int64_t c0 = 0; c0 < I; c0 += chunk) {
        SlotSource src{};
        src.mode = SLOTS_INSTANCES;
        src.n_slots = (int)std::min<int64_t>(chunk, I - c0);
        src.n_instances = I;
        src.refs = (const int64_t *)drefs;
        src.theta = theta;
        src.inputs = p->inputs;
        src.input_stride = p->input_stride;
        src.slot_base = (int)c0;
        const size_t cb = (size_t)src.n_slots * sb;  // bytes of this group's states
        void *psi = bb, *lam = bb + o_lam, *ck = bb + o_ck, *mats = bb + o_mats;
        double *rho = (double *)(bb + o_rho);
        phase_mark(ctx, st);
        s = tiles_forward(ctx, pe, cfg.R, dt, src, psi, mats, true, ncp ? ck : nullptr, every, st,
                          cfg.tc);
        if (s != SV_OK) return s;
        phase_mark(ctx, st);
        cudaError_t e = cudaSuccess;
        if (ddcl_target) {
            e = launch_ddcl_lambda(c128, n, src.n_slots, psi, ddcl_target, lam, Es + c0, st);
            if (e != cudaSuccess) return cuda_fail(e, "JS divergence and its lambda");
        } else {
            s = h_tiles(ctx, obs, n, dt, src.n_slots, psi, lam, Es + c0, st, &pe->host.layout);
            if (s != SV_OK) return s;
        }
        phase_mark(ctx, st);
        SV_CUDA(cudaMemsetAsync(rho, 0, (size_t)src.n_slots * G * 64, st));
        for (int i = npass - 1; i >= 0; --i) {
            // restart psi from the stored forward state after pass i: the
            // reverse pass reads it there and writes psi (no copy)
            const void *psi_in = nullptr;
            if ((i + 1) % every == 0 && i + 1 < npass)
                psi_in = (const char *)ck + (size_t)((i + 1) / every - 1) * cb;
            const TilePass &tp = passes[i];
            const int64_t tiles = (int64_t)src.n_slots << tp.n_tile_bits;
            const uint32_t smem = tile_rev_smem(c128, tp);
            if (smem > 220u * 1024u) return fail(SV_ERR_UNSUPPORTED, "reverse pass needs too much shared memory");
            // psi after this pass is needed only if the next reverse pass
            // un-computes from it (it restarts from a stored state otherwise)
            const bool write_psi = i > 0 && !(i % every == 0 && i < npass);
            e = launch_tile_rev(c128, tp, n, src.n_slots, mats, G, psi, lam, rho,
                                tile_blocks(ctx, tiles), st, psi_in, write_psi);
            if (e != cudaSuccess) return cuda_fail(e, "reverse tile pass");
            // psi (or its stored state) and lambda read, lambda (and psi) written
            ctx->last_rev_bytes += (int64_t)cb * (write_psi ? 4 : 3);
        }
        phase_mark(ctx, st);
        e = launch_group_grads(c128, pe->dev, src, rho, cs, Es + c0, Gs + (size_t)c0 * Pp, st);
        if (e != cudaSuccess) return cuda_fail(e, "per-slot gradients");
    }
    cudaError_t e = launch_adjoint_combine(Gs, Es, I, P, cs, energy_out, loss_out, grad_out, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint combine");
    return SV_OK;
}

// ------------------------------------------------------- uneven batches

// One problem of an uneven batch, planned and placed in the batch's buffer.
struct MultiProblem {
    const sv_problem *p = nullptr;
    PlanEntry *pe = nullptr;
    ObsEntry *obs = nullptr;
    const void *drefs = nullptr;
    int n = 0, I = 0, P = 0, G = 0, npass = 0;
    size_t o_tp = 0, o_psi = 0, o_lam = 0, o_mats = 0, o_rho = 0, o_E = 0, o_G = 0;
    SlotSource src{};
};

// Launches the whole multi-problem adjoint on st (eagerly, or into a
// capture): group matrices and |ref> per problem, the forward sweeps of all
// problems as one persistent launch, lambda = H psi per problem, the reverse
// sweeps as one persistent launch, then per-problem gradients.
struct Sweep {
    size_t o_tasks = 0, o_ticket = 0, o_done = 0;
    int n_tasks = 0, blocks = 0;
    long long n_tickets = 0;
    uint32_t smem = 0;
};

sv_status multi_sequence(DeviceCtx *ctx, std::vector<MultiProblem> &mp, sv_dtype dt, int R,
                         unsigned char *base, const Sweep (&sw)[2], const double *const *theta,
                         double *const *E_out, double *const *L_out, double *const *G_out,
                         cudaStream_t st) {
    const int c128 = dt == SV_C128;
    int *err = device_err(ctx);
    if (!err) return fail(SV_ERR_CUDA, "device error word");
    for (MultiProblem &m : mp) {
        m.src.theta = theta[&m - &mp[0]];
        cudaError_t e = launch_group_mats(c128, m.pe->dev, m.src, base + m.o_mats, st);
        if (e == cudaSuccess) e = launch_init_states(c128, base + m.o_psi, m.n, m.src, st);
        if (e != cudaSuccess) return cuda_fail(e, "uneven batch: group matrices / init");
    }
    const int threads = 1 << (mp[0].pe->tiles[0].t - R);
    for (int rev = 0; rev < 2; ++rev) {
        if (rev) {  // between the sweeps: lambda = H psi, cleared sums
            for (MultiProblem &m : mp) {
                sv_status s = h_tiles(ctx, m.obs, m.n, dt, m.I, base + m.o_psi, base + m.o_lam,
                                      (double *)(base + m.o_E), st, &m.pe->host.layout);
                if (s != SV_OK) return s;
                SV_CUDA(cudaMemsetAsync(base + m.o_rho, 0, (size_t)m.I * m.G * 64, st));
                SV_CUDA(cudaMemsetAsync(base + m.o_G, 0, sizeof(double) * (size_t)m.I * (m.P > 0 ? m.P : 1), st));
            }
        }
        const Sweep &w = sw[rev];
        if (w.n_tasks == 0) continue;
        SV_CUDA(cudaMemsetAsync(base + w.o_ticket, 0, (w.o_done - w.o_ticket) + sizeof(unsigned int) * (size_t)w.n_tasks, st));
        cudaError_t e = launch_tile_sweep(c128, R, rev != 0, (const SweepTask *)(base + w.o_tasks),
                                          w.n_tasks, w.n_tickets,
                                          (unsigned long long *)(base + w.o_ticket),
                                          (unsigned int *)(base + w.o_done), err, w.blocks,
                                          threads, w.smem, st);
        if (e != cudaSuccess)
            return cuda_fail(e, ("uneven batch: persistent " + std::string(rev ? "reverse" : "forward") +
                                 " sweep (" + std::to_string(w.n_tasks) + " passes, " +
                                 std::to_string(w.blocks) + " blocks of " + std::to_string(threads) +
                                 " threads, " + std::to_string(w.smem) + " B shared)").c_str());
    }
    for (size_t j = 0; j < mp.size(); ++j) {
        MultiProblem &m = mp[j];
        const CostSource cs = cost_of(m.p, nullptr);
        const double *Es = (const double *)(base + m.o_E);
        double *Gs = (double *)(base + m.o_G);
        cudaError_t e = launch_group_grads(c128, m.pe->dev, m.src, (const double *)(base + m.o_rho),
                                           cs, Es, Gs, st);
        if (e == cudaSuccess)
            e = launch_adjoint_combine(Gs, Es, m.I, m.P, cs, E_out ? E_out[j] : nullptr,
                                       L_out ? L_out[j] : nullptr, G_out[j], st);
        if (e != cudaSuccess) return cuda_fail(e, "uneven batch: gradients");
    }
    return SV_OK;
}

sv_status multi_adjoint(DeviceCtx *ctx, const sv_problem *problems, int np,
                        const double *const *theta, double *const *E_out, double *const *L_out,
                        double *const *G_out, cudaStream_t st) {
    const sv_dtype dt = problems[0].dtype;
    const int c128 = dt == SV_C128;
    const size_t csz = c128 ? 16 : 8;
    TileCfg cfg{};
    uint64_t key = mix64(0x5e17ull, (uint64_t)np);
    for (int j = 0; j < np; ++j) {
        const sv_problem *p = &problems[j];
        if (p->dtype != dt) return fail(SV_ERR_ARG, "uneven batch: problems differ in dtype");
        if (!wants_tiles(p->circuit->n_qubits, dt, p->opts))
            return fail(SV_ERR_UNSUPPORTED, "uneven batch: every problem must take the tile path");
        TileCfg c{};
        sv_status s = tile_cfg(p->circuit->n_qubits, dt, p->opts, &c);
        if (s != SV_OK) return s;
        if (j == 0) cfg = c;
        else if (c.t != cfg.t || c.R != cfg.R || c.c != cfg.c)
            return fail(SV_ERR_UNSUPPORTED, "uneven batch: problems need one tile shape");
        key = mix64(key, mix64(hash_circuit(*p->circuit), hash_observable(*p->observable)));
        key = mix64(key, (uint64_t)p->n_instances);
        key = mix64(key, (uint64_t)p->cost);
        for (int i = 0; i < p->n_instances; ++i) key = mix64(key, (uint64_t)p->refs[i]);
        for (const void *ptr : {(const void *)theta[j], (const void *)(E_out ? E_out[j] : nullptr),
                                (const void *)(L_out ? L_out[j] : nullptr), (const void *)G_out[j],
                                (const void *)p->inputs, (const void *)p->weights,
                                (const void *)p->targets})
            key = mix64(key, (uint64_t)(uintptr_t)ptr);
        key = mix64(key, (uint64_t)p->input_stride);
    }
    key = mix64(key, mix64((uint64_t)dt, (uint64_t)(cfg.t * 8 + cfg.R)));
    std::unique_ptr<MultiGraph> &g = ctx->graphs[key];
    if (g && g->exec) {
        SV_CUDA(cudaGraphLaunch(g->exec, st));
        return SV_OK;
    }
    // plan every problem and lay out one buffer
    std::vector<MultiProblem> mp(np);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    int max_pass = 0;
    for (int j = 0; j < np; ++j) {
        MultiProblem &m = mp[j];
        m.p = &problems[j];
        m.n = m.p->circuit->n_qubits;
        m.I = m.p->n_instances;
        m.P = m.p->circuit->n_params;
        sv_status s = get_plan(ctx, *m.p->circuit, cfg.R, use_fusion(m.p->opts), dt, &m.pe, cfg.t,
                               cfg.c, use_relabel(m.p->opts));
        if (s == SV_OK) s = get_obs(ctx, *m.p->observable, m.n, dt, &m.obs, st);
        if (s == SV_OK) s = get_array(ctx, m.p->refs, sizeof(int64_t) * m.I, &m.drefs);
        HPlanEntry *hp = nullptr;
        if (s == SV_OK) s = get_hplan(m.obs, m.n, dt, &hp, &m.pe->host.layout);
        if (s != SV_OK) return s;
        m.G = m.pe->dev.n_groups;
        m.npass = (int)m.pe->tiles.size();
        max_pass = std::max(max_pass, m.npass);
        m.src.mode = SLOTS_INSTANCES;
        m.src.n_slots = m.I;
        m.src.n_instances = m.I;
        m.src.refs = (const int64_t *)m.drefs;
        m.src.inputs = m.p->inputs;
        m.src.input_stride = m.p->input_stride;
        m.o_tp = take(sizeof(TilePass) * (size_t)m.npass);
        m.o_psi = take(((size_t)m.I << m.n) * csz);
        m.o_lam = take(((size_t)m.I << m.n) * csz);
        m.o_mats = take((size_t)m.I * m.G * 4 * csz);
        m.o_rho = take((size_t)m.I * m.G * 64);
        m.o_E = take(sizeof(double) * (size_t)m.I);
        m.o_G = take(sizeof(double) * (size_t)m.I * (m.P > 0 ? m.P : 1));
    }
    // sweep task tables: level k of the forward sweep is pass k of every
    // problem that has it, level k of the reverse sweep pass npass - 1 - k;
    // chunks of kSweepChunk tiles take consecutive tickets in level order
    constexpr int kSweepChunk = 16;
    const int threads = 1 << (cfg.t - cfg.R);
    Sweep sw[2];
    std::vector<SweepTask> tasks[2];
    std::vector<std::pair<int, int>> who[2];  // (problem, pass) of each task
    for (int rev = 0; rev < 2; ++rev) {
        std::vector<int> task_of(np * (size_t)max_pass, -1);
        long long tickets = 0;
        for (int k = 0; k < max_pass; ++k)
            for (int j = 0; j < np; ++j) {
                const MultiProblem &m = mp[j];
                if (k >= m.npass) continue;
                const int pi = rev ? m.npass - 1 - k : k;
                const TilePass &tp = m.pe->tiles[pi];
                sw[rev].smem = std::max(sw[rev].smem, tile_sweep_smem(c128, rev != 0, tp));
                SweepTask T{};
                T.n = m.n;
                T.n_slots = m.I;
                T.G = m.G;
                T.dep = k > 0 ? task_of[(size_t)j * max_pass + k - 1] : -1;
                T.tiles = (int64_t)m.I << tp.n_tile_bits;
                T.chunk_tiles = kSweepChunk;
                T.n_chunks = (T.tiles + kSweepChunk - 1) / kSweepChunk;
                T.chunk_begin = tickets;
                tickets += T.n_chunks;
                task_of[(size_t)j * max_pass + k] = (int)tasks[rev].size();
                tasks[rev].push_back(T);
                who[rev].push_back({j, pi});
            }
        Sweep &w = sw[rev];
        w.n_tasks = (int)tasks[rev].size();
        w.n_tickets = tickets;
        if (w.n_tasks == 0) continue;
        if (w.smem > 220u * 1024u) return fail(SV_ERR_UNSUPPORTED, "uneven batch: pass needs too much shared memory");
        const int per_sm = tile_sweep_blocks_per_sm(c128, cfg.R, rev != 0, w.smem, threads);
        if (per_sm < 1) return fail(SV_ERR_UNSUPPORTED, "uneven batch: pass kernel does not fit an SM");
        // resident blocks only: every block that waits holds no ticket of the
        // chunks it waits for
        w.blocks = (int)std::min<long long>((long long)ctx->sms * per_sm, tickets);
        w.o_tasks = take(sizeof(SweepTask) * tasks[rev].size());
        w.o_ticket = take(sizeof(unsigned long long));
        w.o_done = w.o_ticket + sizeof(unsigned long long);
        off = w.o_done;
        take(sizeof(unsigned int) * tasks[rev].size());
    }
    std::unique_ptr<MultiGraph> ng(new MultiGraph());
    if (cudaMalloc(&ng->buf.ptr, off ? off : 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ERR_OOM, "uneven batch: states of all problems do not fit (" +
                                    std::to_string(off >> 20) + " MiB)");
    }
    ng->buf.bytes = off;
    unsigned char *base = (unsigned char *)ng->buf.ptr;
    for (MultiProblem &m : mp)
        SV_CUDA(cudaMemcpy(base + m.o_tp, m.pe->tiles.data(), sizeof(TilePass) * (size_t)m.npass,
                           cudaMemcpyHostToDevice));
    for (int rev = 0; rev < 2; ++rev) {
        for (size_t i = 0; i < tasks[rev].size(); ++i) {
            const MultiProblem &m = mp[who[rev][i].first];
            SweepTask &T = tasks[rev][i];
            T.P = (const TilePass *)(base + m.o_tp) + who[rev][i].second;
            T.mats = base + m.o_mats;
            T.psi = base + m.o_psi;
            T.lam = base + m.o_lam;
            T.rho = (double *)(base + m.o_rho);
        }
        if (!tasks[rev].empty())
            SV_CUDA(cudaMemcpy(base + sw[rev].o_tasks, tasks[rev].data(),
                               sizeof(SweepTask) * tasks[rev].size(), cudaMemcpyHostToDevice));
    }
    // this call runs eagerly; the graph serves the later ones
    sv_status s = multi_sequence(ctx, mp, dt, cfg.R, base, sw, theta, E_out, L_out, G_out, st);
    if (s != SV_OK) return s;
    if (!ctx->capture_stream)
        SV_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    SV_CUDA(cudaStreamSynchronize(st));
    cudaStream_t cap = ctx->capture_stream;
    SV_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    s = multi_sequence(ctx, mp, dt, cfg.R, base, sw, theta, E_out, L_out, G_out, cap);
    set_capturing(false);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
    if (s != SV_OK || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        g = std::move(ng);  // keep the buffer: later calls run eagerly
        return s != SV_OK ? s : cuda_fail(ec, "uneven batch: graph capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&ng->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        ng->exec = nullptr;
        return cuda_fail(ei, "uneven batch: graph instantiation");
    }
    g = std::move(ng);
    return SV_OK;
}

}  // namespace

struct sv_state_s {
    int n = 0, batch = 0;
    sv_dtype dtype = SV_C64;
    void *ptr = nullptr;
    bool owned = false;
    int device = 0;
};

extern "C" {

const char *sv_status_string(sv_status s) {
    switch (s) {
    case SV_OK: return "ok";
    case SV_ERR_ARG: return "invalid argument";
    case SV_ERR_OOM: return "out of device memory";
    case SV_ERR_CUDA: return "CUDA error";
    case SV_ERR_TIMEOUT: return "device-side wait timed out";
    case SV_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *sv_last_error(void) { return g_last_error.c_str(); }

int32_t sv_version(void) { return 1; }

sv_status sv_alloc(sv_state *out, int32_t n, int32_t batch, sv_dtype dtype, void *dev_buf,
                   size_t dev_bytes, sv_stream_t) {
    if (!out) return fail(SV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "bad dtype");
    const int lim = dtype == SV_C128 ? 29 : 30;
    if (n < 1 || n > lim) return fail(SV_ERR_ARG, "n_qubits out of range");
    if (batch < 1) return fail(SV_ERR_ARG, "batch must be >= 1");
    const size_t bytes = (size_t)batch * (size_t(1) << n) * (dtype == SV_C128 ? 16 : 8);
    std::unique_ptr<sv_state_s> s(new sv_state_s());
    s->n = n;
    s->batch = batch;
    s->dtype = dtype;
    cudaGetDevice(&s->device);
    if (dev_buf) {
        if (dev_bytes < bytes) return fail(SV_ERR_ARG, "dev_bytes smaller than the batch");
        if (((uintptr_t)dev_buf & 255) != 0) return fail(SV_ERR_ARG, "dev_buf not 256-byte aligned");
        s->ptr = dev_buf;
    } else {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && bytes > fr)
            return fail(SV_ERR_OOM, "state batch larger than free device memory");
        cudaError_t e = cudaMalloc(&s->ptr, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(state)");
        s->owned = true;
    }
    *out = s.release();
    return SV_OK;
}

sv_status sv_free(sv_state s) {
    if (!s) return SV_OK;
    if (s->owned && s->ptr) cudaFree(s->ptr);
    delete s;
    return SV_OK;
}

sv_status sv_state_info(sv_state s, void **ptr, int32_t *n, int32_t *batch, sv_dtype *dt) {
    if (!s) return fail(SV_ERR_ARG, "state is NULL");
    if (ptr) *ptr = s->ptr;
    if (n) *n = s->n;
    if (batch) *batch = s->batch;
    if (dt) *dt = s->dtype;
    return SV_OK;
}

sv_status sv_apply_circuit_batch(sv_state state, const sv_circuit *circuits, int32_t n_circuits,
                                 const sv_slot *slots, int32_t n_slots, const double *theta,
                                 int32_t theta_stride, const double *inputs,
                                 int32_t input_stride, const sv_plan_opts *opts,
                                 sv_stream_t stream) {
    if (!state) return fail(SV_ERR_ARG, "state is NULL");
    if (!circuits || n_circuits < 1) return fail(SV_ERR_ARG, "no circuits");
    if (n_slots < 0 || n_slots > state->batch) return fail(SV_ERR_ARG, "n_slots out of range");
    if (n_slots > 0 && !slots) return fail(SV_ERR_ARG, "slots is NULL");
    const int64_t dim = int64_t(1) << state->n;
    for (int c = 0; c < n_circuits; ++c) {
        sv_status s = check_circuit(&circuits[c], state->dtype == SV_C128 ? 29 : 30);
        if (s != SV_OK) return s;
        if (circuits[c].n_qubits != state->n)
            return fail(SV_ERR_UNSUPPORTED, "every circuit must have the state's n_qubits");
        if (circuits[c].n_params > 0 && (!theta || theta_stride < circuits[c].n_params))
            return fail(SV_ERR_ARG, "theta/theta_stride too small for a circuit");
        if (circuits[c].input_dim > 0 && (!inputs || input_stride < circuits[c].input_dim))
            return fail(SV_ERR_ARG, "inputs/input_stride too small for a circuit");
    }
    for (int b = 0; b < n_slots; ++b) {
        const sv_slot &sl = slots[b];
        if (sl.circuit < 0 || sl.circuit >= n_circuits) return fail(SV_ERR_ARG, "slot circuit index");
        if (sl.ref < 0 || sl.ref >= dim) return fail(SV_ERR_ARG, "slot reference out of range");
        if (sl.theta_row < 0) return fail(SV_ERR_ARG, "slot theta_row negative");
        if (sl.shift_param >= circuits[sl.circuit].n_params)
            return fail(SV_ERR_ARG, "slot shift_param out of range");
        if (circuits[sl.circuit].input_dim > 0 && sl.input_row < 0)
            return fail(SV_ERR_ARG, "slot needs an input row");
    }
    if (n_slots == 0) return SV_OK;
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    for (int c = 0; c < n_circuits; ++c) {
        // compact the slots of circuit c, keeping their output rows
        std::vector<sv_slot> sub;
        std::vector<int32_t> rows;
        for (int b = 0; b < n_slots; ++b)
            if (slots[b].circuit == c) {
                sub.push_back(slots[b]);
                rows.push_back(b);
            }
        if (sub.empty()) continue;
        if (wants_tiles(state->n, state->dtype, opts)) {
            // tile passes run in place on the state rows of this circuit
            for (size_t k = 1; k < rows.size(); ++k)
                if (rows[k] != rows[0] + (int32_t)k)
                    return fail(SV_ERR_UNSUPPORTED, "states in device memory: the slots of one "
                                                    "circuit must occupy consecutive rows");
            TileCfg cfg{};
            sv_status s = tile_cfg(state->n, state->dtype, opts, &cfg);
            if (s != SV_OK) return s;
            PlanEntry *pe = nullptr;
            s = get_plan(ctx, circuits[c], cfg.R, use_fusion(opts), state->dtype, &pe, cfg.t, cfg.c);
            if (s != SV_OK) return s;
            const void *dslots = nullptr;
            s = get_array(ctx, sub.data(), sub.size() * sizeof(sv_slot), &dslots);
            if (s != SV_OK) return s;
            const size_t csz = state->dtype == SV_C128 ? 16 : 8;
            void *mats = nullptr;
            s = get_big_scratch(ctx, st, sub.size() * pe->dev.n_groups * 4 * csz + 256, &mats);
            if (s != SV_OK) return s;
            SlotSource src{};
            src.mode = SLOTS_EXPLICIT;
            src.n_slots = (int)sub.size();
            src.theta = theta;
            src.theta_stride = theta_stride;
            src.inputs = inputs;
            src.input_stride = input_stride;
            src.slots = (const sv_slot *)dslots;
            char *rows0 = (char *)state->ptr + (size_t)rows[0] * (csz << state->n);
            s = tiles_forward(ctx, pe, cfg.R, state->dtype, src, rows0, mats, true, nullptr, 0, st,
                              cfg.tc);
            if (s != SV_OK) return s;
            continue;
        }
        PlanEntry *plan = nullptr;
        OnchipShape sh{};
        sv_status s = plan_and_shape(ctx, ONCHIP_STORE, circuits[c], state->dtype,
                                     (int)sub.size(), opts, &plan, &sh);
        if (s != SV_OK) return s;
        const void *dslots = nullptr, *drows = nullptr;
        s = get_array(ctx, sub.data(), sub.size() * sizeof(sv_slot), &dslots);
        if (s != SV_OK) return s;
        s = get_array(ctx, rows.data(), rows.size() * sizeof(int32_t), &drows);
        if (s != SV_OK) return s;
        SlotSource src{};
        src.mode = SLOTS_EXPLICIT;
        src.n_slots = (int)sub.size();
        src.theta = theta;
        src.theta_stride = theta_stride;
        src.inputs = inputs;
        src.input_stride = input_stride;
        src.slots = (const sv_slot *)dslots;
        src.rows = (const int32_t *)drows;
        cudaError_t e = launch_onchip_store(state->dtype == SV_C128, sh, plan->dev, src,
                                            state->ptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "apply_circuit_batch launch");
    }
    return SV_OK;
}

sv_status sv_sample(sv_state state, int32_t row, const double *uniforms, int64_t n_shots,
                    int64_t *samples_out, int64_t *counts_out, sv_stream_t stream) {
    if (!state) return fail(SV_ERR_ARG, "state is NULL");
    if (row < 0 || row >= state->batch) return fail(SV_ERR_ARG, "row out of range");
    if (n_shots < 0) return fail(SV_ERR_ARG, "n_shots < 0");
    if (n_shots > 0 && (!uniforms || !samples_out)) return fail(SV_ERR_ARG, "uniforms/samples_out is NULL");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    void *scr = nullptr;
    sv_status s = get_scratch(ctx, st, sample_scratch_bytes(state->n), &scr);
    if (s != SV_OK) return s;
    const size_t csz = state->dtype == SV_C128 ? 16 : 8;
    const void *psi = (const char *)state->ptr + ((size_t)row << state->n) * csz;
    cudaError_t e = launch_sample(state->dtype == SV_C128, state->n, psi, uniforms, n_shots,
                                  samples_out, counts_out, (double *)scr, st);
    return e == cudaSuccess ? SV_OK : cuda_fail(e, "sampling launch");
}

sv_status sv_expect_pauli_sum(sv_state state, const sv_pauli_sum *h, int32_t n_rows, double *out,
                              sv_stream_t stream) {
    if (!state || !h || !out) return fail(SV_ERR_ARG, "NULL argument");
    if (n_rows < 0 || n_rows > state->batch) return fail(SV_ERR_ARG, "n_rows out of range");
    if (h->n_qubits != state->n) return fail(SV_ERR_ARG, "observable qubit count differs");
    if (n_rows == 0) return SV_OK;
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ObsEntry *obs = nullptr;
    sv_status s = get_obs(ctx, *h, state->n, state->dtype, &obs, (cudaStream_t)stream);
    if (s != SV_OK) return s;
    if (wants_tiles(state->n, state->dtype, nullptr))
        return h_tiles(ctx, obs, state->n, state->dtype, n_rows, state->ptr, nullptr, out,
                       (cudaStream_t)stream);
    OnchipShape sh{};
    const char *err = onchip_shape(ONCHIP_EXPECT, state->n, 0, 0, state->dtype == SV_C128, n_rows,
                                   0, 0, &sh, ctx->sms);
    if (err) return fail(SV_ERR_UNSUPPORTED, err);
    cudaError_t e = launch_onchip_expect(state->dtype == SV_C128, sh, state->n,
                                         swz_bits(state->dtype), obs->dev, state->ptr, n_rows,
                                         out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "expect launch");
    return SV_OK;
}

namespace {

// Launches the batched energies of every parameter-shift slot into E[B]
// (and, with `fc`, the gradient assembly in the same launch).
// Energies of parameter-shift slots [slot_begin, slot_begin + B) into E[B].
// The arguments of one on-chip energy launch (recorded instead of launched).
struct EnergyLaunch {
    OnchipShape sh;
    Program prog;
    Observable obs;
    SlotSource src;
    BlockConst bc;
    const void *dtab;
    double *E;
    int32_t c128, valid;
};

sv_status ps_energies_locked(DeviceCtx *ctx, const sv_problem *p, const double *theta, double *E,
                             int B, cudaStream_t st, const FusedCombine *fc = nullptr,
                             int slot_begin = 0, EnergyLaunch *rec = nullptr) {
    const int I = p->n_instances;
    if (wants_tiles(p->circuit->n_qubits, p->dtype, p->opts)) {
        sv_status s = tiles_energies(ctx, p, theta, SLOTS_PARAM_SHIFT, B, E, st, slot_begin);
        if (s != SV_OK || !fc) return s;
        cudaError_t e = launch_ps_combine(E, fc->I, fc->P, fc->cost, fc->lp, fc->energy_out,
                                          fc->loss_out, fc->grad_out, st);
        return e == cudaSuccess ? SV_OK : cuda_fail(e, "param-shift combine launch");
    }
    PlanEntry *plan = nullptr;
    OnchipShape sh{};
    ObsEntry *obs = nullptr;
    sv_status s = get_obs(ctx, *p->observable, p->circuit->n_qubits, p->dtype, &obs, st);
    if (s != SV_OK) return s;
    const Tuned *tn = find_tuned(ctx, p, ONCHIP_ENERGY, B);
    const void *dtab = pick_dtab(obs, p->opts, tn);
    BlockConst bc{};
    s = plan_and_shape(ctx, ONCHIP_ENERGY, *p->circuit, p->dtype, B, p->opts, &plan, &sh, tn, obs,
                       dtab, &bc);
    if (s != SV_OK) return s;
    const void *drefs = nullptr;
    s = get_array(ctx, p->refs, sizeof(int64_t) * I, &drefs);
    if (s != SV_OK) return s;
    SlotSource src{};
    src.mode = SLOTS_PARAM_SHIFT;
    src.n_slots = B;
    src.n_instances = I;
    src.refs = (const int64_t *)drefs;
    src.theta = theta;
    src.inputs = p->inputs;
    src.input_stride = p->input_stride;
    src.slot_base = slot_begin;
    if (rec) {
        std::memset(rec, 0, sizeof(*rec));
        rec->sh = sh;
        rec->prog = plan->dev;
        rec->obs = obs->dev;
        rec->src = src;
        rec->bc = bc;
        rec->dtab = dtab;
        rec->E = E;
        rec->c128 = p->dtype == SV_C128;
        rec->valid = 1;
        return SV_OK;
    }
    cudaError_t e = launch_onchip_energy(p->dtype == SV_C128, sh, plan->dev, obs->dev, src, E, st,
                                         dtab, fc, &bc);
    if (e != cudaSuccess) return cuda_fail(e, "param-shift energy launch");
    return SV_OK;
}

sv_status ps_batch_size(const sv_problem *p, int *B) {
    const int64_t B64 = (int64_t)(2 * (int64_t)p->circuit->n_params + 1) * p->n_instances;
    if (B64 > (int64_t)1 << 30) return fail(SV_ERR_UNSUPPORTED, "too many shifted circuits");
    *B = (int)B64;
    return SV_OK;
}

}  // namespace

sv_status sv_param_shift_energies(const sv_problem *p, const double *theta, double *out,
                                  sv_stream_t stream) {
    sv_status s = check_problem(p, false);
    if (s != SV_OK) return s;
    if (!out) return fail(SV_ERR_ARG, "out is NULL");
    if (p->circuit->n_params > 0 && !theta) return fail(SV_ERR_ARG, "theta is NULL");
    int B = 0;
    s = ps_batch_size(p, &B);
    if (s != SV_OK) return s;
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    return ps_energies_locked(ctx, p, theta, out, B, (cudaStream_t)stream);
}

sv_status sv_param_shift_energies_range(const sv_problem *p, const double *theta,
                                        int32_t slot_begin, int32_t n_slots, double *out,
                                        sv_stream_t stream) {
    sv_status s = check_problem(p, false);
    if (s != SV_OK) return s;
    if (!out && n_slots > 0) return fail(SV_ERR_ARG, "out is NULL");
    if (p->circuit->n_params > 0 && !theta) return fail(SV_ERR_ARG, "theta is NULL");
    int B = 0;
    s = ps_batch_size(p, &B);
    if (s != SV_OK) return s;
    if (slot_begin < 0 || n_slots < 0 || (int64_t)slot_begin + n_slots > B)
        return fail(SV_ERR_ARG, "slot range outside the parameter-shift batch of " +
                                    std::to_string(B) + " circuits");
    if (n_slots == 0) return SV_OK;
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    return ps_energies_locked(ctx, p, theta, out, n_slots, (cudaStream_t)stream, nullptr, slot_begin);
}

sv_status sv_param_shift_combine(const sv_problem *p, const double *energies, double *energy_out,
                                 double *loss_out, double *grad_out, sv_stream_t stream) {
    sv_status s = check_problem(p, true);
    if (s != SV_OK) return s;
    if (!energies) return fail(SV_ERR_ARG, "energies is NULL");
    const int P = p->circuit->n_params;
    if (P > 0 && !grad_out) return fail(SV_ERR_ARG, "grad_out is NULL");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    void *scr = nullptr;
    s = get_scratch(ctx, st, sizeof(double) * (size_t)p->n_instances, &scr);
    if (s != SV_OK) return s;
    cudaError_t e = launch_ps_combine(energies, p->n_instances, P, cost_of(p, nullptr), (double *)scr,
                                      energy_out, loss_out, grad_out, st);
    return e == cudaSuccess ? SV_OK : cuda_fail(e, "param-shift combine launch");
}

sv_status sv_grad_param_shift(const sv_problem *p, const double *theta, double *energy_out,
                              double *loss_out, double *grad_out, sv_stream_t stream) {
    sv_status s = check_problem(p, true);
    if (s != SV_OK) return s;
    const int P = p->circuit->n_params, I = p->n_instances;
    if (P > 0 && (!theta || !grad_out)) return fail(SV_ERR_ARG, "theta/grad_out is NULL");
    int B = 0;
    s = ps_batch_size(p, &B);
    if (s != SV_OK) return s;
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    void *scr = nullptr;
    s = get_scratch(ctx, st, sizeof(double) * ((size_t)B + I), &scr);
    if (s != SV_OK) return s;
    double *E = (double *)scr, *lp = E + B;
    FusedCombine fc{};
    fc.I = I;
    fc.P = P;
    fc.cost = cost_of(p, nullptr);
    fc.lp = lp;
    fc.energy_out = energy_out;
    fc.loss_out = loss_out;
    fc.grad_out = grad_out;
    return ps_energies_locked(ctx, p, theta, E, B, st, &fc);
}

sv_status sv_grad_param_shift_host(const sv_problem *p, const double *theta_host,
                                   double *energy_host, double *loss_host, double *grad_host,
                                   sv_stream_t stream) {
    sv_status s = check_problem(p, true);
    if (s != SV_OK) return s;
    const int P = p->circuit->n_params, I = p->n_instances;
    if (P > 0 && (!theta_host || !grad_host)) return fail(SV_ERR_ARG, "theta/grad is NULL");
    int B = 0;
    s = ps_batch_size(p, &B);
    if (s != SV_OK) return s;
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    // staging, in doubles: [theta P][loss 1][grad P][energies I]
    const size_t nP = (size_t)(P > 0 ? P : 1), n_out = 1 + nP + (size_t)I;
    HostIO *io = nullptr;
    s = get_hostio(ctx, st, sizeof(double) * (nP + n_out), &io);
    if (s != SV_OK) return s;
    void *scr = nullptr;
    s = get_scratch(ctx, st, sizeof(double) * ((size_t)B + I), &scr);
    if (s != SV_OK) return s;
    double *h = (double *)io->host, *d = (double *)io->dev;
    double *E = (double *)scr;
    FusedCombine fc{};
    fc.I = I;
    fc.P = P;
    fc.cost = cost_of(p, nullptr);
    fc.lp = E + B;
    fc.loss_out = d + nP;
    fc.grad_out = d + nP + 1;
    fc.energy_out = d + 2 * nP + 1;
    if (P > 0) std::memcpy(h, theta_host, sizeof(double) * P);
    auto copy_in = [&](cudaStream_t q) {
        return P > 0 ? cudaMemcpyAsync(d, h, sizeof(double) * P, cudaMemcpyHostToDevice, q)
                     : cudaSuccess;
    };
    auto copy_out = [&](cudaStream_t q) {
        return cudaMemcpyAsync(h + nP, d + nP, sizeof(double) * n_out, cudaMemcpyDeviceToHost, q);
    };
    EnergyLaunch L;
    L.valid = 0;
    if (!wants_tiles(p->circuit->n_qubits, p->dtype, p->opts)) {
        s = ps_energies_locked(ctx, p, d, E, B, st, &fc, 0, &L);
        if (s != SV_OK) return s;
    }
    if (!L.valid) {  // states in device memory: the passes launch as they plan
        SV_CUDA(copy_in(st));
        s = ps_energies_locked(ctx, p, d, E, B, st, &fc);
        if (s != SV_OK) return s;
        SV_CUDA(copy_out(st));
    } else {
        // the whole call as one graph, keyed by everything its nodes read
        uint64_t key = hash_bytes(&L, sizeof(L));
        key = mix64(key, hash_bytes(&fc, sizeof(fc)));
        key = mix64(key, mix64((uint64_t)(uintptr_t)h, (uint64_t)(uintptr_t)d));
        key = mix64(key, mix64((uint64_t)P, (uint64_t)n_out));
        // a bounded cache: a caller cycling through many problems (or staging
        // buffers) re-records instead of growing it without limit
        if (ctx->host_graphs.size() >= 64 && !ctx->host_graphs.count(key)) {
            SV_CUDA(cudaDeviceSynchronize());  // no recorded call still running
            ctx->host_graphs.clear();
        }
        std::unique_ptr<HostGraph> &g = ctx->host_graphs[key];
        if (g && g->exec) {
            SV_CUDA(cudaGraphLaunch(g->exec, st));
        } else {
            SV_CUDA(copy_in(st));
            cudaError_t e = launch_onchip_energy(L.c128, L.sh, L.prog, L.obs, L.src, L.E, st, L.dtab,
                                                 &fc, &L.bc);
            if (e != cudaSuccess) return cuda_fail(e, "param-shift energy launch");
            SV_CUDA(copy_out(st));
            if (!g) {  // record the same three steps once for later calls
                g.reset(new HostGraph());
                if (!ctx->capture_stream)
                    SV_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
                cudaStream_t cap = ctx->capture_stream;
                cudaGraph_t graph = nullptr;
                bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    ok = copy_in(cap) == cudaSuccess &&
                         launch_onchip_energy(L.c128, L.sh, L.prog, L.obs, L.src, L.E, cap, L.dtab,
                                              &fc, &L.bc) == cudaSuccess &&
                         copy_out(cap) == cudaSuccess;
                    ok = cudaStreamEndCapture(cap, &graph) == cudaSuccess && ok && graph;
                }
                if (ok) ok = cudaGraphInstantiate(&g->exec, graph, 0) == cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
                if (!ok) {
                    g->exec = nullptr;
                    g->failed = true;
                    cudaGetLastError();  // a refused capture leaves no pending error behind
                }
            }
        }
    }
    SV_CUDA(cudaStreamSynchronize(st));
    if (loss_host) *loss_host = h[nP];
    if (P > 0) std::memcpy(grad_host, h + nP + 1, sizeof(double) * P);
    if (energy_host) std::memcpy(energy_host, h + 2 * nP + 1, sizeof(double) * I);
    return SV_OK;
}

sv_status sv_energies(const sv_problem *p, const double *theta, double *energy_out,
                      double *loss_out, sv_stream_t stream) {
    sv_status s = check_problem(p, loss_out != nullptr);
    if (s != SV_OK) return s;
    const int P = p->circuit->n_params, I = p->n_instances;
    if (!energy_out) return fail(SV_ERR_ARG, "energy_out is NULL");
    if (P > 0 && !theta) return fail(SV_ERR_ARG, "theta is NULL");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    if (wants_tiles(p->circuit->n_qubits, p->dtype, p->opts)) {
        s = tiles_energies(ctx, p, theta, SLOTS_INSTANCES, I, energy_out, st);
        if (s != SV_OK) return s;
        if (loss_out) {
            void *scr = nullptr;
            s = get_scratch(ctx, st, sizeof(double) * I, &scr);
            if (s != SV_OK) return s;
            cudaError_t e = launch_ps_combine(energy_out, I, 0, cost_of(p, nullptr), (double *)scr,
                                              nullptr, loss_out, nullptr, st);
            if (e != cudaSuccess) return cuda_fail(e, "loss launch");
        }
        return SV_OK;
    }
    PlanEntry *plan = nullptr;
    OnchipShape sh{};
    ObsEntry *obs = nullptr;
    s = get_obs(ctx, *p->observable, p->circuit->n_qubits, p->dtype, &obs, st);
    if (s != SV_OK) return s;
    const void *dtab = pick_dtab(obs, p->opts, nullptr);
    BlockConst bc{};
    s = plan_and_shape(ctx, ONCHIP_ENERGY, *p->circuit, p->dtype, I, p->opts, &plan, &sh, nullptr,
                       obs, dtab, &bc);
    if (s != SV_OK) return s;
    const void *drefs = nullptr;
    s = get_array(ctx, p->refs, sizeof(int64_t) * I, &drefs);
    if (s != SV_OK) return s;
    SlotSource src{};
    src.mode = SLOTS_INSTANCES;
    src.n_slots = I;
    src.n_instances = I;
    src.refs = (const int64_t *)drefs;
    src.theta = theta;
    src.inputs = p->inputs;
    src.input_stride = p->input_stride;
    cudaError_t e = launch_onchip_energy(p->dtype == SV_C128, sh, plan->dev, obs->dev, src,
                                         energy_out, st, dtab, nullptr, &bc);
    if (e != cudaSuccess) return cuda_fail(e, "energy launch");
    if (loss_out) {
        void *scr = nullptr;
        s = get_scratch(ctx, st, sizeof(double) * I, &scr);
        if (s != SV_OK) return s;
        e = launch_ps_combine(energy_out, I, 0, cost_of(p, nullptr), (double *)scr, nullptr,
                              loss_out, nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "loss launch");
    }
    return SV_OK;
}

namespace {

// The adjoint gradient with ctx->mu held (arguments checked by the caller).
sv_status adjoint_locked(DeviceCtx *ctx, const sv_problem *p, const double *theta,
                         const double *weights, double *energy_out, double *loss_out,
                         double *grad_out, int checkpoint_every, cudaStream_t st) {
    sv_status s = SV_OK;
    const int P = p->circuit->n_params, I = p->n_instances;
    ctx->last_every = 0;  // on chip unless the tile path records its own
    ctx->last_rev_bytes = 0;
    if (wants_tiles(p->circuit->n_qubits, p->dtype, p->opts))
        return tiles_adjoint(ctx, p, theta, weights, energy_out, loss_out, grad_out,
                             checkpoint_every, st);
    PlanEntry *plan = nullptr;
    OnchipShape sh{};
    ObsEntry *obs = nullptr;
    s = get_obs(ctx, *p->observable, p->circuit->n_qubits, p->dtype, &obs, st);
    if (s != SV_OK) return s;
    BlockConst bc{};
    s = plan_and_shape(ctx, ONCHIP_ADJOINT, *p->circuit, p->dtype, I, p->opts, &plan, &sh,
                       find_tuned(ctx, p, ONCHIP_ADJOINT, I), obs, nullptr, &bc);
    // A deep circuit whose per-group reduced-matrix buffers leave no room for
    // one slot in shared memory runs as tile passes instead (a state of
    // n >= 7 qubits has at least two tiles' worth of amplitudes to split).
    if (s == SV_ERR_UNSUPPORTED && p->circuit->n_qubits >= 7 &&
        !(p->opts && (p->opts->reg_bits > 0 || p->opts->threads_per_block > 0)))
        return tiles_adjoint(ctx, p, theta, weights, energy_out, loss_out, grad_out,
                             checkpoint_every, st);
    if (s != SV_OK) return s;
    const void *drefs = nullptr;
    s = get_array(ctx, p->refs, sizeof(int64_t) * I, &drefs);
    if (s != SV_OK) return s;
    void *scr = nullptr;
    s = get_scratch(ctx, st, sizeof(double) * ((size_t)I * (P > 0 ? P : 1) + I), &scr);
    if (s != SV_OK) return s;
    double *G = (double *)scr, *E = G + (size_t)I * (P > 0 ? P : 1);
    SlotSource src{};
    src.mode = SLOTS_INSTANCES;
    src.n_slots = I;
    src.n_instances = I;
    src.refs = (const int64_t *)drefs;
    src.theta = theta;
    src.inputs = p->inputs;
    src.input_stride = p->input_stride;
    const CostSource cs = cost_of(p, weights);
    cudaError_t e = launch_onchip_adjoint(p->dtype == SV_C128, sh, plan->dev, obs->dev, src, cs,
                                          G, E, st, &bc, obs->dtab.ptr);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    e = launch_adjoint_combine(G, E, I, P, cs, energy_out, loss_out, grad_out, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint combine launch");
    return SV_OK;
}

}  // namespace

sv_status sv_grad_adjoint(const sv_problem *p, const double *theta, const double *weights,
                          double *energy_out, double *loss_out, double *grad_out,
                          int32_t checkpoint_every, sv_stream_t stream) {
    sv_status s = check_problem(p, weights == nullptr);
    if (s != SV_OK) return s;
    if (checkpoint_every < 0) return fail(SV_ERR_ARG, "checkpoint_every must be >= 0");
    const int P = p->circuit->n_params;
    if (P > 0 && (!theta || !grad_out)) return fail(SV_ERR_ARG, "theta/grad_out is NULL");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    return adjoint_locked(ctx, p, theta, weights, energy_out, loss_out, grad_out,
                          checkpoint_every, (cudaStream_t)stream);
}

sv_status sv_grad_adjoint_host(const sv_problem *p, const double *theta_host,
                               double *energy_host, double *loss_host, double *grad_host,
                               int32_t checkpoint_every, sv_stream_t stream) {
    sv_status s = check_problem(p, true);
    if (s != SV_OK) return s;
    if (checkpoint_every < 0) return fail(SV_ERR_ARG, "checkpoint_every must be >= 0");
    const int P = p->circuit->n_params, I = p->n_instances;
    if (P > 0 && (!theta_host || !grad_host)) return fail(SV_ERR_ARG, "theta/grad is NULL");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    // staging, in doubles: [theta P][loss 1][grad P][energies I]
    const size_t nP = (size_t)(P > 0 ? P : 1), n_out = 1 + nP + (size_t)I;
    HostIO *io = nullptr;
    s = get_hostio(ctx, st, sizeof(double) * (nP + n_out), &io);
    if (s != SV_OK) return s;
    double *h = (double *)io->host, *d = (double *)io->dev;
    if (P > 0) {
        std::memcpy(h, theta_host, sizeof(double) * P);
        SV_CUDA(cudaMemcpyAsync(d, h, sizeof(double) * P, cudaMemcpyHostToDevice, st));
    }
    s = adjoint_locked(ctx, p, d, nullptr, d + 2 * nP + 1, d + nP, d + nP + 1, checkpoint_every,
                       st);
    if (s != SV_OK) return s;
    SV_CUDA(cudaMemcpyAsync(h + nP, d + nP, sizeof(double) * n_out, cudaMemcpyDeviceToHost, st));
    SV_CUDA(cudaStreamSynchronize(st));
    if (loss_host) *loss_host = h[nP];
    if (P > 0) std::memcpy(grad_host, h + nP + 1, sizeof(double) * P);
    if (energy_host) std::memcpy(energy_host, h + 2 * nP + 1, sizeof(double) * I);
    return SV_OK;
}

sv_status sv_grad_ddcl(const sv_problem *p, const double *theta, const double *target,
                       double *js_out, double *grad_out, sv_stream_t stream) {
    if (!p || !p->circuit) return fail(SV_ERR_ARG, "problem or circuit is NULL");
    if (!target || !js_out) return fail(SV_ERR_ARG, "target/js_out is NULL");
    sv_status s = check_circuit(p->circuit, p->dtype == SV_C128 ? 29 : 30);
    if (s != SV_OK) return s;
    const int n = p->circuit->n_qubits, P = p->circuit->n_params;
    if (p->n_instances != 1 || !p->refs) return fail(SV_ERR_ARG, "data-driven circuit learning takes one instance");
    if (P > 0 && (!theta || !grad_out)) return fail(SV_ERR_ARG, "theta/grad_out is NULL");
    if (p->circuit->input_dim > 0 && !p->inputs) return fail(SV_ERR_ARG, "inputs are NULL");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    // the tile path at every size (a whole small state is one tile)
    TileCfg cfg{};
    sv_plan_opts o{};
    if (p->opts) o = *p->opts;
    if (o.tile_bits <= 0 && !wants_tiles(n, p->dtype, p->opts)) {
        o.tile_bits = std::min(n, p->dtype == SV_C128 ? 10 : 11);
        if (o.reg_bits <= 0) o.reg_bits = std::max(2, std::min(p->dtype == SV_C128 ? 2 : 4, o.tile_bits - 5));
    }
    s = tile_cfg(n, p->dtype, &o, &cfg);
    if (s != SV_OK) return s;
    const double one = 1.0;
    const void *w1 = nullptr;
    s = get_array(ctx, &one, sizeof(double), &w1);
    if (s != SV_OK) return s;
    sv_problem q = *p;
    q.opts = &o;
    q.cost = SV_COST_LINEAR;
    return tiles_adjoint(ctx, &q, theta, (const double *)w1, js_out, nullptr, grad_out, 0,
                         (cudaStream_t)stream, target, &cfg);
}

sv_status sv_grad_ddcl_param_shift(const sv_problem *p, const double *theta,
                                   const double *target, double *js_out, double *grad_out,
                                   sv_stream_t stream) {
    if (!p || !p->circuit) return fail(SV_ERR_ARG, "problem or circuit is NULL");
    if (!target || !js_out) return fail(SV_ERR_ARG, "target/js_out is NULL");
    sv_status s = check_circuit(p->circuit, p->dtype == SV_C128 ? 29 : 30);
    if (s != SV_OK) return s;
    const int n = p->circuit->n_qubits, P = p->circuit->n_params;
    if (p->n_instances != 1 || !p->refs) return fail(SV_ERR_ARG, "data-driven circuit learning takes one instance");
    if (P > 0 && (!theta || !grad_out)) return fail(SV_ERR_ARG, "theta/grad_out is NULL");
    if (p->circuit->input_dim > 0 && !p->inputs) return fail(SV_ERR_ARG, "inputs are NULL");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    const sv_dtype dt = p->dtype;
    const int c128 = dt == SV_C128;
    // tile passes at every size, as for the adjoint form (identity layout:
    // the derivative table is indexed like the target)
    sv_plan_opts o{};
    if (p->opts) o = *p->opts;
    if (o.tile_bits <= 0 && !wants_tiles(n, dt, p->opts)) {
        o.tile_bits = std::min(n, c128 ? 10 : 11);
        if (o.reg_bits <= 0) o.reg_bits = std::max(2, std::min(c128 ? 2 : 4, o.tile_bits - 5));
    }
    TileCfg cfg{};
    s = tile_cfg(n, dt, &o, &cfg);
    if (s != SV_OK) return s;
    PlanEntry *pe = nullptr;
    s = get_plan(ctx, *p->circuit, cfg.R, use_fusion(&o), dt, &pe, cfg.t, cfg.c, false);
    if (s != SV_OK) return s;
    const void *drefs = nullptr;
    s = get_array(ctx, p->refs, sizeof(int64_t), &drefs);
    if (s != SV_OK) return s;
    const double one = 1.0;
    const void *w1 = nullptr;
    s = get_array(ctx, &one, sizeof(double), &w1);
    if (s != SV_OK) return s;
    const int B = 2 * P + 1;
    const size_t dim = size_t(1) << n;
    void *scr = nullptr;
    s = get_scratch(ctx, st, sizeof(double) * ((size_t)B + 1 + dim), &scr);
    if (s != SV_OK) return s;
    double *E = (double *)scr, *lp = E + B, *D = lp + 1;
    const size_t csz = c128 ? 16 : 8, sb = csz << n;
    const size_t mb = (size_t)pe->dev.n_groups * 4 * csz;
    int64_t chunk = (int64_t)(big_budget(ctx, st) / (sb + mb + 512));
    if (chunk < 1) return fail(SV_ERR_OOM, "one state does not fit in free device memory");
    if (chunk > B) chunk = B;
    if (chunk > 65535) chunk = 65535;
    void *big = nullptr;
    const size_t mats_off = ((size_t)chunk * sb + 255) & ~size_t(255);
    s = get_big_scratch(ctx, st, mats_off + (size_t)chunk * mb + 256, &big);
    if (s != SV_OK) return s;
    SlotSource src{};
    src.mode = SLOTS_PARAM_SHIFT;
    src.n_instances = 1;
    src.refs = (const int64_t *)drefs;
    src.theta = theta;
    src.inputs = p->inputs;
    src.input_stride = p->input_stride;
    // the unshifted circuit (slot 0): JS and the table dJS/dP_theta
    src.n_slots = 1;
    src.slot_base = 0;
    s = tiles_forward(ctx, pe, cfg.R, dt, src, big, (char *)big + mats_off, true, nullptr, 0, st,
                      cfg.tc);
    if (s != SV_OK) return s;
    cudaError_t e = launch_ddcl_diag(c128, n, big, target, D, js_out, st);
    if (e != cudaSuccess) return cuda_fail(e, "JS divergence and its derivative table");
    // every circuit of the batch: <psi_s| diag(dJS/dP_theta) |psi_s>
    for (int64_t c0 = 0; c0 < B; c0 += chunk) {
        src.n_slots = (int)std::min<int64_t>(chunk, B - c0);
        src.slot_base = (int)c0;
        s = tiles_forward(ctx, pe, cfg.R, dt, src, big, (char *)big + mats_off, true, nullptr, 0, st,
                          cfg.tc);
        if (s != SV_OK) return s;
        e = launch_diag_expect(c128, n, src.n_slots, big, D, E + c0, st);
        if (e != cudaSuccess) return cuda_fail(e, "shifted-circuit table expectations");
    }
    CostSource cs{};
    cs.cost = SV_COST_LINEAR;
    cs.n_instances = 1;
    cs.weights = (const double *)w1;
    e = launch_ps_combine(E, 1, P, cs, lp, nullptr, nullptr, P > 0 ? grad_out : nullptr, st);
    return e == cudaSuccess ? SV_OK : cuda_fail(e, "parameter-shift combine launch");
}

sv_status sv_grad_adjoint_multi(const sv_problem *problems, int32_t n_problems,
                                const double *const *theta, double *const *energy_out,
                                double *const *loss_out, double *const *grad_out,
                                sv_stream_t stream) {
    if (!problems || n_problems < 1 || !theta || !grad_out)
        return fail(SV_ERR_ARG, "problems/theta/grad_out is NULL or n_problems < 1");
    for (int j = 0; j < n_problems; ++j) {
        sv_status s = check_problem(&problems[j], true);
        if (s != SV_OK) return s;
        if (problems[j].circuit->n_params > 0 && (!theta[j] || !grad_out[j]))
            return fail(SV_ERR_ARG, "theta[j]/grad_out[j] is NULL");
    }
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    return multi_adjoint(ctx, problems, n_problems, theta, energy_out, loss_out, grad_out,
                         (cudaStream_t)stream);
}

// -------------------------------------------------------------- plain form

namespace {

void host_rotation(int axis, double a, double2 m[4]) {
    const double c = std::cos(0.5 * a), s = std::sin(0.5 * a);
    if (axis == 0) {
        m[0] = make_double2(c, 0); m[1] = make_double2(0, -s); m[2] = make_double2(0, -s); m[3] = make_double2(c, 0);
    } else if (axis == 1) {
        m[0] = make_double2(c, 0); m[1] = make_double2(-s, 0); m[2] = make_double2(s, 0); m[3] = make_double2(c, 0);
    } else {
        m[0] = make_double2(c, -s); m[1] = make_double2(0, 0); m[2] = make_double2(0, 0); m[3] = make_double2(c, s);
    }
}

}  // namespace

sv_status sv_grad_param_shift_plain(const sv_problem *p, const double *theta, double *energy_out,
                                    double *loss_out, double *grad_out, sv_stream_t stream) {
    sv_status s = check_problem(p, true);
    if (s != SV_OK) return s;
    const sv_circuit &c = *p->circuit;
    const int n = c.n_qubits, P = c.n_params, I = p->n_instances;
    if (n > 29) return fail(SV_ERR_UNSUPPORTED, "plain form limited to 29 qubits");
    if (P > 0 && (!theta || !grad_out)) return fail(SV_ERR_ARG, "theta/grad_out is NULL");
    for (int g = 0; g < c.n_gates; ++g) {
        const sv_gate &G = c.gates[g];
        if (G.target < 0 || G.target >= n || G.op < 0 || G.op > SV_GATE_ENC_RZ_ACOS_SQ)
            return fail(SV_ERR_ARG, "bad gate");
        if ((G.op == SV_GATE_CNOT || G.op == SV_GATE_CZ) &&
            (G.control < 0 || G.control >= n || G.control == G.target))
            return fail(SV_ERR_ARG, "bad control");
        if (G.op <= SV_GATE_RZ && G.param >= P) return fail(SV_ERR_ARG, "param out of range");
        if (G.op >= SV_GATE_ENC_RY_ASIN && (G.param < 0 || G.param >= c.input_dim))
            return fail(SV_ERR_ARG, "input column out of range");
    }
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    // The plain form is driven from the host: parameters come back first.
    std::vector<double> th(P), xs;
    if (P) SV_CUDA(cudaMemcpyAsync(th.data(), theta, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
    if (c.input_dim > 0) {
        xs.resize((size_t)I * p->input_stride);
        SV_CUDA(cudaMemcpyAsync(xs.data(), p->inputs, sizeof(double) * xs.size(),
                                cudaMemcpyDeviceToHost, st));
    }
    SV_CUDA(cudaStreamSynchronize(st));
    const int B = (2 * P + 1) * I;
    const size_t dim = size_t(1) << n;
    void *scr = nullptr;
    s = get_scratch(ctx, st, sizeof(double) * ((size_t)B + I) + 16 * dim + 256, &scr);
    if (s != SV_OK) return s;
    double *E = (double *)scr, *lp = E + B;
    double2 *psi = (double2 *)(((uintptr_t)(lp + I) + 255) & ~uintptr_t(255));
    SV_CUDA(cudaMemsetAsync(E, 0, sizeof(double) * B, st));
    std::vector<std::vector<uint32_t>> xz;
    const sv_pauli_sum &h = *p->observable;
    for (int b = 0; b < B; ++b) {
        int inst = b, sp = -1;
        double shift = 0.0;
        if (b >= I) {
            const int bb = b - I, k = bb / (2 * I), r = bb % (2 * I);
            inst = r % I;
            sp = k;
            shift = r < I ? 1.5707963267948966 : -1.5707963267948966;
        }
        cudaError_t e = launch_plain_init(psi, n, p->refs[inst], st);
        if (e != cudaSuccess) return cuda_fail(e, "plain init");
        for (int g = 0; g < c.n_gates; ++g) {
            const sv_gate &G = c.gates[g];
            double2 m[4];
            if (G.op == SV_GATE_CNOT || G.op == SV_GATE_CZ) {
                e = G.op == SV_GATE_CNOT ? launch_plain_cx(psi, n, G.control, G.target, st)
                                         : launch_plain_cz(psi, n, G.control, G.target, st);
                if (e != cudaSuccess) return cuda_fail(e, "plain gate");
                continue;
            }
            switch (G.op) {
            case SV_GATE_RX:
            case SV_GATE_RY:
            case SV_GATE_RZ: {
                double a = G.angle;
                if (G.param >= 0) a = th[G.param] + (G.param == sp ? shift : 0.0);
                host_rotation(G.op - SV_GATE_RX, a, m);
                break;
            }
            case SV_GATE_X:
                m[0] = make_double2(0, 0); m[1] = make_double2(1, 0); m[2] = make_double2(1, 0); m[3] = make_double2(0, 0);
                break;
            case SV_GATE_H: {
                const double r2 = 0.70710678118654752440;
                m[0] = make_double2(r2, 0); m[1] = make_double2(r2, 0); m[2] = make_double2(r2, 0); m[3] = make_double2(-r2, 0);
                break;
            }
            case SV_GATE_ENC_RY_ASIN:
                host_rotation(1, std::asin(xs[(size_t)inst * p->input_stride + G.param]), m);
                break;
            default: {
                const double x = xs[(size_t)inst * p->input_stride + G.param];
                host_rotation(2, std::acos(x * x), m);
                break;
            }
            }
            e = launch_plain_u1(psi, n, G.target, m, st);
            if (e != cudaSuccess) return cuda_fail(e, "plain gate");
        }
        for (int t = 0; t < h.n_terms; ++t) {
            const uint32_t x = (uint32_t)h.x_mask[t], z = (uint32_t)h.z_mask[t];
            e = launch_plain_term(psi, n, x, z, __builtin_popcount(x & z) & 3, h.coeff[t], E + b, st);
            if (e != cudaSuccess) return cuda_fail(e, "plain term");
        }
    }
    cudaError_t e = launch_ps_combine(E, I, P, cost_of(p, nullptr), lp, energy_out, loss_out,
                                      grad_out, st);
    if (e != cudaSuccess) return cuda_fail(e, "plain combine");
    return SV_OK;
}

// Tile shapes (tile bits t, register bits R) for the energies of the
// instances (kinds bit 1) and the adjoint gradient (bit 2) of a problem whose
// states live in device memory: each candidate runs once to plan and warm,
// then the faster of two CUDA-event-timed calls counts.
sv_status tune_tiles(const sv_problem *p, const double *theta, int32_t kinds, cudaStream_t st) {
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    if (p->opts && (p->opts->tile_bits > 0 || p->opts->reg_bits > 0)) return SV_OK;  // fixed by the caller
    const int n = p->circuit->n_qubits, I = p->n_instances, Pp = p->circuit->n_params > 0 ? p->circuit->n_params : 1;
    const bool c128 = p->dtype == SV_C128;
    // (tile bits, register bits, tensor-core blocks)
    const int cand_c64[][3] = {{11, 4, 0}, {11, 3, 0}, {12, 4, 0}, {10, 3, 0}, {10, 4, 0},
                               {11, 4, 1}, {12, 4, 1}};
    const int cand_c128[][3] = {{10, 2, 0}, {10, 3, 0}, {11, 3, 0}, {9, 2, 0}};
    void *out = nullptr;
    const size_t need = sizeof(double) * (2 * (size_t)I + Pp + 2);
    if (cudaMalloc(&out, need) != cudaSuccess) return fail(SV_ERR_OOM, "tuning outputs");
    double *E = (double *)out, *L = E + I, *G = L + 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    sv_status result = SV_OK;
    for (int key : {kTileEnergyKey, kTileAdjointKey}) {
        if (!(kinds & (key == kTileEnergyKey ? 1 : 2))) continue;
        Tuned best;
        best.us = 1e30f;
        const int nc = c128 ? 4 : 7;
        for (int ci = 0; ci < nc; ++ci) {
            const int t = c128 ? cand_c128[ci][0] : cand_c64[ci][0];
            const int R = c128 ? cand_c128[ci][1] : cand_c64[ci][1];
            const int tc = c128 ? cand_c128[ci][2] : cand_c64[ci][2];
            if (t > n || t - R < 5) continue;
            sv_plan_opts o{};
            if (p->opts) o = *p->opts;
            o.tile_bits = t;
            o.reg_bits = R;
            o.tensor_blocks = tc;
            sv_problem q = *p;
            q.opts = &o;
            auto run = [&]() {
                return key == kTileEnergyKey ? sv_energies(&q, theta, E, L, st)
                                             : sv_grad_adjoint(&q, theta, nullptr, E, L, G, 0, st);
            };
            if (run() != SV_OK) continue;  // unsupported shape for this problem
            float tbest = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(e0, st);
                if (run() != SV_OK) break;
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < tbest) tbest = ms;
            }
            if (tbest * 1e3f < best.us) {
                best.us = tbest * 1e3f;
                best.R = R;
                best.tpb = 1 << (t - R);
                best.tc = tc;
            }
        }
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (best.R > 0) ctx->tuned[tune_key(p, key, I)] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return result;
}

sv_status sv_autotune(const sv_problem *p, const double *theta, int32_t kinds,
                      sv_stream_t stream) {
    sv_status s = check_problem(p, true);
    if (s != SV_OK) return s;
    if (p->circuit->n_params > 0 && !theta) return fail(SV_ERR_ARG, "theta is NULL");
    if (kinds & ~3) return fail(SV_ERR_ARG, "kinds must be a combination of 1 and 2");
    const int P = p->circuit->n_params, I = p->n_instances, n = p->circuit->n_qubits;
    if (wants_tiles(n, p->dtype, p->opts)) return tune_tiles(p, theta, kinds, (cudaStream_t)stream);
    int B = 0;
    s = ps_batch_size(p, &B);
    if (s != SV_OK) return s;
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    ObsEntry *obs = nullptr;
    s = get_obs(ctx, *p->observable, n, p->dtype, &obs, st);
    if (s != SV_OK) return s;
    const void *drefs = nullptr;
    s = get_array(ctx, p->refs, sizeof(int64_t) * I, &drefs);
    if (s != SV_OK) return s;
    const size_t need = sizeof(double) * ((size_t)B + (size_t)I * (P > 0 ? P : 1) + 2 * I);
    void *scr = nullptr;
    s = get_scratch(ctx, st, need, &scr);
    if (s != SV_OK) return s;
    double *E = (double *)scr, *G = E + B, *E2 = G + (size_t)I * (P > 0 ? P : 1);
    cudaEvent_t e0, e1;
    SV_CUDA(cudaEventCreate(&e0));
    SV_CUDA(cudaEventCreate(&e1));
    const int rmax = p->dtype == SV_C128 ? 3 : 4;
    const int tpbs[] = {32, 64, 128, 256, 512};
    for (int kind : {ONCHIP_ENERGY, ONCHIP_ADJOINT}) {
        if (!(kinds & (kind == ONCHIP_ENERGY ? 1 : 2))) continue;
        const int slots = kind == ONCHIP_ENERGY ? B : I;
        Tuned best;
        best.us = 1e30f;
        for (int epi = 1; epi <= (kind == ONCHIP_ENERGY && obs->dtab.ptr ? 2 : 1); ++epi)
        for (int R = 1; R <= rmax && R <= n; ++R) {
            for (int tpb : tpbs) {
                sv_plan_opts o{};
                if (p->opts) o = *p->opts;
                o.reg_bits = R;
                o.threads_per_block = tpb;
                PlanEntry *plan = nullptr;
                OnchipShape sh{};
                const void *dt = (kind == ONCHIP_ENERGY && epi == 2) ? obs->dtab.ptr : nullptr;
                BlockConst bc{};
                if (plan_and_shape(ctx, kind, *p->circuit, p->dtype, slots, &o, &plan, &sh, nullptr,
                                   obs, dt, &bc) != SV_OK)
                    continue;
                SlotSource src{};
                src.mode = kind == ONCHIP_ENERGY ? SLOTS_PARAM_SHIFT : SLOTS_INSTANCES;
                src.n_slots = slots;
                src.n_instances = I;
                src.refs = (const int64_t *)drefs;
                src.theta = theta;
                src.inputs = p->inputs;
                src.input_stride = p->input_stride;
                const CostSource cs = cost_of(p, nullptr);
                auto run = [&]() {
                    return kind == ONCHIP_ENERGY
                               ? launch_onchip_energy(p->dtype == SV_C128, sh, plan->dev, obs->dev,
                                                      src, E, st, dt, nullptr, &bc)
                               : launch_onchip_adjoint(p->dtype == SV_C128, sh, plan->dev, obs->dev,
                                                       src, cs, G, E2, st, &bc, obs->dtab.ptr);
                };
                if (run() != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                float tbest = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    SV_CUDA(cudaEventRecord(e0, st));
                    SV_CUDA(run());
                    SV_CUDA(cudaEventRecord(e1, st));
                    SV_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    SV_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < tbest) tbest = ms;
                }
                if (tbest * 1e3f < best.us) {
                    best.us = tbest * 1e3f;
                    best.R = sh.R;
                    best.tpb = sh.S * sh.Ts;
                    best.epi = kind == ONCHIP_ENERGY ? epi : 0;
                }
            }
        }
        if (best.R > 0) ctx->tuned[tune_key(p, kind, slots)] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return SV_OK;
}

sv_status sv_plan_info(const sv_circuit *c, sv_dtype dt, const sv_plan_opts *o, int32_t *on_chip,
                       int32_t *n_passes, int32_t *tile_bits, int32_t *n_stages,
                       int32_t *n_groups) {
    sv_status s = check_circuit(c, dt == SV_C128 ? 29 : 30);
    if (s != SV_OK) return s;
    HostProgram h;
    std::string err;
    const bool tiles = wants_tiles(c->n_qubits, dt, o);
    int t = 0;
    if (tiles) {
        TileCfg cfg{};
        s = tile_cfg(c->n_qubits, dt, o, &cfg);
        if (s != SV_OK) return s;
        t = cfg.t;
        err = plan_passes(*c, cfg.t, cfg.c, cfg.R, use_fusion(o), swz_bits(dt), &h, use_relabel(o));
    } else {
        err = plan_circuit(*c, (o && o->reg_bits > 0) ? o->reg_bits : (dt == SV_C128 ? 3 : 4),
                           use_fusion(o), swz_bits(dt), &h);
    }
    if (!err.empty()) return fail(SV_ERR_ARG, "circuit: " + err);
    if (on_chip) *on_chip = tiles ? 0 : 1;
    if (n_passes) *n_passes = (int32_t)h.passes.size();
    if (tile_bits) *tile_bits = t;
    if (n_stages) *n_stages = (int32_t)h.stages.size();
    if (n_groups) *n_groups = (int32_t)h.groups.size();
    return SV_OK;
}

sv_status sv_h_plan_info(const sv_pauli_sum *h, sv_dtype dt, int32_t *n_passes,
                         int32_t *tile_bits) {
    if (!h) return fail(SV_ERR_ARG, "observable is NULL");
    if (h->n_qubits < 1 || h->n_qubits > 30) return fail(SV_ERR_ARG, "n_qubits must be in [1, 30]");
    HostObservable ho;
    std::string err = plan_observable(*h, h->n_qubits, swz_bits(dt), &ho);
    const int t = h_tile_bits(h->n_qubits, dt);
    HostHPlan hp;
    if (err.empty()) err = plan_h_passes(ho, t, dt == SV_C128 ? 3 : 4, &hp);
    if (!err.empty()) return fail(SV_ERR_ARG, "observable: " + err);
    if (n_passes) *n_passes = (int32_t)hp.passes.size();
    if (tile_bits) *tile_bits = t;
    return SV_OK;
}

sv_status sv_phase_timing(int32_t on) {
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->timing = on != 0;
    ctx->phase_used = 0;
    return SV_OK;
}

sv_status sv_last_phase_ms(float *forward_ms, float *h_ms, float *reverse_ms) {
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->timing || ctx->phase_used < 4 || ctx->phase_used % 4)
        return fail(SV_ERR_ARG, "no timed call since phase timing was turned on");
    float ph[3] = {0.f, 0.f, 0.f};
    for (int c = 0; c < ctx->phase_used; c += 4)
        for (int k = 0; k < 3; ++k) {
            float ms = 0.f;
            SV_CUDA(cudaEventSynchronize(ctx->phase_ev[c + k + 1]));
            SV_CUDA(cudaEventElapsedTime(&ms, ctx->phase_ev[c + k], ctx->phase_ev[c + k + 1]));
            ph[k] += ms;
        }
    if (forward_ms) *forward_ms = ph[0];
    if (h_ms) *h_ms = ph[1];
    if (reverse_ms) *reverse_ms = ph[2];
    return SV_OK;
}

sv_status sv_last_adjoint_info(int32_t *checkpoint_every, int64_t *reverse_bytes) {
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (checkpoint_every) *checkpoint_every = ctx->last_every;
    if (reverse_bytes) *reverse_bytes = ctx->last_rev_bytes;
    return SV_OK;
}

sv_status sv_tuned_shape(const sv_problem *p, int32_t kind, int32_t *reg_bits,
                         int32_t *threads_per_block, float *us) {
    if (!p || !p->circuit || !p->observable) return fail(SV_ERR_ARG, "problem is NULL");
    if (kind != 1 && kind != 2) return fail(SV_ERR_ARG, "kind must be 1 or 2");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    const int B = (2 * p->circuit->n_params + 1) * p->n_instances;
    const Tuned *t = nullptr;
    if (wants_tiles(p->circuit->n_qubits, p->dtype, p->opts))
        t = find_tuned(ctx, p, kind == 1 ? kTileEnergyKey : kTileAdjointKey, p->n_instances);
    else
        t = kind == 1 ? find_tuned(ctx, p, ONCHIP_ENERGY, B)
                      : find_tuned(ctx, p, ONCHIP_ADJOINT, p->n_instances);
    if (!t) return fail(SV_ERR_ARG, "no tuned shape for this problem");
    if (reg_bits) *reg_bits = t->R;
    if (threads_per_block) *threads_per_block = t->tpb;
    if (us) *us = t->us;
    return SV_OK;
}

sv_status sv_sync_status(sv_stream_t stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending error");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->err.ptr) {
        // the word is written only by kernels on any stream: wait for them
        SV_CUDA(cudaDeviceSynchronize());
        int code = 0;
        SV_CUDA(cudaMemcpy(&code, ctx->err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
        if (code != 0) {
            SV_CUDA(cudaMemset(ctx->err.ptr, 0, sizeof(int)));
            return fail(SV_ERR_TIMEOUT, "a bounded device-side wait gave up (code " +
                                            std::to_string(code) +
                                            "); results since the last check are invalid");
        }
    }
    return SV_OK;
}

sv_status sv_tuned_tile(const sv_problem *p, int32_t kind, int32_t *tile_bits,
                        int32_t *reg_bits, int32_t *tensor_blocks, float *us) {
    if (!p || !p->circuit || !p->observable) return fail(SV_ERR_ARG, "problem is NULL");
    if (kind != 1 && kind != 2) return fail(SV_ERR_ARG, "kind must be 1 or 2");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!wants_tiles(p->circuit->n_qubits, p->dtype, p->opts))
        return fail(SV_ERR_ARG, "the problem's states stay on chip: no tile shape");
    const Tuned *t =
        find_tuned(ctx, p, kind == 1 ? kTileEnergyKey : kTileAdjointKey, p->n_instances);
    if (!t) return fail(SV_ERR_ARG, "no tuned tile shape for this problem");
    if (tile_bits) *tile_bits = t->R + __builtin_ctz((unsigned)t->tpb);
    if (reg_bits) *reg_bits = t->R;
    if (tensor_blocks) *tensor_blocks = t->tc;
    if (us) *us = t->us;
    return SV_OK;
}

sv_status sv_debug_wait_expiry(int32_t limit, sv_stream_t stream) {
    if (limit < 1 || limit > (1 << 20)) return fail(SV_ERR_ARG, "limit must be 1..2^20");
    DeviceCtx *ctx = context();
    if (!ctx) return fail(SV_ERR_CUDA, "no CUDA device");
    std::lock_guard<std::mutex> lk(ctx->mu);
    int *err = device_err(ctx);
    if (!err) return fail(SV_ERR_CUDA, "device error word");
    cudaError_t e = launch_wait_expiry(err, (uint32_t)limit, (cudaStream_t)stream);
    return e == cudaSuccess ? SV_OK : cuda_fail(e, "wait-expiry launch");
}

sv_status sv_shutdown(void) {
    svk::noalloc_forget();
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : g_ctx) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(kv.first);
        cudaDeviceSynchronize();
        kv.second.reset();
        cudaSetDevice(cur);
    }
    g_ctx.clear();
    return SV_OK;
}

}  // extern "C"

// Internal hooks for other translation units of the library.
namespace svk {
sv_status record_error(sv_status s, const std::string &msg) { return fail(s, msg); }
sv_status validate_problem(const sv_problem *p, bool need_cost_arrays) {
    return check_problem(p, need_cost_arrays);
}
}  // namespace svk
