// Allocation-free variant of the batched parameter-shift gradient.
//
// sv_grad_param_shift keeps its compiled plan, observable and per-circuit
// energies in device memory that the library allocates with cudaMalloc.
// Some callers cannot let a library do that: their device memory is owned
// by another allocator that must account for every byte (a framework's
// caching allocator), or they must never hit cudaMalloc's implicit device
// synchronisation once their loop is running.  This entry point puts
// everything the call needs beyond the caller's inputs and outputs into one
// fixed, file-scope device array instead, and allocates nothing.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "planner.h"
#include "sv.h"

namespace svk {
sv_status record_error(sv_status s, const std::string &msg);
sv_status validate_problem(const sv_problem *p, bool need_cost_arrays);
}  // namespace svk

using namespace svk;

// The scratch: every GPU that loads the library holds these bytes until the
// process exits.  Host code must never pass `g_noalloc_scratch` itself to a
// kernel (in host code the name is a host-side stand-in, not a device
// address); it uses the address obtained below with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SV_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[kMaxDevices];  // device address of the array, per device

// Once per device, with that device current.  sv_shutdown() forgets the
// addresses (svk::noalloc_forget), so that a caller who reset a device and
// then shut the library down gets the address in the new context.
sv_status noalloc_setup(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return record_error(SV_ERR_CUDA, std::string("cudaGetSymbolAddress(noalloc scratch): ") +
                                                 cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return SV_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

namespace svk {
void noalloc_forget() {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    for (auto &p : g_noalloc_ptr) p = nullptr;
}
}  // namespace svk

extern "C" sv_status sv_grad_param_shift_noalloc(const sv_problem *p, const double *theta,
                                                 double *energy_out, double *loss_out,
                                                 double *grad_out, sv_stream_t stream) {
    sv_status s = validate_problem(p, true);
    if (s != SV_OK) return s;
    const int P = p->circuit->n_params, I = p->n_instances;
    if (P > 0 && (!theta || !grad_out)) return record_error(SV_ERR_ARG, "theta/grad_out is NULL");
    const int64_t B64 = (int64_t)(2 * (int64_t)P + 1) * I;
    const int swz = p->dtype == SV_C128 ? 3 : 4;
    const int c128 = p->dtype == SV_C128;
    cudaStream_t st = (cudaStream_t)stream;
    // The plan is copied from a host vector released on return: a captured
    // copy would read freed memory on every replay, so capture is refused.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(st, &cap);
    if (ce != cudaSuccess)
        return record_error(SV_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    if (cap != cudaStreamCaptureStatusNone)
        return record_error(SV_ERR_UNSUPPORTED,
                            "sv_grad_param_shift_noalloc cannot be captured into a CUDA graph "
                            "(it uploads a host-side plan on every call)");
    const int onchip_max = c128 ? 12 : 13;
    if (p->circuit->n_qubits > onchip_max)
        return record_error(SV_ERR_UNSUPPORTED,
                            "sv_grad_param_shift_noalloc runs the on-chip engine only: at most " +
                                std::to_string(onchip_max) + " qubits for " +
                                (c128 ? "complex128" : "complex64") + ", got " +
                                std::to_string(p->circuit->n_qubits));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return record_error(SV_ERR_CUDA, "no usable current CUDA device");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return record_error(SV_ERR_CUDA, "cannot read the device's SM count");
    const sv_plan_opts *o = p->opts;
    const int reg = (o && o->reg_bits > 0) ? o->reg_bits : 0;
    const int tpb = (o && o->threads_per_block > 0) ? o->threads_per_block : 0;
    const bool fuse = !(o && o->no_fusion);

    // Plan on the host only.
    OnchipShape pre{}, sh{};
    const char *err = onchip_shape(ONCHIP_ENERGY, p->circuit->n_qubits, 0, P, c128,
                                   (int)(B64 > (1 << 30) ? 1 : B64), reg, tpb, &pre, sms);
    if (err) return record_error(SV_ERR_UNSUPPORTED, err);
    HostProgram hp;
    std::string perr = plan_circuit(*p->circuit, pre.R, fuse, swz, &hp);
    if (!perr.empty()) return record_error(SV_ERR_ARG, "circuit: " + perr);
    HostObservable ho;
    perr = plan_observable(*p->observable, p->circuit->n_qubits, swz, &ho);
    if (!perr.empty()) return record_error(SV_ERR_ARG, "observable: " + perr);

    // Everything in one blob laid out inside the scratch array.
    std::vector<unsigned char> blob;
    auto put = [&](const void *src, size_t n) {
        const size_t off = align256(blob.size());
        blob.resize(off + n);
        if (n) memcpy(blob.data() + off, src, n);
        return off;
    };
    const size_t o_st = put(hp.stages.data(), hp.stages.size() * sizeof(Stage));
    const size_t o_op = put(hp.ops.data(), hp.ops.size() * sizeof(Op));
    const size_t o_gr = put(hp.groups.data(), hp.groups.size() * sizeof(Group));
    const size_t o_me = put(hp.members.data(), hp.members.size() * sizeof(Member));
    const size_t o_tg = put(ho.tgroups.data(), ho.tgroups.size() * sizeof(TermGroup));
    const size_t o_tm = put(ho.terms.data(), ho.terms.size() * sizeof(Term));
    const size_t o_rf = put(p->refs, sizeof(int64_t) * (size_t)I);
    const size_t o_E = align256(blob.size());
    const size_t need = o_E + align256(sizeof(double) * (size_t)B64) + sizeof(double) * (size_t)I;
    if (B64 > (1 << 30) || need > (size_t)SV_NOALLOC_SCRATCH_BYTES)
        return record_error(SV_ERR_UNSUPPORTED,
                            "problem needs " + std::to_string(need) +
                                " bytes of scratch; the allocation-free entry point holds at most " +
                                std::to_string((size_t)SV_NOALLOC_SCRATCH_BYTES));
    const int B = (int)B64;
    err = onchip_shape(ONCHIP_ENERGY, p->circuit->n_qubits, (int)hp.groups.size(), P, c128, B,
                       reg, tpb, &sh, sms);
    if (err) return record_error(SV_ERR_UNSUPPORTED, err);

    unsigned char *base = nullptr;
    s = noalloc_setup(dev, &base);
    if (s != SV_OK) return s;
    // From pageable host memory: the copy is staged before this returns, so
    // `blob` may be released afterwards.
    e = cudaMemcpyAsync(base, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return record_error(SV_ERR_CUDA, std::string("plan upload: ") + cudaGetErrorString(e));

    Program prog{};
    prog.n = hp.n;
    prog.R = hp.R;
    prog.n_stages = (int)hp.stages.size();
    prog.n_groups = (int)hp.groups.size();
    prog.n_params = hp.n_params;
    prog.input_dim = hp.input_dim;
    prog.swz_bits = hp.swz_bits;
    prog.stages = (const Stage *)(base + o_st);
    prog.ops = (const Op *)(base + o_op);
    prog.groups = (const Group *)(base + o_gr);
    prog.members = (const Member *)(base + o_me);
    Observable obs{};
    obs.n_tgroups = (int)ho.tgroups.size();
    obs.n_terms = (int)ho.terms.size();
    obs.real = 1;
    for (const Term &tm : ho.terms) obs.real &= (tm.phase & 1) == 0;
    obs.tgroups = (const TermGroup *)(base + o_tg);
    obs.terms = (const Term *)(base + o_tm);
    double *E = (double *)(base + o_E);
    double *lp = (double *)(base + o_E + align256(sizeof(double) * (size_t)B));

    SlotSource src{};
    src.mode = SLOTS_PARAM_SHIFT;
    src.n_slots = B;
    src.n_instances = I;
    src.refs = (const int64_t *)(base + o_rf);
    src.theta = theta;
    src.inputs = p->inputs;
    src.input_stride = p->input_stride;
    e = launch_onchip_energy(c128, sh, prog, obs, src, E, st);
    if (e != cudaSuccess)
        return record_error(SV_ERR_CUDA, std::string("energy launch: ") + cudaGetErrorString(e));
    CostSource cs{};
    cs.cost = p->cost;
    cs.n_instances = I;
    cs.weights = p->weights;
    cs.targets = p->targets;
    e = launch_ps_combine(E, I, P, cs, lp, energy_out, loss_out, grad_out, st);
    if (e != cudaSuccess)
        return record_error(SV_ERR_CUDA, std::string("combine launch: ") + cudaGetErrorString(e));
    return SV_OK;
}
