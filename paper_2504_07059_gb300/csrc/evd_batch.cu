// evd_batch.cu -- C ABI of the batch of independent lattices (evd_batch.h).
//
// Host side: member validation and constants (the single-lattice helpers),
// the work list, the per-member FP64 mass reductions, replay of runs of steps
// from a captured CUDA graph, and the schedule autotuner.  The per-node work
// is the general step's (evd_batch_kernels.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "evd.h"
#include "evd_batch.h"
#include "evd_device.cuh"
#include "evd_internal.h"

using evd::BatchArgs;
using evd::BatchItem;
using evd::HostParams;
using evd::MAXS;
using evd::MemberInfo;

namespace {

constexpr int FLAG_MASS = 1, FLAG_RAW = 2;   // must match the device-side flags
constexpr int kMaxGraphs = 4;

thread_local std::string g_batch_error;

struct GraphEntry {
    int signature;            // cur * 4 + (corr_pending + 1) at the start of the run
    cudaGraphExec_t exec;
    long long nodes;          // kernels per replay
    int end_cur, end_pending, end_applied;
};

}  // namespace

struct evd_batch {
    int lattice, precision, Q, D, n;
    size_t elem;
    std::vector<HostParams> hp;
    std::vector<MemberInfo> info;
    long long buf_elems;
    size_t buf_bytes;
    void* buf[2];
    int cur;            // buf[cur] holds f*_t of every member
    bool prev_raw;      // buf[cur ^ 1] holds f_t itself (right after initialisation)
    bool ready;
    long long t;
    cudaStream_t stream;
    cudaStream_t cap;   // private stream used only to capture graphs
    int device, sm_count;
    void* params_d;     // Params<T>[n]
    MemberInfo* info_d;
    BatchItem* items_d;
    int n_items;
    size_t items_cap;
    double* part;       // [items][MAXS] per-item mass partials
    size_t part_cap;
    double* small;      // target, corr[0], corr[1], mass_out: [n][MAXS] each
    unsigned* seed_ctr; // {step counter, CTAs done} seeding the dithered rounding (in small)
    double *target, *corr[2], *mass_out;
    unsigned* err_flag;
    int mc_every, corr_pending, corr_applied;
    int item_sites, ctas_per_sm, grid;
    int graph_steps;
    std::vector<GraphEntry> graphs;
    long long launches;
    double* staging;
    size_t staging_bytes;
    long long tot_sites, tot_ssites;
    std::string err;
};

namespace {

evd_status fail(evd_batch* b, evd_status s, const std::string& msg)
{
    if (b) b->err = msg;
    else g_batch_error = msg;
    return s;
}

evd_status cuda_fail(evd_batch* b, cudaError_t e, const char* where)
{
    return fail(b, EVD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define BK(b, call)                                                    \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((b), e_, #call);       \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

// Initial species masses sum_x x_i M_i n of every member in FP64, one warp
// per member in a fixed order, so that they (and the deviation references
// derived from them) do not depend on the schedule.
__global__ void __launch_bounds__(256)
evd_k_batch_field_mass(const MemberInfo* __restrict__ info, int n_members, const double* __restrict__ x,
                       const double* __restrict__ nf, double* __restrict__ out)
{
    const int m = (blockIdx.x * 256 + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (m >= n_members) return;   // whole warps
    const MemberInfo mi = info[m];
    for (int i = 0; i < MAXS; ++i) {
        double s = 0.0;
        if (i < mi.ns)
            for (int node = lane; node < mi.sites; node += 32) {
                const double n = nf ? nf[mi.soff + node] : 1.0;
                s += x[mi.xoff + (long long)i * mi.sites + node] * mi.M[i] * n;
            }
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) out[m * MAXS + i] = s;
    }
}

// Per-member sums of the item partials in a fixed order (one warp per
// member).  With target: out = (target - sum) / sites, the per-node
// correction the next step re-injects; else out = sum.
__global__ void __launch_bounds__(256)
evd_k_batch_finish(const double* __restrict__ part, const MemberInfo* __restrict__ info, int n_members,
                   const double* __restrict__ target, double* __restrict__ out)
{
    const int m = (blockIdx.x * 256 + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (m >= n_members) return;   // whole warps
    const MemberInfo mi = info[m];
    for (int i = 0; i < MAXS; ++i) {
        double s = 0.0;
        if (i < mi.ns)
            for (int it = mi.item_begin + lane; it < mi.item_end; it += 32) s += part[(long long)it * MAXS + i];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) {
            double r = 0.0;
            if (i < mi.ns) r = target ? (target[m * MAXS + i] - s) / s : s;
            out[m * MAXS + i] = r;
        }
    }
}

namespace {

BatchArgs args_of(const evd_batch* b)
{
    return BatchArgs{b->items_d, b->n_items, b->params_d, b->info_d, b->grid,
                     b->precision == EVD_FP64 ? nullptr : b->seed_ctr};
}

cudaError_t dispatch_step(const evd_batch* b, cudaStream_t st, const void* fin, void* fout, int flags,
                          const double* corr)
{
    const BatchArgs a = args_of(b);
    switch (b->precision * 2 + b->lattice) {
        case 0: return evd::BatchLaunch<0, 0>::step(a, fin, fout, b->part, b->err_flag, flags, corr, st);
        case 1: return evd::BatchLaunch<0, 1>::step(a, fin, fout, b->part, b->err_flag, flags, corr, st);
        case 2: return evd::BatchLaunch<1, 0>::step(a, fin, fout, b->part, b->err_flag, flags, corr, st);
        case 3: return evd::BatchLaunch<1, 1>::step(a, fin, fout, b->part, b->err_flag, flags, corr, st);
        case 4: return evd::BatchLaunch<2, 0>::step(a, fin, fout, b->part, b->err_flag, flags, corr, st);
        case 5: return evd::BatchLaunch<2, 1>::step(a, fin, fout, b->part, b->err_flag, flags, corr, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_readout(const evd_batch* b, const void* fin, int flags, double* x, double* rho, double* u,
                             double* ui, const double* corr)
{
    const BatchArgs a = args_of(b);
    cudaStream_t st = b->stream;
    switch (b->precision * 2 + b->lattice) {
        case 0: return evd::BatchLaunch<0, 0>::readout(a, fin, flags, x, rho, u, ui, b->part, b->err_flag, corr, st);
        case 1: return evd::BatchLaunch<0, 1>::readout(a, fin, flags, x, rho, u, ui, b->part, b->err_flag, corr, st);
        case 2: return evd::BatchLaunch<1, 0>::readout(a, fin, flags, x, rho, u, ui, b->part, b->err_flag, corr, st);
        case 3: return evd::BatchLaunch<1, 1>::readout(a, fin, flags, x, rho, u, ui, b->part, b->err_flag, corr, st);
        case 4: return evd::BatchLaunch<2, 0>::readout(a, fin, flags, x, rho, u, ui, b->part, b->err_flag, corr, st);
        case 5: return evd::BatchLaunch<2, 1>::readout(a, fin, flags, x, rho, u, ui, b->part, b->err_flag, corr, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_init(const evd_batch* b, const double* x, const double* n)
{
    const BatchArgs a = args_of(b);
    cudaStream_t st = b->stream;
    void* fp = b->buf[1];
    void* fc = b->buf[0];
    switch (b->precision * 2 + b->lattice) {
        case 0: return evd::BatchLaunch<0, 0>::init(a, x, n, fp, fc, b->part, b->err_flag, st);
        case 1: return evd::BatchLaunch<0, 1>::init(a, x, n, fp, fc, b->part, b->err_flag, st);
        case 2: return evd::BatchLaunch<1, 0>::init(a, x, n, fp, fc, b->part, b->err_flag, st);
        case 3: return evd::BatchLaunch<1, 1>::init(a, x, n, fp, fc, b->part, b->err_flag, st);
        case 4: return evd::BatchLaunch<2, 0>::init(a, x, n, fp, fc, b->part, b->err_flag, st);
        case 5: return evd::BatchLaunch<2, 1>::init(a, x, n, fp, fc, b->part, b->err_flag, st);
    }
    return cudaErrorInvalidValue;
}

evd_status finish(evd_batch* b, cudaStream_t st, const double* target, double* out)
{
    b->launches += 1;
    const int blocks = (b->n * 32 + 255) / 256;
    evd_k_batch_finish<<<blocks, 256, 0, st>>>(b->part, b->info_d, b->n, target, out);
    BK(b, cudaGetLastError());
    return EVD_OK;
}

void destroy_graphs(evd_batch* b)
{
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

// Work list for the schedule: items of item_sites consecutive sites, members
// in order (a member's items are contiguous, which the mass reduction uses).
evd_status set_schedule(evd_batch* b, int item_sites, int ctas_per_sm)
{
    std::vector<BatchItem> items;
    for (int m = 0; m < b->n; ++m) {
        MemberInfo& mi = b->info[m];
        mi.item_begin = (int)items.size();
        for (long long node0 = 0; node0 < mi.sites; node0 += item_sites) {
            const int cnt = (int)std::min<long long>(item_sites, mi.sites - node0);
            items.push_back(BatchItem{m, (int)node0, cnt, mi.ns});
            if (items.size() >= (size_t)1 << 30) return fail(b, EVD_ERR_ARG, "too many work items");
        }
        mi.item_end = (int)items.size();
    }
    if (items.size() > b->items_cap) {
        if (b->items_d) cudaFree(b->items_d);
        b->items_d = nullptr;
        b->items_cap = 0;
        BK(b, cudaMalloc((void**)&b->items_d, items.size() * sizeof(BatchItem)));
        b->items_cap = items.size();
    }
    if (items.size() * MAXS > b->part_cap) {
        if (b->part) cudaFree(b->part);
        b->part = nullptr;
        b->part_cap = 0;
        BK(b, cudaMalloc((void**)&b->part, items.size() * MAXS * sizeof(double)));
        b->part_cap = items.size() * MAXS;
    }
    BK(b, cudaMemcpyAsync(b->items_d, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                          b->stream));
    BK(b, cudaMemcpyAsync(b->info_d, b->info.data(), b->n * sizeof(MemberInfo), cudaMemcpyHostToDevice, b->stream));
    BK(b, cudaStreamSynchronize(b->stream));   // the host vectors go out of scope
    b->n_items = (int)items.size();
    b->item_sites = item_sites;
    b->ctas_per_sm = ctas_per_sm;
    const long long persistent = (long long)ctas_per_sm * b->sm_count;
    b->grid = (ctas_per_sm == 0 || persistent >= b->n_items) ? b->n_items : (int)persistent;
    destroy_graphs(b);
    return EVD_OK;
}

// The members' constants on the device, in the arithmetic type of the
// precision (double for FP64, float otherwise).
evd_status upload_params(evd_batch* b)
{
    std::vector<char> host;
    if (b->precision == EVD_FP64) {
        host.resize(b->n * sizeof(evd::Params<double>));
        for (int m = 0; m < b->n; ++m) {
            const evd::Params<double> p = evd::to_params<double>(b->hp[m]);
            std::memcpy(host.data() + m * sizeof(p), &p, sizeof(p));
        }
    } else {
        host.resize(b->n * sizeof(evd::Params<float>));
        for (int m = 0; m < b->n; ++m) {
            const evd::Params<float> p = evd::to_params<float>(b->hp[m]);
            std::memcpy(host.data() + m * sizeof(p), &p, sizeof(p));
        }
    }
    BK(b, cudaMemcpyAsync(b->params_d, host.data(), host.size(), cudaMemcpyHostToDevice, b->stream));
    BK(b, cudaStreamSynchronize(b->stream));
    return EVD_OK;
}

evd_status ensure_staging(evd_batch* b, size_t bytes)
{
    if (b->staging_bytes >= bytes) return EVD_OK;
    if (b->staging) cudaFree(b->staging);
    b->staging = nullptr;
    b->staging_bytes = 0;
    BK(b, cudaMalloc((void**)&b->staging, bytes));
    b->staging_bytes = bytes;
    return EVD_OK;
}

// One step on stream st from the given state; returns the state after it.
struct StepState {
    int cur, pending, applied;
    long long t;
};

evd_status enqueue_step(evd_batch* b, cudaStream_t st, StepState& s)
{
    // every mc_every steps the step kernel also reduces the species masses of
    // f_t; the deficit from the FP64 targets is re-injected in the next step
    const bool measure = b->mc_every > 0 && ((s.t + 1) % b->mc_every == 0);
    const int apply = s.pending;
    b->launches += 1;
    BK(b, dispatch_step(b, st, b->buf[s.cur], b->buf[s.cur ^ 1], measure ? FLAG_MASS : 0,
                        apply >= 0 ? b->corr[apply] : nullptr));
    s.applied = apply;
    s.pending = -1;
    if (measure) {
        const int slot = (apply == 0) ? 1 : 0;
        evd_status r = finish(b, st, b->target, b->corr[slot]);
        if (r != EVD_OK) return r;
        s.pending = slot;
    }
    s.cur ^= 1;
    s.t += 1;
    return EVD_OK;
}

// Graph of graph_steps steps starting from state s (captured once per start
// signature on the private stream, replayed on the batch's stream).
evd_status graph_for(evd_batch* b, const StepState& s, const GraphEntry** out)
{
    const int sig = s.cur * 4 + (s.pending + 1);
    for (const auto& g : b->graphs)
        if (g.signature == sig) {
            *out = &g;
            return EVD_OK;
        }
    *out = nullptr;
    if ((int)b->graphs.size() >= kMaxGraphs) return EVD_OK;
    const long long before = b->launches;
    BK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    StepState z = s;
    evd_status r = EVD_OK;
    for (int k = 0; k < b->graph_steps && r == EVD_OK; ++k) r = enqueue_step(b, b->cap, z);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->cap, &graph);
    const long long nodes = b->launches - before;
    b->launches = before;   // captured, not launched
    if (r != EVD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return r;
    }
    if (ee != cudaSuccess) return cuda_fail(b, ee, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_fail(b, ei, "cudaGraphInstantiate");
    b->graphs.push_back(GraphEntry{sig, exec, nodes, z.cur, z.pending, z.applied});
    *out = &b->graphs.back();
    return EVD_OK;
}

evd_status readout(evd_batch* b, double* x, double* rho, double* u, double* ui)
{
    const double* cr = (!b->prev_raw && b->corr_applied >= 0) ? b->corr[b->corr_applied] : nullptr;
    b->launches += 1;
    BK(b, dispatch_readout(b, b->buf[b->cur ^ 1], b->prev_raw ? FLAG_RAW : 0, x, rho, u, ui, cr));
    return finish(b, b->stream, nullptr, b->mass_out);
}

evd_status check_word(evd_batch* b)
{
    unsigned w = 0;
    BK(b, cudaMemcpyAsync(&w, b->err_flag, sizeof(w), cudaMemcpyDeviceToHost, b->stream));
    BK(b, cudaStreamSynchronize(b->stream));
    if (w) return fail(b, EVD_ERR_UNSTABLE, "a member became unstable (rho_i <= 0 or tau_ij <= 0 / non-finite)");
    return EVD_OK;
}

void free_all(evd_batch* b)
{
    destroy_graphs(b);
    for (int k = 0; k < 2; ++k)
        if (b->buf[k]) cudaFree(b->buf[k]);
    if (b->params_d) cudaFree(b->params_d);
    if (b->info_d) cudaFree(b->info_d);
    if (b->items_d) cudaFree(b->items_d);
    if (b->part) cudaFree(b->part);
    if (b->small) cudaFree(b->small);
    if (b->staging) cudaFree(b->staging);
    if (b->cap) cudaStreamDestroy(b->cap);
}

}  // namespace

extern "C" {

evd_status evd_batch_create(int lattice, int precision, const evd_member* members, int n_members,
                            void* cuda_stream, evd_batch** out)
{
    if (out) *out = nullptr;
    if (!out) return fail(nullptr, EVD_ERR_ARG, "out must not be NULL");
    if (!members || n_members < 1) return fail(nullptr, EVD_ERR_ARG, "need at least one member");
    if (lattice != EVD_D2Q9 && lattice != EVD_D3Q19) return fail(nullptr, EVD_ERR_ARG, "unknown lattice");
    if (precision < EVD_FP64 || precision > EVD_FP16_STORE) return fail(nullptr, EVD_ERR_ARG, "unknown precision");
    evd_batch* b = new evd_batch();
    b->lattice = lattice;
    b->precision = precision;
    b->Q = lattice == EVD_D2Q9 ? 9 : 19;
    b->D = lattice == EVD_D2Q9 ? 2 : 3;
    b->n = n_members;
    b->elem = evd::elem_size(precision);
    b->stream = (cudaStream_t)cuda_stream;
    b->hp.resize(n_members);
    b->info.resize(n_members);
    long long foff = 0, xoff = 0, soff = 0;
    for (int m = 0; m < n_members; ++m) {
        const evd_member& mb = members[m];
        const evd_grid g{lattice, precision, mb.nx, mb.ny, mb.nz, mb.wall_mask};
        std::string msg;
        if (mb.species.flags) msg = "the corrective forcing terms are not supported in a batch";
        else if (mb.species.n_species > evd::MAXS_FAST) msg = "batch members take at most 3 species";
        if (!msg.empty() || !evd::validate(&g, &mb.species, msg)) {
            delete b;
            return fail(nullptr, EVD_ERR_ARG, "member " + std::to_string(m) + ": " + msg);
        }
        evd::fill_params(b->hp[m], &g, &mb.species);
        MemberInfo& mi = b->info[m];
        std::memset(&mi, 0, sizeof(mi));
        mi.sites = b->hp[m].nsites;
        mi.ns = mb.species.n_species;
        mi.foff = foff;
        mi.xoff = xoff;
        mi.soff = soff;
        mi.uoff = soff * b->D;
        mi.uioff = xoff * b->D;
        for (int i = 0; i < mi.ns; ++i) mi.M[i] = mb.species.molar_mass[i];
        foff += (long long)evd::buffer_planes(lattice, precision, mi.ns) * b->hp[m].pstride;
        xoff += (long long)mi.ns * mi.sites;
        soff += mi.sites;
    }
    b->buf_elems = foff;
    b->buf_bytes = (size_t)foff * b->elem;
    b->tot_sites = soff;
    b->tot_ssites = xoff;
    b->mc_every = precision == EVD_FP64 ? 0 : (precision == EVD_FP32 ? 8 : 1);
    b->corr_pending = b->corr_applied = -1;
    b->graph_steps = 8;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&b->buf[k], b->buf_bytes);
    const size_t pbytes = (size_t)n_members *
                          (precision == EVD_FP64 ? sizeof(evd::Params<double>) : sizeof(evd::Params<float>));
    if (e == cudaSuccess) e = cudaMalloc(&b->params_d, pbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->info_d, n_members * sizeof(MemberInfo));
    const size_t arr = (size_t)n_members * MAXS;
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->small, 4 * arr * sizeof(double) + 256);
    if (e != cudaSuccess) {
        const std::string msg = std::string("allocation: ") + cudaGetErrorString(e);
        free_all(b);
        delete b;
        return fail(nullptr, EVD_ERR_CUDA, msg);
    }
    b->target = b->small;
    b->corr[0] = b->small + arr;
    b->corr[1] = b->small + 2 * arr;
    b->mass_out = b->small + 3 * arr;
    b->err_flag = (unsigned*)(b->small + 4 * arr);
    b->seed_ctr = (unsigned*)((char*)(b->small + 4 * arr) + 128);
    evd_status s = set_schedule(b, 512, 8);
    if (s == EVD_OK) s = upload_params(b);
    if (s == EVD_OK) {
        e = cudaMemsetAsync(b->small, 0, 4 * arr * sizeof(double) + 256, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) s = cuda_fail(b, e, "cudaMemsetAsync");
    }
    if (s != EVD_OK) {
        g_batch_error = b->err;
        free_all(b);
        delete b;
        return s;
    }
    *out = b;
    return EVD_OK;
}

evd_status evd_batch_sizes(const evd_batch* b, long long* sites, long long* species_sites)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (sites) *sites = b->tot_sites;
    if (species_sites) *species_sites = b->tot_ssites;
    return EVD_OK;
}

evd_status evd_batch_set_fields(evd_batch* b, const double* x, const double* n)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (!x) return fail(b, EVD_ERR_ARG, "x must not be NULL");
    for (long long k = 0; k < b->tot_ssites; ++k)
        if (!(x[k] > 0.0) || !std::isfinite(x[k])) return fail(b, EVD_ERR_ARG, "mole fractions must be > 0");
    if (n)
        for (long long k = 0; k < b->tot_sites; ++k)
            if (!(n[k] > 0.0) || !std::isfinite(n[k])) return fail(b, EVD_ERR_ARG, "number density must be > 0");
    DeviceGuard dg(b->device);
    const size_t nx = (size_t)b->tot_ssites, nn = (size_t)b->tot_sites;
    evd_status s = ensure_staging(b, (nx + nn) * sizeof(double));
    if (s != EVD_OK) return s;
    double* xd = b->staging;
    double* nd = n ? b->staging + nx : nullptr;
    BK(b, cudaMemcpyAsync(xd, x, nx * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    if (n) BK(b, cudaMemcpyAsync(nd, n, nn * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    // FP64 initial species masses: the correction targets and, for deviation
    // storage, the reference densities (mass / sites)
    b->launches += 1;
    evd_k_batch_field_mass<<<(b->n * 32 + 255) / 256, 256, 0, b->stream>>>(b->info_d, b->n, xd, nd, b->target);
    BK(b, cudaGetLastError());
    if (b->precision != EVD_FP64) {
        std::vector<double> m((size_t)b->n * MAXS);
        BK(b, cudaMemcpyAsync(m.data(), b->target, m.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        BK(b, cudaStreamSynchronize(b->stream));
        for (int k = 0; k < b->n; ++k) {
            HostParams& h = b->hp[k];
            for (int i = 0; i < MAXS; ++i)
                for (int c = 0; c < 3; ++c)
                    h.ref[i][c] = (i < h.ns && b->precision == EVD_FP32) ? h.wl[c] * m[(size_t)k * MAXS + i] / h.nsites
                                                                         : 0.0;
        }
        s = upload_params(b);
        if (s != EVD_OK) return s;
    }
    BK(b, cudaMemsetAsync(b->err_flag, 0, sizeof(unsigned), b->stream));
    BK(b, cudaMemsetAsync(b->seed_ctr, 0, 2 * sizeof(unsigned), b->stream));   // step t + 1 draws seed t + 1
    b->launches += 1;
    BK(b, dispatch_init(b, xd, nd));
    b->cur = 0;
    b->prev_raw = true;
    b->ready = true;
    b->corr_pending = b->corr_applied = -1;
    b->t = 0;
    BK(b, cudaStreamSynchronize(b->stream));
    return check_word(b);
}

evd_status evd_batch_step(evd_batch* b, long long nsteps)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return fail(b, EVD_ERR_ARG, "nsteps must be >= 0");
    if (!b->ready) return fail(b, EVD_ERR_STATE, "evd_batch_set_fields has not been called");
    DeviceGuard dg(b->device);
    StepState s{b->cur, b->corr_pending, b->corr_applied, b->t};
    long long left = nsteps;
    while (left > 0) {
        const bool aligned = b->mc_every == 0 || s.t % b->mc_every == 0;
        if (b->graph_steps > 0 && left >= b->graph_steps && aligned) {
            const GraphEntry* g = nullptr;
            evd_status r = graph_for(b, s, &g);
            if (r != EVD_OK) return r;
            if (g) {
                BK(b, cudaGraphLaunch(g->exec, b->stream));
                b->launches += g->nodes;
                s.cur = g->end_cur;
                s.pending = g->end_pending;
                s.applied = g->end_applied;
                s.t += b->graph_steps;
                left -= b->graph_steps;
                b->cur = s.cur; b->corr_pending = s.pending; b->corr_applied = s.applied; b->t = s.t;
                b->prev_raw = false;
                continue;
            }
        }
        evd_status r = enqueue_step(b, b->stream, s);
        if (r != EVD_OK) return r;
        left -= 1;
        b->cur = s.cur; b->corr_pending = s.pending; b->corr_applied = s.applied; b->t = s.t;
        b->prev_raw = false;
    }
    return EVD_OK;
}

evd_status evd_batch_readout_device(evd_batch* b, double* x, double* rho, double* u, double* ui)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (!b->ready) return fail(b, EVD_ERR_STATE, "evd_batch_set_fields has not been called");
    DeviceGuard dg(b->device);
    return readout(b, x, rho, u, ui);
}

static evd_status readout_host(evd_batch* b, double* x, double* rho, double* u, double* ui)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (!b->ready) return fail(b, EVD_ERR_STATE, "evd_batch_set_fields has not been called");
    DeviceGuard dg(b->device);
    const size_t nx = (size_t)b->tot_ssites, nu = (size_t)b->tot_sites * b->D, nui = (size_t)b->tot_ssites * b->D;
    const size_t need = (x ? nx : 0) + (rho ? nx : 0) + (u ? nu : 0) + (ui ? nui : 0);
    evd_status s = ensure_staging(b, std::max<size_t>(need, 1) * sizeof(double));
    if (s != EVD_OK) return s;
    double* p = b->staging;
    double* xd = x ? p : nullptr;
    p += x ? nx : 0;
    double* rd = rho ? p : nullptr;
    p += rho ? nx : 0;
    double* ud = u ? p : nullptr;
    p += u ? nu : 0;
    double* uid = ui ? p : nullptr;
    s = readout(b, xd, rd, ud, uid);
    if (s != EVD_OK) return s;
    if (x) BK(b, cudaMemcpyAsync(x, xd, nx * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (rho) BK(b, cudaMemcpyAsync(rho, rd, nx * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (u) BK(b, cudaMemcpyAsync(u, ud, nu * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (ui) BK(b, cudaMemcpyAsync(ui, uid, nui * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BK(b, cudaStreamSynchronize(b->stream));
    return check_word(b);
}

evd_status evd_batch_get_mole_fractions(evd_batch* b, double* x)
{
    if (b && !x) return fail(b, EVD_ERR_ARG, "x must not be NULL");
    return readout_host(b, x, nullptr, nullptr, nullptr);
}

evd_status evd_batch_get_densities(evd_batch* b, double* rho)
{
    if (b && !rho) return fail(b, EVD_ERR_ARG, "rho must not be NULL");
    return readout_host(b, nullptr, rho, nullptr, nullptr);
}

evd_status evd_batch_get_velocities(evd_batch* b, double* u, double* ui)
{
    if (b && !u && !ui) return fail(b, EVD_ERR_ARG, "u and ui are both NULL");
    return readout_host(b, nullptr, nullptr, u, ui);
}

evd_status evd_batch_get_species_mass(evd_batch* b, double* mass)
{
    if (b && !mass) return fail(b, EVD_ERR_ARG, "mass must not be NULL");
    evd_status s = readout_host(b, nullptr, nullptr, nullptr, nullptr);
    if (s != EVD_OK) return s;
    BK(b, cudaMemcpyAsync(mass, b->mass_out, (size_t)b->n * MAXS * sizeof(double), cudaMemcpyDeviceToHost,
                          b->stream));
    BK(b, cudaStreamSynchronize(b->stream));
    return EVD_OK;
}

evd_status evd_batch_set_schedule(evd_batch* b, int item_sites, int ctas_per_sm)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (item_sites < 128 || item_sites > 65536 || item_sites % 128 != 0)
        return fail(b, EVD_ERR_ARG, "item_sites must be a multiple of 128 in 128..65536");
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return fail(b, EVD_ERR_ARG, "ctas_per_sm must be 0..32");
    DeviceGuard dg(b->device);
    BK(b, cudaStreamSynchronize(b->stream));
    return set_schedule(b, item_sites, ctas_per_sm);
}

evd_status evd_batch_get_schedule(const evd_batch* b, int* item_sites, int* ctas_per_sm)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (item_sites) *item_sites = b->item_sites;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    return EVD_OK;
}

evd_status evd_batch_autotune(evd_batch* b, int steps_per_trial, int* item_sites, int* ctas_per_sm)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (!b->ready) return fail(b, EVD_ERR_STATE, "evd_batch_set_fields has not been called");
    if (steps_per_trial < 2 || steps_per_trial > 64 || steps_per_trial % 2 != 0)
        return fail(b, EVD_ERR_ARG, "steps_per_trial must be even, 2..64");
    DeviceGuard dg(b->device);
    // the trials step a copy of the populations and of the dither step
    // counter; both are put back after
    void* backup = nullptr;
    BK(b, cudaMalloc(&backup, 2 * b->buf_bytes + 16));
    char* bk = (char*)backup;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    evd_status r = EVD_OK;
    int best_i = b->item_sites, best_c = b->ctas_per_sm;
    float best_ms = 1e30f;
    cudaError_t e = cudaMemcpyAsync(bk, b->buf[0], b->buf_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bk + b->buf_bytes, b->buf[1], b->buf_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bk + 2 * b->buf_bytes, b->seed_ctr, 8, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) r = cuda_fail(b, e, "autotune setup");
    const int sizes[] = {128, 256, 512, 1024, 2048};
    const int ctas[] = {0, 2, 4, 8, 16};
    for (int si = 0; si < 5 && r == EVD_OK; ++si)
        for (int ci = 0; ci < 5 && r == EVD_OK; ++ci) {
            r = set_schedule(b, sizes[si], ctas[ci]);
            if (r != EVD_OK) break;
            int c = b->cur;
            auto run = [&](int k) -> cudaError_t {
                for (int j = 0; j < k; ++j) {
                    b->launches += 1;
                    const cudaError_t ex = dispatch_step(b, b->stream, b->buf[c], b->buf[c ^ 1], 0, nullptr);
                    if (ex != cudaSuccess) return ex;
                    c ^= 1;
                }
                return cudaSuccess;
            };
            e = run(2);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess) e = run(steps_per_trial);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                r = cuda_fail(b, e, "autotune trial");
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best_i = sizes[si];
                best_c = ctas[ci];
            }
        }
    evd_status r2 = set_schedule(b, best_i, best_c);
    if (r == EVD_OK) r = r2;
    e = cudaMemcpyAsync(b->buf[0], bk, b->buf_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->buf[1], bk + b->buf_bytes, b->buf_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->seed_ctr, bk + 2 * b->buf_bytes, 8, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess && r == EVD_OK) r = cuda_fail(b, e, "autotune restore");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(backup);
    if (r != EVD_OK) return r;
    if (item_sites) *item_sites = best_i;
    if (ctas_per_sm) *ctas_per_sm = best_c;
    return check_word(b);
}

evd_status evd_batch_set_graph(evd_batch* b, int steps_per_graph)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (steps_per_graph != 0 &&
        (steps_per_graph < 2 || steps_per_graph > 1024 || steps_per_graph % 2 != 0 ||
         (b->mc_every > 0 && steps_per_graph % b->mc_every != 0)))
        return fail(b, EVD_ERR_ARG, "steps_per_graph must be 0, or even in 2..1024 and a multiple of the "
                                    "mass-correction interval");
    DeviceGuard dg(b->device);
    BK(b, cudaStreamSynchronize(b->stream));
    destroy_graphs(b);
    b->graph_steps = steps_per_graph;
    return EVD_OK;
}

evd_status evd_batch_set_mass_correction(evd_batch* b, int every)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    if (every < 0) return fail(b, EVD_ERR_ARG, "every must be >= 0");
    DeviceGuard dg(b->device);
    BK(b, cudaStreamSynchronize(b->stream));
    destroy_graphs(b);
    b->mc_every = every;
    if (every > 0 && b->graph_steps % every != 0) b->graph_steps = every % 2 == 0 ? every : 2 * every;
    return EVD_OK;
}

long long evd_batch_time(const evd_batch* b) { return b ? b->t : -1; }

long long evd_batch_launch_count(const evd_batch* b) { return b ? b->launches : -1; }

evd_status evd_batch_check(evd_batch* b)
{
    if (!b) return fail(nullptr, EVD_ERR_ARG, "batch is NULL");
    DeviceGuard dg(b->device);
    return check_word(b);
}

evd_status evd_batch_destroy(evd_batch* b)
{
    if (!b) return EVD_OK;
    {
        DeviceGuard dg(b->device);
        cudaStreamSynchronize(b->stream);
        free_all(b);
    }
    delete b;
    return EVD_OK;
}

const char* evd_batch_last_error(const evd_batch* b)
{
    return b ? b->err.c_str() : g_batch_error.c_str();
}

}  // extern "C"
