// evd_api.cu -- the C ABI of libevd (declared in include/evd.h): context
// management, validation, host-side constants, launches and readouts.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "evd.h"
#include "evd_internal.h"

using evd::HostParams;
using evd::MAXS;

namespace {

constexpr int FLAG_MASS = 1, FLAG_RAW = 2;   // must match the device-side flags
constexpr int BLOCK = 128;                   // must match the device-side block size
constexpr long long PLANE_ALIGN = 64;        // elements; every plane starts 128-byte aligned
constexpr int kTmaRows = 1;                  // default rows per tile of the TMA step

thread_local std::string g_create_error;

}  // namespace

void evd::set_thread_error(const std::string& msg) { g_create_error = msg; }
const char* evd::thread_error() { return g_create_error.c_str(); }

// Storage encodings: 0 raw double, 1 float deviations from one reference per
// species, 2 half deviations from the node's own (half) density, 3 float
// deviations from the node's own density kept in the rest plane.
enum : int { ENC_F64 = 0, ENC_F32 = 1, ENC_F16 = 2, ENC_F32N = 3 };

struct evd_ctx {
    HostParams hp;
    int lattice, precision, ns, Q, D;
    int enc;          // storage encoding in effect (ENC_*)
    int ref_mode;     // EVD_REF_AUTO / _SPECIES / _NODE (float storage)
    int nx, ny, nz, nsites;
    size_t elem;
    long long pstride;
    size_t buf_bytes;
    void* buf[2];
    bool own_bufs;
    int cur;          // buf[cur] holds f*_t
    bool prev_raw;    // buf[cur ^ 1] holds f_t itself (right after initialisation)
    bool ready;
    long long t;
    cudaStream_t stream;
    int device;
    int nblocks;
    double* mass_part;   // [nblocks][ns]
    double* mass_out;    // [ns]
    double* m_target;    // [ns] initial species masses (FP64)
    double* corr[2];     // [ns] per-node mass corrections (two slots)
    unsigned* err_flag;
    unsigned long long* range;   // [2][ns] min / max species density of an initial field (bits of positive doubles)
    void* small;         // one allocation holding the six arrays above
    int mc_every;        // mass correction every k steps (0 = off)
    bool tma_ok;         // the TMA-staged step can run this configuration
    int kernel;          // EVD_KERNEL_GENERAL or EVD_KERNEL_TMA
    int tma_blocks;      // grid of the TMA step
    int tma_ty;          // rows per tile of the TMA step (1, 2 or 4)
    int adj_mode = EVD_ADJOINT_REVERSE;   // how evd_loss_gradient transposes the collision
    int adj_forward = EVD_FP64;           // storage of the adjoint's forward pass
    unsigned wall_mask;                   // as given at creation
    std::vector<double> sp_M, sp_D;       // the species table as given at creation
    double sp_tau1, sp_g[3];
    int last_parts;      // mass partials written by the last measuring launch
    CUtensorMap tma[2][evd::TmaLaunch::NGROUPS];   // per population buffer, per storage group
    float* lumps;        // App. A coefficients per wall class, species, direction (TMA step)
    void* kf;            // per-node force field [3][nsites] in the arithmetic type, or nullptr
    void* rhof;          // [ns + 1][nsites] densities of f_t for the gradient terms, or nullptr
    int corr_pending;    // slot of a computed, not yet applied correction, or -1
    int corr_applied;    // slot the last step applied (the readout applies it too), or -1
    long long launches;  // kernels launched by this context
    double* staging;     // device scratch for host transfers, grown on demand
    size_t staging_bytes;
    std::string err;
};

namespace {

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

evd_status fail(evd_ctx* c, evd_status s, const std::string& msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

evd_status cuda_fail(evd_ctx* c, cudaError_t e, const char* where)
{
    return fail(c, EVD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(ctx, call)                                                  \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);     \
    } while (0)

}  // namespace

namespace evd {

size_t elem_size(int precision)
{
    return precision == EVD_FP64 ? 8 : (precision == EVD_FP32 ? 4 : 2);
}

// Checks every documented precondition; fills msg on failure.
bool validate(const evd_grid* g, const evd_species* s, std::string& msg)
{
    if (!g || !s) { msg = "grid and species must not be NULL"; return false; }
    if (g->lattice != EVD_D2Q9 && g->lattice != EVD_D3Q19) { msg = "unknown lattice"; return false; }
    if (g->precision < EVD_FP64 || g->precision > EVD_FP16_STORE) { msg = "unknown precision"; return false; }
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) { msg = "grid extents must be >= 1"; return false; }
    if (g->lattice == EVD_D2Q9 && g->nz != 1) { msg = "D2Q9 needs nz == 1"; return false; }
    const long long n = (long long)g->nx * g->ny * g->nz;
    if (n >= (1LL << 31)) { msg = "nx*ny*nz must be below 2^31"; return false; }
    if (g->wall_mask & ~0x3Fu) { msg = "unknown wall_mask bits"; return false; }
    for (int k = 0; k < 3; ++k) {
        const unsigned w = (g->wall_mask >> (2 * k)) & 3u;
        if (w == 1u || w == 2u) { msg = "a dimension must be periodic or walled at both ends"; return false; }
    }
    if (g->lattice == EVD_D2Q9 && (g->wall_mask & 0x30u)) { msg = "D2Q9 has no z walls"; return false; }
    if (s->n_species < 1 || s->n_species > EVD_MAX_SPECIES) { msg = "n_species must be 1..6"; return false; }
    if (g->lattice == EVD_D3Q19 && s->n_species > EVD_MAX_SPECIES_D3Q19) {
        msg = "D3Q19 takes at most 3 species";
        return false;
    }
    if (!s->molar_mass) { msg = "molar_mass is NULL"; return false; }
    for (int i = 0; i < s->n_species; ++i) {
        if (!(s->molar_mass[i] > 0.0) || !std::isfinite(s->molar_mass[i])) { msg = "molar masses must be > 0"; return false; }
        if (i > 0 && s->molar_mass[i] < s->molar_mass[i - 1]) { msg = "molar masses must be non-decreasing"; return false; }
    }
    if (s->n_species > 1) {
        if (!s->diffusivity) { msg = "diffusivity is NULL"; return false; }
        const int N = s->n_species;
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) {
                const double a = s->diffusivity[i * N + j], b = s->diffusivity[j * N + i];
                if (!(a > 0.0) || !std::isfinite(a)) { msg = "diffusivities must be > 0"; return false; }
                if (std::fabs(a - b) > 1e-12 * std::fabs(a)) { msg = "diffusivity matrix must be symmetric"; return false; }
            }
    }
    if (!(s->tau1 > 0.5) || !std::isfinite(s->tau1)) { msg = "tau1 must be > 1/2"; return false; }
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(s->g[k])) { msg = "g must be finite"; return false; }
    if (g->lattice == EVD_D2Q9 && s->g[2] != 0.0) { msg = "D2Q9 needs g[2] == 0"; return false; }
    if (s->flags & ~(EVD_FORCE_S_DIFF | EVD_FORCE_S_P | EVD_FORCE_S_RHO)) { msg = "unknown species flags"; return false; }
    if (s->flags && g->lattice != EVD_D2Q9) {
        msg = "the corrective forcing terms are implemented for D2Q9";
        return false;
    }
    if (s->flags && s->n_species > evd::MAXS_FAST) {
        msg = "the corrective forcing terms take at most 3 species";
        return false;
    }
    return true;
}

long long plane_stride(const evd_grid* g)
{
    const long long n = (long long)g->nx * g->ny * g->nz;
    return (n + PLANE_ALIGN - 1) / PLANE_ALIGN * PLANE_ALIGN;
}

// Planes of a population buffer: one per (species, direction), plus one per
// species holding the node densities that half storage decodes with.
int buffer_planes(int lattice, int precision, int ns)
{
    const int Q = lattice == EVD_D2Q9 ? 9 : 19;
    return ns * Q + (precision == EVD_FP16_STORE ? ns : 0);
}

size_t buffer_bytes(const evd_grid* g, const evd_species* s)
{
    return (size_t)plane_stride(g) * (size_t)buffer_planes(g->lattice, g->precision, s->n_species) *
           elem_size(g->precision);
}

// Constants of the scheme for this run (double precision).
//   c_i = sqrt(M_1/M_i)                                  Eq. (speed_DLS)
//   c_s,i^2 = c_i^2 / 3
//   tau_i from (tau_i - 1/2) c_s,i^2 = (tau_1 - 1/2) c_s,1^2   (equal viscosity)
//   1-D interpolation weights for a component s = c_i along the motion:
//     upstream node  W(s;+1) = s(1+s)/2,  centre W(s;0) = 1 - s^2,
//     downstream     W(s;-1) = -s(1-s)/2  (Eq. Second_order_spatial_interpolation)
//   2 n^2 M_i M_j / (p dt) = n * 6 M_i M_j / M_1 with p = n M_1 c_s,1^2
void fill_params(HostParams& h, const evd_grid* g, const evd_species* s)
{
    std::memset(&h, 0, sizeof(h));
    h.lattice = g->lattice;
    h.precision = g->precision;
    h.ns = s->n_species;
    h.nx = g->nx; h.ny = g->ny; h.nz = g->nz;
    h.nsites = g->nx * g->ny * g->nz;
    h.pstride = plane_stride(g);
    h.flags = s->flags;
    h.wait_polls = kWaitPolls;
    for (int k = 0; k < 3; ++k) {
        h.wall[k] = ((g->wall_mask >> (2 * k)) & 3u) ? 1 : 0;
        h.g[k] = s->g[k];
    }
    if (g->lattice == EVD_D2Q9) { h.wl[0] = 4.0 / 9.0; h.wl[1] = 1.0 / 9.0; h.wl[2] = 1.0 / 36.0; }
    else { h.wl[0] = 1.0 / 3.0; h.wl[1] = 1.0 / 18.0; h.wl[2] = 1.0 / 36.0; }
    // Float arithmetic: constants whose sums must be exactly one (lattice
    // weights, 1 - 1/tau + 1/tau, the 1-D interpolation weights) are put on
    // the 2^-24 grid, where the float values are exact and the sums are
    // exactly one.  Rounded independently they bias the species mass by up to
    // ~3e-8 per step.
    const bool on_grid = g->precision != EVD_FP64;
    const double q = 16777216.0;
    auto grid24 = [&](double v) { return on_grid ? std::nearbyint(v * q) / q : v; };
    if (on_grid) {
        const int n1 = g->lattice == EVD_D2Q9 ? 4 : 6, n2 = g->lattice == EVD_D2Q9 ? 4 : 12;
        h.wl[1] = grid24(h.wl[1]);
        h.wl[2] = grid24(h.wl[2]);
        h.wl[0] = 1.0 - n1 * h.wl[1] - n2 * h.wl[2];
    }
    // The lattice's second moment m2 = sum_a w_a e_ax^2 (1/3 for both
    // lattices; with grid-rounded weights it is 1/3 + O(1e-8)).
    const double m2 = !on_grid ? 1.0 / 3.0
                               : (g->lattice == EVD_D2Q9 ? 2.0 * h.wl[1] + 4.0 * h.wl[2] : 2.0 * h.wl[1] + 8.0 * h.wl[2]);
    const double M1 = s->molar_mass[0];
    const double cs2_1 = 1.0 / 3.0;
    for (int i = 0; i < h.ns; ++i) {
        const double Mi = s->molar_mass[i];
        const double c = std::sqrt(M1 / Mi);
        const double cs2_ref = c * c / 3.0;
        const double tau = 0.5 + (s->tau1 - 0.5) * (cs2_1 / cs2_ref);
        h.M[i] = Mi;
        h.Minv[i] = 1.0 / Mi;
        h.c[i] = c;
        h.unit[i] = (c == 1.0) ? 1 : 0;
        h.inv_cs2[i] = 1.0 / cs2_ref;
        h.c_inv_cs2[i] = c / cs2_ref;
        h.c_inv_cs2_lo[i] = 0.0;
        if (on_grid) {
            // The collision keeps the species momentum sum_a e_a f_a only if
            // c k m2 = 1, k = c / c_s^2 the factor of e.u in the equilibrium
            // (sum_a e_a f^eq_a = rho u c k m2 with u = c j / rho).  With
            // float c and k and the rounded weights c k m2 - 1 is up to
            // ~5e-7, and every collision scales the momentum by that much:
            // over 10^4 steps slow pressure waves grow or decay by ~1e-3 and
            // move a diffusion front by a few 1e-5 in mole fraction.  So k =
            // 1 / (c m2) for the float c, held as a float pair k_hi + k_lo
            // (c k m2 = 1 to ~1e-14), and c_s^2 = c^2 m2.
            const double cf = (double)(float)c;
            const double k = 1.0 / (cf * m2);
            h.c_inv_cs2[i] = (double)(float)k;
            h.c_inv_cs2_lo[i] = (double)(float)(k - h.c_inv_cs2[i]);
            h.inv_cs2[i] = 1.0 / (cf * cf * m2);
        }
        h.tau_inv[i] = grid24(1.0 / tau);
        h.omt[i] = on_grid ? 1.0 - h.tau_inv[i] : 1.0 - 1.0 / tau;
        h.sfac[i] = 1.0 - 1.0 / (2.0 * tau);
        h.w1[i][0] = c * (1.0 + c) / 2.0;
        h.w1[i][1] = 1.0 - c * c;
        h.w1[i][2] = -c * (1.0 - c) / 2.0;
        if (on_grid) {
            h.w1[i][0] = grid24(h.w1[i][0]);
            h.w1[i][2] = grid24(h.w1[i][2]);
            h.w1[i][1] = 1.0 - h.w1[i][0] - h.w1[i][2];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) h.w2[i][a][b] = h.w1[i][a] * h.w1[i][b];
        for (int j = 0; j < h.ns; ++j) {
            h.MM[i][j] = 6.0 * Mi * s->molar_mass[j] / M1;
            h.iD[i][j] = (i == j) ? 0.0 : 1.0 / s->diffusivity[i * h.ns + j];
        }
    }
}

}  // namespace evd

namespace {

using evd::buffer_bytes;
using evd::buffer_planes;
using evd::elem_size;
using evd::fill_params;
using evd::plane_stride;
using evd::validate;

// Seed of the dithered rounding of the step that makes f*_t (t >= 1).
unsigned step_seed(long long t)
{
    return (unsigned)((unsigned long long)t * 2654435761ull) | 1u;
}

// Global deviation references of float storage (half storage keeps one per
// node instead; FP64 stores populations as they are).
void set_reference(evd_ctx* c, const double* rho_ref)
{
    for (int i = 0; i < MAXS; ++i)
        for (int k = 0; k < 3; ++k)
            c->hp.ref[i][k] = (c->enc != ENC_F32 || i >= c->ns) ? 0.0 : c->hp.wl[k] * rho_ref[i];
}

// Float storage: deviations from one reference per species (the TMA step
// implements it) unless a species' density varies by more than a factor
// kNodeRefContrast over the initial field, where they are taken from each
// node's own density (a depleted species would otherwise keep the float
// precision of the species mean, not of its own density).  The caller's
// choice (evd_set_reference_mode) overrides.  lo / hi: the smallest and
// largest density of each species over the field.
constexpr double kNodeRefContrast = 2.0;

void choose_encoding(evd_ctx* c, const double* lo, const double* hi)
{
    if (c->precision != EVD_FP32) return;
    bool node = c->ref_mode == EVD_REF_NODE;
    if (c->ref_mode == EVD_REF_AUTO)
        for (int i = 0; i < c->ns; ++i)
            if (!(hi[i] <= kNodeRefContrast * lo[i])) node = true;
    c->enc = node ? ENC_F32N : ENC_F32;
}

// The TMA-staged step runs this context's steps: chosen, a uniform force,
// and an encoding it implements (not the node-reference float encoding).
bool tma_active(const evd_ctx* c)
{
    return c->kernel == EVD_KERNEL_TMA && !c->kf && c->enc != ENC_F32N;
}

cudaError_t launch_step(evd_ctx* c, const void* fin, void* fout, int flags, const double* corr)
{
    const HostParams& h = c->hp;
    double* mp = c->mass_part;
    unsigned* e = c->err_flag;
    cudaStream_t st = c->stream;
    c->launches += 1;
    if (tma_active(c)) {
        const int in = (fin == c->buf[0]) ? 0 : 1;
        c->last_parts = evd::TmaLaunch::parts(h, c->tma_ty);
        if (c->precision == EVD_FP32)
            return evd::launch_step_tma<1>(h, c->tma_ty, c->tma[in], fin, fout, mp, e, flags, corr, c->lumps, st);
        return evd::launch_step_tma<2>(h, c->tma_ty, c->tma[in], fin, fout, mp, e, flags, corr, c->lumps, st);
    }
    c->last_parts = c->nblocks;
    if (h.flags) {   // corrective forcing terms (D2Q9): densities of f_t first when gradients are needed
        if (h.rhof) {
            c->launches += 1;
            const cudaError_t ed = c->enc == ENC_F64  ? evd::CorrLaunch<0>::density(h, fin, corr, st)
                                 : c->enc == ENC_F32  ? evd::CorrLaunch<1>::density(h, fin, corr, st)
                                 : c->enc == ENC_F32N ? evd::CorrLaunch<3>::density(h, fin, corr, st)
                                                      : evd::CorrLaunch<2>::density(h, fin, corr, st);
            if (ed != cudaSuccess) return ed;
        }
        if (c->enc == ENC_F64) return evd::CorrLaunch<0>::step(h, fin, fout, mp, e, flags, corr, st);
        if (c->enc == ENC_F32) return evd::CorrLaunch<1>::step(h, fin, fout, mp, e, flags, corr, st);
        if (c->enc == ENC_F32N) return evd::CorrLaunch<3>::step(h, fin, fout, mp, e, flags, corr, st);
        return evd::CorrLaunch<2>::step(h, fin, fout, mp, e, flags, corr, st);
    }
    switch (c->enc * 2 + c->lattice) {
        case 0: return evd::Launch<0, 0>::step(h, fin, fout, mp, e, flags, corr, st);
        case 1: return evd::Launch<0, 1>::step(h, fin, fout, mp, e, flags, corr, st);
        case 2: return evd::Launch<1, 0>::step(h, fin, fout, mp, e, flags, corr, st);
        case 3: return evd::Launch<1, 1>::step(h, fin, fout, mp, e, flags, corr, st);
        case 4: return evd::Launch<2, 0>::step(h, fin, fout, mp, e, flags, corr, st);
        case 5: return evd::Launch<2, 1>::step(h, fin, fout, mp, e, flags, corr, st);
        case 6: return evd::Launch<3, 0>::step(h, fin, fout, mp, e, flags, corr, st);
        case 7: return evd::Launch<3, 1>::step(h, fin, fout, mp, e, flags, corr, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_readout(evd_ctx* c, const void* fin, int flags, double* x, double* rho, double* u,
                           double* ui, double* fpop)
{
    const HostParams& h = c->hp;
    double* mp = c->mass_part;
    unsigned* e = c->err_flag;
    cudaStream_t st = c->stream;
    // f_t as the last step saw it includes the correction that step applied
    const double* cr = (!(flags & FLAG_RAW) && c->corr_applied >= 0) ? c->corr[c->corr_applied] : nullptr;
    c->launches += 1;
    switch (c->enc * 2 + c->lattice) {
        case 0: return evd::Launch<0, 0>::readout(h, fin, flags, x, rho, u, ui, fpop, mp, e, cr, st);
        case 1: return evd::Launch<0, 1>::readout(h, fin, flags, x, rho, u, ui, fpop, mp, e, cr, st);
        case 2: return evd::Launch<1, 0>::readout(h, fin, flags, x, rho, u, ui, fpop, mp, e, cr, st);
        case 3: return evd::Launch<1, 1>::readout(h, fin, flags, x, rho, u, ui, fpop, mp, e, cr, st);
        case 4: return evd::Launch<2, 0>::readout(h, fin, flags, x, rho, u, ui, fpop, mp, e, cr, st);
        case 5: return evd::Launch<2, 1>::readout(h, fin, flags, x, rho, u, ui, fpop, mp, e, cr, st);
        case 6: return evd::Launch<3, 0>::readout(h, fin, flags, x, rho, u, ui, fpop, mp, e, cr, st);
        case 7: return evd::Launch<3, 1>::readout(h, fin, flags, x, rho, u, ui, fpop, mp, e, cr, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_init(evd_ctx* c, const double* x, const double* n, const double* fsrc)
{
    const HostParams& h = c->hp;
    void* prev = c->buf[c->cur ^ 1];
    void* cur = c->buf[c->cur];
    double* mp = c->mass_part;
    unsigned* e = c->err_flag;
    cudaStream_t st = c->stream;
    c->launches += 1;
    switch (c->enc * 2 + c->lattice) {
        case 0: return evd::Launch<0, 0>::init(h, x, n, fsrc, prev, cur, mp, e, st);
        case 1: return evd::Launch<0, 1>::init(h, x, n, fsrc, prev, cur, mp, e, st);
        case 2: return evd::Launch<1, 0>::init(h, x, n, fsrc, prev, cur, mp, e, st);
        case 3: return evd::Launch<1, 1>::init(h, x, n, fsrc, prev, cur, mp, e, st);
        case 4: return evd::Launch<2, 0>::init(h, x, n, fsrc, prev, cur, mp, e, st);
        case 5: return evd::Launch<2, 1>::init(h, x, n, fsrc, prev, cur, mp, e, st);
        case 6: return evd::Launch<3, 0>::init(h, x, n, fsrc, prev, cur, mp, e, st);
        case 7: return evd::Launch<3, 1>::init(h, x, n, fsrc, prev, cur, mp, e, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// Fixed-order sum of per-block partials [nblocks][ns]: thread t adds blocks
// t, t+1024, ... in order, then a fixed binary tree.  Writes the totals to
// out[ns], or, when target != nullptr, the relative deficit
// (target_i - total_i) / total_i that the next step re-injects in proportion
// to each node's density.
__global__ void __launch_bounds__(1024)
evd_k_mass_finish(const double* __restrict__ part, int nblocks, int ns, const double* __restrict__ target,
                  double inv_nsites, double* __restrict__ out)
{
    __shared__ double sm[1024];
    for (int i = 0; i < ns; ++i) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += 1024) s += part[(long long)b * ns + i];
        sm[threadIdx.x] = s;
        __syncthreads();
        for (int w = 512; w > 0; w >>= 1) {
            if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[i] = target ? (target[i] - sm[0]) / sm[0] : sm[0];
        __syncthreads();
    }
}

// Smallest and largest species density x_i M_i n of an initial field,
// per species: range[i] and range[ns + i] receive the bit patterns of the
// positive doubles (which order as unsigned integers), by atomic min / max.
__global__ void __launch_bounds__(128)
evd_k_field_range(const double* __restrict__ x, const double* __restrict__ nf, int nsites, int ns,
                  const evd::MassTable mt, unsigned long long* __restrict__ range)
{
    const int node = blockIdx.x * 128 + threadIdx.x;
    const bool active = node < nsites;
    const double* M = mt.M;
    const double n = active ? (nf ? nf[node] : 1.0) : 1.0;
    for (int i = 0; i < ns; ++i) {
        const double v = active ? x[(long long)i * nsites + node] * M[i] * n : 0.0;
        double lo = active ? v : __longlong_as_double(0x7fefffffffffffffLL), hi = active ? v : 0.0;
        for (int off = 16; off > 0; off >>= 1) {
            lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, off));
            hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, off));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(range + i, (unsigned long long)__double_as_longlong(lo));
            atomicMax(range + ns + i, (unsigned long long)__double_as_longlong(hi));
        }
    }
}

// Per-block partials of sum_x x_i M_i n (the initial species masses).
__global__ void __launch_bounds__(128)
evd_k_field_mass(const double* __restrict__ x, const double* __restrict__ nf, int nsites, int ns,
                 const evd::MassTable mt, double* __restrict__ part)
{
    __shared__ double sm[evd::MAXS][4];
    const int node = blockIdx.x * 128 + threadIdx.x;
    const bool active = node < nsites;
    const double* M = mt.M;
    const double n = active ? (nf ? nf[node] : 1.0) : 0.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < ns; ++i) {
        double v = active ? x[(long long)i * nsites + node] * M[i] * n : 0.0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sm[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < ns) {
        double t = 0.0;
        for (int w = 0; w < 4; ++w) t += sm[threadIdx.x][w];
        part[(long long)blockIdx.x * ns + threadIdx.x] = t;
    }
}

namespace {

evd_status ensure_staging(evd_ctx* c, size_t bytes)
{
    if (c->staging_bytes >= bytes) return EVD_OK;
    if (c->staging) cudaFree(c->staging);
    c->staging = nullptr;
    c->staging_bytes = 0;
    CK(c, cudaMalloc((void**)&c->staging, bytes));
    c->staging_bytes = bytes;
    return EVD_OK;
}

evd_status finish_mass(evd_ctx* c, double* out, const double* target = nullptr, int parts = -1)
{
    c->launches += 1;
    evd_k_mass_finish<<<1, 1024, 0, c->stream>>>(c->mass_part, parts < 0 ? c->nblocks : parts, c->ns, target,
                                                 1.0 / (double)c->nsites, out);
    CK(c, cudaGetLastError());
    return EVD_OK;
}

// Tensor maps of the TMA-staged step: each population buffer seen as a 4-D
// tensor (x, y, z, plane).  D3Q19 planes are stored [group][species][direction
// in group] (groups of directions that move in the same dimensions); one map
// per group, whose box is the tile plus a one-node halo in the in-plane
// dimensions the group moves in (x halo widened to 16 bytes each side, the
// TMA alignment), one z-plane, and all NS * group-size planes of the group.
// Returns false when the configuration needs the general kernel: another
// lattice or precision, periodic x or y, rows that are not a multiple of 16
// bytes, or no driver entry point.
// D3Q19 unit vectors in the library's direction order (include/evd.h).
const int kE19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                         {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                         {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                         {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

int opp19(int a)
{
    for (int b = 0; b < 19; ++b)
        if (kE19[b][0] == -kE19[a][0] && kE19[b][1] == -kE19[a][1] && kE19[b][2] == -kE19[a][2]) return b;
    return 0;
}

// App. A lumped weight of direction b leaving a node of the given wall class
// (lo/hi per dimension): the push weight bound for solid nodes that stays at
// the node, in b itself (into_self) or in its opposite.  The rule: stays in
// b unless b heads into the crossed wall(s), e_b . d_s > 0.
double lump_weight(const HostParams& h, int i, int b, const bool lo[3], const bool hi[3], bool into_self)
{
    double acc = 0.0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int d[3] = {dx, dy, dz};
                bool skip = false, crossed = false;
                int dot = 0;
                double w = 1.0;
                for (int k = 0; k < 3; ++k) {
                    const int e = kE19[b][k];
                    if (e == 0) {
                        if (d[k] != 0) skip = true;
                        continue;
                    }
                    w *= h.w1[i][d[k] == e ? 0 : (d[k] == 0 ? 1 : 2)];
                    const bool cr = (d[k] == 1 && hi[k]) || (d[k] == -1 && lo[k]);
                    crossed |= cr;
                    if (cr) dot += e * d[k];
                }
                if (skip || !crossed) continue;
                if ((dot > 0) != into_self) acc += w;
            }
    return acc;
}

// Table [27 wall classes][ns][19] of (L_self, L_opp) floats for the TMA step.
// Per (wall class, species, direction): the App. A lumped weights L_self,
// L_opp, and K - 1 where K is the sum of every weight feeding that population
// (the fluid stencil weights and both lumps); float storage, which gathers
// deviations from a reference, adds the reference times K - 1.
bool build_lumps(evd_ctx* c)
{
    const int n = 27 * c->ns * 19 * 4;
    float* host = new float[n];
    for (int cls = 0; cls < 27; ++cls) {
        const int cc[3] = {cls % 3, (cls / 3) % 3, cls / 9};
        bool lo[3], hi[3];
        for (int k = 0; k < 3; ++k) { lo[k] = cc[k] == 1; hi[k] = cc[k] == 2; }
        for (int i = 0; i < c->ns; ++i)
            for (int a = 0; a < 19; ++a) {
                float* t = host + ((cls * c->ns + i) * 19 + a) * 4;
                const double ls = a ? lump_weight(c->hp, i, a, lo, hi, true) : 0.0;
                const double lop = a ? lump_weight(c->hp, i, opp19(a), lo, hi, false) : 0.0;
                double kin = 1.0;   // fluid stencil weights: product of masked 1-D sums
                for (int k = 0; k < 3; ++k) {
                    const int e = kE19[a][k];
                    if (e == 0) continue;
                    double sk = 0.0;
                    for (int o = -1; o <= 1; ++o) {
                        if ((o == -1 && lo[k]) || (o == 1 && hi[k])) continue;
                        sk += c->hp.w1[i][o == -e ? 0 : (o == 0 ? 1 : 2)];
                    }
                    kin *= sk;
                }
                t[0] = (float)ls;
                t[1] = (float)lop;
                t[2] = (float)(kin + ls + lop - 1.0);
                t[3] = 0.0f;
            }
    }
    bool ok = cudaMalloc((void**)&c->lumps, n * sizeof(float)) == cudaSuccess &&
              cudaMemcpy(c->lumps, host, n * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    delete[] host;
    return ok;
}

bool tma_setup(evd_ctx* c)
{
    if (c->lattice != EVD_D3Q19 || c->precision == EVD_FP64 || c->ns > evd::MAXS_FAST) return false;
    if (!c->hp.wall[0] || !c->hp.wall[1]) return false;
    if (c->nx < 2 || c->ny < 2 || (c->hp.wall[2] && c->nz < 2)) return false;
    const int planes = buffer_planes(c->lattice, c->precision, c->ns);
    if ((long long)planes * c->pstride >= (1LL << 31)) return false;
    const size_t elem = c->elem;
    if (((size_t)c->nx * elem) % 16 != 0) return false;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const int TY = c->tma_ty, TX = evd::TmaLaunch::TX;
    const int XP = (int)(16 / elem);
    // storage groups: halo class (bit 0 x, bit 1 y) and planes per species;
    // group 7 is the node densities of half storage (planes ns * 19 + i)
    const int gcls[8] = {0, 0, 1, 1, 2, 2, 3, 3};
    const int gsize[8] = {1, 2, 2, 4, 2, 4, 4, 1};
    const int ngroups = c->precision == EVD_FP16_STORE ? 8 : 7;
    const cuuint64_t dims[4] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, (cuuint64_t)c->nz, (cuuint64_t)planes};
    const cuuint64_t strides[3] = {(cuuint64_t)c->nx * elem, (cuuint64_t)c->nx * c->ny * elem,
                                   (cuuint64_t)c->pstride * elem};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int b = 0; b < 2; ++b)
        for (int g = 0; g < ngroups; ++g) {
            const int cls = gcls[g];
            const cuuint32_t box[4] = {(cuuint32_t)((cls & 1) ? TX + 2 * XP : TX),
                                       (cuuint32_t)((cls & 2) ? TY + 2 : TY), 1,
                                       (cuuint32_t)(c->ns * gsize[g])};
            const CUresult r = encode(&c->tma[b][g],
                                      c->precision == EVD_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                                      4, c->buf[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return false;
        }
    return build_lumps(c);
}

evd_status create_common(const evd_grid* grid, const evd_species* species, void* stream, void* pa,
                         void* pb, size_t bytes_each, evd_ctx** out)
{
    if (!out) return fail(nullptr, EVD_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    std::string msg;
    if (!validate(grid, species, msg)) return fail(nullptr, EVD_ERR_ARG, msg);
    evd_ctx* c = new evd_ctx();
    c->lattice = grid->lattice;
    c->precision = grid->precision;
    c->ns = species->n_species;
    c->Q = grid->lattice == EVD_D2Q9 ? 9 : 19;
    c->D = grid->lattice == EVD_D2Q9 ? 2 : 3;
    c->nx = grid->nx; c->ny = grid->ny; c->nz = grid->nz;
    c->nsites = grid->nx * grid->ny * grid->nz;
    c->elem = elem_size(grid->precision);
    c->pstride = plane_stride(grid);
    c->buf_bytes = buffer_bytes(grid, species);
    c->stream = (cudaStream_t)stream;
    c->nblocks = (c->nsites + BLOCK - 1) / BLOCK;
    fill_params(c->hp, grid, species);
    c->wall_mask = grid->wall_mask;
    c->sp_M.assign(species->molar_mass, species->molar_mass + c->ns);
    if (c->ns > 1) c->sp_D.assign(species->diffusivity, species->diffusivity + c->ns * c->ns);
    else c->sp_D.assign(1, 0.0);
    c->sp_tau1 = species->tau1;
    for (int k = 0; k < 3; ++k) c->sp_g[k] = species->g[k];
    double zero[MAXS] = {0, 0, 0};
    set_reference(c, zero);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) { delete c; return cuda_fail(nullptr, e, "cudaGetDevice"); }
    if (pa || pb) {
        if (!pa || !pb || pa == pb) { delete c; return fail(nullptr, EVD_ERR_ARG, "need two distinct buffers"); }
        if (bytes_each < c->buf_bytes) { delete c; return fail(nullptr, EVD_ERR_ARG, "buffers too small"); }
        if (((uintptr_t)pa | (uintptr_t)pb) & 255u) { delete c; return fail(nullptr, EVD_ERR_ARG, "buffers must be 256-byte aligned"); }
        c->buf[0] = pa; c->buf[1] = pb; c->own_bufs = false;
    } else {
        c->own_bufs = true;
        for (int b = 0; b < 2; ++b) {
            e = cudaMalloc(&c->buf[b], c->buf_bytes);
            if (e != cudaSuccess) {
                if (b == 1) cudaFree(c->buf[0]);
                delete c;
                return cuda_fail(nullptr, e, "cudaMalloc(populations)");
            }
        }
    }
    if (c->hp.flags & (EVD_FORCE_S_P | EVD_FORCE_S_RHO)) {
        // densities of f_t at every node, for the gradient terms
        const size_t rb = (size_t)(c->ns + 1) * c->nsites * (c->precision == EVD_FP64 ? sizeof(double) : sizeof(float));
        e = cudaMalloc(&c->rhof, rb);
        if (e != cudaSuccess) {
            if (c->own_bufs) { cudaFree(c->buf[0]); cudaFree(c->buf[1]); }
            delete c;
            return cuda_fail(nullptr, e, "cudaMalloc(density field)");
        }
        c->hp.rhof = c->rhof;
    }
    c->ref_mode = EVD_REF_AUTO;
    c->enc = c->precision == EVD_FP64 ? ENC_F64 : c->precision == EVD_FP32 ? ENC_F32 : ENC_F16;
    c->tma_ty = kTmaRows;
    c->tma_ok = tma_setup(c);
    c->kernel = c->tma_ok ? EVD_KERNEL_TMA : EVD_KERNEL_GENERAL;
    c->tma_blocks = c->tma_ok ? evd::TmaLaunch::grid(c->hp, c->tma_ty) : 0;
    // partials for either tile height, so that evd_set_tile_rows never reallocates
    const int max_tma = c->tma_ok ? evd::TmaLaunch::parts(c->hp, 1) : 0;
    const int max_parts = c->nblocks > max_tma ? c->nblocks : max_tma;
    const size_t part_bytes = ((size_t)max_parts * c->ns * sizeof(double) + 255) / 256 * 256;
    e = cudaMalloc(&c->small, part_bytes + 6 * 256);
    if (e != cudaSuccess) {
        if (c->own_bufs) { cudaFree(c->buf[0]); cudaFree(c->buf[1]); }
        delete c;
        return cuda_fail(nullptr, e, "cudaMalloc(scratch)");
    }
    c->mass_part = (double*)c->small;
    c->mass_out = (double*)((char*)c->small + part_bytes);
    c->m_target = (double*)((char*)c->small + part_bytes + 256);
    c->corr[0] = (double*)((char*)c->small + part_bytes + 512);
    c->corr[1] = (double*)((char*)c->small + part_bytes + 768);
    c->err_flag = (unsigned*)((char*)c->small + part_bytes + 1024);
    c->range = (unsigned long long*)((char*)c->small + part_bytes + 1280);
    c->corr_pending = c->corr_applied = -1;
    // FP16 storage rounding moves the species mass by ~1e-7 per step on rough
    // fields, so it is corrected every step; FP32 drifts ~1e-9 per step
    c->mc_every = (c->precision == EVD_FP64) ? 0 : (c->precision == EVD_FP32 ? 8 : 1);
    e = cudaMemsetAsync(c->err_flag, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) {
        evd_destroy(c);
        return cuda_fail(nullptr, e, "cudaMemsetAsync");
    }
    *out = c;
    return EVD_OK;
}

evd_status readout_to_host(evd_ctx* c, double* x_h, double* rho_h, double* u_h, double* ui_h)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!c->ready) return fail(c, EVD_ERR_STATE, "set_fields has not been called");
    DeviceGuard dg(c->device);
    const size_t n = (size_t)c->nsites;
    const size_t sx = x_h ? c->ns * n : 0, sr = rho_h ? c->ns * n : 0, su = u_h ? c->D * n : 0,
                 sui = ui_h ? c->ns * c->D * n : 0;
    evd_status s = ensure_staging(c, (sx + sr + su + sui + 1) * sizeof(double));
    if (s != EVD_OK) return s;
    double* d = c->staging;
    double *dx = x_h ? d : nullptr, *dr = rho_h ? d + sx : nullptr, *du = u_h ? d + sx + sr : nullptr,
           *dui = ui_h ? d + sx + sr + su : nullptr;
    s = evd_readout_device(c, dx, dr, du, dui);
    if (s != EVD_OK) return s;
    if (x_h) CK(c, cudaMemcpyAsync(x_h, dx, sx * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (rho_h) CK(c, cudaMemcpyAsync(rho_h, dr, sr * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (u_h) CK(c, cudaMemcpyAsync(u_h, du, su * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (ui_h) CK(c, cudaMemcpyAsync(ui_h, dui, sui * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return evd_check(c);
}

}  // namespace

extern "C" {

int evd_version(void) { return EVD_API_VERSION; }

size_t evd_required_bytes(const evd_grid* grid, const evd_species* species)
{
    std::string msg;
    if (!validate(grid, species, msg)) return 0;
    return buffer_bytes(grid, species);
}

evd_status evd_create(const evd_grid* grid, const evd_species* species, void* cuda_stream, evd_ctx** out)
{
    return create_common(grid, species, cuda_stream, nullptr, nullptr, 0, out);
}

evd_status evd_create_with_buffers(const evd_grid* grid, const evd_species* species, void* cuda_stream,
                                   void* pop_a, void* pop_b, size_t bytes_each, evd_ctx** out)
{
    if (!pop_a || !pop_b) {
        if (out) *out = nullptr;
        return fail(nullptr, EVD_ERR_ARG, "pop_a and pop_b must not be NULL");
    }
    return create_common(grid, species, cuda_stream, pop_a, pop_b, bytes_each, out);
}

evd_status evd_set_stream(evd_ctx* ctx, void* cuda_stream)
{
    if (!ctx) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    ctx->stream = (cudaStream_t)cuda_stream;
    return EVD_OK;
}

evd_status evd_set_fields_device(evd_ctx* c, const double* x_dev, const double* n_dev)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!x_dev) return fail(c, EVD_ERR_ARG, "x must not be NULL");
    DeviceGuard dg(c->device);
    // initial species masses sum_x x_i M_i n in FP64: the target of the mass
    // correction and, for deviation storage, the reference densities
    c->launches += 1;
    evd::MassTable mt;
    for (int i = 0; i < MAXS; ++i) mt.M[i] = c->hp.M[i];
    evd_k_field_mass<<<c->nblocks, 128, 0, c->stream>>>(x_dev, n_dev, c->nsites, c->ns, mt, c->mass_part);
    CK(c, cudaGetLastError());
    evd_status s0 = finish_mass(c, c->m_target);
    if (s0 != EVD_OK) return s0;
    if (c->precision == EVD_FP32 && c->ref_mode == EVD_REF_AUTO) {
        // the density range of each species decides the float encoding
        CK(c, cudaMemsetAsync(c->range, 0xff, c->ns * sizeof(unsigned long long), c->stream));
        CK(c, cudaMemsetAsync(c->range + c->ns, 0, c->ns * sizeof(unsigned long long), c->stream));
        c->launches += 1;
        evd_k_field_range<<<c->nblocks, 128, 0, c->stream>>>(x_dev, n_dev, c->nsites, c->ns, mt, c->range);
        CK(c, cudaGetLastError());
    }
    if (c->precision != EVD_FP64) {
        double m[MAXS] = {0, 0, 0}, ref[MAXS] = {0, 0, 0};
        unsigned long long rg[2 * MAXS] = {};
        CK(c, cudaMemcpyAsync(m, c->m_target, c->ns * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (c->precision == EVD_FP32 && c->ref_mode == EVD_REF_AUTO)
            CK(c, cudaMemcpyAsync(rg, c->range, 2 * c->ns * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                  c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        double lo[MAXS], hi[MAXS];
        for (int i = 0; i < c->ns; ++i) {
            if (!(m[i] > 0.0)) return fail(c, EVD_ERR_ARG, "initial species mass must be > 0");
            ref[i] = m[i] / c->nsites;
            std::memcpy(&lo[i], &rg[i], sizeof(double));
            std::memcpy(&hi[i], &rg[c->ns + i], sizeof(double));
        }
        choose_encoding(c, lo, hi);
        set_reference(c, ref);
    }
    CK(c, cudaMemsetAsync(c->err_flag, 0, sizeof(unsigned), c->stream));
    c->cur = 0;
    CK(c, launch_init(c, x_dev, n_dev, nullptr));
    c->prev_raw = true;
    c->ready = true;
    c->corr_pending = c->corr_applied = -1;
    c->t = 0;
    return EVD_OK;
}

evd_status evd_set_fields(evd_ctx* c, const double* x_host, const double* n_host)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!x_host) return fail(c, EVD_ERR_ARG, "x must not be NULL");
    const size_t n = (size_t)c->nsites;
    for (size_t k = 0; k < c->ns * n; ++k)
        if (!(x_host[k] > 0.0) || !std::isfinite(x_host[k])) return fail(c, EVD_ERR_ARG, "mole fractions must be > 0");
    if (n_host)
        for (size_t k = 0; k < n; ++k)
            if (!(n_host[k] > 0.0) || !std::isfinite(n_host[k])) return fail(c, EVD_ERR_ARG, "number density must be > 0");
    DeviceGuard dg(c->device);
    evd_status s = ensure_staging(c, (c->ns * n + n) * sizeof(double));
    if (s != EVD_OK) return s;
    CK(c, cudaMemcpyAsync(c->staging, x_host, c->ns * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (n_host)
        CK(c, cudaMemcpyAsync(c->staging + c->ns * n, n_host, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    s = evd_set_fields_device(c, c->staging, n_host ? c->staging + c->ns * n : nullptr);
    if (s != EVD_OK) return s;
    CK(c, cudaStreamSynchronize(c->stream));
    return evd_check(c);
}

evd_status evd_set_populations(evd_ctx* c, const double* f_host)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!f_host) return fail(c, EVD_ERR_ARG, "f must not be NULL");
    DeviceGuard dg(c->device);
    const size_t n = (size_t)c->nsites, total = (size_t)c->ns * c->Q * n;
    double m[MAXS] = {0, 0, 0}, ref[MAXS] = {0, 0, 0}, lo[MAXS], hi[MAXS];
    for (int i = 0; i < c->ns; ++i) {
        lo[i] = HUGE_VAL;
        hi[i] = 0.0;
        for (size_t q = 0; q < n; ++q) {
            double r = 0.0;
            for (int a = 0; a < c->Q; ++a) r += f_host[((size_t)i * c->Q + a) * n + q];
            m[i] += r;
            lo[i] = std::min(lo[i], r);
            hi[i] = std::max(hi[i], r);
        }
        if (!(m[i] > 0.0)) return fail(c, EVD_ERR_ARG, "species mass must be > 0");
        ref[i] = m[i] / n;
    }
    if (c->precision != EVD_FP64) {
        choose_encoding(c, lo, hi);
        set_reference(c, ref);
    }
    CK(c, cudaMemcpyAsync(c->m_target, m, c->ns * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->corr_pending = c->corr_applied = -1;
    evd_status s = ensure_staging(c, total * sizeof(double));
    if (s != EVD_OK) return s;
    CK(c, cudaMemcpyAsync(c->staging, f_host, total * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (!c->ready) CK(c, cudaMemsetAsync(c->err_flag, 0, sizeof(unsigned), c->stream));
    CK(c, launch_init(c, nullptr, nullptr, c->staging));
    c->prev_raw = true;
    c->ready = true;
    CK(c, cudaStreamSynchronize(c->stream));
    return evd_check(c);
}

evd_status evd_step(evd_ctx* c, long long nsteps)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(c, EVD_ERR_ARG, "nsteps must be >= 0");
    if (!c->ready) return fail(c, EVD_ERR_STATE, "set_fields has not been called");
    DeviceGuard dg(c->device);
    for (long long k = 0; k < nsteps; ++k) {
        // every mc_every steps the step kernel also reduces the species masses
        // of f_t; the deficit from the FP64 targets is re-injected uniformly
        // in the next step
        const bool measure = c->mc_every > 0 && ((c->t + 1) % c->mc_every == 0);
        // reduced storage dithers its rounding with a fresh seed every step
        c->hp.seed = c->precision == EVD_FP64 ? 0u : step_seed(c->t + 1);
        const int apply = c->corr_pending;
        CK(c, launch_step(c, c->buf[c->cur], c->buf[c->cur ^ 1], measure ? FLAG_MASS : 0,
                          apply >= 0 ? c->corr[apply] : nullptr));
        c->corr_applied = apply;
        c->corr_pending = -1;
        if (measure) {
            const int slot = (apply == 0) ? 1 : 0;
            evd_status s = finish_mass(c, c->corr[slot], c->m_target, c->last_parts);
            if (s != EVD_OK) return s;
            c->corr_pending = slot;
        }
        c->cur ^= 1;
        c->prev_raw = false;
        c->t += 1;
    }
    return EVD_OK;
}

evd_status evd_readout_device(evd_ctx* c, double* x, double* rho, double* u, double* ui)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!c->ready) return fail(c, EVD_ERR_STATE, "set_fields has not been called");
    DeviceGuard dg(c->device);
    CK(c, launch_readout(c, c->buf[c->cur ^ 1], c->prev_raw ? FLAG_RAW : 0, x, rho, u, ui, nullptr));
    return finish_mass(c, c->mass_out);
}

evd_status evd_get_mole_fractions(evd_ctx* c, double* x_host)
{
    if (!x_host) return fail(c, EVD_ERR_ARG, "x must not be NULL");
    return readout_to_host(c, x_host, nullptr, nullptr, nullptr);
}

evd_status evd_get_densities(evd_ctx* c, double* rho_host)
{
    if (!rho_host) return fail(c, EVD_ERR_ARG, "rho must not be NULL");
    return readout_to_host(c, nullptr, rho_host, nullptr, nullptr);
}

evd_status evd_get_velocities(evd_ctx* c, double* u_mix_host, double* u_species_host)
{
    if (!u_mix_host && !u_species_host) return fail(c, EVD_ERR_ARG, "no output given");
    return readout_to_host(c, nullptr, nullptr, u_mix_host, u_species_host);
}

evd_status evd_species_mass_device(evd_ctx* c, double* m_dev)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!m_dev) return fail(c, EVD_ERR_ARG, "m must not be NULL");
    if (!c->ready) return fail(c, EVD_ERR_STATE, "set_fields has not been called");
    DeviceGuard dg(c->device);
    CK(c, launch_readout(c, c->buf[c->cur ^ 1], c->prev_raw ? FLAG_RAW : 0, nullptr, nullptr, nullptr,
                         nullptr, nullptr));
    return finish_mass(c, m_dev);
}

evd_status evd_get_species_mass(evd_ctx* c, double* m_host)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!m_host) return fail(c, EVD_ERR_ARG, "m must not be NULL");
    evd_status s = evd_species_mass_device(c, c->mass_out);
    if (s != EVD_OK) return s;
    DeviceGuard dg(c->device);
    CK(c, cudaMemcpyAsync(m_host, c->mass_out, c->ns * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return evd_check(c);
}

evd_status evd_get_populations(evd_ctx* c, double* f_host)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!f_host) return fail(c, EVD_ERR_ARG, "f must not be NULL");
    if (!c->ready) return fail(c, EVD_ERR_STATE, "set_fields has not been called");
    DeviceGuard dg(c->device);
    const size_t total = (size_t)c->ns * c->Q * c->nsites;
    double* tmp = nullptr;
    CK(c, cudaMalloc((void**)&tmp, total * sizeof(double)));
    cudaError_t e = launch_readout(c, c->buf[c->cur ^ 1], c->prev_raw ? FLAG_RAW : 0, nullptr, nullptr, nullptr,
                                   nullptr, tmp);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f_host, tmp, total * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "evd_get_populations");
    return evd_check(c);
}

long long evd_time(const evd_ctx* c) { return c ? c->t : -1; }

evd_status evd_check(evd_ctx* c)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    DeviceGuard dg(c->device);
    unsigned flag = 0;
    CK(c, cudaMemcpyAsync(&flag, c->err_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (flag) {
        std::string m = "unstable state:";
        if (flag & 1u) m += " non-positive or NaN species density;";
        if (flag & 2u) m += " non-positive or non-finite cross relaxation time;";
        if (flag & 4u) return fail(c, EVD_ERR_TIMEOUT, "a device-side wait for a tile copy gave up");
        return fail(c, EVD_ERR_UNSTABLE, m);
    }
    return EVD_OK;
}

long long evd_launch_count(const evd_ctx* c) { return c ? c->launches : -1; }

evd_status evd_set_kernel(evd_ctx* c, int kernel)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (kernel == EVD_KERNEL_AUTO) kernel = c->tma_ok ? EVD_KERNEL_TMA : EVD_KERNEL_GENERAL;
    if (kernel == EVD_KERNEL_TMA && !c->tma_ok)
        return fail(c, EVD_ERR_ARG, "the TMA-staged step needs D3Q19, FP32 or FP16 storage, walls in x and y "
                                    "and rows of a multiple of 16 bytes");
    if (kernel != EVD_KERNEL_GENERAL && kernel != EVD_KERNEL_TMA) return fail(c, EVD_ERR_ARG, "unknown kernel");
    if (kernel == EVD_KERNEL_TMA && c->kf)
        return fail(c, EVD_ERR_ARG, "the TMA-staged step takes a uniform body force only (a force field is set)");
    c->kernel = kernel;
    return EVD_OK;
}

int evd_get_kernel(const evd_ctx* c) { return c ? (tma_active(c) ? EVD_KERNEL_TMA : EVD_KERNEL_GENERAL) : 0; }

evd_status evd_set_reference_mode(evd_ctx* c, int mode)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (mode != EVD_REF_AUTO && mode != EVD_REF_SPECIES && mode != EVD_REF_NODE)
        return fail(c, EVD_ERR_ARG, "mode must be EVD_REF_AUTO, EVD_REF_SPECIES or EVD_REF_NODE");
    c->ref_mode = mode;
    return EVD_OK;
}

int evd_get_reference_mode(const evd_ctx* c)
{
    if (!c) return -1;
    return c->enc == ENC_F32N || c->enc == ENC_F16 ? EVD_REF_NODE : c->enc == ENC_F32 ? EVD_REF_SPECIES : EVD_REF_AUTO;
}

evd_status evd_set_force_field(evd_ctx* c, const double* k_host)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    DeviceGuard dg(c->device);
    CK(c, cudaStreamSynchronize(c->stream));
    if (!k_host) {
        if (c->kf) cudaFree(c->kf);
        c->kf = nullptr;
        c->hp.kf = nullptr;
        return EVD_OK;
    }
    const size_t n = (size_t)c->nsites;
    for (size_t q = 0; q < (size_t)c->D * n; ++q)
        if (!std::isfinite(k_host[q])) return fail(c, EVD_ERR_ARG, "force field values must be finite");
    const bool dbl = c->precision == EVD_FP64;
    const size_t bytes = 3 * n * (dbl ? sizeof(double) : sizeof(float));
    if (!c->kf) CK(c, cudaMalloc(&c->kf, bytes));
    // [3][nsites] in the arithmetic type; D2Q9 has no z component
    std::vector<char> host(bytes, 0);
    for (int k = 0; k < c->D; ++k)
        for (size_t q = 0; q < n; ++q) {
            if (dbl) ((double*)host.data())[k * n + q] = k_host[k * n + q];
            else ((float*)host.data())[k * n + q] = (float)k_host[k * n + q];
        }
    CK(c, cudaMemcpy(c->kf, host.data(), bytes, cudaMemcpyHostToDevice));
    c->hp.kf = c->kf;
    return EVD_OK;
}

evd_status evd_set_adjoint_mode(evd_ctx* c, int mode)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (mode != EVD_ADJOINT_REVERSE && mode != EVD_ADJOINT_DUAL)
        return fail(c, EVD_ERR_ARG, "mode must be EVD_ADJOINT_REVERSE or EVD_ADJOINT_DUAL");
    c->adj_mode = mode;
    return EVD_OK;
}

evd_status evd_set_adjoint_forward(evd_ctx* c, int precision)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (precision != EVD_FP64 && precision != EVD_FP32)
        return fail(c, EVD_ERR_ARG, "the adjoint's forward pass runs in EVD_FP64 or EVD_FP32");
    c->adj_forward = precision;
    return EVD_OK;
}

evd_status evd_set_tile_rows(evd_ctx* c, int rows)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (rows != 1 && rows != 2 && rows != 4) return fail(c, EVD_ERR_ARG, "rows must be 1, 2 or 4");
    if (!c->tma_ok) return fail(c, EVD_ERR_ARG, "the TMA-staged step does not apply to this configuration");
    if (rows == c->tma_ty) return EVD_OK;
    DeviceGuard dg(c->device);
    CK(c, cudaStreamSynchronize(c->stream));
    const int old = c->tma_ty;
    if (c->lumps) { cudaFree(c->lumps); c->lumps = nullptr; }
    c->tma_ty = rows;
    if (!tma_setup(c)) {
        c->tma_ty = old;
        tma_setup(c);
        return fail(c, EVD_ERR_CUDA, "could not rebuild the tile copies");
    }
    c->tma_blocks = evd::TmaLaunch::grid(c->hp, rows);
    return EVD_OK;
}

evd_status evd_set_wait_limit(evd_ctx* c, int polls)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    c->hp.wait_polls = polls < 0 ? evd::kWaitPolls : polls;
    return EVD_OK;
}

evd_status evd_set_mass_correction(evd_ctx* c, int every)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (every < 0) return fail(c, EVD_ERR_ARG, "every must be >= 0");
    c->mc_every = every;
    if (every == 0) c->corr_pending = -1;
    return EVD_OK;
}

evd_status evd_get_target_mass(evd_ctx* c, double* m_host)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!m_host) return fail(c, EVD_ERR_ARG, "m must not be NULL");
    if (!c->ready) return fail(c, EVD_ERR_STATE, "set_fields has not been called");
    DeviceGuard dg(c->device);
    CK(c, cudaMemcpyAsync(m_host, c->m_target, c->ns * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return EVD_OK;
}

namespace {

// Device buffers released together on every exit path.
struct DevBufs {
    std::vector<void*> p;
    ~DevBufs()
    {
        for (void* q : p) cudaFree(q);
    }
    cudaError_t alloc(size_t bytes, void** out)
    {
        *out = nullptr;
        cudaError_t e = cudaMalloc(out, bytes);
        if (e == cudaSuccess) p.push_back(*out);
        return e;
    }
};

}  // namespace

evd_status evd_loss_gradient(evd_ctx* c, const double* x0, const double* n0, long long nsteps, const double* target,
                             int checkpoint_every, double* loss, double* dL_dD, double* dL_dg)
{
    if (!c) return fail(nullptr, EVD_ERR_ARG, "ctx is NULL");
    if (!x0 || !target || !loss) return fail(c, EVD_ERR_ARG, "x0, target and loss must not be NULL");
    if (c->lattice != EVD_D2Q9 || c->precision != EVD_FP64)
        return fail(c, EVD_ERR_ARG, "the adjoint is implemented for D2Q9 with FP64 storage");
    if (c->ns > evd::MAXS_FAST) return fail(c, EVD_ERR_ARG, "the adjoint takes at most 3 species");
    if (c->kf || c->hp.flags || c->mc_every)
        return fail(c, EVD_ERR_ARG, "the adjoint takes a uniform g, no corrective terms, no mass correction");
    if (nsteps < 1) return fail(c, EVD_ERR_ARG, "nsteps must be >= 1");
    if (checkpoint_every < 0) return fail(c, EVD_ERR_ARG, "checkpoint_every must be >= 0");
    const long long N = nsteps;
    long long K = checkpoint_every;
    if (K == 0) {   // about sqrt(N) checkpoints of about sqrt(N) steps each
        K = 1;
        while (K * K < N) ++K;
    }
    if (K > N) K = N;
    evd_status s = evd_set_fields(c, x0, n0);
    if (s != EVD_OK) return s;
    DeviceGuard dg(c->device);
    const size_t bb = c->buf_bytes;
    const size_t n = (size_t)c->nsites;
    const int np = evd::AdjLaunch::nparams(c->ns);
    const long long ncp = (N - 1) / K + 1;          // checkpoints f*_0, f*_K, ...
    DevBufs mem;
    // FP32 forward: an internal float context (node references, no mass
    // correction) runs the forward pass and recomputes the segments with the
    // same dither seeds; each state the reverse sweep needs is decoded to
    // doubles.  The reverse sweep itself runs in FP64 either way.
    struct Owned {
        evd_ctx* p = nullptr;
        ~Owned() { if (p) evd_destroy(p); }
    } fcp;
    const bool f32 = c->adj_forward == EVD_FP32;
    if (f32) {
        const evd_grid g32{c->lattice, EVD_FP32, c->nx, c->ny, c->nz, c->wall_mask};
        evd_species s32{c->ns, c->sp_M.data(), c->sp_D.data(), c->sp_tau1, {c->sp_g[0], c->sp_g[1], c->sp_g[2]}, 0u};
        s = create_common(&g32, &s32, c->stream, nullptr, nullptr, 0, &fcp.p);
        if (s != EVD_OK) return fail(c, s, std::string("FP32 forward context: ") + g_create_error);
        fcp.p->ref_mode = EVD_REF_NODE;
        fcp.p->mc_every = 0;
        s = evd_set_fields(fcp.p, x0, n0);
        if (s != EVD_OK) return fail(c, s, std::string("FP32 forward: ") + fcp.p->err);
    }
    evd_ctx* fc = fcp.p;
    void* dec = nullptr;   // a decoded state (FP32 forward)
    if (f32) CK(c, mem.alloc(bb, &dec));
    auto as_f64 = [&](const void* state) -> const double* {
        if (!f32) return (const double*)state;
        c->launches += 1;
        const cudaError_t e = evd::DecodeLaunch::f32n_to_f64(fc->hp, state, (double*)dec, c->stream);
        return e == cudaSuccess ? (const double*)dec : nullptr;
    };
    void *f0 = nullptr, *lam_f = nullptr, *lam_s = nullptr, *xd = nullptr, *nd = nullptr, *dldx = nullptr,
         *part = nullptr, *grad = nullptr;
    CK(c, mem.alloc(bb, &f0));
    CK(c, mem.alloc(bb, &lam_f));
    CK(c, mem.alloc(bb, &lam_s));
    CK(c, mem.alloc(c->ns * n * sizeof(double), &xd));
    if (n0) CK(c, mem.alloc(n * sizeof(double), &nd));
    CK(c, mem.alloc(c->ns * n * sizeof(double), &dldx));
    CK(c, mem.alloc((size_t)evd::AdjLaunch::nblocks(c->hp) * np * sizeof(double), &part));
    CK(c, mem.alloc(np * sizeof(double), &grad));
    std::vector<void*> cp(ncp, nullptr), seg(K, nullptr);
    const size_t sb = f32 ? fc->buf_bytes : bb;   // bytes of a stored state
    for (auto& q : cp) CK(c, mem.alloc(sb, &q));
    for (auto& q : seg) CK(c, mem.alloc(sb, &q));
    evd_ctx* fw = f32 ? fc : c;   // the context that runs the forward pass
    cudaStream_t st = c->stream;
    CK(c, cudaMemcpyAsync(xd, x0, c->ns * n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (n0) CK(c, cudaMemcpyAsync(nd, n0, n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(c, cudaMemsetAsync(grad, 0, np * sizeof(double), st));
    // forward: f_0 and the checkpoints, then N steps to the state the loss reads
    CK(c, cudaMemcpyAsync(f0, c->buf[c->cur ^ 1], bb, cudaMemcpyDeviceToDevice, st));
    CK(c, cudaMemcpyAsync(cp[0], fw->buf[fw->cur], sb, cudaMemcpyDeviceToDevice, st));
    for (long long t = 1; t <= N; ++t) {
        s = evd_step(fw, 1);
        if (s != EVD_OK) return f32 ? fail(c, s, std::string("FP32 forward: ") + fc->err) : s;
        if (t < N && t % K == 0) CK(c, cudaMemcpyAsync(cp[t / K], fw->buf[fw->cur], sb, cudaMemcpyDeviceToDevice, st));
    }
    // the loss: row averages of the mole fractions of f_N against the target
    std::vector<double> x(c->ns * n), g(c->ns * n, 0.0);
    s = readout_to_host(fw, x.data(), nullptr, nullptr, nullptr);
    if (s != EVD_OK) return f32 ? fail(c, s, std::string("FP32 forward: ") + fc->err) : s;
    double L = 0.0;
    for (int i = 0; i < c->ns; ++i)
        for (int y = 0; y < c->ny; ++y) {
            double m = 0.0;
            for (int xx = 0; xx < c->nx; ++xx) m += x[(size_t)i * n + (size_t)y * c->nx + xx];
            m /= c->nx;
            const double r = m - target[(size_t)i * c->ny + y];
            L += r * r;
            for (int xx = 0; xx < c->nx; ++xx) g[(size_t)i * n + (size_t)y * c->nx + xx] = 2.0 * r / c->nx;
        }
    *loss = L;
    CK(c, cudaMemcpyAsync(dldx, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    // reverse sweep: lambda_N, then lambda*_{N-1} = G^T lambda_N
    const HostParams& h = c->hp;
    c->launches += 2;
    const double* fN1 = as_f64(fw->buf[fw->cur ^ 1]);   // f*_{N-1}
    if (!fN1) return cuda_fail(c, cudaGetLastError(), "decode");
    CK(c, evd::AdjLaunch::readout(h, fN1, (const double*)dldx, (double*)lam_f, st));
    CK(c, evd::AdjLaunch::gather_t(h, (const double*)lam_f, (double*)lam_s, st));
    long long seg_id = -1;
    for (long long t = N - 1; t >= 1; --t) {
        // f*_{t-1}, recomputed from its checkpoint with the rest of its segment
        const long long j = (t - 1) / K;
        if (j != seg_id) {
            CK(c, cudaMemcpyAsync(seg[0], cp[j], sb, cudaMemcpyDeviceToDevice, st));
            const long long last = std::min(j * K + K - 1, N - 2);
            for (long long q = 1; q <= last - j * K; ++q) {
                // the forward's step to f*_{jK+q}, with its dither seed
                if (f32) fc->hp.seed = step_seed(j * K + q);
                CK(c, launch_step(fw, seg[q - 1], seg[q], 0, nullptr));
            }
            seg_id = j;
        }
        const double* fprev = as_f64(seg[(t - 1) - j * K]);
        if (!fprev) return cuda_fail(c, cudaGetLastError(), "decode");
        c->launches += 3;
        CK(c, evd::AdjLaunch::collide(h, fprev, false, (const double*)lam_s, (double*)lam_f, (double*)part,
                                      (double*)grad, c->adj_mode == EVD_ADJOINT_DUAL, st));
        CK(c, evd::AdjLaunch::gather_t(h, (const double*)lam_f, (double*)lam_s, st));
    }
    // t = 0: f*_0 = C(f_0), and f_0 itself depends on g
    c->launches += 4;
    CK(c, evd::AdjLaunch::collide(h, (const double*)f0, true, (const double*)lam_s, (double*)lam_f, (double*)part,
                                  (double*)grad, c->adj_mode == EVD_ADJOINT_DUAL, st));
    CK(c, evd::AdjLaunch::init_g(h, (const double*)xd, (const double*)nd, (const double*)lam_f, (double*)part,
                                 (double*)grad, st));
    std::vector<double> gr(np);
    CK(c, cudaMemcpyAsync(gr.data(), grad, np * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(c, cudaStreamSynchronize(st));
    s = evd_check(c);
    if (s != EVD_OK) return s;
    if (f32 && (s = evd_check(fc)) != EVD_OK) return fail(c, s, std::string("FP32 forward: ") + fc->err);
    if (dL_dD) {
        for (int q = 0; q < c->ns * c->ns; ++q) dL_dD[q] = 0.0;
        int m = 0;
        for (int i = 0; i < c->ns; ++i)
            for (int k = i + 1; k < c->ns; ++k, ++m) dL_dD[i * c->ns + k] = dL_dD[k * c->ns + i] = gr[m];
    }
    if (dL_dg) {
        dL_dg[0] = gr[np - 2];
        dL_dg[1] = gr[np - 1];
        dL_dg[2] = 0.0;
    }
    return EVD_OK;
}

evd_status evd_destroy(evd_ctx* c)
{
    if (!c) return EVD_OK;
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->own_bufs) {
        cudaFree(c->buf[0]);
        cudaFree(c->buf[1]);
    }
    if (c->small) cudaFree(c->small);
    if (c->staging) cudaFree(c->staging);
    if (c->lumps) cudaFree(c->lumps);
    if (c->kf) cudaFree(c->kf);
    if (c->rhof) cudaFree(c->rhof);
    delete c;
    return EVD_OK;
}

const char* evd_last_error(const evd_ctx* c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
