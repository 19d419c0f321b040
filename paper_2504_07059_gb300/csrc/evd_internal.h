// evd_internal.h -- host-side parameter block and kernel launchers shared by
// the C ABI (evd_api.cu) and the per-precision kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <string>

#include "evd.h"

namespace evd {

// Sets the message evd_last_error(NULL) returns on this thread.
void set_thread_error(const std::string& msg);
const char* thread_error();

constexpr int MAXS = 6;        // species of the general kernel (D2Q9)
constexpr int MAXS_FAST = 3;   // species of the TMA step, the batch, D3Q19, the
                               // corrective terms and the adjoint

// Molar masses passed by value to the field kernels.
struct MassTable {
    double M[MAXS];
};

// Per-run constants in double; each precision casts them to its own type.
struct HostParams {
    int lattice, ns, precision;
    int nx, ny, nz, nsites;
    long long pstride;       // elements between consecutive (species, direction) planes
    int wall[3];
    int unit[MAXS];
    double c[MAXS], inv_cs2[MAXS], c_inv_cs2[MAXS];
    double c_inv_cs2_lo[MAXS];   // float arithmetic: c_inv_cs2 + c_inv_cs2_lo = 1 / (c m2) (0 in FP64)
    double tau_inv[MAXS], omt[MAXS], sfac[MAXS];
    double Minv[MAXS], M[MAXS];
    double MM[MAXS][MAXS], iD[MAXS][MAXS];
    double g[3];
    double w1[MAXS][3], w2[MAXS][3][3];
    double wl[3];
    double ref[MAXS][3];
    const void* kf;          // device [3][nsites] force field in the arithmetic type, or nullptr
    unsigned flags;          // corrective forcing terms (EVD_FORCE_S_DIFF / _S_P / _S_RHO)
    const void* rhof;        // device [ns + 1][nsites] densities of f_t for the gradient terms
    int wait_polls;          // polls of a TMA-step wait for a tile copy before it gives up
    unsigned seed;           // per-step seed of the dithered rounding (0: off)
};

// Default of HostParams::wait_polls: far longer than any tile copy takes.
constexpr int kWaitPolls = 1 << 22;

// Host-side checks and constants shared by the single-lattice context and the
// batch of lattices (evd_api.cu).
size_t elem_size(int precision);
bool validate(const evd_grid* g, const evd_species* s, std::string& msg);
long long plane_stride(const evd_grid* g);
int buffer_planes(int lattice, int precision, int ns);
size_t buffer_bytes(const evd_grid* g, const evd_species* s);
void fill_params(HostParams& h, const evd_grid* g, const evd_species* s);

// Kernel launchers, one explicit specialisation per storage precision
// (0 double, 1 float deviation, 2 half deviation) and lattice (0 D2Q9,
// 1 D3Q19), each in its own translation unit.
template <int PREC, int LAT>
struct Launch {
    static cudaError_t step(const HostParams& h, const void* fin, void* fout, double* mass_part,
                            unsigned* err, int flags, const double* corr, cudaStream_t st);
    static cudaError_t readout(const HostParams& h, const void* fin, int flags, double* x, double* rho,
                               double* u, double* ui, double* fpop, double* mass_part, unsigned* err,
                               const double* corr, cudaStream_t st);
    static cudaError_t init(const HostParams& h, const double* x, const double* n, const double* fsrc,
                            void* fprev, void* fcur, double* mass_part, unsigned* err, cudaStream_t st);
};

// Batched step: work items are ranges of consecutive sites of one member.
struct BatchItem {
    int member, node0, count, ns;
};

// Where member m lives: element offset of its populations in a population
// buffer, and offsets of its fields in the concatenated readout arrays.
struct MemberInfo {
    long long foff;    // populations (elements)
    long long xoff;    // x, rho: [ns][sites]
    long long soff;    // n: [sites]
    long long uoff;    // u: [D][sites]
    long long uioff;   // ui: [ns][D][sites]
    int sites, ns, item_begin, item_end;
    double M[MAXS];    // molar masses (FP64, for the initial-mass reduction)
};

struct BatchArgs {
    const BatchItem* items;
    int n_items;
    const void* params;      // Params<T>[members] on the device
    const MemberInfo* info;  // [members] on the device
    int grid;                // CTAs of the step launch (persistent when < n_items)
    unsigned* seed;          // {step counter, CTAs done}: seeds the dithered rounding, or nullptr
};

template <int PREC, int LAT>
struct BatchLaunch {
    static cudaError_t step(const BatchArgs& a, const void* fin, void* fout, double* part, unsigned* err,
                            int flags, const double* corr, cudaStream_t st);
    static cudaError_t readout(const BatchArgs& a, const void* fin, int flags, double* x, double* rho,
                               double* u, double* ui, double* part, unsigned* err, const double* corr,
                               cudaStream_t st);
    static cudaError_t init(const BatchArgs& a, const double* x, const double* n, void* fprev, void* fcur,
                            double* part, unsigned* err, cudaStream_t st);
};

// The D2Q9 step with the corrective forcing terms: a density pre-pass into
// h.rhof, then the step with the gradient terms (only D2Q9 translation units
// define these).
template <int PREC>
struct CorrLaunch {
    static cudaError_t density(const HostParams& h, const void* fin, const double* corr, cudaStream_t st);
    static cudaError_t step(const HostParams& h, const void* fin, void* fout, double* mass_part, unsigned* err,
                            int flags, const double* corr, cudaStream_t st);
};

// Kernels of the discrete adjoint (D2Q9, FP64): lambda_t = C^T lambda*_t with
// the parameter gradient accumulated into grad[nparams] (D_ij for i < j, then
// g_x, g_y); lambda*_{t-1} = G^T lambda_t; the readout and initial-state
// terms.  part: scratch of nblocks * nparams doubles.
struct AdjLaunch {
    static int nparams(int ns);
    static int nblocks(const HostParams& h);
    static cudaError_t collide(const HostParams& h, const double* fin, bool raw, const double* lam_star,
                               double* lam_f, double* part, double* grad, bool dual, cudaStream_t st);
    static cudaError_t gather_t(const HostParams& h, const double* lam_f, double* lam_star, cudaStream_t st);
    static cudaError_t readout(const HostParams& h, const double* fin, const double* dldx, double* lam_f,
                               cudaStream_t st);
    static cudaError_t init_g(const HostParams& h, const double* x0, const double* n0, const double* lam0,
                              double* part, double* grad, cudaStream_t st);
};

// Post-collision populations of a float node-reference buffer (D2Q9) as
// doubles in the double-precision plane layout (same plane stride): f_a =
// w_a rho + g_a, the rest f_0 = w_0 rho - sum of the others' g (the adjoint's
// FP32-forward mode reads its states this way).  h: the float context's
// constants.
struct DecodeLaunch {
    static cudaError_t f32n_to_f64(const HostParams& h, const void* fin, double* fout, cudaStream_t st);
};

inline int grid_blocks(const HostParams& h, int block) { return (h.nsites + block - 1) / block; }

// The D3Q19 step with TMA-staged tiles (float and half storage only).
// maps points to the seven tensor maps (CUtensorMap, 128 bytes each) of the
// input buffer, one per storage group of directions.
struct TmaLaunch {
    static constexpr int TX = 32, SLOTS = 4, NGROUPS = 8;   // at most 8 tensor maps per buffer
    // rows per tile: 4 (one CTA per SM) or 2 (two CTAs per SM)
    static int zchunk(const HostParams& h) { return h.nz < 32 ? h.nz : 32; }
    static int grid(const HostParams& h, int ty)
    {
        const int ntx = (h.nx + TX - 1) / TX, nty = (h.ny + ty - 1) / ty, zc = zchunk(h);
        return ntx * nty * ((h.nz + zc - 1) / zc);
    }
    // mass partials of a step at tile height ty
    static int parts(const HostParams& h, int ty) { return grid(h, ty); }
};

// lumps: App. A coefficients [27 wall classes][ns][19] x (L_self, L_opp,
// K - 1, 0) as float4; wall class = cx + 3 cy + 9 cz with c = 0 interior, 1 at the
// low wall, 2 at the high wall of that dimension.
template <int PREC>
cudaError_t launch_step_tma(const HostParams& h, int ty, const void* maps, const void* fin, void* fout,
                            double* mass_part, unsigned* err, int flags, const double* corr,
                            const float* lumps, cudaStream_t st);

}  // namespace evd
