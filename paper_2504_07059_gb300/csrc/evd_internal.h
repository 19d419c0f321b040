// evd_internal.h -- host-side parameter block and kernel launchers shared by
// the C ABI (evd_api.cu) and the per-precision kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>

namespace evd {

// Sets the message evd_last_error(NULL) returns on this thread.
void set_thread_error(const std::string& msg);

constexpr int MAXS = 3;

// Per-run constants in double; each precision casts them to its own type.
struct HostParams {
    int lattice, ns, precision;
    int nx, ny, nz, nsites;
    long long pstride;       // elements between consecutive (species, direction) planes
    int wall[3];
    int unit[MAXS];
    double c[MAXS], inv_cs2[MAXS], c_inv_cs2[MAXS];
    double tau_inv[MAXS], omt[MAXS], sfac[MAXS];
    double Minv[MAXS], M[MAXS];
    double MM[MAXS][MAXS], iD[MAXS][MAXS];
    double g[3];
    double w1[MAXS][3], w2[MAXS][3][3];
    double wl[3];
    double ref[MAXS][3];
};

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

inline int grid_blocks(const HostParams& h, int block) { return (h.nsites + block - 1) / block; }

}  // namespace evd
