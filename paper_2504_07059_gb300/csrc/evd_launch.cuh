// evd_launch.cuh -- (lattice, species count) dispatch of the kernel templates
// for one storage type S and arithmetic type T: 1 to 3 species on both
// lattices, 4 to 6 on D2Q9.
#pragma once

#include "evd_device.cuh"

namespace evd {

#define EVD_DISPATCH(KERNEL, ...)                                                    \
    if (h.lattice != LAT) return cudaErrorInvalidValue;                              \
    switch (h.ns) {                                                                  \
        case 1: KERNEL<LAT, 1, S, T><<<grid, BLOCK, 0, st>>>(__VA_ARGS__); break;    \
        case 2: KERNEL<LAT, 2, S, T><<<grid, BLOCK, 0, st>>>(__VA_ARGS__); break;    \
        case 3: KERNEL<LAT, 3, S, T><<<grid, BLOCK, 0, st>>>(__VA_ARGS__); break;    \
        case 4: if constexpr (LAT == 0) {                                            \
                    KERNEL<LAT, 4, S, T><<<grid, BLOCK, 0, st>>>(__VA_ARGS__); break; \
                } return cudaErrorInvalidValue;                                      \
        case 5: if constexpr (LAT == 0) {                                            \
                    KERNEL<LAT, 5, S, T><<<grid, BLOCK, 0, st>>>(__VA_ARGS__); break; \
                } return cudaErrorInvalidValue;                                      \
        case 6: if constexpr (LAT == 0) {                                            \
                    KERNEL<LAT, 6, S, T><<<grid, BLOCK, 0, st>>>(__VA_ARGS__); break; \
                } return cudaErrorInvalidValue;                                      \
        default: return cudaErrorInvalidValue;                                       \
    }

template <int LAT, typename S, typename T>
cudaError_t dispatch_step(const HostParams& h, const void* fin, void* fout, double* mass_part,
                          unsigned* err, int flags, const double* corr, cudaStream_t st)
{
    const Params<T> p = to_params<T>(h);
    const int grid = grid_blocks(h, BLOCK);
    if (grid == 0) return cudaSuccess;
    EVD_DISPATCH(k_step, p, (const S*)fin, (S*)fout, mass_part, err, flags, corr)
    return cudaGetLastError();
}

template <int LAT, typename S, typename T>
cudaError_t dispatch_readout(const HostParams& h, const void* fin, int flags, double* x, double* rho,
                             double* u, double* ui, double* fpop, double* mass_part, unsigned* err,
                             const double* corr, cudaStream_t st)
{
    const Params<T> p = to_params<T>(h);
    const int grid = grid_blocks(h, BLOCK);
    if (grid == 0) return cudaSuccess;
    EVD_DISPATCH(k_readout, p, (const S*)fin, flags, x, rho, u, ui, fpop, mass_part, err, corr)
    return cudaGetLastError();
}

template <int LAT, typename S, typename T>
cudaError_t dispatch_init(const HostParams& h, const double* x, const double* n, const double* fsrc,
                          void* fprev, void* fcur, double* mass_part, unsigned* err, cudaStream_t st)
{
    const Params<T> p = to_params<T>(h);
    const int grid = grid_blocks(h, BLOCK);
    if (grid == 0) return cudaSuccess;
    EVD_DISPATCH(k_init, p, x, n, fsrc, (S*)fprev, (S*)fcur, mass_part, err)
    return cudaGetLastError();
}

#undef EVD_DISPATCH

}  // namespace evd

#define EVD_DEFINE_LAUNCHERS(PREC, LAT, S, T)                                                              \
    namespace evd {                                                                                   \
    template <>                                                                                       \
    cudaError_t Launch<PREC, LAT>::step(const HostParams& h, const void* fin, void* fout, double* mp,      \
                                   unsigned* err, int flags, const double* corr, cudaStream_t st)     \
    {                                                                                                 \
        return dispatch_step<LAT, S, T>(h, fin, fout, mp, err, flags, corr, st);                      \
    }                                                                                                 \
    template <>                                                                                       \
    cudaError_t Launch<PREC, LAT>::readout(const HostParams& h, const void* fin, int flags, double* x,     \
                                      double* rho, double* u, double* ui, double* fpop, double* mp,   \
                                      unsigned* err, const double* corr, cudaStream_t st)             \
    {                                                                                                 \
        return dispatch_readout<LAT, S, T>(h, fin, flags, x, rho, u, ui, fpop, mp, err, corr, st);    \
    }                                                                                                 \
    template <>                                                                                       \
    cudaError_t Launch<PREC, LAT>::init(const HostParams& h, const double* x, const double* n,             \
                                   const double* fsrc, void* fprev, void* fcur, double* mp,           \
                                   unsigned* err, cudaStream_t st)                                    \
    {                                                                                                 \
        return dispatch_init<LAT, S, T>(h, x, n, fsrc, fprev, fcur, mp, err, st);                          \
    }                                                                                                 \
    }

#define EVD_DEFINE_TMA_LAUNCHER(PREC, S)                                                              \
    namespace evd {                                                                                   \
    template <>                                                                                       \
    cudaError_t launch_step_tma<PREC>(const HostParams& h, int ty, const void* maps, const void* fin, \
                                      void* fout, double* mp, unsigned* err, int flags,               \
                                      const double* corr, const float* lumps, cudaStream_t st)        \
    {                                                                                                 \
        return dispatch_step_tma<S>(h, ty, maps, fin, fout, mp, err, flags, corr, lumps, st);         \
    }                                                                                                 \
    }

#define EVD_DEFINE_CORR_LAUNCHERS(PREC, S, T)                                                         \
    namespace evd {                                                                                   \
    template <>                                                                                       \
    cudaError_t CorrLaunch<PREC>::density(const HostParams& h, const void* fin, const double* corr,   \
                                          cudaStream_t st)                                            \
    {                                                                                                 \
        constexpr int LAT = 0;                                                                        \
        using St = S;                                                                                 \
        using Tt = T;                                                                                 \
        const Params<T> p = to_params<T>(h);                                                          \
        const int grid = grid_blocks(h, BLOCK);                                                       \
        if (grid == 0) return cudaSuccess;                                                            \
        EVD_CORR_DISPATCH(k_density, p, (const S*)fin, (T*)h.rhof, corr)                              \
        return cudaGetLastError();                                                                    \
    }                                                                                                 \
    template <>                                                                                       \
    cudaError_t CorrLaunch<PREC>::step(const HostParams& h, const void* fin, void* fout, double* mp,  \
                                       unsigned* err, int flags, const double* corr, cudaStream_t st) \
    {                                                                                                 \
        constexpr int LAT = 0;                                                                        \
        using St = S;                                                                                 \
        using Tt = T;                                                                                 \
        const Params<T> p = to_params<T>(h);                                                          \
        const int grid = grid_blocks(h, BLOCK);                                                       \
        if (grid == 0) return cudaSuccess;                                                            \
        EVD_CORR_DISPATCH(k_step_corr, p, (const S*)fin, (S*)fout, mp, err, flags, corr)               \
        return cudaGetLastError();                                                                    \
    }                                                                                                 \
    }

#define EVD_CORR_DISPATCH(KERNEL, ...)                                                                \
    switch (h.ns) {                                                                                   \
        case 1: KERNEL<LAT, 1, St, Tt><<<grid, BLOCK, 0, st>>>(__VA_ARGS__); break;                   \
        case 2: KERNEL<LAT, 2, St, Tt><<<grid, BLOCK, 0, st>>>(__VA_ARGS__); break;                   \
        case 3: KERNEL<LAT, 3, St, Tt><<<grid, BLOCK, 0, st>>>(__VA_ARGS__); break;                   \
        default: return cudaErrorInvalidValue;                                                        \
    }
