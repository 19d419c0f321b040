// evd_tma_launch.cuh -- species-count dispatch and launch of the TMA step.
#pragma once

#include "evd_launch.cuh"
#include "evd_tma.cuh"

namespace evd {

template <int NS, typename S, int TY>
cudaError_t launch_tma_ns(const HostParams& h, const TmaMaps& maps, const void* fin, void* fout, double* mp,
                          unsigned* err, int flags, const double* corr, const float* lumps, cudaStream_t st)
{
    // ring slots: as many as leave room, next to the exchange and the wall
    // terms, for the CTAs per SM the tile height targets (four of one row,
    // two of two rows, one of four)
    constexpr int SLOTS = sizeof(S) == 4 ? (TY == 1 ? 2 : 3) : (TY == 1 ? 3 : TmaLaunch::SLOTS);
    using L = TmaLayout<NS, S, TY, SLOTS>;
    auto kern = k_step_tma<NS, S, TY, SLOTS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::total_bytes);
    if (e != cudaSuccess) return e;
    const Params<float> p = to_params<float>(h);
    const int ntx = (h.nx + TTX - 1) / TTX, nty = (h.ny + TY - 1) / TY;
    const dim3 block(L::threads);
    const int grid = TmaLaunch::grid(h, TY);
    kern<<<grid, block, L::total_bytes, st>>>(maps, p, (const S*)fin, (S*)fout, mp, err, flags, corr,
                                              (const float4*)lumps, ntx, nty, TmaLaunch::zchunk(h), h.wait_polls);
    return cudaGetLastError();
}

template <typename S>
cudaError_t dispatch_step_tma(const HostParams& h, int ty, const void* maps, const void* fin, void* fout,
                              double* mp, unsigned* err, int flags, const double* corr, const float* lumps,
                              cudaStream_t st)
{
    if (h.lattice != 1 || !h.wall[0] || !h.wall[1]) return cudaErrorInvalidValue;
    const TmaMaps& m = *reinterpret_cast<const TmaMaps*>(maps);
    switch (h.ns * 8 + ty) {
        case 1 * 8 + 1: return launch_tma_ns<1, S, 1>(h, m, fin, fout, mp, err, flags, corr, lumps, st);
        case 2 * 8 + 1: return launch_tma_ns<2, S, 1>(h, m, fin, fout, mp, err, flags, corr, lumps, st);
        case 3 * 8 + 1: return launch_tma_ns<3, S, 1>(h, m, fin, fout, mp, err, flags, corr, lumps, st);
        case 1 * 8 + 2: return launch_tma_ns<1, S, 2>(h, m, fin, fout, mp, err, flags, corr, lumps, st);
        case 2 * 8 + 2: return launch_tma_ns<2, S, 2>(h, m, fin, fout, mp, err, flags, corr, lumps, st);
        case 3 * 8 + 2: return launch_tma_ns<3, S, 2>(h, m, fin, fout, mp, err, flags, corr, lumps, st);
        case 1 * 8 + 4: return launch_tma_ns<1, S, 4>(h, m, fin, fout, mp, err, flags, corr, lumps, st);
        case 2 * 8 + 4: return launch_tma_ns<2, S, 4>(h, m, fin, fout, mp, err, flags, corr, lumps, st);
        case 3 * 8 + 4: return launch_tma_ns<3, S, 4>(h, m, fin, fout, mp, err, flags, corr, lumps, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace evd
