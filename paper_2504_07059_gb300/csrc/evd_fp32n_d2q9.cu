// Float storage of deviations from each node's own density (kept in the rest
// plane), float arithmetic, D2Q9.
#include "evd_launch.cuh"
EVD_DEFINE_LAUNCHERS(3, 0, f32n, float)
EVD_DEFINE_CORR_LAUNCHERS(3, f32n, float)

namespace evd {
cudaError_t DecodeLaunch::f32n_to_f64(const HostParams& h, const void* fin, double* fout, cudaStream_t st)
{
    const Params<float> p = to_params<float>(h);
    const int grid = grid_blocks(h, BLOCK);
    if (grid == 0) return cudaSuccess;
    switch (h.ns) {
        case 1: k_decode_f32n<0, 1><<<grid, BLOCK, 0, st>>>(p, (const f32n*)fin, fout); break;
        case 2: k_decode_f32n<0, 2><<<grid, BLOCK, 0, st>>>(p, (const f32n*)fin, fout); break;
        case 3: k_decode_f32n<0, 3><<<grid, BLOCK, 0, st>>>(p, (const f32n*)fin, fout); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
}  // namespace evd
