// Float storage of deviations from each node's own density (kept in the rest
// plane), float arithmetic, D3Q19.
#include "evd_launch.cuh"
EVD_DEFINE_LAUNCHERS(3, 1, f32n, float)
