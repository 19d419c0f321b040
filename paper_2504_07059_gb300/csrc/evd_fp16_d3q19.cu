// Half storage of f - w_a rho~_i(x) (node densities), float arithmetic, D3Q19.
#include "evd_tma_launch.cuh"
EVD_DEFINE_LAUNCHERS(2, 1, __half, float)
EVD_DEFINE_TMA_LAUNCHER(2, __half)
