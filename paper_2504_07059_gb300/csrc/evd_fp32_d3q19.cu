// Float storage of f - w_a rho_ref_i, float arithmetic, D3Q19.
#include "evd_tma_launch.cuh"
EVD_DEFINE_LAUNCHERS(1, 1, float, float)
EVD_DEFINE_TMA_LAUNCHER(1, float)
