// Half storage of f - w_a rho~_i(x) (node densities), float arithmetic, D2Q9.
#include "evd_launch.cuh"
EVD_DEFINE_LAUNCHERS(2, 0, __half, float)
EVD_DEFINE_CORR_LAUNCHERS(2, __half, float)
