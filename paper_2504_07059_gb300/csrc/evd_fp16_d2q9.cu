// Half storage of f - w_a rho_ref_i, float arithmetic, D2Q9.
#include "evd_launch.cuh"
EVD_DEFINE_LAUNCHERS(2, 0, __half, float)
EVD_DEFINE_CORR_LAUNCHERS(2, __half, float)
