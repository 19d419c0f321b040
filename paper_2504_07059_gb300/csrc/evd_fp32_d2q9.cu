// Float storage of f - w_a rho_ref_i, float arithmetic, D2Q9.
#include "evd_launch.cuh"
EVD_DEFINE_LAUNCHERS(1, 0, float, float)
EVD_DEFINE_CORR_LAUNCHERS(1, float, float)
