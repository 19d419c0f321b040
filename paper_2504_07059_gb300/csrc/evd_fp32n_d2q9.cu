// Float storage of deviations from each node's own density (kept in the rest
// plane), float arithmetic, D2Q9.
#include "evd_launch.cuh"
EVD_DEFINE_LAUNCHERS(3, 0, f32n, float)
EVD_DEFINE_CORR_LAUNCHERS(3, f32n, float)
