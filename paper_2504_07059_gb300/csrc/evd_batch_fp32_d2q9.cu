// Batched step kernels, fp32 storage (deviations from each node's density), D2Q9.
#include "evd_batch_kernels.cuh"
EVD_DEFINE_BATCH_LAUNCHERS(1, 0, f32n, float)
