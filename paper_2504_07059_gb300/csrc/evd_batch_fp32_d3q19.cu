// Batched step kernels, fp32 storage (deviations from each node's density), D3Q19.
#include "evd_batch_kernels.cuh"
EVD_DEFINE_BATCH_LAUNCHERS(1, 1, f32n, float)
