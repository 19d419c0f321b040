// Batched step kernels, fp64 storage, D3Q19.
#include "evd_batch_kernels.cuh"
EVD_DEFINE_BATCH_LAUNCHERS(0, 1, double, double)
