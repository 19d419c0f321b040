// Batched step kernels, fp16 storage, D3Q19.
#include "evd_batch_kernels.cuh"
EVD_DEFINE_BATCH_LAUNCHERS(2, 1, __half, float)
