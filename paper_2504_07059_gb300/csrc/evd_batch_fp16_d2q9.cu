// Batched step kernels, fp16 storage, D2Q9.
#include "evd_batch_kernels.cuh"
EVD_DEFINE_BATCH_LAUNCHERS(2, 0, __half, float)
