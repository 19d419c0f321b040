// Batched step kernels, fp64 storage, D2Q9.
#include "evd_batch_kernels.cuh"
EVD_DEFINE_BATCH_LAUNCHERS(0, 0, double, double)
