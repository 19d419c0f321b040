// Double storage, double arithmetic (the parity path), D3Q19.
#include "evd_launch.cuh"
EVD_DEFINE_LAUNCHERS(0, 1, double, double)
