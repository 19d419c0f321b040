// Double storage, double arithmetic (the parity path), D2Q9.
#include "evd_launch.cuh"
EVD_DEFINE_LAUNCHERS(0, 0, double, double)
EVD_DEFINE_CORR_LAUNCHERS(0, double, double)
