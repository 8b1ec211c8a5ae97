// Instantiations of the n <= 256 fine kernels (kd_fine2.cuh): float, n = 16 32 64.
#include "kd_fine_sets.cuh"

KD_FINE2_INSTANTIATE(float, 16)
KD_FINE2_INSTANTIATE(float, 32)
KD_FINE2_INSTANTIATE(float, 64)
