// Instantiations of the n <= 256 fine kernels (kd_fine2.cuh): float, n = 128.
#include "kd_fine_sets.cuh"

KD_FINE2_INSTANTIATE(float, 128)
