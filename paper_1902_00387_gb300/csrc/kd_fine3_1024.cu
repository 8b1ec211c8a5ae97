// Instantiations of the n = 512, 1024 fine kernels (kd_fine3.cuh): float, n = 1024.
#include "kd_fine_sets.cuh"

KD_FINE3_INSTANTIATE(float, 1024)
