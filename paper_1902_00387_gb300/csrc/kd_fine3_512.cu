// Instantiations of the n = 512, 1024 fine kernels (kd_fine3.cuh): float, n = 512.
#include "kd_fine3.cuh"

KD_FINE3_INSTANTIATE(float, 512)
