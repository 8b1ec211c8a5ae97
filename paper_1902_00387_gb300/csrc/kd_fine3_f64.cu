// Instantiations of the n = 512, 1024 fine kernels (kd_fine3.cuh): double, n = 512 1024.
#include "kd_fine_sets.cuh"

KD_FINE3_INSTANTIATE(double, 512)
KD_FINE3_INSTANTIATE(double, 1024)
