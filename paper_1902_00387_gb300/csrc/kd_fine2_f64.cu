// Instantiations of the n <= 256 fine kernels (kd_fine2.cuh): double, n = 16 32 64 128 256.
#include "kd_fine_sets.cuh"

KD_FINE2_INSTANTIATE(double, 16)
KD_FINE2_INSTANTIATE(double, 32)
KD_FINE2_INSTANTIATE(double, 64)
KD_FINE2_INSTANTIATE(double, 128)
KD_FINE2_INSTANTIATE(double, 256)
