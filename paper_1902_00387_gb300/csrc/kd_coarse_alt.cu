// The alternative halo exchanges of the coarse-solver cluster kernel (CoarseArgs::halo
// = 1: point-to-point st.async + mbarrier; 2: pull after a split cluster barrier), in
// their own translation unit so that the library's units compile in parallel.
#include "kd_coarse.h"
#include "kd_coarse_kernel.cuh"

namespace kd {

cudaError_t coarse_alt_allow_nonportable(int prec) {
  cudaError_t e = prec == 0 ? cluster_allow_nonportable<float, 1>() : cluster_allow_nonportable<double, 1>();
  if (e == cudaSuccess) e = prec == 0 ? cluster_allow_nonportable<float, 2>() : cluster_allow_nonportable<double, 2>();
  return e;
}

cudaError_t coarse_alt_set_smem(int prec, int bytes) {
  cudaError_t e = prec == 0 ? cluster_set_smem<float, 1>(bytes) : cluster_set_smem<double, 1>(bytes);
  if (e == cudaSuccess) e = prec == 0 ? cluster_set_smem<float, 2>(bytes) : cluster_set_smem<double, 2>(bytes);
  return e;
}

cudaError_t coarse_alt_launch(int prec, const cudaLaunchConfig_t& cfg, int mpt, const CoarseArgs& a, int CS, int H) {
  if (a.halo == 1)
    return prec == 0 ? cluster_launch<float, 1>(cfg, mpt, a, CS, H) : cluster_launch<double, 1>(cfg, mpt, a, CS, H);
  return prec == 0 ? cluster_launch<float, 2>(cfg, mpt, a, CS, H) : cluster_launch<double, 2>(cfg, mpt, a, CS, H);
}

}  // namespace kd
