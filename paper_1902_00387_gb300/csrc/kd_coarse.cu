// Classical coarse propagator G (Sec. 3.2, Sec. 5.2: the same equations on the coarse
// N_C grid with the coarse step) as one persistent thread-block cluster per field for
// coarse sets of side <= 88 (coarse grids up to 128) with portable clusters, and up to
// 127 (grids up to 190) with 16-block clusters,
// fused with the Fourier restriction of the fine input and, in the Parareal sweep,
// with the FP64 update U_{n+1} = F + (G_new - G_old) and the defect of Eq. 9.
//
// The explicit term is evaluated as the exact spectral convolution
//     w_hat(k) = sum_q u_hat(q, t) x b_hat(k - q),   q in {(+-1, 0), (0, +-1)},
// followed by the curl i k3 x w_hat on the dealiased set (two complex products per
// neighbour: the flows' modes satisfy u_y = -+ i u_z at q = +-x, u_z = -+ i u_x at q = +-y).  The flow has only those
// four Fourier modes and n/3 + 1 < n/2, so the pseudo-spectral product of the fine
// kernels has no aliasing and this is the same discrete operator (equal to round-off).
//
// Layout: the stage values live in shared memory with a one-mode ring of zeros around
// the kept square; the IMEX RK443 state X0 and accumulators R2..R4 of each mode live in
// the registers of the thread that owns the mode.
#include "kd_coarse_kernel.cuh"

namespace kd {

// cluster split of a P-row coarse square: CS blocks of H rows (H <= 8 for P <= 64,
// H <= 11 for P <= 88; 16 blocks of H <= 8 rows for P <= 127)
// clusters of more than 8 blocks need the non-portable size opt-in (granted in prepare)
static int g_max_cluster = 8;

static void cluster_shape(int P, int* CS, int* H, int req = 0) {
  int cs = req > 0 ? req : (P + 5) / 6;
  if (cs > g_max_cluster) cs = g_max_cluster;
  if (req == 0 && cs > 8) cs = 8;
  if (cs < 1) cs = 1;
  *H = (P + cs - 1) / cs;
  *CS = cs;
}

constexpr int kMaxPhaseSlots = 8192;   // staged flow phases (512 steps x 4 stages x 4)

static size_t cluster_smem(int prec, int P, int nsteps, int* phase_slots, int req = 0) {
  const int L = P + 2;
  int CS, H;
  cluster_shape(P, &CS, &H, req);
  const size_t es = prec == 0 ? 4 : 8;
  const size_t base = (size_t)2 * 3 * (H + 2) * L * 2 * es;
  const int slots = nsteps * 16 <= kMaxPhaseSlots ? nsteps * 16 : 0;
  *phase_slots = slots;
  return base + (size_t)slots * es;
}

// modes per thread needed for a P-row square (0: unsupported)
// modes per thread of a block (1: CCB1 threads; 2, 4: CCB threads); 0 if the rows of a
// block do not fit
static int modes_per_thread(int P, int req = 0) {
  int CS, H;
  cluster_shape(P, &CS, &H, req);
  if (H * P <= CCB) return 2;
  if (H * P <= CCB1) return 1;
  if (H * P <= 2 * CCB) return 2;
  if (H * P <= 4 * CCB) return 4;
  return 0;
}

bool coarse_cluster_fits(int P, int cs) {
  return P >= 1 && cs >= 0 && cs <= g_max_cluster && (cs == 0 || cs <= P) && modes_per_thread(P, cs) > 0;
}

// smallest cluster larger than the default that holds a P-row square (0: none)
static int min_fitting_cluster(int P) {
  for (int cs = 9; cs <= g_max_cluster; ++cs)
    if (coarse_cluster_fits(P, cs)) return cs;
  return 0;
}

// the default shape, or (squares above 88 rows) the smallest larger cluster that holds them
bool coarse_conv_supported(int P) { return P >= 1 && (modes_per_thread(P) > 0 || min_fitting_cluster(P) > 0); }

template <typename T>
static cudaError_t prepare_T() {
  const int prec = sizeof(T) == 4 ? 0 : 1;
  // 16-block clusters where the device grants them (every variant)
  if (cluster_allow_nonportable<T, 0>() == cudaSuccess && coarse_alt_allow_nonportable(prec) == cudaSuccess)
    g_max_cluster = 16;
  cudaGetLastError();
  int slots = 0;
  int bytes = 0;   // the largest shared-memory need over every supported square and cluster size
  for (int P = 1; P <= 128; ++P)
    for (int cs = 0; cs <= g_max_cluster; ++cs)
      if (coarse_cluster_fits(P, cs)) {
        const int b = (int)cluster_smem(prec, P, 512, &slots, cs);
        if (b > bytes) bytes = b;
      }
  const cudaError_t e = cluster_set_smem<T, 0>(bytes);
  return e != cudaSuccess ? e : coarse_alt_set_smem(prec, bytes);
}

cudaError_t coarse_prepare(int prec) { return prec == 0 ? prepare_T<float>() : prepare_T<double>(); }

static int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 132;
  }
  return sms;
}

// Default cluster size: the per-stage time is a fixed barrier / latency part plus a part
// proportional to the rows of a block, so a few fields take the largest clusters that all
// fit on the GPU at once (~3 rows per block, up to 16 blocks); larger batches keep ~6 rows
// per block (at most 8) so that more clusters run concurrently.
static int auto_cluster(int P, int batch) {
  if (g_max_cluster >= 16 && batch * 16 <= sm_count()) {
    const int cs = (P + 2) / 3 < 16 ? (P + 2) / 3 : 16;
    if (cs > 8 && coarse_cluster_fits(P, cs)) return cs;
  }
  return modes_per_thread(P) > 0 ? 0 : min_fitting_cluster(P);
}

template <typename T>
static int launch_cluster(const CoarseArgs& a0, int batch, cudaStream_t st) {
  CoarseArgs a = a0;
  const int req = a.cluster > 0 && coarse_cluster_fits(a.Pc, a.cluster) ? a.cluster : auto_cluster(a.Pc, batch);
  int CS, H, slots;
  cluster_shape(a.Pc, &CS, &H, req);
  const size_t sm = cluster_smem(sizeof(T) == 4 ? 0 : 1, a.Pc, a.nsteps, &slots, req);
  a.phase_smem = slots;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(CS * batch), 1, 1);
  const int mpt = modes_per_thread(a.Pc, req);
  cfg.blockDim = dim3(mpt == 1 ? CCB1 : CCB, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = a.halo == 0 ? cluster_launch<T, 0>(cfg, mpt, a, CS, H)
                                    : coarse_alt_launch(sizeof(T) == 4 ? 0 : 1, cfg, mpt, a, CS, H);
  return e == cudaSuccess ? 1 : -1;
}

int coarse_conv_launch(int prec, const CoarseArgs& a, int batch, cudaStream_t st) {
  if (!coarse_conv_supported(a.Pc) || batch <= 0) return -1;
  return prec == 0 ? launch_cluster<float>(a, batch, st) : launch_cluster<double>(a, batch, st);
}

}  // namespace kd
