/*
 * kd.h -- C ABI of the GB300 Parareal library for the 2.5D kinematic dynamo.
 *
 * The library integrates the monochromatic induction equation (Sec. 2, Eq. 1 with
 * B = b(x, y, t) exp(i kz z)):
 *
 *     d b / dt = nabla_k x (u x b) + Rm^-1 (nabla^2 - kz^2) b,   nabla_k = (d_x, d_y, i kz),
 *
 * on the periodic square [0, 2 pi)^2 for the Roberts flow (Sec. 2.1) or the
 * Galloway-Proctor circularly polarised flow (Sec. 2.2), with a Fourier
 * pseudo-spectral discretisation (2/3 dealiasing) and the IMEX Runge-Kutta scheme
 * RK443 (Sec. 4), and runs Parareal (Sec. 3, Eq. 8) on one GPU.
 *
 * Conventions shared by every call:
 *  - A field is complex [3][n][n] = [component x,y,z][ky][kx] of spectral
 *    coefficients b_hat(k) with b(x) = sum_k b_hat(k) exp(i k.x); indices are in FFT
 *    order (index i <-> wavenumber i for i < n/2, i - n otherwise).  Complex numbers
 *    are interleaved (re, im) doubles (complex128) or floats (complex64).
 *  - Modes outside the dealiased square |kx|, |ky| <= n/3 are ignored on input and
 *    written as zero on output.
 *  - The caller owns every buffer it passes; the library never frees them.  The
 *    context owns its workspace, tables and CUDA graphs.
 *  - Work is enqueued on the stream given to kd_create (NULL = legacy default
 *    stream).  Calls documented as synchronous wait for that stream.
 *  - Errors are return codes; kd_last_error() gives a message.  CUDA failures map
 *    to KD_ECUDA.  A context is not thread-safe.
 */
#ifndef KD_H_
#define KD_H_

#include <stddef.h> /* size_t */

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kd_ctx kd_ctx;

typedef enum {
  KD_OK = 0,
  KD_EINVAL = 1,        /* bad argument */
  KD_ENOMEM = 2,        /* device allocation failed */
  KD_ECUDA = 3,         /* CUDA runtime error */
  KD_ENOTCONV = 4,      /* Parareal reached k_max with sigma > tol (results still written) */
  KD_ETIMEOUT = 5,      /* a bounded device-side wait ran out */
  KD_ENONFINITE = 6,    /* NaN or Inf met in a norm */
  KD_EUNSUPPORTED = 7   /* valid request the library does not implement */
} kd_status;

enum { KD_FLOW_ROBERTS = 0, KD_FLOW_GALLOWAY_PROCTOR = 1, KD_FLOW_NONE = 2 };
enum { KD_C64 = 0, KD_C128 = 1 };
enum { KD_COARSE_CLASSICAL = 0, KD_COARSE_LEARNED = 1 };
/* How kd_parareal_run evaluates the fine values F(U^k_n) of its parallel step:
 * DIRECT propagates U^k_n itself (a complex64 fine propagator then leaves round-off
 * noise of ~1e-7 per slice in every iterate, which floors the defect sigma near
 * sqrt(n_slices) x 1e-7); INCREMENT uses the linearity of F in b,
 * F(U^k) = F(U^{k-1}) + F(U^k - U^{k-1}), propagating only the FP64 increment in the
 * fine precision and accumulating in FP64, so sigma keeps falling below that floor.
 * Both are the same iteration in exact arithmetic; DIRECT keeps the bitwise
 * finite-termination property (after k iterations slices 0..k equal kd_fine_serial). */
enum { KD_FINE_DIRECT = 0, KD_FINE_INCREMENT = 1 };
/* Evaluation of the explicit term by the fine propagator.  The flow has Fourier modes
 * |q| = 1 only, so with the 2/3 rule the pseudo-spectral product u x b has no aliasing
 * and equals the spectral convolution sum_q u_hat(q) x b_hat(k - q) exactly; the two
 * operators differ by round-off. */
enum { KD_FINE_FFT = 0, KD_FINE_CONV = 1 };
/* IMEX Runge-Kutta scheme of the fine step (Sec. 4, Sec. 5.1): Ascher-Ruuth-Spiteri
 * (4,4,3), (2,2,2) or (1,1,1); the coarse propagator always steps with RK443. */
enum { KD_RK443 = 0, KD_RK222 = 1, KD_RK111 = 2 };

#define KD_MAX_SLICES 1024
#define KD_MAX_ITERS 256

/* Problem and discretisation parameters (Sec. 2, Sec. 4, Table 1). */
typedef struct {
  int flow;            /* KD_FLOW_*; NONE (u = 0) leaves pure diffusion */
  int n;               /* fine grid side, even (kept set |kx|, |ky| <= n/3).  KD_FINE_FFT:
                          n = 16, 32, ..., 1024 and 96, 160, 192 (32 R, R = 3, 5, 6: mixed
                          radix; Table 1's N_F = 160) transform on n itself; any other even
                          n <= 286 on the smallest mixed-radix side m >= 2 (n/3) + 2: the flow
                          has only the wavenumbers +-1, so m points resolve u x b on the kept
                          set without aliasing, exactly as n points do (n = 240, the 3/2-padded
                          grid of 160 kept modes, runs on m = 192).  KD_FINE_CONV: even
                          n <= 190 */
  double kz;           /* wavenumber along the invariant direction (the paper's kx for GP) */
  double Rm;           /* magnetic Reynolds number (Eq. 2), > 0 */
  double dt_fine;      /* fine step delta t (upper bound; see kd_parareal_run) */
  int prec_fine;       /* KD_C64 or KD_C128 arithmetic of the fine propagator */
  int n_coarse;        /* coarse grid side N_C, even, 16 <= N_C <= n: the cluster solver when
                          its dealiased set fits (N_C <= 190), else the FFT fine kernels (a
                          side they take, as for n) */
  double dt_coarse;    /* coarse step Delta t (upper bound) */
  int prec_coarse;     /* KD_C64 or KD_C128 arithmetic of the classical coarse propagator */
  int coarse_kind;     /* KD_COARSE_CLASSICAL or KD_COARSE_LEARNED (needs kd_learned_init and
                          fine_form KD_FINE_INCREMENT; falls back to the classical propagator) */
  int learned_modes;   /* m > 0: coarse mode set kx, ky in [-floor(m/2), m - floor(m/2)) (inside
                          |k| <= n/3, m <= 64; odd m = 2K+1 gives the square |k| <= K), used by
                          the learned operator AND by the classical coarse propagator ("same
                          truncation"); 0: the dealiased set of the n_coarse grid */
  int fine_form;       /* KD_FINE_DIRECT or KD_FINE_INCREMENT (kd_parareal_run) */
  int fine_operator;   /* KD_FINE_FFT (pseudo-spectral: FFT, u x b on the grid, FFT) or
                          KD_FINE_CONV: the same discrete operator evaluated as the exact
                          4-mode spectral convolution in a persistent cluster kernel (one
                          launch for all steps; even n <= 190, i.e. at most 127 kept modes
                          a side; RK443 only) */
  int fine_scheme;     /* KD_RK443 (default), KD_RK222 or KD_RK111 */
} kd_params;

/* Create a context for one problem: the initial-value problem of Sec. 3 (the induction
 * equation of Sec. 2 Eq. 1 with the flow, kz and Rm of params) with its fine and coarse
 * discretisations; the set-up step of the Parareal algorithms of Sec. 4.1 (the
 * communicators and solvers each process creates there are this context's tables and
 * workspace here).  `cuda_stream` is a cudaStream_t (may be NULL).  Allocates the grid
 * tables on the current device.  Returns KD_EINVAL for unsupported sizes and KD_ECUDA /
 * KD_ENOMEM on device failures. */
kd_status kd_create(const kd_params* params, void* cuda_stream, kd_ctx** out);

/* Release every resource of the context (waits for its stream first).  NULL is a no-op.
 * No counterpart in the paper (resource management of this library). */
kd_status kd_destroy(kd_ctx* ctx);

/* Fine propagator F (Sec. 3): advance `batch` independent fields by `nsteps` RK443
 * steps of params.dt_fine, every field in the same launches.
 *   b_in, b_out : device, [batch][3][n][n] complex in params.prec_fine; may alias.
 *   t0          : device double[batch]; absolute start time of each field (step s of
 *                 field i evaluates the flow at t0[i] + (s + c_j) dt; matters for GP).
 * Asynchronous on the context stream.  nsteps = 0 copies the masked input. */
kd_status kd_fine_batched(kd_ctx* ctx, const void* b_in, void* b_out, const double* t0,
                          int nsteps, int batch);

/* The fine propagator of kd_fine_batched on fields in HOST memory: the batch moves in
 * chunks, the copy in of a chunk, its propagation and the copy out of the previous chunk
 * overlapping on three streams (two device slots per direction, allocated on first use
 * and kept).  chunk > 0: chunks of that many fields (the last one ragged); chunk = 0: a
 * graded plan, chunks doubling from ceil(batch / 32) fields up to batch / 4, then back
 * down (a short pipeline fill and drain, large batches for the steps in between; 8, 16,
 * 32, 48, 48, 48, 32, 16, 8 for 256 fields).  Same values as kd_fine_batched, field by
 * field.  No counterpart in the paper (host I/O of this library).
 *   h_in, h_out : host, [batch][3][n][n] complex in params.prec_fine (page-locked memory
 *                 lets the copies overlap; pageable memory works, slower); may alias.
 *   t0          : host double[batch] start times.
 * Synchronous: returns when h_out holds the result. */
kd_status kd_fine_batched_host(kd_ctx* ctx, const void* h_in, void* h_out, const double* t0,
                               int nsteps, int batch, int chunk);

/* The kept-mode layout of a field: [3][P][P] complex in params.prec_fine, P = 2K + 1,
 * K = floor(n / 3); entry [c][iy][ix] holds component c of the coefficient of
 * (kx, ky) = (ix - K, iy - K).  These are the modes the 2/3 rule keeps (Sec. 3: the
 * dealiased pseudo-spectral discretisation), the only coefficients a fine step reads or
 * writes: a field in the [3][n][n] layout of kd_fine_batched is this array with zeros
 * around it (wavenumber k < 0 at index k + n).
 *
 * kd_fine_batched_kept: kd_fine_batched on device fields in the kept-mode layout; the
 * same values, field by field.  No counterpart in the paper (a storage layout of this
 * library).  The steps run in place on c_out (c_in is first copied there unless the two
 * are the same buffer; partly overlapping buffers are not allowed).
 *   c_in, c_out : device, [batch][3][P][P] complex in params.prec_fine, aligned to the
 *                 complex element (KD_EINVAL otherwise).
 *   t0          : device double[batch], as in kd_fine_batched.
 * Asynchronous on the context stream.  nsteps = 0 copies the input. */
kd_status kd_fine_batched_kept(kd_ctx* ctx, const void* c_in, void* c_out, const double* t0,
                               int nsteps, int batch);

/* kd_fine_batched_host on fields in the kept-mode layout: the chunks (`chunk` as in
 * kd_fine_batched_host) move through four device slots, each chunk stepped in place
 * in its slot, its copy in, its steps and the copy out of earlier chunks overlapping on
 * three streams.  3 P^2 instead of 3 n^2 complex per field cross the host link.  Same
 * values as kd_fine_batched_kept.  No counterpart in the paper (host I/O of this library).
 *   h_in, h_out : host, [batch][3][P][P] complex in params.prec_fine (page-locked memory
 *                 lets the copies overlap); may alias.
 *   t0          : host double[batch] start times.
 * Synchronous: returns when h_out holds the result. */
kd_status kd_fine_batched_host_kept(kd_ctx* ctx, const void* h_in, void* h_out, const double* t0,
                                    int nsteps, int batch, int chunk);

/* Classical coarse propagator G (Sec. 3.2, Sec. 5.2): restrict each field to the
 * N_C grid (Fourier truncation), take `nsteps` RK443 steps of params.dt_coarse in
 * params.prec_coarse, prolong (zero-pad) back to n.
 *   b_in, b_out : device, [batch][3][n][n] complex128; may alias.
 *   t0          : device double[batch] start times.
 * Asynchronous on the context stream. */
kd_status kd_coarse(kd_ctx* ctx, const double* b_in, double* b_out, const double* t0,
                    int nsteps, int batch);

typedef struct {
  int k_con;                           /* iterations done (= first k with sigma <= tol) */
  int converged;                       /* 1 if sigma <= tol was reached */
  int n_fine_steps;                    /* fine steps per slice S = ceil(dT / dt_fine) */
  int n_coarse_steps;                  /* coarse steps per slice */
  double dt_fine_used;                 /* dT / S */
  double dt_coarse_used;
  double sigma[KD_MAX_ITERS];          /* Eq. 9 defect after iteration k (index k-1) */
  double energy[KD_MAX_SLICES + 1];    /* E(t_n) = sum |b_hat|^2 of the final iterate */
  double growth_rate;                  /* slope of 0.5 ln E over t >= T/2 */
  double ms_total;                     /* device time of the whole run */
  double ms_fine;                      /* parallel fine sweeps */
  double ms_coarse;                    /* serial coarse sweeps incl. the initial one */
  int fallback_used;                   /* learned coarse propagator replaced by the classical one */
  long long n_launches;                /* kernels launched by this call */
  double true_err[KD_MAX_ITERS];       /* with kd_set_reference: |U^k_N - b_ref| / |b_ref| after
                                          iteration k (index k - 1); -1 otherwise */
} kd_parareal_stats;

/* Parareal (Sec. 3, Eq. 8; Algorithms of Sec. 4.1) over [0, T] with n_slices slices
 * of dT = T / n_slices.  Fine: S = ceil(dT / dt_fine) steps of dT / S from
 * t_n = n dT; coarse: ceil(dT / dt_coarse) steps.  Iterate 0 is the serial coarse
 * sweep; iteration k+1 sets U_{n+1} = F(U^k_n) + (G(U^{k+1}_n) - G(U^k_n)) with the
 * fine values of all slices computed in one batched propagation and the update in
 * FP64.  Stops when sigma (Eq. 9) <= tol or after k_max iterations.
 *   b0       : complex128 [3][n][n], host or device pointer.
 *   u_slices : complex128 [n_slices+1][3][n][n] output (host or device), or NULL.
 *   stats    : host, may be NULL.
 * Synchronous.  Returns KD_ENOTCONV if tol was not reached (outputs still valid). */
kd_status kd_parareal_run(kd_ctx* ctx, const double* b0, double T, int n_slices, int k_max,
                          double tol, double* u_slices, kd_parareal_stats* stats);

/* Reference field for the relative error of every Parareal iterate (Sec. 5.1 measures
 * solutions by their relative error against a reference solution; here next to the
 * defect of Eq. 9): b_ref (complex128 [3][n][n], host or device), e.g. the serial fine
 * solution at t = T from kd_fine_serial; kd_parareal_run then fills stats->true_err with
 * |U^k_N - b_ref| / |b_ref| (last slice, FP64, fixed-order reduction).  Not computed by
 * the pipelined iterations.  NULL removes the reference.  Synchronous. */
kd_status kd_set_reference(kd_ctx* ctx, const double* b_ref);

/* Checkpoint / resume of kd_parareal_run: continue Parareal from the iterate U^{k_done}
 * of an earlier run (u_init, complex128 [n_slices+1][3][n][n], host or device, e.g. the
 * u_slices that run returned after k_done iterations; slices 0..k_done of it are the
 * exact fine solution, u_init[0] is b0).  Iterations k_done + 1 .. k_max follow, the
 * first fine sweep in direct form, and give the values the uninterrupted run gives to
 * FP32 round-off.  k_done = 0 starts Parareal from an arbitrary initial iterate instead of
 * the coarse sweep.  stats->sigma[k - 1] holds the defects of the resumed iterations
 * (0 for k <= k_done).  fine_form must be KD_FINE_INCREMENT (else KD_EUNSUPPORTED);
 * otherwise as kd_parareal_run. */
kd_status kd_parareal_resume(kd_ctx* ctx, const double* u_init, int k_done, double T, int n_slices, int k_max,
                             double tol, double* u_slices, kd_parareal_stats* stats);

/* Thread blocks per cluster of the persistent coarse solver (coarse sets up to 88 modes
 * a side): 0 = the default (a batch of fields that fits the GPU in clusters of 16: ~3 rows
 * per block, up to 16 blocks; larger batches: ~6 rows per block, at most 8), else 1..8 (1..16 where the
 * device allows non-portable cluster sizes) when the rows of a block fit its
 * modes-per-thread budget.  Fewer blocks mean cheaper cluster
 * barriers and more work per block.  KD_EINVAL if the coarse set does not fit. */
kd_status kd_set_coarse_cluster(kd_ctx* ctx, int blocks);

/* How the blocks of a coarse-solver cluster exchange the halo rows after each of the
 * 4 stages of an RK443 step (the classical G, Sec. 3.2 / 5.2, and the KD_FINE_CONV
 * operator).  KD_SYNC_CLUSTER (default): the first and last rows are stored into the
 * neighbours' halo rows through distributed shared memory, then a cluster-wide barrier.
 * KD_SYNC_P2P: each block pushes those rows with st.async, counted on the receiver's
 * mbarrier, and waits only for its own halos (bounded wait; a halo that never arrives
 * makes the outputs NaN, which the callers report as KD_ENONFINITE).  KD_SYNC_PULL: no
 * halo copies; the cluster barrier is split (arrive after a stage's stores, wait before
 * the first and last rows of the next stage, the rows between computed meanwhile) and the
 * neighbours' rows are read in place.  All give identical results bit for bit.  KD_EINVAL
 * for another mode. */
enum { KD_SYNC_CLUSTER = 0, KD_SYNC_P2P = 1, KD_SYNC_PULL = 2 };
kd_status kd_set_coarse_sync(kd_ctx* ctx, int mode);

/* Pipelined iterations of kd_parareal_run (default chunks = 0: off): the parallel step of
 * iteration k + 1 runs in `chunks` slice chunks on a low-priority stream and overlaps the
 * serial sweep of iteration k, which runs on a high-priority stream; chunk j starts once
 * the sweep has passed its last slice, and the next sweep waits for each chunk before its
 * first slice.  The parallel step is computed before the defect of iteration k is known
 * and discarded if the run stops there.  The results are those of the unpipelined order
 * bit for bit.  It pays when a chunk's fine work is few launches (KD_FINE_CONV); with the
 * FFT operator every chunk repeats all the step launches on a smaller batch.  KD_EINVAL
 * for chunks outside [0, 16]. */
kd_status kd_set_overlap(kd_ctx* ctx, int chunks);

/* Serial fine solution at the slice boundaries, U_{n+1} = F(U_n) with each slice
 * restarted at t_n = n dT exactly as in kd_parareal_run (the solution Parareal
 * converges to, Sec. 3.1).  Same arguments and step rule as kd_parareal_run.  The fine
 * kernels run with a launch plan autotuned for one field (once per context; the
 * batched plan of kd_set_plan / kd_autotune is left unchanged).  Synchronous. */
kd_status kd_fine_serial(kd_ctx* ctx, const double* b0, double T, int n_slices,
                         double* u_slices);

/* Magnetic energy E_i = sum_{c,k} |b_hat|^2 of `count` complex128 fields
 * ([count][3][n][n], device) into device double[count].  Deterministic order.
 * Asynchronous. */
kd_status kd_energy(kd_ctx* ctx, const double* fields, int count, double* energy_out);

/* Growth rate (Table 1 "Growth Rate"; Sec. 1): least-squares slope of 0.5 ln E(t_i)
 * over the samples with t_i >= fit_from, where t_i = i T / (n_samples - 1) and
 * E_i = kd_energy of u_slices[i].
 *   u_slices : device complex128 [n_samples][3][n][n].
 *   rate_out : host double.
 * Synchronous.  KD_ENONFINITE if an energy is 0, NaN or Inf. */
kd_status kd_growth_rate(kd_ctx* ctx, const double* u_slices, int n_samples, double T,
                         double fit_from, double* rate_out);

/* ------------------------------------------------------------------------------------
 * Learned coarse propagator (a coarse-solver strategy in the sense of Sec. 3.2).
 * A complex-linear map W_p on the mode set kx, ky in [-m/2, m/2) x 3 components
 * (nc = 3 m^2 complex unknowns, m = params.learned_modes), one per flow phase
 * p = slice index mod n_phase (the Galloway-Proctor flow has period 2 pi; a slice of
 * length slice_T starts at phase p when it starts at t = p slice_T).  Operators are
 * stored in BF16 as [Re W; Im W] ([2 nc][nc]) and applied with FP32 accumulation.
 * Vectors on the set ("learned vectors") are device complex FP32 [3][m][m] (ky-major),
 * interleaved (re, im).  The fine solution decides: pairs (x, F x) come from the
 * fine propagator, and kd_learned_eval compares W_p and the classical coarse
 * propagator against them; phases whose operator loses fall back to the classical one.
 * ------------------------------------------------------------------------------------ */

/* Operators are stored with rows padded to a multiple of 8 columns internally; every
 * matrix crossing this interface is [2 nc][nc].
 * W_p := the classical coarse propagator on the learned set over one slice from
 * t = p slice_T (built by applying it to every unit vector).  Synchronous. */
kd_status kd_learned_init(kd_ctx* ctx, int n_phase, double slice_T);

/* y_i = R F(P x_i): the fine propagator over one slice from t = phase[i] slice_T applied
 * to the learned vector x_i prolonged to the fine grid, restricted back to the set.
 *   x, y : device learned vectors [n]; phase : host int[n] in [0, n_phase).  Synchronous. */
kd_status kd_learned_pairs(kd_ctx* ctx, const float* x, int n, const int* phase, float* y);

enum { KD_TRAIN_ADAM = 0, KD_TRAIN_MOMENTUM = 1, KD_TRAIN_MINNORM = 2 };

/* Train every W_p on its pairs, starting from W_classical, on
 *   L = (1/m) sum_i |W x_i - y_i|^2 + weight_decay |W - W_classical|^2;
 * forward product and gradient 2/m (W X - Y) X^H are BF16 tensor-core GEMMs with FP32
 * accumulation, master weights FP32.  method:
 *   KD_TRAIN_ADAM      Adam (beta 0.9 / 0.999), step lr with cosine decay to 0;
 *   KD_TRAIN_MOMENTUM  heavy-ball gradient descent (momentum 0.9), step lr / lambda with
 *                      lambda = (2/m) sum |x_i|^2 (lr <= 1); its updates stay in the span
 *                      of the training inputs, which matters when pairs are fewer than
 *                      the 3 m^2 unknowns of a row (Adam's per-weight scaling does not).
 *   KD_TRAIN_MINNORM   the minimiser in closed form (epochs and lr unused):
 *                      W = W0 + (Y - W0 X)(X^H X + m weight_decay I)^-1 X^H, X, Y the pairs
 *                      of a phase as columns (m <= 4096 of them); with weight_decay = 0 the
 *                      smallest change of W0 that maps every training input onto its
 *                      output (W0 X in FP64 from the classical propagator, X^H X summed in
 *                      FP32 per 32 unknowns and in FP64 across, its Cholesky inverse in FP64
 *                      on the host, the correction GEMM in BF16 on the tensor cores).
 *                      KD_EINVAL when the inputs of a phase are linearly dependent and
 *                      weight_decay is 0. loss_out is not written.
 *   loss_out : host double[n_phase * epochs] data loss per phase and epoch (may be NULL).
 * Synchronous. */
kd_status kd_learned_train(kd_ctx* ctx, const float* x, const float* y, const int* phase, int n, int epochs, float lr,
                           float weight_decay, int method, double* loss_out);

/* Relative L2 errors per phase of the learned operator and of the classical coarse
 * propagator against held-out pairs (host double[n_phase] each; -1 for phases without
 * pairs).  Marks a phase's operator unusable when it is worse than the classical one.
 * Synchronous. */
kd_status kd_learned_eval(kd_ctx* ctx, const float* x, const float* y, const int* phase, int n, double* err_learned,
                          double* err_classical);

/* Loss and gradient of the training objective for a given stacked FP32 operator W
 * ([2 nc][nc], device) and regulariser centre W0 (device or NULL = 0), through the same
 * kernels as kd_learned_train: *loss_out (host), grad_out (device FP32 [2 nc][nc],
 * [d/dRe W; d/dIm W]).  Needs params.learned_modes > 0 only.  Synchronous. */
kd_status kd_learned_loss_grad(kd_ctx* ctx, const float* W, const float* W0, float weight_decay, const float* x,
                               const float* y, int n, double* loss_out, float* grad_out);

/* Checkpoint of the learned operators: copy W_phase out (BF16 [2 nc][nc], host or
 * device) with its usability flag (valid: 1 when kd_learned_eval found it no worse than
 * the classical propagator; may be NULL), or load one in, e.g. from a previous run, with
 * the flag the caller gives (the Parareal sweep uses W_phase only when it is set).  The
 * padding of the internal rows stays zero.  Synchronous.  KD_EINVAL before
 * kd_learned_init or for a phase outside [0, n_phase). */
kd_status kd_learned_get(kd_ctx* ctx, int phase, void* W, int* valid);
kd_status kd_learned_set(kd_ctx* ctx, int phase, const void* W, int valid);

/* y_i = W_phase x_i for n learned vectors (device).  Asynchronous. */
kd_status kd_learned_apply(kd_ctx* ctx, const float* x, float* y, int phase, int n);

/* Size of the device scratch array used by kd_fine_batched_static (32 MiB). */
#define KD_STATIC_SCRATCH_BYTES 33554432

/* kd_fine_batched_static: the same fine propagator as kd_fine_batched, for callers that
 * must not allocate device memory -- for example a library embedded in a host
 * application whose memory pool already owns the GPU's memory, or a latency-critical
 * loop that cannot afford cudaMalloc's implicit device synchronisation.  It needs no
 * context: it takes the parameters directly and makes no cudaMalloc, cudaFree or
 * other allocating call.  (The paper has no counterpart; this is an integration aid.)
 *
 *   params      : as for kd_create; only flow, n, kz, Rm, dt_fine and prec_fine are used.
 *   b_in, b_out : device, [batch][3][n][n] complex in params->prec_fine; may alias.
 *   t0          : device double[batch], start time of each field.
 *   cuda_stream : cudaStream_t the work is enqueued on (NULL = legacy default stream).
 *
 * The workspace lives in one file-scope device array of KD_STATIC_SCRATCH_BYTES that
 * every GPU loading the library keeps until the process exits.  A request needs
 *   256-byte-aligned sums of: 3 n complex-or-real table entries, A x batch x 3 x P^2
 *   and 2 x batch x 3 x P x n complex values (P = 2 (n/3) + 1; A = 5 for complex64:
 *   state, its low part and three stage accumulators; A = 4 for complex128), plus for
 *   the Galloway-Proctor flow batch x nsteps x 16 reals of flow phases,
 * in the bytes of prec_fine (e.g. about 1.38 MB per complex64 field at n = 128, so at
 * most 24 fields of the Roberts flow fit); larger requests return KD_EINVAL with a message on
 * stderr and enqueue nothing.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) on the current device; the first call on a device, and the
 * first call after cudaDeviceReset gave it a new context, also set the kernels'
 * shared-memory limits; make such a call before any stream capture.  All
 * calls share the one array: calls that can overlap on the GPU (different streams
 * without ordering, several host threads) race and corrupt each other's results.
 * Every part of the array a call reads is written earlier in the same call, so the
 * previous call's contents never leak into a result.  Asynchronous; returns
 * KD_EINVAL or KD_ECUDA on failure. */
kd_status kd_fine_batched_static(const kd_params* params, const void* b_in, void* b_out, const double* t0,
                                 int nsteps, int batch, void* cuda_stream);

/* Growth rate by power iteration of the fine propagator over [t0, t0 + tau] (Sec. 1: the
 * leading eigenvalue for a steady flow, the leading Floquet multiplier for a time-periodic
 * one with tau = its period): b <- M b / |M b| from b0 (complex128 [3][n][n], host or
 * device), rate_k = ln(|M b| / |b|) / tau, until |rate_k - rate_{k-1}| <= tol or max_iter
 * iterations.  The fine steps are ceil(tau / dt_fine) steps of the context's fine
 * precision; norms are FP64.  rate: the last estimate; iters (may be NULL): iterations
 * taken; b_out (may be NULL): the normalised final vector (complex128 [3][n][n]).
 * Synchronous.  KD_ENOTCONV if tol was not reached (outputs still written),
 * KD_ENONFINITE on a zero or non-finite norm. */
kd_status kd_growth_power(kd_ctx* ctx, const double* b0, double t0, double tau, int max_iter, double tol,
                          double* rate, int* iters, double* b_out);

/* Leading eigenvalues of the fine propagator M over [t0, t0 + tau] by restarted Arnoldi
 * (Sec. 1: the growth rate is Re lambda of the leading eigenvalue for a steady flow,
 * ln|mu| / period of the leading Floquet multiplier for a time-periodic one).  Unlike the
 * power iteration it converges for a small gap between the leading |mu| and finds complex
 * multipliers (oscillating modes).  A Krylov space of dimension m is built from b0
 * (complex128 [3][n][n], host or device; its dealiased part) with FP64 basis vectors and
 * Gram-Schmidt done twice; the Ritz values of largest modulus are accepted when the
 * relative residual |H[m][m-1]| |y[m-1]| / |theta| of each of the nev leading ones is
 * <= tol; otherwise the run restarts from the sum of their Ritz vectors, at most
 * `restarts` times.  M is ceil(tau / dt_fine) fine steps of the context's operator and
 * precision.
 *   mu    : out, double[nev][2], the multipliers (re, im) by decreasing modulus; for a
 *           steady flow lambda = log(mu) / tau (principal branch: take tau with
 *           |Im lambda| tau < pi)
 *   rate  : out (may be NULL), double[nev], ln|mu| / tau
 *   iters : out (may be NULL), restarts used
 *   b_out : out (may be NULL), complex128 [3][n][n], the leading Ritz vector (unit norm)
 * 2 <= m <= KD_ARNOLDI_MAX_M, 1 <= nev < m, restarts >= 1, tol >= 0, else KD_EINVAL.
 * Synchronous; allocates (m + 1) compact FP64 fields for the call.  KD_ENOTCONV if tol
 * was not reached (outputs hold the last estimates), KD_ENONFINITE on a zero or
 * non-finite vector. */
#define KD_ARNOLDI_MAX_M 64
kd_status kd_growth_arnoldi(kd_ctx* ctx, const double* b0, double t0, double tau, int m, int nev, int restarts,
                            double tol, double* mu, double* rate, int* iters, double* b_out);

/* The BF16 GEMM of the learned operator's training (Sec. 3.2's learned G; the forward
 * product W X and the gradient product (W X - Y) X^T): C[M][N] = A[M][K] Bt[N][K]^T with
 * A and Bt row-major BF16 (K innermost, K a multiple of 8, base addresses 16-byte
 * aligned), C row-major FP32 with row
 * stride ldc >= N; all device pointers.  KD_GEMM_TCGEN05 (default for training): 5th-
 * generation tensor cores, tcgen05.mma into a tensor-memory accumulator, 128 x 256 tiles
 * (128 x 128 where the wide tiles would be fewer than two per SM);
 * KD_GEMM_MMA_SYNC: the warp-level mma.sync kernel.  Synchronous on cuda_stream (NULL =
 * legacy default stream).  KD_EINVAL for bad arguments, KD_ECUDA on a launch failure or a
 * bounded wait inside the kernel that ran out. */
enum { KD_GEMM_TCGEN05 = 0, KD_GEMM_MMA_SYNC = 1 };
kd_status kd_gemm_bf16_tn(const void* A, const void* Bt, float* C, int M, int N, int K, int ldc, int engine,
                          void* cuda_stream);

/* CUDA graphs for the Parareal fine sweeps of the FFT operator (default on; not used
 * with kd_set_overlap's pipelined iterations): the ~8 S launches of one sweep shape
 * (first slice, slices, steps, step, form, launch plan) are captured once into a graph
 * and replayed on a stream of the context, fenced by events against the context stream;
 * any device allocation of the context invalidates the captured graphs.  Off: direct
 * launches.  Same values either way. */
kd_status kd_set_graphs(kd_ctx* ctx, int enable);

/* Engine of the GEMMs in kd_learned_train / kd_learned_loss_grad (default KD_GEMM_TCGEN05). */
kd_status kd_set_learned_gemm(kd_ctx* ctx, int engine);

/* Self-test of the bounded device-side waits (failure detection without a GPU fault):
 * one CTA waits on an mbarrier phase with the same bounded-wait helper the kernels use;
 * arrive = 1 gives it its arrival (KD_OK), arrive = 0 gives it none, and the wait gives up
 * after max_ms milliseconds (0 < max_ms <= 1000) with KD_ETIMEOUT, the device still
 * usable.  Synchronous on cuda_stream. */
kd_status kd_selftest_wait(int arrive, double max_ms, void* cuda_stream);

/* Allocation limit of a context (failure injection of device out-of-memory without
 * exhausting the GPU, and a memory budget for callers that share it).  No counterpart in
 * the paper.  The limit caps the device bytes the context holds in its own buffers (grid
 * tables, fine and coarse workspaces, Parareal arrays, staging; not CUDA's own objects
 * such as streams, events and graph executables, nor the static array of
 * kd_fine_batched_static).  max_bytes = 0 removes it (the default); a limit below what the
 * context already holds keeps those buffers and refuses new ones.  A call that needs a
 * buffer beyond the limit returns KD_ENOMEM, as a failed cudaMalloc does, with
 * kd_last_error naming the buffer, its size, the bytes held and the limit; the context
 * stays usable, and the same call succeeds once the limit allows it.  Contexts that
 * kd_sweep_create makes for itself are not affected.  kd_get_alloc_bytes returns the bytes
 * held and the limit (either pointer may be NULL).  Both are host-only: no CUDA call. */
kd_status kd_set_alloc_limit(kd_ctx* ctx, size_t max_bytes);
kd_status kd_get_alloc_bytes(kd_ctx* ctx, size_t* held, size_t* limit);

/* The host routine that kd_growth_arnoldi uses for its small dense eigenproblem, exposed
 * for checking: eigenvalues of an m x m complex upper Hessenberg matrix h (row-major,
 * interleaved re / im; entries below the subdiagonal must be zero) by the shifted QR
 * algorithm, into eig[m][2] in the order of the Schur form's diagonal; vec (may be NULL):
 * the unit eigenvectors as columns of an m x m complex matrix (row-major, interleaved).
 * No GPU involved.  KD_EINVAL for bad arguments, KD_ENOTCONV if QR did not converge. */
kd_status kd_hessenberg_eig(int m, const double* h, double* eig, double* vec);

/* ------------------------------------------------------------------------------------
 * Slice blocks for Parareal over several ranks (the paper's time communicator, Sec. 4.1
 * Algorithms 1-3): rank r owns the contiguous slices [lo, lo + n_local) of n_slices.  The
 * host drives the iteration and moves one boundary state per sweep between ranks:
 *
 *   kd_block_init(ctx, lo, n_local, T, n_slices)
 *   rank 0: kd_block_set_initial(ctx, b0)
 *   k = 0:  rank > 0 receives U_lo -> kd_block_set_boundary;  kd_block_sweep(ctx, 0, NULL);
 *           kd_block_get_boundary -> send U_hi to rank + 1
 *   k >= 1: kd_block_fine(ctx, k) (parallel step, no communication); receive U_lo and
 *           kd_block_set_boundary (rank > 0); kd_block_sweep(ctx, k, &sigma) (the rank
 *           holding the last slice gets the Eq. 9 defect); send U_hi; broadcast sigma.
 *
 * The arithmetic is that of kd_parareal_run with fine_form KD_FINE_INCREMENT (required);
 * one rank holding all slices reproduces it.  Boundary states are FP64 compact fields of
 * kd_block_boundary_bytes() bytes (host or device buffers).  States are returned by
 * kd_block_get_state (local index 0..n_local, complex128 [3][n][n]).  Synchronous.  The
 * learned coarse propagator is used where it passed validation, without the fallback
 * rule of kd_parareal_run. */
kd_status kd_block_init(kd_ctx* ctx, int lo, int n_local, double T, int n_slices);
size_t kd_block_boundary_bytes(kd_ctx* ctx);
kd_status kd_block_set_initial(kd_ctx* ctx, const double* b0);
kd_status kd_block_set_boundary(kd_ctx* ctx, const double* u_lo);
kd_status kd_block_get_boundary(kd_ctx* ctx, double* u_hi);
kd_status kd_block_fine(kd_ctx* ctx, int k);
kd_status kd_block_sweep(kd_ctx* ctx, int k, double* sigma);
kd_status kd_block_get_state(kd_ctx* ctx, int local_index, double* u);

/* ------------------------------------------------------------------------------------
 * Launch plans and the autotuner.
 *
 * The fine step's column and row kernels exist in several variants per grid and
 * precision (columns or rows per thread block; the row kernel's stage update run from
 * shared memory or from registers).  A plan is the pair (col, row) of variant indices;
 * {0, 0} is the default, except on the complex64 grid n = 1024, whose default is the
 * warp-transform pair {5, 7}.  grid: 0 = the fine grid n, 1 = the coarse grid n_coarse. */
enum { KD_GRID_FINE = 0, KD_GRID_COARSE = 1 };

/* Number of column / row variants of the context's grid.  KD_EINVAL for a bad grid. */
kd_status kd_plan_variants(kd_ctx* ctx, int grid, int* n_col, int* n_row);
/* Set / read the plan of a grid.  KD_EINVAL if an index is out of range. */
kd_status kd_set_plan(kd_ctx* ctx, int grid, int col, int row);
kd_status kd_get_plan(kd_ctx* ctx, int grid, int* col, int* row);

/* Launch the fine step's kernels as programmatic dependent launches (enable = 1, the
 * default): each kernel may start while its predecessor drains and waits on the device
 * before it reads the predecessor's output.  enable = 0 uses ordinary launches. */
kd_status kd_set_dependent_launch(kd_ctx* ctx, int enable);

/* Autotune the plan of a grid for batches of `batch` fields: if `cache_path` (may be
 * NULL) names a JSON file holding an entry for (device name, n, precision, batch rounded
 * up to a power of two), that entry's plan is used; otherwise every (col, row) pair is
 * timed with CUDA events over `nsteps` fine steps (after one untimed step) on seeded
 * workspace data, the fastest is set and, with cache_path, written to the file (other
 * entries are kept).  ms_per_step (may be NULL) receives the chosen plan's time, or -1
 * when it came from the cache.  Synchronous.  KD_EINVAL for bad arguments, KD_ECUDA on
 * device failures; an unreadable or malformed cache file is ignored and rewritten. */
kd_status kd_autotune(kd_ctx* ctx, int grid, int batch, int nsteps, const char* cache_path,
                      double* ms_per_step);

/* ------------------------------------------------------------------------------------
 * Batched sweep of independent Parareal problems (instances of different grids, flows,
 * kz and Rm; Sec. 3 applied to each).  Instances are grouped by (n, n_coarse); within a
 * group every instance's slices advance together in the same batched fine launches (each
 * field with its own dt, kz, Rm and flow, fields ordered by decreasing step count so that
 * the fields still stepping are a prefix of the batch), and the serial sweeps of all
 * instances run together slice by slice.  Fine propagator complex64, classical coarse
 * propagator complex64 on the n_coarse grid, the increment form of the correction
 * (U_{n+1} = F(U_n) accumulated + G(U_n - U_n^prev)) and the defect in FP64.  An instance
 * stops iterating when its defect reaches tol (or at k_max) while the others go on. */
typedef struct {
  int flow;            /* KD_FLOW_* */
  int n;               /* fine grid side, power of two in [16, 1024] */
  double kz, Rm;
  double dt_fine;      /* fine step; the slice length is split into ceil(dT / dt_fine) equal steps */
  int n_coarse;        /* coarse grid side, power of two in [16, n] */
  double dt_coarse;    /* coarse step (rounded like dt_fine) */
} kd_instance;

typedef struct {
  int status;              /* KD_OK, KD_ENOTCONV or KD_ENONFINITE for this instance */
  int k_con;               /* iterations taken */
  int n_fine_steps, n_coarse_steps;
  double dt_fine_used, dt_coarse_used;
  double sigma[KD_MAX_ITERS];  /* Eq. 9 defect after iteration k (index k-1) */
  double growth_rate;      /* 0.5 d ln E / dt fitted over t >= T/2 at the slice boundaries */
} kd_instance_result;

typedef struct {
  int n_groups;
  double ms_total, ms_fine, ms_coarse;
  long long n_launches;
  double fine_dof_steps;   /* sum over fine launches of 3 n^2 x fields x steps actually advanced */
} kd_sweep_stats;

/* Run Parareal with n_slices slices of T / n_slices on every instance.  b0[i]: instance
 * i's initial field, complex128 [3][n_i][n_i] (host or device pointer).  u_final (may be
 * NULL, entries may be NULL): receives instance i's final-iterate state at t = T in the
 * same layout.  results[n_inst] (may be NULL), stats (may be NULL).  tune_cache (may be
 * NULL): JSON cache of kd_autotune; when given, each group's fine plan is autotuned (or
 * read from the cache) before the run.  Synchronous on cuda_stream.  Returns KD_OK when
 * every instance converged, KD_ENOTCONV if some did not (outputs still written),
 * KD_ENONFINITE if an instance's defect was not finite, KD_EINVAL / KD_ENOMEM / KD_ECUDA
 * otherwise; err (may be NULL, >= 256 bytes) receives a message. */
kd_status kd_sweep_run(const kd_instance* inst, int n_inst, const double* const* b0, double T, int n_slices,
                       int k_max, double tol, const char* tune_cache, double* const* u_final,
                       kd_instance_result* results, kd_sweep_stats* stats, void* cuda_stream, char* err);

/* A prepared sweep of the same kind (kd_sweep_run is kd_sweep_create, one kd_sweep_exec and
 * kd_sweep_destroy).  kd_sweep_create groups the instances by (n, n_coarse) and makes
 * each group's context, device buffers and workspaces once (KD_EINVAL for invalid
 * instances or sizes, KD_ENOMEM / KD_ECUDA on device failures; err as above); the object
 * is owned by the library until kd_sweep_destroy (NULL is a no-op).  kd_sweep_exec runs
 * the Parareal iterations of every instance from b0 (arguments and results as in
 * kd_sweep_run; tune_cache is read on the first exec only) and may be called any number
 * of times.  The parallel fine step of each (iteration, set of unconverged instances) is
 * captured into a CUDA graph the first time it occurs and replayed when it recurs, e.g.
 * in a repeated exec of the same initial fields; kd_sweep_set_graphs(sw, 0) launches it
 * directly instead (same values).  Same numerics as Eq. 8 / Eq. 9 per instance, as in
 * kd_sweep_run. */
typedef struct kd_sweep kd_sweep;
kd_status kd_sweep_create(const kd_instance* inst, int n_inst, double T, int n_slices, void* cuda_stream,
                          kd_sweep** out, char* err);
kd_status kd_sweep_exec(kd_sweep* sw, const double* const* b0, int k_max, double tol, const char* tune_cache,
                        double* const* u_final, kd_instance_result* results, kd_sweep_stats* stats, char* err);
kd_status kd_sweep_set_graphs(kd_sweep* sw, int enable);
kd_status kd_sweep_destroy(kd_sweep* sw);

/* Number of kernels this context has launched since kd_create (-1 for NULL). */
long long kd_launch_count(kd_ctx* ctx);

/* Event timing of the fine propagator's kernels (instrumentation; not needed for
 * results).  kd_profile(ctx, 1) resets the counters and brackets every launch of the
 * fine-grid column kernel (index 0) and row kernel (index 1) with CUDA events on the
 * context stream; kd_profile(ctx, 0) stops.  kd_profile_read waits for the recorded
 * events and returns the summed device milliseconds ms[2] and launch counts
 * launches[2] since the last reset.  Synchronous. */
kd_status kd_profile(kd_ctx* ctx, int enable);
kd_status kd_profile_read(kd_ctx* ctx, double* ms, long long* launches);

/* Message of the last error on this context ("" if none).  Valid until the next call.
 * No counterpart in the paper (diagnostics of this library). */
const char* kd_last_error(kd_ctx* ctx);

/* Library version string. */
const char* kd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KD_H_ */
