// Learned coarse propagator: a complex-linear map W_p on a square mode set
// k in [-K, P - K)^2 x 3 components (nc = 3 P^2 complex unknowns), one per flow
// phase.  Stored "stacked": W = [Re W; Im W] as a real [2 nc][nc] matrix, so that
//   [A; B] [x_r x_i] = [[A x_r, A x_i], [B x_r, B x_i]],  W x = (A x_r - B x_i) + i (B x_r + A x_i).
// Vectors on the set are complex FP32, layout [3][P][P] interleaved (re, im).  Operator
// rows are padded to ld = nc rounded up to a multiple of 8 (zero columns), so that rows
// start on 16-byte boundaries for the vector loads and the GEMM's K-tiles.
#pragma once
#include <cuda_bf16.h>

#include "kd_common.cuh"

namespace kd {

// x[b] = restriction of (U[b] - Uprev[b]) (or U[b] if Uprev == NULL) from the fine
// compact FP64 layout (set Kf, Pf) to the learned set (K, P).
int learned_gather(const double* U, const double* Uprev, int Kf, int Pf, float* x, int K, int P, int batch,
                   cudaStream_t st);
// U_next = (init ? 0 : Fv) + prolong(y) over the fine compact set, FP64, with fixed-order
// per-block sums of |U_next - U_next_old|^2, |U_next|^2 into partials (if not NULL).
// Returns the number of blocks (for finish_sigma) or a negative value on error.
int learned_update(const double* Fv, const float* y, int K, int P, double* Unext, int Kf, int Pf, int init,
                   double* partials, cudaStream_t st);
// learned-set complex FP32 <-> fine compact complex (precision prec: 0 c64, 1 c128)
int learned_to_fine(const float* x, int K, int P, void* X, int prec, int Kf, int Pf, long batch, cudaStream_t st);
int fine_to_learned(const void* X, int prec, int Kf, int Pf, float* y, int K, int P, long batch, cudaStream_t st);
// learned-set complex FP64 (coarse-solver layout) <-> complex FP32
int learned_f32_to_f64(const float* x, double* d, long n_complex, cudaStream_t st);
int learned_f64_to_f32(const double* d, float* x, long n_complex, cudaStream_t st);
// unit vectors e_j (j < count, j0 offset) in the learned-set complex FP64 layout: [count][nc]
int learned_unit_vectors(double* d, int nc, int j0, int count, cudaStream_t st);
// columns j0..j0+count of the complex matrix, given as g64[count][nc] (g64[j] = G e_j),
// into the stacked FP32 matrix W[2 nc][nc]
int learned_columns(const double* g64, int nc, int ld, int j0, int count, float* W, cudaStream_t st);

// y[f] = W x[f] for `batch` fields; W stacked BF16 [2 nc][ld] (row-major), FP32 accumulate
cudaError_t learned_gemv_prepare(int ld_max);
int learned_gemv(const __nv_bfloat16* W, const float* x, float* y, int nc, int ld, int batch, cudaStream_t st);

// C[M][N] (FP32, row stride ldc) = A[M][K] . Bt[N][K]^T, A and Bt BF16 row-major with K
// contiguous (K a multiple of 8); tensor-core mma, FP32 accumulate.
int gemm_bf16_tn(const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C, int M, int N, int K, int ldc,
                 cudaStream_t st);
// The same product on the tcgen05 tensor cores (kd_gemm_tc.cu): TMEM accumulator, 128-byte
// swizzled K-major operand tiles; *err (device int) is set if a bounded wait ran out.
int gemm_bf16_tn_tc(const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C, int M, int N, int K, int ldc,
                    int* err, cudaStream_t st);

// training helpers (m pairs, nc complex unknowns)
// Xs[2m][ld]  rows n: Re x_n, rows m + n: Im x_n (zero beyond nc)  (forward B operand)
// XtT[nc][2m] row j: (Re x_n[j])_n, (Im x_n[j])_n                    (gradient B operand)
int learned_pack_x(const float* x, int m, int nc, int ld, __nv_bfloat16* Xs, __nv_bfloat16* XtT, cudaStream_t st);
// yT[nc][m] complex FP32 from y[m][nc]
int learned_transpose_y(const float* y, int m, int nc, float* yT, cudaStream_t st);
// from C1[2nc][2m] = W_stack . Xs^T: residual R = W x_n - y_n, loss partials (per-block
// sum of |R|^2 into partials), and the gradient A operand
// A2[2nc][2m]: row j: (R_r, R_i), row nc + j: (R_i, -R_r)
int learned_residual(const float* C1, const float* yT, int m, int nc, __nv_bfloat16* A2, double* partials,
                     cudaStream_t st);
// Adam step on the stacked FP32 master weights with gradient
//   g = scale * C2 + 2 wd (W - W0)
// m1, v updated; Wbf = bf16(W); also per-block sums of |W - W0|^2 (if partials2).
int learned_adam(float* W, const float* W0, const float* C2, float* m1, float* v, __nv_bfloat16* Wbf, long count,
                 float scale, float wd, float lr, float beta1, float beta2, float eps, int step, double* partials2,
                 cudaStream_t st);
// heavy-ball step: g as above, v = mu v + g, W -= eta v, Wbf = bf16(W)
int learned_momentum(float* W, const float* W0, const float* C2, float* v, __nv_bfloat16* Wbf, long count,
                     float scale, float wd, float eta, float mu, cudaStream_t st);
// plain gradient (no update): grad = scale * C2 + 2 wd (W - W0)   (W0 may be NULL)
int learned_grad(const float* W, const float* W0, const float* C2, float* grad, long count, float scale, float wd,
                 cudaStream_t st);
int f32_to_bf16(const float* x, __nv_bfloat16* y, long count, cudaStream_t st);
// sum of `count` doubles in fixed order -> out[0]
int sum_partials(const double* p, int count, double* out, cudaStream_t st);
// relative errors: out[0] = sum |a - b|^2, out[1] = sum |b|^2 over `count` floats
int diff_norms(const float* a, const float* b, long count, double* partials, cudaStream_t st);
// minimum-norm correction W = W0 + (Y - W0 X)(X^H X + lambda I)^-1 X^H (KD_TRAIN_MINNORM):
// G = X^H X, complex FP64 [m][m], of the learned vectors x [m][nc]
int learned_gram(const float* x, int m, int nc, double* G, cudaStream_t st);
// R = y - g (g the classical outputs in FP64), complex FP32, n_complex values
int learned_resid64(const float* y, const double* g, float* R, long n_complex, cudaStream_t st);
// A = R Ginv (Ginv complex FP32 [m][m]) as the gradient GEMM's left operand A2 [2 nc][2 mp]
// (the layout learned_residual writes), zero in the padding columns n >= m, split in two
// BF16 terms A2 + A2lo (A2lo = the rounding error of A2), so that the correction GEMM
// A X^H keeps ~16 bits where its terms cancel
int learned_minnorm_operand(const float* R, const float* Ginv, int m, int mp, int nc, __nv_bfloat16* A2,
                            __nv_bfloat16* A2lo, cudaStream_t st);
// the rounding error x - bf16(x) of learned_pack_x's XtT operand, same layout
int learned_pack_x_lo(const float* x, int m, int nc, __nv_bfloat16* XtTlo, cudaStream_t st);
// Wbf = bf16(W0 + D0 + D1 + D2)
int learned_add_bf16(const float* W0, const float* D0, const float* D1, const float* D2, __nv_bfloat16* Wbf,
                     long count, cudaStream_t st);

}  // namespace kd
