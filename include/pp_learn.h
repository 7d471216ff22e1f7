/*
 * pp_learn.h -- kernels of the learned warm start for shooting: a POD basis of periodic
 * states and an MLP that predicts POD coefficients of the periodic initial state from the
 * motion parameters.  (The paper starts shooting from the steady state or from fixed-point
 * iterations, Sec. 6.1; this learned initial guess is an addition whose quality is judged
 * by the shooting residual it starts from, with cold-start shooting as the fallback.)
 *
 * All pointers are DEVICE pointers; matrices are row-major; work is issued on `stream`
 * (a cudaStream_t, NULL = default stream).  Return 0, PP_LEARN_EINVAL or PP_LEARN_ECUDA.
 */
#ifndef PP_LEARN_H
#define PP_LEARN_H

#ifdef __cplusplus
extern "C" {
#endif

#define PP_LEARN_EINVAL -1
#define PP_LEARN_ECUDA -6

/* C = alpha op(A) op(B) + beta C with op(A) m x k, op(B) k x n; ta/tb = 1 transposes
   (A stored k x m, B stored n x k).  FP32 (network layers) and FP64 (POD Gram matrix,
   modes and projections). */
int pp_gemm_f32(int m, int n, int k, float alpha, const float* A, int lda, int ta, const float* B, int ldb, int tb,
                float beta, float* C, int ldc, void* stream);
int pp_gemm_f64(int m, int n, int k, double alpha, const double* A, int lda, int ta, const double* B, int ldb,
                int tb, double beta, double* C, int ldc, void* stream);
/* Z[r][c] += b[c]; H = GELU(Z) (gelu_on = 1, GELU(z) = z Phi(z)) or H = Z (0). */
int pp_bias_act_f32(int rows, int cols, float* Z, const float* b, float* H, int gelu_on, void* stream);
/* dZ = dH * GELU'(Z), elementwise over n values. */
int pp_gelu_backward_f32(int n, const float* Z, const float* dH, float* dZ, void* stream);
/* db[c] = sum_r dZ[r][c] (bias gradient). */
int pp_colsum_f32(int rows, int cols, const float* dZ, float* db, void* stream);
/* loss[0] = mean((Y - T)^2) over n values; dY = 2 (Y - T) / n. */
int pp_mse_f32(int n, const float* Y, const float* T, float* dY, float* loss, void* stream);
/* Adam step (step >= 1 counts from 1) on n parameters with moments m1, m2. */
int pp_adam_f32(int n, float* w, const float* g, float* m1, float* m2, float lr, float b1, float b2, float eps,
                int step, void* stream);
/* Eigen-decomposition of a symmetric n x n matrix A (n <= 4096, overwritten) by cyclic
   Jacobi rotations in the parallel round-robin ordering: V (n x n) receives the eigenvectors
   as columns, w (n) the eigenvalues (unsorted); stops when the off-diagonal norm is <= tol
   times the Frobenius norm or after max_sweeps.  sweeps: DEVICE int or NULL.  n <= 256 runs
   in one thread block with the test on the device; larger n runs one CTA per rotation pair
   and round (columns, then rows), tests the norms on the host once per sweep (the call
   then synchronizes the stream) and allocates (n + 2) doubles of device scratch. */
int pp_syevj_f64(int n, double* A, double* V, double* w, double tol, int max_sweeps, int* sweeps, void* stream);

#ifdef __cplusplus
}
#endif
#endif
