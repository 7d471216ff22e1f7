// Kernels of the learned warm start (POD of periodic states + MLP predicting the POD
// coefficients from the motion parameters):
//  - tiled dense GEMM, FP32 (network) and FP64 (snapshot Gram matrix, modes, projections),
//    C = alpha op(A) op(B) + beta C, row-major;
//  - bias + GELU forward (pre-activation kept), GELU backward, bias-gradient column sums;
//  - mean-squared-error loss and gradient;
//  - Adam update;
//  - one-CTA cyclic Jacobi eigensolver for a small symmetric matrix (POD Gram matrix).
// The C ABI is declared in include/pp_learn.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/pp_learn.h"
#include "prof.h"
#include "../../include/pp_prof.h"

namespace {

constexpr int TILE = 16;

// row-major element of op(A) (m x k): A is m x k (ta = 0) or k x m (ta = 1)
template <class T>
__device__ __forceinline__ T at(const T* A, int lda, int r, int c, int trans) {
  return trans ? A[(size_t)c * lda + r] : A[(size_t)r * lda + c];
}

template <class T>
__global__ void k_gemm(int m, int n, int k, T alpha, const T* __restrict__ A, int lda, int ta,
                       const T* __restrict__ B, int ldb, int tb, T beta, T* __restrict__ C, int ldc) {
  __shared__ T As[TILE][TILE + 1];
  __shared__ T Bs[TILE][TILE + 1];
  const int r = blockIdx.y * TILE + threadIdx.y;
  const int c = blockIdx.x * TILE + threadIdx.x;
  T acc = T(0);
  for (int k0 = 0; k0 < k; k0 += TILE) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    As[threadIdx.y][threadIdx.x] = (r < m && ka < k) ? at(A, lda, r, ka, ta) : T(0);
    Bs[threadIdx.y][threadIdx.x] = (kb < k && c < n) ? at(B, ldb, kb, c, tb) : T(0);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < TILE; ++t) acc += As[threadIdx.y][t] * Bs[t][threadIdx.x];
    __syncthreads();
  }
  if (r < m && c < n) {
    T* out = C + (size_t)r * ldc + c;
    *out = alpha * acc + (beta != T(0) ? beta * *out : T(0));
  }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  // d/dz [z Phi(z)] = Phi(z) + z phi(z)
  const float Phi = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float phi = 0.39894228040143268f * expf(-0.5f * z * z);
  return Phi + z * phi;
}

// Z[r, c] += b[c]; H = gelu(Z) (act = 1) or H = Z (act = 0)
__global__ void k_bias_act(int rows, int cols, float* Z, const float* b, float* H, int act) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const float z = Z[i] + b[i % cols];
  Z[i] = z;
  H[i] = act ? gelu(z) : z;
}

// dZ = dH * gelu'(Z)
__global__ void k_gelu_back(int n, const float* Z, const float* dH, float* dZ) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dZ[i] = dH[i] * gelu_grad(Z[i]);
}

// db[c] = sum_r dZ[r, c]  (one thread per column, fixed order)
__global__ void k_colsum32(int rows, int cols, const float* dZ, float* db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.0f;
  for (int r = 0; r < rows; ++r) s += dZ[(size_t)r * cols + c];
  db[c] = s;
}

// loss = mean((Y - T)^2) over all entries; dY = 2 (Y - T) / count.  One block.
__global__ void k_mse(int n, const float* Y, const float* Tg, float* dY, float* loss) {
  __shared__ float red[256];
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = Y[i] - Tg[i];
    s += d * d;
    dY[i] = 2.0f * d / (float)n;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / (float)n;
}

__global__ void k_adam(int n, float* w, const float* g, float* m1, float* m2, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi;
  const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = v;
  w[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

// Cyclic Jacobi eigensolver for a symmetric n x n matrix (row-major, n <= 256) in one CTA:
// parallel round-robin ordering (n/2 disjoint rotations per round), rotations applied to
// the working matrix and accumulated into V.  Stops when the off-diagonal Frobenius norm
// is below tol times the Frobenius norm, or after max_sweeps sweeps.
__global__ void __launch_bounds__(256) k_syevj(int n, double* A, double* V, double* w, double tol, int max_sweeps,
                                                int* sweeps_done) {
  __shared__ int pairs[256][2];
  __shared__ double cs[128], sn[128];
  __shared__ double red[256];
  __shared__ int s_done;
  const int tid = threadIdx.x;
  const int m = (n + 1) / 2 * 2;  // even count for the tournament (index n is a dummy)
  for (int i = tid; i < n * n; i += blockDim.x) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncthreads();
  double fro = 0.0;
  for (int i = tid; i < n * n; i += blockDim.x) fro += A[i] * A[i];
  red[tid] = fro;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  const double fro_all = sqrt(red[0]);
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int i = tid; i < n * n; i += blockDim.x)
      if (i / n != i % n) off += A[i] * A[i];
    red[tid] = off;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (tid < o) red[tid] += red[tid + o];
      __syncthreads();
    }
    if (tid == 0) s_done = sqrt(red[0]) <= tol * fro_all ? 1 : 0;
    __syncthreads();
    if (s_done) break;
    for (int round = 0; round < m - 1; ++round) {
      // round-robin pairing: position 0 fixed, the others rotate
      if (tid < m / 2) {
        int a = tid == 0 ? 0 : 1 + (tid - 1 + round) % (m - 1);
        int b = 1 + (m - 2 - tid + round) % (m - 1);
        if (a > b) {
          int t = a;
          a = b;
          b = t;
        }
        pairs[tid][0] = a;
        pairs[tid][1] = b;
      }
      __syncthreads();
      if (tid < m / 2) {
        const int p = pairs[tid][0], q = pairs[tid][1];
        double c = 1.0, s = 0.0;
        if (q < n && p != q) {
          const double apq = A[(size_t)p * n + q];
          if (apq != 0.0) {
            const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J (J rotates columns p, q)
      for (int idx = tid; idx < (m / 2) * n; idx += blockDim.x) {
        const int pr = idx / n, r = idx % n;
        const int p = pairs[pr][0], q = pairs[pr][1];
        if (q >= n) continue;
        const double c = cs[pr], s = sn[pr];
        const double ap = A[(size_t)r * n + p], aq = A[(size_t)r * n + q];
        A[(size_t)r * n + p] = c * ap - s * aq;
        A[(size_t)r * n + q] = s * ap + c * aq;
        const double vp = V[(size_t)r * n + p], vq = V[(size_t)r * n + q];
        V[(size_t)r * n + p] = c * vp - s * vq;
        V[(size_t)r * n + q] = s * vp + c * vq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = tid; idx < (m / 2) * n; idx += blockDim.x) {
        const int pr = idx / n, col = idx % n;
        const int p = pairs[pr][0], q = pairs[pr][1];
        if (q >= n) continue;
        const double c = cs[pr], s = sn[pr];
        const double ap = A[(size_t)p * n + col], aq = A[(size_t)q * n + col];
        A[(size_t)p * n + col] = c * ap - s * aq;
        A[(size_t)q * n + col] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < n; i += blockDim.x) w[i] = A[(size_t)i * n + i];
  if (tid == 0 && sweeps_done) *sweeps_done = sweep;
}

// ---- multi-CTA cyclic Jacobi for n > 256 (same ordering and rotations as k_syevj).
// Round r of the round-robin tournament pairs the m = n (+1 if odd) indices into m/2
// disjoint (p, q).  Columns phase: one CTA per pair computes the pair's rotation from
// A_pp, A_qq, A_pq -- entries of columns p and q, which only this CTA changes in this
// phase -- then rotates columns p, q of A and V over all rows.  Rows phase: one CTA per
// pair rotates rows p, q of A with the stored rotation.
__device__ __forceinline__ void round_pair(int m, int round, int pr, int& p, int& q) {
  int a = pr == 0 ? 0 : 1 + (pr - 1 + round) % (m - 1);
  int b = 1 + (m - 2 - pr + round) % (m - 1);
  p = a < b ? a : b;
  q = a < b ? b : a;
}

__global__ void __launch_bounds__(512) k_jacobi_cols(int n, int m, int round, double* A, double* V, double* cs,
                                                     double* sn) {
  const int pr = blockIdx.x;
  int p, q;
  round_pair(m, round, pr, p, q);
  __shared__ double s_c, s_s;
  if (threadIdx.x == 0) {
    double c = 1.0, s = 0.0;
    if (q < n) {
      const double apq = A[(size_t)p * n + q];
      if (apq != 0.0) {
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        c = 1.0 / sqrt(1.0 + t * t);
        s = t * c;
      }
    }
    s_c = c;
    s_s = s;
    cs[pr] = c;
    sn[pr] = s;
  }
  __syncthreads();
  if (q >= n) return;
  const double c = s_c, s = s_s;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double ap = A[(size_t)r * n + p], aq = A[(size_t)r * n + q];
    A[(size_t)r * n + p] = c * ap - s * aq;
    A[(size_t)r * n + q] = s * ap + c * aq;
    const double vp = V[(size_t)r * n + p], vq = V[(size_t)r * n + q];
    V[(size_t)r * n + p] = c * vp - s * vq;
    V[(size_t)r * n + q] = s * vp + c * vq;
  }
}

__global__ void __launch_bounds__(512) k_jacobi_rows(int n, int m, int round, double* A, const double* cs,
                                                     const double* sn) {
  const int pr = blockIdx.x;
  int p, q;
  round_pair(m, round, pr, p, q);
  if (q >= n) return;
  const double c = cs[pr], s = sn[pr];
  for (int col = threadIdx.x; col < n; col += blockDim.x) {
    const double ap = A[(size_t)p * n + col], aq = A[(size_t)q * n + col];
    A[(size_t)p * n + col] = c * ap - s * aq;
    A[(size_t)q * n + col] = s * ap + c * aq;
  }
}

// out[0] = off-diagonal sum of squares, out[1] = Frobenius sum of squares (one CTA, fixed order)
__global__ void __launch_bounds__(1024) k_jacobi_norms(int n, const double* A, double* out) {
  __shared__ double r0[1024], r1[1024];
  double off = 0.0, all = 0.0;
  for (int64_t i = threadIdx.x; i < (int64_t)n * n; i += blockDim.x) {
    const double a = A[i];
    all += a * a;
    if (i / n != i % n) off += a * a;
  }
  r0[threadIdx.x] = off;
  r1[threadIdx.x] = all;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o];
      r1[threadIdx.x] += r1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = r0[0];
    out[1] = r1[0];
  }
}

__global__ void k_jacobi_finish(int n, const double* A, double* w, int* sweeps, int sw) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) w[i] = A[(size_t)i * n + i];
  if (sweeps && blockIdx.x == 0 && threadIdx.x == 0) *sweeps = sw;
}

__global__ void k_identity(int n, double* V) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n * n; i += (int64_t)gridDim.x * blockDim.x)
    V[i] = (i / n == i % n) ? 1.0 : 0.0;
}

int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

extern "C" {

int pp_gemm_f32(int m, int n, int k, float alpha, const float* A, int lda, int ta, const float* B, int ldb, int tb,
                float beta, float* C, int ldc, void* stream) {
  if (m <= 0 || n <= 0 || k <= 0 || !A || !B || !C) return PP_LEARN_EINVAL;
  pp::ProfScope ps(PP_K_OTHER, (cudaStream_t)stream);
  dim3 grid((n + TILE - 1) / TILE, (m + TILE - 1) / TILE), block(TILE, TILE);
  k_gemm<float><<<grid, block, 0, (cudaStream_t)stream>>>(m, n, k, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc);
  return cudaGetLastError() == cudaSuccess ? 0 : PP_LEARN_ECUDA;
}

int pp_gemm_f64(int m, int n, int k, double alpha, const double* A, int lda, int ta, const double* B, int ldb, int tb,
                double beta, double* C, int ldc, void* stream) {
  if (m <= 0 || n <= 0 || k <= 0 || !A || !B || !C) return PP_LEARN_EINVAL;
  pp::ProfScope ps(PP_K_OTHER, (cudaStream_t)stream);
  dim3 grid((n + TILE - 1) / TILE, (m + TILE - 1) / TILE), block(TILE, TILE);
  k_gemm<double><<<grid, block, 0, (cudaStream_t)stream>>>(m, n, k, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc);
  return cudaGetLastError() == cudaSuccess ? 0 : PP_LEARN_ECUDA;
}

int pp_bias_act_f32(int rows, int cols, float* Z, const float* b, float* H, int gelu_on, void* stream) {
  if (rows <= 0 || cols <= 0) return PP_LEARN_EINVAL;
  pp::ProfScope ps(PP_K_OTHER, (cudaStream_t)stream);
  k_bias_act<<<blocks_for((int64_t)rows * cols, 256), 256, 0, (cudaStream_t)stream>>>(rows, cols, Z, b, H, gelu_on);
  return cudaGetLastError() == cudaSuccess ? 0 : PP_LEARN_ECUDA;
}

int pp_gelu_backward_f32(int n, const float* Z, const float* dH, float* dZ, void* stream) {
  if (n <= 0) return PP_LEARN_EINVAL;
  pp::ProfScope ps(PP_K_OTHER, (cudaStream_t)stream);
  k_gelu_back<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, Z, dH, dZ);
  return cudaGetLastError() == cudaSuccess ? 0 : PP_LEARN_ECUDA;
}

int pp_colsum_f32(int rows, int cols, const float* dZ, float* db, void* stream) {
  if (rows <= 0 || cols <= 0) return PP_LEARN_EINVAL;
  pp::ProfScope ps(PP_K_OTHER, (cudaStream_t)stream);
  k_colsum32<<<blocks_for(cols, 128), 128, 0, (cudaStream_t)stream>>>(rows, cols, dZ, db);
  return cudaGetLastError() == cudaSuccess ? 0 : PP_LEARN_ECUDA;
}

int pp_mse_f32(int n, const float* Y, const float* Tg, float* dY, float* loss, void* stream) {
  if (n <= 0) return PP_LEARN_EINVAL;
  pp::ProfScope ps(PP_K_OTHER, (cudaStream_t)stream);
  k_mse<<<1, 256, 0, (cudaStream_t)stream>>>(n, Y, Tg, dY, loss);
  return cudaGetLastError() == cudaSuccess ? 0 : PP_LEARN_ECUDA;
}

int pp_adam_f32(int n, float* w, const float* g, float* m1, float* m2, float lr, float b1, float b2, float eps,
                int step, void* stream) {
  if (n <= 0 || step < 1) return PP_LEARN_EINVAL;
  pp::ProfScope ps(PP_K_OTHER, (cudaStream_t)stream);
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, w, g, m1, m2, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? 0 : PP_LEARN_ECUDA;
}

int pp_syevj_f64(int n, double* A, double* V, double* w, double tol, int max_sweeps, int* sweeps, void* stream) {
  using namespace pp;
  if (n <= 0 || n > 4096 || !A || !V || !w) return PP_LEARN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (n <= 256) {
    ProfScope ps(PP_K_OTHER, st);
    k_syevj<<<1, 256, 0, st>>>(n, A, V, w, tol, max_sweeps, sweeps);
    return cudaGetLastError() == cudaSuccess ? 0 : PP_LEARN_ECUDA;
  }
  // multi-CTA sweeps, the convergence test on the host once per sweep
  const int m = (n + 1) / 2 * 2;
  double* scratch = nullptr;  // cs [m/2] | sn [m/2] | norms [2]
  if (cudaMalloc(&scratch, sizeof(double) * (m + 2)) != cudaSuccess) return PP_LEARN_ECUDA;
  double* cs = scratch;
  double* sn = scratch + m / 2;
  double* nrm = scratch + m;
  double h[2] = {0.0, 0.0};
  int sweep = 0, rc = 0;
  {
    ProfScope ps(PP_K_OTHER, st);
    k_identity<<<blocks_for((int64_t)n * n, 256), 256, 0, st>>>(n, V);
  }
  for (;; ++sweep) {
    {
      ProfScope ps(PP_K_OTHER, st);
      k_jacobi_norms<<<1, 1024, 0, st>>>(n, A, nrm);
    }
    if (cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = PP_LEARN_ECUDA;
      break;
    }
    if (sweep >= max_sweeps || sqrt(h[0]) <= tol * sqrt(h[1])) break;
    for (int round = 0; round < m - 1; ++round) {
      {
        ProfScope ps(PP_K_OTHER, st);
        k_jacobi_cols<<<m / 2, 512, 0, st>>>(n, m, round, A, V, cs, sn);
      }
      ProfScope ps(PP_K_OTHER, st);
      k_jacobi_rows<<<m / 2, 512, 0, st>>>(n, m, round, A, cs, sn);
    }
    if (cudaGetLastError() != cudaSuccess) {
      rc = PP_LEARN_ECUDA;
      break;
    }
  }
  if (rc == 0) {
    ProfScope ps(PP_K_OTHER, st);
    k_jacobi_finish<<<blocks_for(n, 256), 256, 0, st>>>(n, A, w, sweeps, sweep);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = PP_LEARN_ECUDA;
  }
  cudaFree(scratch);
  return rc;
}

}  // extern "C"
