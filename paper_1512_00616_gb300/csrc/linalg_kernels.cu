// Batched element-block linear algebra and Krylov vector kernels (FP64).
//
//  - k_block_inverse: A_e = detB_e Mref (x) I4 - c J_ee, the diagonal block of
//    the DIRK stage matrix M - a_ii dt dr/du, inverted in shared memory by
//    Gauss-Jordan elimination with partial pivoting.  The inverse is the
//    block-Jacobi preconditioner of the stage solves; stored explicitly so that
//    each application (normal for the primal and tangent sweeps, transposed for
//    the adjoint sweep, Eq. uns-disc-adj-dirk2) is one dense block matvec
//    streamed from HBM instead of two dependent triangular solves.
//  - k_stage_matvec: y = alpha M x + beta J x (or beta J^T x) over the block-
//    sparse element Jacobian (diagonal + 3 face-neighbour blocks).
//  - Krylov vector kernels: fused multi-dot products with a deterministic
//    two-level reduction (per-block partials, summed in block order by the
//    last block to finish), used by the classical Gram-Schmidt (twice) Arnoldi.
#include "pp_internal.h"
#include "prof.h"
#include "../../include/pp_prof.h"

namespace pp {

namespace {

constexpr int INV_THREADS = 256;
constexpr int MV_WARPS = 4;
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs
constexpr int kChunk = 4;

__global__ void __launch_bounds__(INV_THREADS)
    k_block_inverse(DevMesh m, DevTables tb, const double* __restrict__ J, double c, double* __restrict__ Ainv,
                    int* status) {
  __shared__ double A[kMaxNb][kMaxNb + 1];
  __shared__ double colk[kMaxNb];
  __shared__ int piv[kMaxNb];
  __shared__ int s_p;
  const int e = blockIdx.x, tid = threadIdx.x;
  const int nb = tb.nb, Np = tb.Np;
  const size_t nb2 = (size_t)nb * nb;
  const double* Je = J + (size_t)e * 4 * nb2;  // diagonal slot
  const double detB = m.detB[e];
  for (int ent = tid; ent < nb * nb; ent += INV_THREADS) {
    int col = ent / nb, row = ent - col * nb;
    int a = row / Np, i = row - a * Np, b = col / Np, j = col - b * Np;
    double mass = (a == b) ? detB * tb.Mref[i * Np + j] : 0.0;
    A[row][col] = mass - c * Je[ent];
  }
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < nb; i += 32) {
        double v = fabs(A[i][k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        s_p = bi;
        piv[k] = bi;
        if (!(best > 0.0) || !isfinite(best)) atomicOr(status, 1);
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
      for (int j = tid; j < nb; j += INV_THREADS) {
        double t = A[k][j];
        A[k][j] = A[p][j];
        A[p][j] = t;
      }
    __syncthreads();
    const double pinv = 1.0 / A[k][k];
    __syncthreads();
    if (tid == 0) A[k][k] = 1.0;
    __syncthreads();
    for (int j = tid; j < nb; j += INV_THREADS) A[k][j] *= pinv;
    for (int i = tid; i < nb; i += INV_THREADS) colk[i] = A[i][k];
    __syncthreads();
    for (int ent = tid; ent < nb * nb; ent += INV_THREADS) {
      int i = ent / nb, j = ent - i * nb;
      if (i == k) continue;
      double f = colk[i];
      double v = (j == k) ? 0.0 : A[i][j];
      A[i][j] = v - f * A[k][j];
    }
    __syncthreads();
  }
  // undo the row pivoting: inverse(P A) * P, P = S_{nb-1} ... S_0 -> swap columns k, piv[k] for k descending
  for (int i = tid; i < nb; i += INV_THREADS) {
    for (int k = nb - 1; k >= 0; --k) {
      int p = piv[k];
      if (p != k) {
        double t = A[i][k];
        A[i][k] = A[i][p];
        A[i][p] = t;
      }
    }
  }
  __syncthreads();
  double* out = Ainv + (size_t)e * nb2;
  for (int ent = tid; ent < nb * nb; ent += INV_THREADS) {
    int col = ent / nb, row = ent - col * nb;
    out[ent] = A[row][col];
  }
}

// y_e = alpha M_e x_e + beta (J x)_e  or  beta (J^T x)_e
__global__ void __launch_bounds__(MV_WARPS * 32)
    k_stage_matvec(DevMesh m, DevTables tb, const double* __restrict__ J, double alpha, double beta,
                   const double* __restrict__ x, double* __restrict__ y, int trans) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * MV_WARPS + warp;
  if (e >= m.ne) return;
  const int nb = tb.nb, Np = tb.Np;
  const size_t nb2 = (size_t)nb * nb;
  const double* xe = x + (size_t)e * nb;
  for (int r = lane; r < nb; r += 32) {
    double acc = 0.0;
    if (alpha != 0.0) {
      int a = r / Np, i = r - a * Np;
      double s = 0.0;
      for (int j = 0; j < Np; ++j) s += tb.Mref[i * Np + j] * xe[a * Np + j];
      acc = alpha * m.detB[e] * s;
    }
    if (beta != 0.0) {
      double s = 0.0;
      if (!trans) {
        for (int slot = 0; slot < 4; ++slot) {
          int src = e;
          if (slot > 0) {
            src = m.nbr[3 * e + slot - 1];
            if (src < 0) continue;
          }
          const double* Jb = J + ((size_t)e * 4 + slot) * nb2 + r;
          const double* xs = x + (size_t)src * nb;
          for (int cc = 0; cc < nb; ++cc) s += Jb[(size_t)cc * nb] * xs[cc];
        }
      } else {
        const double* Jb = J + ((size_t)e * 4) * nb2 + (size_t)r * nb;
        for (int cc = 0; cc < nb; ++cc) s += Jb[cc] * xe[cc];
        for (int f = 0; f < 3; ++f) {
          int e2 = m.nbr[3 * e + f];
          if (e2 < 0) continue;
          int g = m.nbrface[3 * e + f];
          const double* J2 = J + ((size_t)e2 * 4 + 1 + g) * nb2 + (size_t)r * nb;
          const double* x2 = x + (size_t)e2 * nb;
          for (int cc = 0; cc < nb; ++cc) s += J2[cc] * x2[cc];
        }
      }
      acc += beta * s;
    }
    y[(size_t)e * nb + r] = acc;
  }
}

__global__ void __launch_bounds__(MV_WARPS * 32)
    k_block_apply(int ne, int nb, const double* __restrict__ Ainv, const double* __restrict__ x,
                  double* __restrict__ y, int trans) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * MV_WARPS + warp;
  if (e >= ne) return;
  const size_t nb2 = (size_t)nb * nb;
  const double* A = Ainv + (size_t)e * nb2;
  const double* xe = x + (size_t)e * nb;
  double acc[2] = {0.0, 0.0};
  if (!trans) {
    for (int cc = 0; cc < nb; ++cc) {
      double xc = xe[cc];
      if (lane < nb) acc[0] += A[(size_t)cc * nb + lane] * xc;
      if (lane + 32 < nb) acc[1] += A[(size_t)cc * nb + lane + 32] * xc;
    }
  } else {
    for (int h = 0; h < 2; ++h) {
      int r = lane + 32 * h;
      if (r >= nb) break;
      const double* Ar = A + (size_t)r * nb;
      double s = 0.0;
      for (int cc = 0; cc < nb; ++cc) s += Ar[cc] * xe[cc];
      acc[h] = s;
    }
  }
  __syncwarp();
  if (lane < nb) y[(size_t)e * nb + lane] = acc[0];
  if (lane + 32 < nb) y[(size_t)e * nb + lane + 32] = acc[1];
}

__global__ void k_lincomb(int64_t n, double* y, int nterms, double c0, double c1, double c2, double c3,
                          const double* x0, const double* x1, const double* x2, const double* x3) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = c0 * x0[i];
    if (nterms > 1) s += c1 * x1[i];
    if (nterms > 2) s += c2 * x2[i];
    if (nterms > 3) s += c3 * x3[i];
    y[i] = s;
  }
}

__global__ void k_scale(int64_t n, double* y, double a, const double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// block-wide sum of k <= kChunk values; result valid in thread 0
__device__ __forceinline__ void block_sum(double* v, int k, double (*sh)[RED_THREADS / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < k; ++j) {
    double s = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sh[j][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int w = 0; w < RED_THREADS / 32; ++w) s += sh[j][w];
      v[j] = s;
    }
  __syncthreads();
}

// last-block finalisation: out[j] = sum_b partial[b*k + j] in block order
__device__ __forceinline__ void finish(int k, double* partial, unsigned* counter, double* out) {
  __shared__ bool last;
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) s += ((volatile double*)partial)[(size_t)b * k + j];
    out[j] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// mode 0: out = V^T w;  mode 1: w -= V h, out = V^T w;  mode 2: w -= V h, out[0] = w.w;  mode 3: out[0] = V_0 . w
__global__ void __launch_bounds__(RED_THREADS)
    k_krylov(int mode, int64_t n, const double* __restrict__ V, int64_t ldv, int k, const double* __restrict__ h,
             double* __restrict__ w, double* __restrict__ out, double* __restrict__ partial, unsigned* counter) {
  __shared__ double sh[kChunk][RED_THREADS / 32];
  const int64_t stride = (int64_t)gridDim.x * RED_THREADS;
  const int64_t i0 = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x;
  if (mode == 1 || mode == 2) {
    for (int64_t i = i0; i < n; i += stride) {
      double s = w[i];
      for (int j = 0; j < k; ++j) s -= h[j] * V[j * ldv + i];
      w[i] = s;
    }
  }
  const int nout = (mode == 2 || mode == 3) ? 1 : k;
  for (int j0 = 0; j0 < nout; j0 += kChunk) {
    int kc = min(kChunk, nout - j0);
    double acc[kChunk] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = i0; i < n; i += stride) {
      double wi = w[i];
      if (mode == 2) {
        acc[0] += wi * wi;
      } else {
        for (int j = 0; j < kc; ++j) acc[j] += V[(j0 + j) * ldv + i] * wi;
      }
    }
    block_sum(acc, kc, sh);
    if (threadIdx.x == 0)
      for (int j = 0; j < kc; ++j) partial[(size_t)blockIdx.x * nout + j0 + j] = acc[j];
  }
  finish(nout, partial, counter, out);
}

// out[j] = sum_e per_elem[e*k + j]
__global__ void __launch_bounds__(RED_THREADS)
    k_colsum(int ne, int k, const double* __restrict__ pe, double* out, double* partial, unsigned* counter) {
  __shared__ double sh[kChunk][RED_THREADS / 32];
  for (int j0 = 0; j0 < k; j0 += kChunk) {
    int kc = min(kChunk, k - j0);
    double acc[kChunk] = {0.0, 0.0, 0.0, 0.0};
    for (int e = blockIdx.x * RED_THREADS + threadIdx.x; e < ne; e += gridDim.x * RED_THREADS)
      for (int j = 0; j < kc; ++j) acc[j] += pe[(size_t)e * k + j0 + j];
    block_sum(acc, kc, sh);
    if (threadIdx.x == 0)
      for (int j = 0; j < kc; ++j) partial[(size_t)blockIdx.x * k + j0 + j] = acc[j];
  }
  finish(k, partial, counter, out);
}

int vec_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 4 * 152 ? (b < 1 ? 1 : b) : 4 * 152);
}

int red_blocks(int64_t n) {
  int64_t b = (n + RED_THREADS - 1) / RED_THREADS;
  return (int)(b < RED_BLOCKS ? (b < 1 ? 1 : b) : RED_BLOCKS);
}

}  // namespace

int reduction_blocks() { return RED_BLOCKS; }

cudaError_t launch_block_inverse(const DevMesh& m, const DevTables& tb, const double* J, double c, double* Ainv,
                                 int* status, cudaStream_t st) {
  ProfScope ps(PP_K_BLOCK_INVERSE, st);
  k_block_inverse<<<m.ne, INV_THREADS, 0, st>>>(m, tb, J, c, Ainv, status);
  return cudaGetLastError();
}

cudaError_t launch_stage_matvec(const DevMesh& m, const DevTables& tb, const double* J, double alpha, double beta,
                                const double* x, double* y, int trans, cudaStream_t st) {
  ProfScope ps(PP_K_STAGE_MATVEC, st);
  k_stage_matvec<<<(m.ne + MV_WARPS - 1) / MV_WARPS, MV_WARPS * 32, 0, st>>>(m, tb, J, alpha, beta, x, y, trans);
  return cudaGetLastError();
}

cudaError_t launch_block_apply(const DevMesh& m, int nb, const double* Ainv, const double* x, double* y, int trans,
                               cudaStream_t st) {
  ProfScope ps(PP_K_BLOCK_APPLY, st);
  k_block_apply<<<(m.ne + MV_WARPS - 1) / MV_WARPS, MV_WARPS * 32, 0, st>>>(m.ne, nb, Ainv, x, y, trans);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(int64_t n, double* y, int nterms, const double* c, const double* const* x,
                           cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_lincomb<<<vec_blocks(n), 256, 0, st>>>(n, y, nterms, c[0], nterms > 1 ? c[1] : 0.0, nterms > 2 ? c[2] : 0.0,
                                           nterms > 3 ? c[3] : 0.0, x[0], nterms > 1 ? x[1] : nullptr,
                                           nterms > 2 ? x[2] : nullptr, nterms > 3 ? x[3] : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_scale(int64_t n, double* y, double a, const double* x, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_scale<<<vec_blocks(n), 256, 0, st>>>(n, y, a, x);
  return cudaGetLastError();
}

cudaError_t launch_mdot(int64_t n, const double* V, int64_t ldv, int k, const double* w, double* out,
                        double* partial, unsigned* counter, cudaStream_t st) {
  ProfScope ps(PP_K_KRYLOV, st);
  k_krylov<<<red_blocks(n), RED_THREADS, 0, st>>>(0, n, V, ldv, k, nullptr, const_cast<double*>(w), out, partial,
                                                  counter);
  return cudaGetLastError();
}

cudaError_t launch_update_mdot(int64_t n, const double* V, int64_t ldv, int k, const double* h, double* w,
                               double* out, double* partial, unsigned* counter, cudaStream_t st) {
  ProfScope ps(PP_K_KRYLOV, st);
  k_krylov<<<red_blocks(n), RED_THREADS, 0, st>>>(1, n, V, ldv, k, h, w, out, partial, counter);
  return cudaGetLastError();
}

cudaError_t launch_update_norm2(int64_t n, const double* V, int64_t ldv, int k, const double* h, double* w,
                                double* out, double* partial, unsigned* counter, cudaStream_t st) {
  ProfScope ps(PP_K_KRYLOV, st);
  k_krylov<<<red_blocks(n), RED_THREADS, 0, st>>>(2, n, V, ldv, k, h, w, out, partial, counter);
  return cudaGetLastError();
}

cudaError_t launch_dot(int64_t n, const double* x, const double* y, double* out, double* partial,
                       unsigned* counter, cudaStream_t st) {
  ProfScope ps(PP_K_KRYLOV, st);
  k_krylov<<<red_blocks(n), RED_THREADS, 0, st>>>(3, n, x, 0, 1, nullptr, const_cast<double*>(y), out, partial,
                                                  counter);
  return cudaGetLastError();
}

cudaError_t launch_colsum(int ne, int k, const double* per_elem, double* out, double* partial, unsigned* counter,
                          cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_colsum<<<red_blocks(ne), RED_THREADS, 0, st>>>(ne, k, per_elem, out, partial, counter);
  return cudaGetLastError();
}

}  // namespace pp
