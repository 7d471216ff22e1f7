// Batched element-block linear algebra and Krylov vector kernels, templated on the
// storage/arithmetic type S (double for the FP64 path, float for the inner solves of
// the mixed-precision path).
//
//  - k_block_inverse<S>: A_e = detB_e Mref (x) I4 - c J_ee (the diagonal block of the
//    DIRK stage matrix M - a_ii dt dr/du, assembled in FP64) inverted in shared memory
//    by Gauss-Jordan elimination with partial pivoting in precision S.  The inverse is
//    the block-Jacobi preconditioner of the stage solves; it is stored explicitly (and
//    transposed) so that every application, normal for the primal / tangent sweeps and
//    transposed for the adjoint sweep (Eq. uns-disc-adj-dirk2), is one dense block
//    matvec streamed from HBM.
//  - k_stage_matvec<S>: y = alpha M x + beta J x (or J^T x) over the block-sparse
//    element Jacobian (diagonal + 3 face-neighbour blocks).
//  - k_transpose_blocks: per element, the transposed blocks of its block-column, so
//    that J^T x runs through the same row-streaming kernel as J x.
//  - k_cgs<KB, S>: fused classical Gram-Schmidt passes of the Arnoldi step (a second pass
//    only when the first cancels more than half of |w|^2), with a deterministic
//    reduction (warp, CTA, then the CTA that finishes last in a fixed order), and the
//    GMRES Givens update fused into the norm pass.
//
// GB300 note: its FP64 pipe issues ~2 DFMA per clock per SM, so FP64 block products are
// ALU-bound (~21 us for the 4 x 40 x 40 x 2048 Jacobian product) before they are
// HBM-bound; the same products in FP32 are bandwidth-bound.
#include "pp_internal.h"
#include "prof.h"
#include "../../include/pp_prof.h"

namespace pp {

namespace {

constexpr int INV_THREADS = 256;
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 152;  // one block per SM keeps the finishing reduction short

// ------------------------------------------------------------------ block inverse
template <class S>
__global__ void __launch_bounds__(INV_THREADS)
    k_block_inverse(DevMesh m, DevTables tb, const double* __restrict__ J, double c, S* __restrict__ Ainv,
                    S* __restrict__ AinvT, int* status) {
  __shared__ S A[kMaxNb][kMaxNb + 1];
  __shared__ S colk[kMaxNb];
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
    A[row][col] = S(mass - c * Je[ent]);
  }
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (tid < 32) {
      S best = S(-1);
      int bi = k;
      for (int i = k + tid; i < nb; i += 32) {
        S v = fabs(A[i][k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        S ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        s_p = bi;
        piv[k] = bi;
        if (!(best > S(0)) || !isfinite((double)best)) atomicOr(status, 1);
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
      for (int j = tid; j < nb; j += INV_THREADS) {
        S t = A[k][j];
        A[k][j] = A[p][j];
        A[p][j] = t;
      }
    __syncthreads();
    const S pinv = S(1) / A[k][k];
    __syncthreads();
    if (tid == 0) A[k][k] = S(1);
    __syncthreads();
    for (int j = tid; j < nb; j += INV_THREADS) A[k][j] *= pinv;
    for (int i = tid; i < nb; i += INV_THREADS) colk[i] = A[i][k];
    __syncthreads();
    for (int ent = tid; ent < nb * nb; ent += INV_THREADS) {
      int i = ent / nb, j = ent - i * nb;
      if (i == k) continue;
      S f = colk[i];
      S v = (j == k) ? S(0) : A[i][j];
      A[i][j] = v - f * A[k][j];
    }
    __syncthreads();
  }
  // undo the row pivoting: inverse(P A) * P, P = S_{nb-1} ... S_0 -> swap columns k, piv[k] for k descending
  for (int i = tid; i < nb; i += INV_THREADS) {
    for (int k = nb - 1; k >= 0; --k) {
      int p = piv[k];
      if (p != k) {
        S t = A[i][k];
        A[i][k] = A[i][p];
        A[i][p] = t;
      }
    }
  }
  __syncthreads();
  S* out = Ainv + (size_t)e * nb2;
  S* outT = AinvT ? AinvT + (size_t)e * nb2 : nullptr;
  for (int ent = tid; ent < nb * nb; ent += INV_THREADS) {
    int col = ent / nb, row = ent - col * nb;
    out[ent] = A[row][col];
    if (outT) outT[ent] = A[col][row];
  }
}

// ------------------------------------------------------------------ warp reduce-scatter
template <int CNT, int O, class T>
__device__ __forceinline__ void rs_step(T* v, int lane) {
  if constexpr (O > 0) {
    if constexpr (CNT > 1) {
      constexpr int half = CNT / 2;
      const bool upper = (lane & O) != 0;
#pragma unroll
      for (int t = 0; t < half; ++t) {
        const T send = upper ? v[t] : v[t + half];
        const T keep = upper ? v[t + half] : v[t];
        v[t] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      rs_step<half, O / 2, T>(v, lane);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
      rs_step<1, O / 2, T>(v, lane);
    }
  }
}

// Warp reduce-scatter of KB (power of two, <= 32) per-lane values: afterwards lane l
// holds the warp sum of value (l >> (5 - log2 KB)) in v[0] (31 shuffles for KB = 32).
template <int KB, class T>
__device__ __forceinline__ void warp_reduce_scatter(T* v, int lane) {
  rs_step<KB, 16, T>(v, lane);
}

template <int KB>
struct ILog2 {
  static constexpr int value = KB >= 32 ? 5 : KB >= 16 ? 4 : KB >= 8 ? 3 : KB >= 4 ? 2 : KB >= 2 ? 1 : 0;
};

// ------------------------------------------------------------------ block products
// Warp-per-block products with compile-time block size NB = 4 Np.  Normal: lanes over
// rows, the input values read with warp-uniform loads into registers, columns streamed
// (column-major, coalesced).  Transposed: output r is the dot product of the contiguous
// column r with the input, so lanes run over the column and a reduce-scatter across the
// warp delivers 32 outputs at a time.
template <int NB, class S>
struct BlockOps {
  static constexpr int H = (NB + 31) / 32;

  __device__ static __forceinline__ void load(const S* x, int lane, S xr[H]) {
#pragma unroll
    for (int h = 0; h < H; ++h) xr[h] = (lane + 32 * h < NB) ? x[lane + 32 * h] : S(0);
  }

  __device__ static __forceinline__ void mv_x(const S* __restrict__ B, const S* __restrict__ x, int lane,
                                              S acc[H]) {
    S xc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) xc[c] = __ldg(x + c);
#pragma unroll
    for (int c = 0; c < NB; ++c) {
#pragma unroll
      for (int h = 0; h < H; ++h)
        if (lane + 32 * h < NB) acc[h] += __ldg(B + (size_t)c * NB + lane + 32 * h) * xc[c];
    }
  }

  template <int NQ>
  __device__ static __forceinline__ void mvt(const S* const (&Bq)[NQ], const S (&xq)[NQ][H], int lane, S out[H]) {
#pragma unroll
    for (int b = 0; b < H; ++b) {
      constexpr int KB = 32;
      S acc[KB];
#pragma unroll
      for (int t = 0; t < KB; ++t) acc[t] = S(0);
      const int r0 = 32 * b;
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        if (r0 + t < NB) {
          S part = S(0);
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            if (!Bq[q]) continue;
            const S* col = Bq[q] + (size_t)(r0 + t) * NB;
#pragma unroll
            for (int h = 0; h < H; ++h)
              if (lane + 32 * h < NB) part += col[lane + 32 * h] * xq[q][h];
          }
          acc[t] = part;
        }
      }
      warp_reduce_scatter<KB, S>(acc, lane);
      out[b] = acc[0];
    }
  }
};

// One CTA (4 warps) per element; warp q handles block q of the element row (q = 0 the
// diagonal block, q = 1..3 the face neighbours); the 4 partial rows meet in shared memory.
template <int NB, bool TRANS, class S>
__global__ void __launch_bounds__(128)
    k_stage_matvec(DevMesh m, DevTables tb, const S* __restrict__ J, double alpha, double beta,
                   const S* __restrict__ x, S* __restrict__ y) {
  using Ops = BlockOps<NB, S>;
  constexpr int H = Ops::H;
  constexpr size_t nb2 = (size_t)NB * NB;
  __shared__ S part[4][NB];
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x;
  S s[H];
#pragma unroll
  for (int h = 0; h < H; ++h) s[h] = S(0);
  if (beta != 0.0) {
    const S* B = nullptr;
    const S* xs = x + (size_t)e * NB;
    if (q == 0) {
      B = J + ((size_t)e * 4) * nb2;
    } else {
      const int e2 = m.nbr[3 * e + q - 1];
      if (e2 >= 0) {
        B = TRANS ? J + ((size_t)e2 * 4 + 1 + m.nbrface[3 * e + q - 1]) * nb2 : J + ((size_t)e * 4 + q) * nb2;
        xs = x + (size_t)e2 * NB;
      }
    }
    if (B) {
      if constexpr (!TRANS) {
        Ops::mv_x(B, xs, lane, s);
      } else {
        S xr[H];
        Ops::load(xs, lane, xr);
        const S* Bq[1] = {B};
        S xq[1][H];
#pragma unroll
        for (int h = 0; h < H; ++h) xq[0][h] = xr[h];
        Ops::template mvt<1>(Bq, xq, lane, s);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < H; ++h)
    if (lane + 32 * h < NB) part[q][lane + 32 * h] = S(beta) * s[h];
  __syncthreads();
  const int Np = NB / 4;
  const S* xe = x + (size_t)e * NB;
  for (int r = threadIdx.x; r < NB; r += 128) {
    S acc = part[0][r] + part[1][r] + part[2][r] + part[3][r];
    if (alpha != 0.0) {
      const int a = r / Np, i = r - a * Np;
      S mm = S(0);
      for (int jj = 0; jj < Np; ++jj) mm += S(tb.Mref[i * Np + jj]) * xe[a * Np + jj];
      acc += S(alpha * m.detB[e]) * mm;
    }
    y[(size_t)e * NB + r] = acc;
  }
}

// One CTA (4 warps) per element: normal product with the columns split over the warps,
// transposed product with the outputs split over the warps.
template <int NB, bool TRANS, class S>
__global__ void __launch_bounds__(128)
    k_block_apply(int ne, const S* __restrict__ Ainv, const S* __restrict__ x, S* __restrict__ y) {
  constexpr int H = (NB + 31) / 32;
  constexpr int CW = (NB + 3) / 4;  // columns (or outputs) per warp
  __shared__ S part[4][NB];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x;
  const S* A = Ainv + (size_t)e * NB * NB;
  const S* xe = x + (size_t)e * NB;
  if constexpr (!TRANS) {
    S acc[H];
#pragma unroll
    for (int h = 0; h < H; ++h) acc[h] = S(0);
#pragma unroll
    for (int cc = 0; cc < CW; ++cc) {
      const int c = w * CW + cc;
      if (c < NB) {
        const S xc = __ldg(xe + c);
#pragma unroll
        for (int h = 0; h < H; ++h)
          if (lane + 32 * h < NB) acc[h] += __ldg(A + (size_t)c * NB + lane + 32 * h) * xc;
      }
    }
#pragma unroll
    for (int h = 0; h < H; ++h)
      if (lane + 32 * h < NB) part[w][lane + 32 * h] = acc[h];
  } else {
    S xr[H];
#pragma unroll
    for (int h = 0; h < H; ++h) xr[h] = (lane + 32 * h < NB) ? xe[lane + 32 * h] : S(0);
#pragma unroll
    for (int rr = 0; rr < CW; ++rr) {
      const int r = w * CW + rr;
      S p = S(0);
      if (r < NB) {
        const S* col = A + (size_t)r * NB;
#pragma unroll
        for (int h = 0; h < H; ++h)
          if (lane + 32 * h < NB) p += col[lane + 32 * h] * xr[h];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if (r < NB && lane == 0) part[w][r] = p;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < NB; r += 128)
    y[(size_t)e * NB + r] = TRANS ? part[r / CW][r] : part[0][r] + part[1][r] + part[2][r] + part[3][r];
}

// JT[e][q] = (block of J in block-row src_q(e), block-column e)^T, column-major, so that
// J^T x is the same block-row product as J x with JT in place of J.  q = 0: J_ee;
// q = 1+f: J_{e2,e} = J[e2][1 + nbrface(e,f)], e2 = nbr(e,f); zero on boundary faces.
// One CTA per (element, slot), tile staged in shared memory; the output type may be
// narrower than the input (FP64 -> FP32 copy for the mixed-precision path).
template <class Si, class So>
__global__ void __launch_bounds__(256)
    k_transpose_blocks(DevMesh m, int nb, const Si* __restrict__ J, So* __restrict__ JT) {
  __shared__ Si T[kMaxNb][kMaxNb + 1];
  const int e = blockIdx.x >> 2, q = blockIdx.x & 3;
  const size_t nb2 = (size_t)nb * nb;
  So* dst = JT + ((size_t)e * 4 + q) * nb2;
  const Si* src = nullptr;
  if (q == 0) {
    src = J + ((size_t)e * 4) * nb2;
  } else {
    const int e2 = m.nbr[3 * e + q - 1];
    if (e2 >= 0) src = J + ((size_t)e2 * 4 + 1 + m.nbrface[3 * e + q - 1]) * nb2;
  }
  if (!src) {
    for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) dst[i] = So(0);
    return;
  }
  for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
    const int col = i / nb, row = i - col * nb;
    T[row][col] = src[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
    const int col = i / nb, row = i - col * nb;  // (row, col) of the transpose
    dst[i] = So(T[col][row]);
  }
}

// Preconditioner folded into the stage operator (one CTA per element face, both nb x nb
// operands staged in shared memory, column-major in and out):
//   BN[e][f] = -c J[e][1+f] Ainv[e2]                    e2 = nbr(e, f)
//   BT[e][f] = (-c Ainv[e2] J[e2][1+g])^T              g = nbrface(e, f)
// so that (M - cJ) D^{-1} = I + BN and (M - cJ)^T D^{-T} = I + BT, with D = M - c J_ee the
// block diagonal (Ainv its inverse) and BN, BT zero on boundary faces.
template <int NB, class S>
__global__ void __launch_bounds__(256)
    k_fold_blocks(DevMesh m, const S* __restrict__ J, const S* __restrict__ Ainv, double c, S* __restrict__ BN,
                  S* __restrict__ BT) {
  extern __shared__ __align__(16) unsigned char fsm_raw[];
  S* P = reinterpret_cast<S*>(fsm_raw);
  S* Q = P + NB * NB;
  constexpr int nb2 = NB * NB;
  const int e = blockIdx.x / 3, f = blockIdx.x - 3 * (blockIdx.x / 3);
  const int e2 = m.nbr[3 * e + f];
  S* outN = BN ? BN + ((size_t)e * 3 + f) * nb2 : nullptr;
  S* outT = BT ? BT + ((size_t)e * 3 + f) * nb2 : nullptr;
  if (e2 < 0) {
    for (int i = threadIdx.x; i < nb2; i += blockDim.x) {
      if (outN) outN[i] = S(0);
      if (outT) outT[i] = S(0);
    }
    return;
  }
  for (int pass = 0; pass < 2; ++pass) {
    S* out = pass == 0 ? outN : outT;
    if (!out) continue;
    const S* Pg = pass == 0 ? J + ((size_t)e * 4 + 1 + f) * nb2 : Ainv + (size_t)e2 * nb2;
    const S* Qg = pass == 0 ? Ainv + (size_t)e2 * nb2 : J + ((size_t)e2 * 4 + 1 + m.nbrface[3 * e + f]) * nb2;
    __syncthreads();
    for (int i = threadIdx.x; i < nb2; i += blockDim.x) {
      P[i] = Pg[i];
      Q[i] = Qg[i];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb2; idx += blockDim.x) {
      const int cc = idx / NB, r = idx - cc * NB;  // output (r, cc), column-major
      S a0 = S(0), a1 = S(0);
      if (pass == 0) {
        // (P Q)(r, cc) = sum_k P(r, k) Q(k, cc)
#pragma unroll 8
        for (int k = 0; k < NB; k += 2) {
          a0 += P[k * NB + r] * Q[cc * NB + k];
          a1 += P[(k + 1) * NB + r] * Q[cc * NB + k + 1];
        }
      } else {
        // ((P Q)^T)(r, cc) = (P Q)(cc, r) = sum_k P(cc, k) Q(k, r)
#pragma unroll 8
        for (int k = 0; k < NB; k += 2) {
          a0 += P[k * NB + cc] * Q[r * NB + k];
          a1 += P[(k + 1) * NB + cc] * Q[r * NB + k + 1];
        }
      }
      out[idx] = S(-c) * (a0 + a1);
    }
  }
}

// ------------------------------------------------------------------ vector kernels
template <class S>
__global__ void k_lincomb(int64_t n, S* y, int nterms, double c0, double c1, double c2, double c3, const S* x0,
                          const S* x1, const S* x2, const S* x3) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    S s = S(c0) * x0[i];
    if (nterms > 1) s += S(c1) * x1[i];
    if (nterms > 2) s += S(c2) * x2[i];
    if (nterms > 3) s += S(c3) * x3[i];
    y[i] = s;
  }
}

template <class S>
__global__ void k_scale_dev(int64_t n, S* y, const double* a, const S* x) {
  const S s = S(a[0]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = s * x[i];
}

template <class Si, class So>
__global__ void k_cast(int64_t n, So* y, const Si* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = So(x[i]);
}

// ------------------------------------------------------------------ reductions
// block partial sums of KB per-thread values -> partial[blockIdx*ld + j0 + t], t < kb
template <int KB, class S>
__device__ __forceinline__ void block_partials(S* v, int kb, double* partial, int ld, int j0) {
  __shared__ double red[32][RED_THREADS / 32 + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_reduce_scatter<KB, S>(v, lane);
  constexpr int sh = 5 - ILog2<KB>::value;
  if ((lane & ((1 << sh) - 1)) == 0) red[lane >> sh][warp] = (double)v[0];
  __syncthreads();
  if (threadIdx.x < kb) {
    double s = 0.0;
    for (int w = 0; w < RED_THREADS / 32; ++w) s += red[threadIdx.x][w];
    partial[(size_t)blockIdx.x * ld + j0 + threadIdx.x] = s;
  }
  __syncthreads();
}

// Last-block finalisation: out[j] = sum_b partial[b*k + j].  Warp w reduces outputs
// j = w, w + nwarps, ...; lanes stride over the block partials and a fixed xor
// butterfly combines them, so the summation order is fixed (deterministic).
// Returns true in the block that finished the reduction.
__device__ __forceinline__ bool finish(int k, double* partial, unsigned* counter, double* out) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < k; j += nw) {
    double s = 0.0;
    for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(partial + (size_t)b * k + j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[j] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
  __syncthreads();
  return true;
}

struct GivensArgs {
  int j, m;
  const double* h1;
  const double* h2;
  double* H;
  double* cs;
  double* sn;
  double* g;
  double* stat;  // {res, tol, hn, 1/hn, beta, 1/beta, flag, j}
  double shift = 0.0;  // added to H(j, j): Arnoldi ran on A - shift I
};

// Hessenberg column j = h1 + h2 (+ shift on the diagonal) and norm hn, previous rotations, new rotation, residual
// estimate |g[j+1]| and stop flag (1 converged, 2 breakdown, 4 non-finite).  Loads are
// staged in shared memory by the whole block; the rotation chain runs on one thread.
__device__ __forceinline__ void givens_update(const GivensArgs& a, double nrm2) {
  __shared__ double col[72], c_s[72], s_s[72];
  const int j = a.j, m = a.m;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    col[i] = a.h1[i] + a.h2[i];
    if (i == j) col[i] += a.shift;
    if (i < j) {
      c_s[i] = a.cs[i];
      s_s[i] = a.sn[i];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double hn = sqrt(fmax(nrm2, 0.0));
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double t = c_s[i] * col[i] + s_s[i] * col[i + 1];
      col[i + 1] = -s_s[i] * col[i] + c_s[i] * col[i + 1];
      col[i] = t;
    }
    const double rr = hypot(col[j], col[j + 1]);
    const double c = rr > 0.0 ? col[j] / rr : 1.0, s = rr > 0.0 ? col[j + 1] / rr : 0.0;
    a.cs[j] = c;
    a.sn[j] = s;
    col[j] = rr;
    col[j + 1] = 0.0;
    const double gj = a.g[j];
    a.g[j + 1] = -s * gj;
    a.g[j] = c * gj;
    const double res = fabs(s * gj);
    a.stat[0] = res;
    a.stat[2] = hn;
    a.stat[3] = hn > 0.0 ? 1.0 / hn : 0.0;
    double flag = 0.0;
    if (res <= a.stat[1]) flag = 1.0;
    if (hn == 0.0) flag = 2.0;
    if (!isfinite(hn) || !isfinite(res)) flag = 4.0;
    a.stat[6] = flag;
    a.stat[7] = (double)j;
  }
  __syncthreads();
  double* Hc = a.H + (size_t)j * (m + 1);
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) Hc[i] = col[i];
}

// ------------------------------------------------------------------ Gram-Schmidt kernels
// One kernel per classical Gram-Schmidt pass of the Arnoldi step:
//   mode 0: out = V^T w (and out[k] = w.w when self is set)
//   mode 1: w -= V h, then out = V^T w
//   mode 2: w -= V h, then out[0] = w.w (and the Givens update when gv.H is set)
//   mode 3: out[0] = V_0 . w
// GB300 issues about 1.7 FP64 FMAs per clock per SM, so every FP64 instruction counts:
// at most one CTA per SM, each thread accumulates several vector entries before the
// single warp reduce-scatter, and the unrolled loops run over KB = k rounded up to a
// multiple of 4.  For k <= KB (up to 40) the k basis entries of an index are loaded once
// (all in flight together) and serve both the update and the dots.  Reduction, in a
// fixed order at every level so that results are bitwise reproducible: warp
// reduce-scatter -> CTA partials -> the CTA that finishes last sums the CTA partials.
constexpr int CGS_T = 256;
constexpr int CGS_MAX_BLOCKS = 152;
constexpr int CGS_MAXK = 64;
constexpr int CGS_MAXKB = 40;

template <int KB>
struct Pow2Up {
  static constexpr int value =
      KB <= 1 ? 1 : KB <= 2 ? 2 : KB <= 4 ? 4 : KB <= 8 ? 8 : KB <= 16 ? 16 : KB <= 32 ? 32 : 64;
};

// v[KB] per thread -> bp[j0 + t] (shared), t < kb; all CTA threads call it.  KB <= 64:
// a 64-wide reduction runs as two 32-wide halves.
template <int KB, class S>
__device__ __forceinline__ void cta_reduce(S* v, int kb, double* bp, int j0) {
  if constexpr (KB > 32) {
    cta_reduce<32, S>(v, kb < 32 ? kb : 32, bp, j0);
    if (kb > 32) cta_reduce<32, S>(v + 32, kb - 32, bp, j0 + 32);
  } else {
    __shared__ double red[32][CGS_T / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce_scatter<KB, S>(v, lane);
    constexpr int sh = 5 - ILog2<KB>::value;
    if ((lane & ((1 << sh) - 1)) == 0) red[lane >> sh][warp] = (double)v[0];
    __syncthreads();
    if (threadIdx.x < kb) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < CGS_T / 32; ++w) s += red[threadIdx.x][w];
      bp[j0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// cta_reduce over KB (a multiple of 4, <= 40) values split into power-of-two pieces
// (40 = 32 + 8, 28 = 16 + 8 + 4, ...): a reduce-scatter of P values costs about P FP64 adds
// per lane, so the pieces cost about KB adds instead of the next power of two.
template <int KB, int J0, class S>
__device__ __forceinline__ void cta_reduce_pieces(S* v, int k, double* bp) {
  if constexpr (KB > 0) {
    constexpr int P = KB >= 32 ? 32 : (1 << ILog2<KB>::value);
    const int valid = k - J0 < P ? k - J0 : P;
    cta_reduce<P, S>(v + J0, valid > 0 ? valid : 0, bp, J0);
    cta_reduce_pieces<KB - P, J0 + P, S>(v, k, bp);
  }
}

// Grid level of the reduction of the CTA partials bp[0..nk).  Returns true in the one
// CTA that holds the final sums in out[] (the last CTA to arrive).  The last CTA splits
// the partial rows into CGS_T / nk' chunks per output, loads each chunk with all loads
// in flight, and sums the chunk totals in chunk order (a fixed order: reproducible).
__device__ __forceinline__ bool cgs_finish(int nk, const double* bp, double* partial, unsigned* counter,
                                           double* out) {
  __shared__ double chunk[CGS_T];
  for (int t = threadIdx.x; t < nk; t += CGS_T) partial[(size_t)blockIdx.x * nk + t] = bp[t];
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1u);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const int nb = gridDim.x;
  int nc = CGS_T / nk;  // chunks per output
  if (nc > 32) nc = 32;
  if (nc > nb) nc = nb;
  if (nc < 1) nc = 1;
  const int per = (nb + nc - 1) / nc;
  for (int t = threadIdx.x; t < nk * nc; t += CGS_T) {
    const int j = t / nc, c = t - j * nc;
    const int b0 = c * per, b1 = min(nb, b0 + per);
    double a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = 0.0;
    int b = b0;
    for (; b + 7 < b1; b += 8) {
#pragma unroll
      for (int r = 0; r < 8; ++r) a[r] += __ldcg(partial + (size_t)(b + r) * nk + j);
    }
    for (; b < b1; ++b) a[0] += __ldcg(partial + (size_t)b * nk + j);
    chunk[t] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nk; j += CGS_T) {
    double s = 0.0;
    for (int c = 0; c < nc; ++c) s += chunk[j * nc + c];
    out[j] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
  __syncthreads();
  return true;
}

// Second Gram-Schmidt pass needed?  |w - V h1|^2 = |w|^2 - |h1|^2 in exact arithmetic; the
// pass is repeated when more than half of |w|^2 cancelled (|w - V h1| < |w| / sqrt 2).  Every
// caller (every CTA of every pass) evaluates the same expression on the same coefficients in
// the same order, so all take the same decision.  Warp 0 of the block calls it; returns
// |h1|^2 in hh.
__device__ __forceinline__ bool reorth_needed_warp0(const double* h1, double w2, int k, double& hh) {
  double s = 0.0;
  for (int t = threadIdx.x; t < k; t += 32) s += h1[t] * h1[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  hh = s;
  return !(s <= 0.5 * w2);
}

template <class S>
struct CgsArgs {
  int mode;           // 0 dots, 1 update + dots, 2 update + norm, 3 single dot
  int self;           // mode 0: also out[k] = w.w
  int64_t n;
  const S* V;
  int64_t ldv;
  int k;
  const double* h;    // update coefficients (modes 1, 2)
  const double* chk;  // non-null: selective reorthogonalization on chk[0..k), chk[k] = |w|^2 before
  S* w;
  double* out;
  double* out_nrm;    // mode 1 without reorthogonalization: |w|^2 goes here, out[0..k) = 0
  double* partial;
  unsigned* counter;
  GivensArgs gv;
};

template <int KB, class S>
__global__ void __launch_bounds__(CGS_T, 1) k_cgs(CgsArgs<S> a) {
  constexpr int K2 = Pow2Up<KB>::value;
  __shared__ double hs[CGS_MAXK + 1];
  __shared__ double bp[CGS_MAXK + 1];
  __shared__ int s_need;
  const int k = a.k;
  const int64_t n = a.n;
  const S* __restrict__ V = a.V;
  S* __restrict__ w = a.w;
  const int64_t ldv = a.ldv;
  int mode = a.mode;
  bool to_norm = false;
  if (a.chk) {
    // second pass needed?  (same decision in every CTA, see reorth_needed_warp0)
    if (threadIdx.x < 32) {
      double hh;
      const bool nd = reorth_needed_warp0(a.chk, a.chk[k], k, hh);
      if (threadIdx.x == 0) s_need = nd ? 1 : 0;
    }
    __syncthreads();
    const bool need = s_need != 0;
    if (mode == 2 && !need) return;  // the second pass was not needed: nothing left to do
    if (mode == 1 && !need) {        // update with h1, then the norm instead of a second pass
      mode = 2;
      to_norm = true;
    }
  }
  const bool upd = (mode == 1 || mode == 2);
  for (int t = threadIdx.x; t < CGS_MAXK; t += CGS_T) hs[t] = (upd && t < k) ? a.h[t] : 0.0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * CGS_T;
  const int64_t i0 = (int64_t)blockIdx.x * CGS_T + threadIdx.x;
  const bool self = (mode == 0 && a.self);
  const int nk = (mode == 0 || mode == 1) ? k : 1;
  S accs[1] = {S(0)};
  if (k <= KB) {
    S acc[K2];
#pragma unroll
    for (int t = 0; t < K2; ++t) acc[t] = S(0);
    for (int64_t i = i0; i < n; i += stride) {
      S v[KB];
#pragma unroll
      for (int t = 0; t < KB; ++t) v[t] = (t < k) ? V[(int64_t)t * ldv + i] : S(0);
      S s = w[i];
      if (upd) {
#pragma unroll
        for (int t = 0; t < KB; ++t) s -= S(hs[t]) * v[t];
        w[i] = s;
      }
      if (mode == 2) {
        acc[0] += s * s;
      } else if (mode == 3) {
        acc[0] += v[0] * s;
      } else {
#pragma unroll
        for (int t = 0; t < KB; ++t) acc[t] += v[t] * s;
        if (self) accs[0] += s * s;
      }
    }
    if (nk == 1) cta_reduce<1, S>(acc, 1, bp, 0);
    else cta_reduce<K2, S>(acc, nk, bp, 0);
  } else {
    // k > KB: update in chunks of KB loads, then one dot pass per chunk (re-reads)
    if (upd) {
      for (int64_t i = i0; i < n; i += stride) {
        S s = w[i];
        for (int c0 = 0; c0 < k; c0 += KB) {
          S v[KB];
#pragma unroll
          for (int t = 0; t < KB; ++t) v[t] = (c0 + t < k) ? V[(int64_t)(c0 + t) * ldv + i] : S(0);
#pragma unroll
          for (int t = 0; t < KB; ++t) s -= S(hs[c0 + t]) * v[t];
        }
        w[i] = s;
      }
    }
    if (mode == 2) {
      S acc[1] = {S(0)};
      for (int64_t i = i0; i < n; i += stride) {
        const S s = w[i];
        acc[0] += s * s;
      }
      cta_reduce<1, S>(acc, 1, bp, 0);
    } else {
      for (int c0 = 0; c0 < k; c0 += KB) {
        S acc[K2];
#pragma unroll
        for (int t = 0; t < K2; ++t) acc[t] = S(0);
        for (int64_t i = i0; i < n; i += stride) {
          const S s = w[i];
#pragma unroll
          for (int t = 0; t < KB; ++t)
            if (c0 + t < k) acc[t] += V[(int64_t)(c0 + t) * ldv + i] * s;
          if (self && c0 == 0) accs[0] += s * s;
        }
        cta_reduce<K2, S>(acc, min(KB, k - c0), bp, c0);
      }
    }
  }
  if (self) cta_reduce<1, S>(accs, 1, bp, k);
  double* out = to_norm ? a.out_nrm : a.out;
  if (!cgs_finish(nk + (self ? 1 : 0), bp, a.partial, a.counter, out)) return;
  if (to_norm) {
    for (int t = threadIdx.x; t < k; t += CGS_T) a.out[t] = 0.0;  // no second-pass coefficients
    __syncthreads();
  }
  if (mode == 2 && a.gv.H) givens_update(a.gv, out[0]);
}

// ------------------------------------------------------------------ fused Arnoldi step
// One cooperative launch per Arnoldi step (replaces the three Gram-Schmidt launches, the
// host copy of the convergence record and the scaling launch).  Every CTA stays resident
// (cooperative launch, one CTA per SM at most) and the passes are separated by grid
// barriers; after each barrier EVERY CTA sums the CTA partials itself, in one fixed order
// (warp w sums outputs w, w + 8, ...; lanes stride over the CTAs, then a xor butterfly),
// so all CTAs hold bitwise the same coefficients and no CTA waits for a last-arriving one.
// Passes (k <= KB basis vectors in registers):
//   1. h1 = V^T w and |w|^2 (one exchange)
//   2. if at most half of |w|^2 cancelled (|h1|^2 <= |w|^2 / 2, the selective
//      reorthogonalization test): v_k = (w - V h1) / sqrt(|w|^2 - |h1|^2), no further
//      exchange; else w -= V h1, h2 = V^T w (exchange), w -= V h2, |w|^2 (exchange),
//      v_k = w / |w|
// and CTA 0 applies the Givens update and writes the convergence record to the pinned
// host ring.  Barrier waits are bounded (about a second);
// an expired wait sets the error word, the convergence flag 8 and ends the kernel.
constexpr unsigned long long kArnBarrierNs = 1000000000ull;
constexpr int ARN_LD = CGS_MAXKB + 2;       // partial rows (outputs) per exchange
constexpr int ARN_NB = CGS_MAX_BLOCKS;      // partial columns (CTAs)
// barrier words, each on its own 128-byte line: arrival count (u32), release epoch (u64),
// error word (u32)
constexpr int ARN_BAR_COUNT = 0, ARN_BAR_EPOCH = 32, ARN_BAR_ERROR = 64, ARN_BAR_WORDS = 96;

template <class S>
struct ArnArgs {
  int64_t n;
  const S* V;
  int64_t ldv;
  int k;
  S* w;                 // A v_{k-1} on entry; w - V (h1 + h2) on exit
  S* vnext;             // V column k on exit: w / |w|
  double* h1;
  double* h2;
  double* nrm;
  double* partial;      // [2][ARN_LD][ARN_NB], alternating between exchanges
  unsigned* bar;        // ARN_BAR_WORDS words (see above), zero before the first launch
  double* host_stat;    // device alias of the pinned ring slot (or null)
  GivensArgs gv;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier number `target` of this launch (epochs continue across launches).  Thread 0
// of each CTA arrives with an acquire-release add (its CTA's partials, ordered by the
// preceding __syncthreads, become visible with it); the last arrival resets the count and
// publishes the epoch with a release store; the others poll the epoch with acquire loads,
// for at most kArnBarrierNs.
__device__ __forceinline__ bool arn_grid_barrier(unsigned* bar, unsigned long long target) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int good = 1;
    unsigned long long* epoch = reinterpret_cast<unsigned long long*>(bar + ARN_BAR_EPOCH);
    const unsigned prev = atom_add_acq_rel_u32(bar + ARN_BAR_COUNT, 1u);
    if (prev == gridDim.x - 1u) {
      st_relaxed_u32(bar + ARN_BAR_COUNT, 0u);
      st_release_u64(epoch, target);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned it = 0;
      while (ld_acquire_u64(epoch) < target) {
        if ((++it & 255u) == 0u && global_ns() - t0 > kArnBarrierNs) {
          atomicExch(bar + ARN_BAR_ERROR, 1u);
          good = 0;
          break;
        }
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// CTA partials bp[0..nk) -> column blockIdx.x of the region, grid barrier, then every CTA
// forms out[j] = sum_b region[j][b] (out in shared memory), in the same order everywhere.
__device__ __forceinline__ bool arn_exchange(int nk, const double* bp, double* region, unsigned* bar,
                                             unsigned long long target, double* out) {
  for (int t = threadIdx.x; t < nk; t += CGS_T) region[(size_t)t * ARN_NB + blockIdx.x] = bp[t];
  if (!arn_grid_barrier(bar, target)) return false;
  constexpr int NW = CGS_T / 32;
  constexpr int R = (ARN_NB + 31) / 32;
  constexpr int Q = (ARN_LD + NW - 1) / NW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nb = gridDim.x;
  // outputs of this warp: j = warp + NW q for q < nq (warp-uniform, so only the warps and
  // rounds that own an output spend FP64 adds; GB300 issues about 1.7 FP64 adds per clock
  // per SM, so the reduction of the partials is not free)
  const int nq = nk > warp ? (nk - warp + NW - 1) / NW : 0;
  double s[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    double acc = 0.0;
    if (q < nq) {
      const double* col = region + (size_t)(warp + NW * q) * ARN_NB;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int b = lane + 32 * r;
        if (b < nb) acc += __ldcg(col + b);
      }
    }
    s[q] = acc;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (q < nq) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
      if (lane == 0) out[warp + NW * q] = s[q];
    }
  }
  __syncthreads();
  return true;
}

template <int KB, class S>
__global__ void __launch_bounds__(CGS_T, 1) k_arnoldi(ArnArgs<S> a) {
  __shared__ double bp[CGS_MAXK + 1];
  __shared__ double red[CGS_MAXKB + 1];  // result of the last exchange
  __shared__ double hA[KB], hB[KB];      // h1, h2 (zero beyond k)
  __shared__ int s_need;
  const int k = a.k;
  const int64_t n = a.n;
  const S* __restrict__ V = a.V;
  S* __restrict__ w = a.w;
  const int64_t ldv = a.ldv;
  // contiguous, balanced slices (a multiple of 32 entries per CTA): every CTA reaches the
  // barriers with the same work, where a grid-stride loop leaves the first n mod (grid x
  // CGS_T) / CGS_T CTAs with one more entry per thread than the rest
  const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
  const int64_t lo = (int64_t)blockIdx.x * chunk < n ? (int64_t)blockIdx.x * chunk : n;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  const int64_t stride = CGS_T;
  const int64_t i0 = lo + threadIdx.x;
  double* region0 = a.partial;
  double* region1 = a.partial + (size_t)ARN_LD * ARN_NB;
  // epoch before this launch's first barrier (stable: it only moves inside a barrier,
  // which no CTA passes before every CTA has read it here)
  __shared__ unsigned long long s_epoch;
  if (threadIdx.x == 0)
    s_epoch = ld_acquire_u64(reinterpret_cast<const unsigned long long*>(a.bar + ARN_BAR_EPOCH));
  __syncthreads();
  const unsigned long long e0 = s_epoch;
  bool ok;
  // pass 1: h1 = V^T w, |w|^2
  {
    S acc[KB], accs[1] = {S(0)};
#pragma unroll
    for (int t = 0; t < KB; ++t) acc[t] = S(0);
    for (int64_t i = i0; i < hi; i += stride) {
      S v[KB];
#pragma unroll
      for (int t = 0; t < KB; ++t) v[t] = (t < k) ? V[(int64_t)t * ldv + i] : S(0);
      const S s = w[i];
#pragma unroll
      for (int t = 0; t < KB; ++t) acc[t] += v[t] * s;
      accs[0] += s * s;
    }
    cta_reduce_pieces<KB, 0, S>(acc, k, bp);
    cta_reduce<1, S>(accs, 1, bp, k);
  }
  ok = arn_exchange(k + 1, bp, region0, a.bar, e0 + 1, red);
  double nrm2 = 0.0;
  S* __restrict__ vn = a.vnext;
  if (ok) {
    __shared__ double s_hh;
    if (threadIdx.x < 32) {
      double hh;
      const bool nd = reorth_needed_warp0(red, red[k], k, hh);
      if (threadIdx.x == 0) {
        s_need = nd ? 1 : 0;
        s_hh = hh;
      }
    }
    for (int t = threadIdx.x; t < KB; t += CGS_T) {
      hA[t] = t < k ? red[t] : 0.0;
      hB[t] = 0.0;
    }
    __syncthreads();
    const bool need = s_need != 0;
    if (!need) {
      // at most half of |w|^2 cancelled: one update, and |w - V h1|^2 = |w|^2 - |h1|^2 (the
      // basis is orthonormal to working precision; the subtraction keeps at least half),
      // so v_k = (w - V h1) / |w - V h1| needs no second reduction
      nrm2 = red[k] - s_hh;
      const double hn = sqrt(fmax(nrm2, 0.0));
      const S inv = S(hn > 0.0 ? 1.0 / hn : 0.0);
      for (int64_t i = i0; i < hi; i += stride) {
        S v[KB];
#pragma unroll
        for (int t = 0; t < KB; ++t) v[t] = (t < k) ? V[(int64_t)t * ldv + i] : S(0);
        S s = w[i];
#pragma unroll
        for (int t = 0; t < KB; ++t) s -= S(hA[t]) * v[t];
        vn[i] = inv * s;
      }
    } else {
      // pass 2: w -= V h1, h2 = V^T w
      {
        S acc[KB];
#pragma unroll
        for (int t = 0; t < KB; ++t) acc[t] = S(0);
        for (int64_t i = i0; i < hi; i += stride) {
          S v[KB];
#pragma unroll
          for (int t = 0; t < KB; ++t) v[t] = (t < k) ? V[(int64_t)t * ldv + i] : S(0);
          S s = w[i];
#pragma unroll
          for (int t = 0; t < KB; ++t) s -= S(hA[t]) * v[t];
          w[i] = s;
#pragma unroll
          for (int t = 0; t < KB; ++t) acc[t] += v[t] * s;
        }
        cta_reduce_pieces<KB, 0, S>(acc, k, bp);
      }
      ok = arn_exchange(k, bp, region1, a.bar, e0 + 2, red);
      if (ok) {
        for (int t = threadIdx.x; t < k; t += CGS_T) hB[t] = red[t];
        __syncthreads();
        // pass 3: w -= V h2, |w|^2
        S acc[1] = {S(0)};
        for (int64_t i = i0; i < hi; i += stride) {
          S v[KB];
#pragma unroll
          for (int t = 0; t < KB; ++t) v[t] = (t < k) ? V[(int64_t)t * ldv + i] : S(0);
          S s = w[i];
#pragma unroll
          for (int t = 0; t < KB; ++t) s -= S(hB[t]) * v[t];
          w[i] = s;
          acc[0] += s * s;
        }
        cta_reduce<1, S>(acc, 1, bp, 0);
        ok = arn_exchange(1, bp, region0, a.bar, e0 + 3, red);
      }
      if (ok) {
        nrm2 = red[0];
        const double hn = sqrt(fmax(nrm2, 0.0));
        const S inv = S(hn > 0.0 ? 1.0 / hn : 0.0);
        for (int64_t i = i0; i < hi; i += stride) vn[i] = inv * w[i];
      }
    }
  }
  if (!ok) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.gv.stat[6] = 8.0;
      if (a.host_stat) {
        for (int t = 0; t < 8; ++t) a.host_stat[t] = a.gv.stat[t];
      }
    }
    return;
  }
  if (blockIdx.x != 0) return;
  for (int t = threadIdx.x; t < k; t += CGS_T) {
    a.h1[t] = hA[t];
    a.h2[t] = hB[t];
  }
  if (threadIdx.x == 0) a.nrm[0] = nrm2;
  __syncthreads();
  givens_update(a.gv, nrm2);
  if (threadIdx.x == 0 && a.host_stat) {
    for (int t = 0; t < 8; ++t) a.host_stat[t] = a.gv.stat[t];
  }
}

// out[j] = sum_e per_elem[e*k + j], k <= 8
__global__ void __launch_bounds__(RED_THREADS)
    k_colsum(int ne, int k, const double* __restrict__ pe, double* out, double* partial, unsigned* counter) {
  double acc[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) acc[t] = 0.0;
  for (int e = blockIdx.x * RED_THREADS + threadIdx.x; e < ne; e += gridDim.x * RED_THREADS)
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (t < k) acc[t] += pe[(size_t)e * k + t];
  block_partials<8, double>(acc, k, partial, k, 0);
  finish(k, partial, counter, out);
}

// GMRES bookkeeping on the device (one thread): stat = {res, tol, hn, inv_hn, beta, inv_beta, flag, j}
__global__ void k_gmres_init(const double* bb, double rtol, double atol, int first, int m, double* g, double* stat) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double beta = sqrt(fmax(bb[0], 0.0));
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  if (first) stat[1] = fmax(rtol * beta, atol);
  stat[0] = beta;
  stat[4] = beta;
  stat[5] = beta > 0.0 ? 1.0 / beta : 0.0;
  stat[6] = (beta <= stat[1]) ? 1.0 : 0.0;
  if (!isfinite(beta)) stat[6] = 4.0;
  stat[7] = -1.0;
}

// y = -(H^{-1} g) on the leading ncols x ncols triangle (negated for the fused update
// kernel).  The triangle is staged in shared memory; column-oriented back substitution,
// one column per step, the remaining right-hand side updated by the whole block in a
// fixed order (each entry by one thread).
__global__ void __launch_bounds__(256) k_gmres_backsolve(int ncols, int m, const double* H, const double* g,
                                                         double* y) {
  __shared__ double Hs[64 * 65];
  __shared__ double rhs[64];
  for (int idx = threadIdx.x; idx < ncols * ncols; idx += blockDim.x) {
    const int c = idx / ncols, r = idx - c * ncols;
    Hs[c * 65 + r] = H[(size_t)c * (m + 1) + r];
  }
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) rhs[i] = g[i];
  __syncthreads();
  for (int i = ncols - 1; i >= 0; --i) {
    const double d = Hs[i * 65 + i];
    const double yi = d != 0.0 ? rhs[i] / d : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) y[i] = -yi;
    for (int r = threadIdx.x; r < i; r += blockDim.x) rhs[r] -= Hs[i * 65 + r] * yi;
    __syncthreads();
  }
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

template <class S>
cudaError_t launch_block_inverse(const DevMesh& m, const DevTables& tb, const double* J, double c, S* Ainv, S* AinvT,
                                 int* status, cudaStream_t st) {
  ProfScope ps(PP_K_BLOCK_INVERSE, st);
  k_block_inverse<S><<<m.ne, INV_THREADS, 0, st>>>(m, tb, J, c, Ainv, AinvT, status);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_stage_matvec(const DevMesh& m, const DevTables& tb, const S* J, double alpha, double beta,
                                const S* x, S* y, int trans, cudaStream_t st) {
  ProfScope ps(sizeof(S) == 8 ? PP_K_STAGE_MATVEC : PP_K_STAGE_MATVEC32, st);
  if (!trans && beta != 0.0 && stream_rows_supported<S>(tb.nb, J, x, y))
    return launch_stream_rows<S>(m, tb, tb.nb, 4, J, alpha, beta, x, y, st);
  const int g = m.ne, b = 128;
#define PP_SMV(NBV)                                                                        \
  case NBV:                                                                                \
    if (trans) k_stage_matvec<NBV, true, S><<<g, b, 0, st>>>(m, tb, J, alpha, beta, x, y);  \
    else k_stage_matvec<NBV, false, S><<<g, b, 0, st>>>(m, tb, J, alpha, beta, x, y);       \
    break;
  switch (tb.nb) {
    PP_SMV(12)
    PP_SMV(24)
    PP_SMV(40)
    PP_SMV(60)
    default: return cudaErrorInvalidValue;
  }
#undef PP_SMV
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_block_apply(const DevMesh& m, int nb, const S* Ainv, const S* x, S* y, int trans,
                               cudaStream_t st) {
  ProfScope ps(sizeof(S) == 8 ? PP_K_BLOCK_APPLY : PP_K_BLOCK_APPLY32, st);
  if (!trans && stream_rows_supported<S>(nb, Ainv, x, y)) {
    DevTables none{};
    return launch_stream_rows<S>(m, none, nb, 1, Ainv, 0.0, 1.0, x, y, st);
  }
  const int g = m.ne, b = 128;
#define PP_BAP(NBV)                                                             \
  case NBV:                                                                     \
    if (trans) k_block_apply<NBV, true, S><<<g, b, 0, st>>>(m.ne, Ainv, x, y);   \
    else k_block_apply<NBV, false, S><<<g, b, 0, st>>>(m.ne, Ainv, x, y);        \
    break;
  switch (nb) {
    PP_BAP(12)
    PP_BAP(24)
    PP_BAP(40)
    PP_BAP(60)
    default: return cudaErrorInvalidValue;
  }
#undef PP_BAP
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_fold_blocks(const DevMesh& m, int nb, const S* J, const S* Ainv, double c, S* BN, S* BT,
                               cudaStream_t st) {
  ProfScope ps(PP_K_FOLD, st);
  const size_t smem = sizeof(S) * 2 * nb * nb;
#define PP_FOLD(NBV)                                                                                     \
  case NBV: {                                                                                            \
    static const cudaError_t attr =                                                                      \
        cudaFuncSetAttribute(k_fold_blocks<NBV, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (attr != cudaSuccess) return attr;                                                                \
    k_fold_blocks<NBV, S><<<m.ne * 3, 256, smem, st>>>(m, J, Ainv, c, BN, BT);                           \
    break;                                                                                               \
  }
  switch (nb) {
    PP_FOLD(12)
    PP_FOLD(24)
    PP_FOLD(40)
    PP_FOLD(60)
    default:
      return cudaErrorInvalidValue;
  }
#undef PP_FOLD
  return cudaGetLastError();
}

template <class Si, class So>
cudaError_t launch_transpose_blocks(const DevMesh& m, int nb, const Si* J, So* JT, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_transpose_blocks<Si, So><<<m.ne * 4, 256, 0, st>>>(m, nb, J, JT);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_lincomb(int64_t n, S* y, int nterms, const double* c, const S* const* x, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_lincomb<S><<<vec_blocks(n), 256, 0, st>>>(n, y, nterms, c[0], nterms > 1 ? c[1] : 0.0, nterms > 2 ? c[2] : 0.0,
                                              nterms > 3 ? c[3] : 0.0, x[0], nterms > 1 ? x[1] : nullptr,
                                              nterms > 2 ? x[2] : nullptr, nterms > 3 ? x[3] : nullptr);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_scale_dev(int64_t n, S* y, const double* a, const S* x, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_scale_dev<S><<<vec_blocks(n), 256, 0, st>>>(n, y, a, x);
  return cudaGetLastError();
}

template <class Si, class So>
cudaError_t launch_cast(int64_t n, So* y, const Si* x, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_cast<Si, So><<<vec_blocks(n), 256, 0, st>>>(n, y, x);
  return cudaGetLastError();
}

cudaError_t launch_gmres_init(const double* bb, double rtol, double atol, int first, int m, double* g, double* stat,
                              cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_gmres_init<<<1, 32, 0, st>>>(bb, rtol, atol, first, m, g, stat);
  return cudaGetLastError();
}

cudaError_t launch_gmres_backsolve(int ncols, int m, const double* H, const double* g, double* y, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_gmres_backsolve<<<1, 256, 0, st>>>(ncols, m, H, g, y);
  return cudaGetLastError();
}

// One CTA per SM at most (fewer for short vectors).
int cgs_blocks(int64_t n) {
  static const int cap = [] {  // thread-safe static initialization; one device per process
    int dev = 0, sms = CGS_MAX_BLOCKS;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int c = sms < CGS_MAX_BLOCKS ? sms : CGS_MAX_BLOCKS;
    return c < 1 ? 1 : c;
  }();
  int64_t b = (n + CGS_T - 1) / CGS_T;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

template <class S>
cudaError_t launch_cgs(const CgsArgs<S>& a, cudaStream_t st, int kind = -1) {
  ProfScope ps(kind >= 0 ? kind : (sizeof(S) == 8 ? PP_K_KRYLOV : PP_K_KRYLOV32), st);
  if (a.k < 1 || a.k > CGS_MAXK) return cudaErrorInvalidValue;
  const int g = cgs_blocks(a.n);
  switch ((a.k + 3) / 4) {
#define PP_CGS(Q) \
  case Q:         \
    k_cgs<4 * Q, S><<<g, CGS_T, 0, st>>>(a); \
    break;
    PP_CGS(1)
    PP_CGS(2)
    PP_CGS(3)
    PP_CGS(4)
    PP_CGS(5)
    PP_CGS(6)
    PP_CGS(7)
    PP_CGS(8)
    PP_CGS(9)
    PP_CGS(10)
    default:
      k_cgs<32, S><<<g, CGS_T, 0, st>>>(a);  // k > 40: chunked path
#undef PP_CGS
  }
  return cudaGetLastError();
}

template <class S>
CgsArgs<S> cgs_args(int mode, int64_t n, const S* V, int64_t ldv, int k, const double* h, S* w, double* out,
                    double* partial, unsigned* counter) {
  CgsArgs<S> a{};
  a.mode = mode;
  a.n = n;
  a.V = V;
  a.ldv = ldv;
  a.k = k;
  a.h = h;
  a.w = w;
  a.out = out;
  a.partial = partial;
  a.counter = counter;
  return a;
}

template <class S>
cudaError_t launch_mdot(int64_t n, const S* V, int64_t ldv, int k, const S* w, double* out, double* partial,
                        unsigned* counter, cudaStream_t st) {
  return launch_cgs<S>(cgs_args<S>(0, n, V, ldv, k, nullptr, const_cast<S*>(w), out, partial, counter), st);
}

template <class S>
cudaError_t launch_update_mdot(int64_t n, const S* V, int64_t ldv, int k, const double* h, S* w, double* out,
                               double* partial, unsigned* counter, cudaStream_t st) {
  return launch_cgs<S>(cgs_args<S>(1, n, V, ldv, k, h, w, out, partial, counter), st);
}

template <class S>
cudaError_t launch_update_norm2(int64_t n, const S* V, int64_t ldv, int k, const double* h, S* w, double* out,
                                double* partial, unsigned* counter, cudaStream_t st) {
  return launch_cgs<S>(cgs_args<S>(2, n, V, ldv, k, h, w, out, partial, counter), st);
}

template <class S>
cudaError_t launch_update_norm2_givens(int64_t n, const S* V, int64_t ldv, int k, const double* h, S* w, double* out,
                                       double* partial, unsigned* counter, int j, int m, const double* h1,
                                       const double* h2, double* H, double* cs, double* sn, double* g, double* stat,
                                       cudaStream_t st) {
  CgsArgs<S> a = cgs_args<S>(2, n, V, ldv, k, h, w, out, partial, counter);
  a.gv = GivensArgs{j, m, h1, h2, H, cs, sn, g, stat};
  return launch_cgs<S>(a, st);
}

template <class S>
cudaError_t launch_arnoldi_ortho(int64_t n, const S* V, int64_t ldv, int k, S* w, double* h1, double* h2,
                                 double* nrm, double* partial, unsigned* counter, int j, int m, double* H, double* cs,
                                 double* sn, double* g, double* stat, double shift, cudaStream_t st) {
  const GivensArgs gv{j, m, h1, h2, H, cs, sn, g, stat, shift};
  const int kind = sizeof(S) == 8 ? PP_K_ARNOLDI : PP_K_ARNOLDI32;
  // algorithmic traffic of one classical Gram-Schmidt pass: V and w read for the projections,
  // V and w read and w written for the update and norm
  prof_add_bytes(kind, (2.0 * k + 3.0) * (double)n * sizeof(S), 3);
  // pass 1: h1 = V^T w and |w|^2
  CgsArgs<S> a = cgs_args<S>(0, n, V, ldv, k, nullptr, w, h1, partial, counter);
  a.self = 1;
  cudaError_t e = launch_cgs<S>(a, st, kind);
  if (e != cudaSuccess) return e;
  // pass 2: w -= V h1; then h2 = V^T w if reorthogonalization is needed, else |w|^2 + Givens
  a = cgs_args<S>(1, n, V, ldv, k, h1, w, h2, partial, counter);
  a.chk = h1;
  a.out_nrm = nrm;
  a.gv = gv;
  if ((e = launch_cgs<S>(a, st, kind)) != cudaSuccess) return e;
  // pass 3 (only if needed): w -= V h2, |w|^2 + Givens
  a = cgs_args<S>(2, n, V, ldv, k, h2, w, nrm, partial, counter);
  a.chk = h1;
  a.gv = gv;
  return launch_cgs<S>(a, st, kind);
}

template <class S>
cudaError_t launch_arnoldi_step(int64_t n, const S* V, int64_t ldv, int k, S* w, S* vnext, double* h1, double* h2,
                                double* nrm, double* arn_partial, unsigned* arn_bar, double* host_stat, int j, int m,
                                double* H, double* cs, double* sn, double* g, double* stat, double shift,
                                cudaStream_t st) {
  if (k < 1 || k > CGS_MAXKB) return cudaErrorInvalidValue;
  const int kind = sizeof(S) == 8 ? PP_K_ARNOLDI : PP_K_ARNOLDI32;
  // algorithmic traffic of the common path: V and w read for the projections, V and w
  // read and v_k written for the update and scaling (a second pass, when the
  // reorthogonalization test asks for it, is not counted)
  prof_add_bytes(kind, (2.0 * k + 3.0) * (double)n * sizeof(S), 1);
  ProfScope ps(kind, st);
  ArnArgs<S> a{};
  a.n = n;
  a.V = V;
  a.ldv = ldv;
  a.k = k;
  a.w = w;
  a.vnext = vnext;
  a.h1 = h1;
  a.h2 = h2;
  a.nrm = nrm;
  a.partial = arn_partial;
  a.bar = arn_bar;
  a.host_stat = host_stat;
  a.gv = GivensArgs{j, m, h1, h2, H, cs, sn, g, stat, shift};
  // grid <= SM count and one CTA per SM: every CTA is resident, which the cooperative launch
  // checks (it fails rather than start a grid that could wait on a CTA that never runs)
  const int grid = cgs_blocks(n);
  void* args[] = {&a};
  cudaError_t e = cudaSuccess;
  switch ((k + 3) / 4) {
#define PP_ARN(Q)                                                                                   \
  case Q:                                                                                           \
    e = cudaLaunchCooperativeKernel((const void*)k_arnoldi<4 * Q, S>, dim3(grid), dim3(CGS_T), args, 0, st); \
    break;
    PP_ARN(1)
    PP_ARN(2)
    PP_ARN(3)
    PP_ARN(4)
    PP_ARN(5)
    PP_ARN(6)
    PP_ARN(7)
    PP_ARN(8)
    PP_ARN(9)
    PP_ARN(10)
#undef PP_ARN
    default:
      return cudaErrorInvalidValue;
  }
  return e;
}

size_t arnoldi_partial_words() { return (size_t)2 * ARN_NB * ARN_LD; }
int arnoldi_barrier_words() { return ARN_BAR_WORDS; }
int arnoldi_barrier_error_word() { return ARN_BAR_ERROR; }

template <class S>
cudaError_t launch_dot(int64_t n, const S* x, const S* y, double* out, double* partial, unsigned* counter,
                       cudaStream_t st) {
  return launch_cgs<S>(cgs_args<S>(3, n, x, 0, 1, nullptr, const_cast<S*>(y), out, partial, counter), st);
}

cudaError_t launch_colsum(int ne, int k, const double* per_elem, double* out, double* partial, unsigned* counter,
                          cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_colsum<<<red_blocks(ne), RED_THREADS, 0, st>>>(ne, k, per_elem, out, partial, counter);
  return cudaGetLastError();
}

cudaError_t launch_scale(int64_t n, double* y, double a, const double* x, cudaStream_t st) {
  const double c[1] = {a};
  const double* xs[1] = {x};
  return launch_lincomb<double>(n, y, 1, c, xs, st);
}

// ------------------------------------------------------------------ explicit instantiations
#define PP_INST(S)                                                                                                    \
  template cudaError_t launch_block_inverse<S>(const DevMesh&, const DevTables&, const double*, double, S*, S*,     \
                                               int*, cudaStream_t);                                                 \
  template cudaError_t launch_stage_matvec<S>(const DevMesh&, const DevTables&, const S*, double, double, const S*, \
                                              S*, int, cudaStream_t);                                               \
  template cudaError_t launch_block_apply<S>(const DevMesh&, int, const S*, const S*, S*, int, cudaStream_t);       \
  template cudaError_t launch_lincomb<S>(int64_t, S*, int, const double*, const S* const*, cudaStream_t);           \
  template cudaError_t launch_scale_dev<S>(int64_t, S*, const double*, const S*, cudaStream_t);                     \
  template cudaError_t launch_mdot<S>(int64_t, const S*, int64_t, int, const S*, double*, double*, unsigned*,       \
                                      cudaStream_t);                                                                \
  template cudaError_t launch_update_mdot<S>(int64_t, const S*, int64_t, int, const double*, S*, double*, double*,  \
                                             unsigned*, cudaStream_t);                                              \
  template cudaError_t launch_update_norm2<S>(int64_t, const S*, int64_t, int, const double*, S*, double*, double*, \
                                              unsigned*, cudaStream_t);                                             \
  template cudaError_t launch_fold_blocks<S>(const DevMesh&, int, const S*, const S*, double, S*, S*,         \
                                             cudaStream_t);                                                     \
  template cudaError_t launch_arnoldi_step<S>(int64_t, const S*, int64_t, int, S*, S*, double*, double*, double*,    \
                                             double*, unsigned*, double*, int, int, double*, double*, double*,      \
                                             double*, double*, double, cudaStream_t);                               \
  template cudaError_t launch_arnoldi_ortho<S>(int64_t, const S*, int64_t, int, S*, double*, double*, double*,  \
                                                 double*, unsigned*, int, int, double*, double*, double*, double*,  \
                                                 double*, double, cudaStream_t);                                    \
  template cudaError_t launch_update_norm2_givens<S>(int64_t, const S*, int64_t, int, const double*, S*, double*,   \
                                                     double*, unsigned*, int, int, const double*, const double*,    \
                                                     double*, double*, double*, double*, double*, cudaStream_t);    \
  template cudaError_t launch_dot<S>(int64_t, const S*, const S*, double*, double*, unsigned*, cudaStream_t);
PP_INST(double)
PP_INST(float)
#undef PP_INST
template cudaError_t launch_transpose_blocks<double, double>(const DevMesh&, int, const double*, double*,
                                                             cudaStream_t);
template cudaError_t launch_transpose_blocks<double, float>(const DevMesh&, int, const double*, float*, cudaStream_t);
template cudaError_t launch_cast<double, float>(int64_t, float*, const double*, cudaStream_t);
template cudaError_t launch_cast<float, double>(int64_t, double*, const float*, cudaStream_t);

}  // namespace pp
