// Block-row streaming products staged through shared memory by the Tensor Memory
// Accelerator's bulk-copy engine (cp.async.bulk + mbarrier transaction counts).
//
//  y_e = alpha detB_e (Mref (x) I4) x_e + beta sum_q B_{e,q} x_{src(e,q)}     NBLK = 4
//  y_e = A_e x_e                                                              NBLK = 1
//  y_e = x_e + sum_f B_{e,f} x_{nbr(e,f)}                                     NBLK = 3
//
// NBLK = 4 is the DIRK stage operator M - a_ii dt dr/du of Eq. dirk2 (diagonal block and
// the three face-neighbour blocks of the element row; the Jacobian J[e][q] is stored as
// contiguous column-major nb x nb blocks).  NBLK = 1 is the block-Jacobi preconditioner
// application (explicit inverse A_e of the diagonal block).  NBLK = 3 is the stage
// operator with the block-Jacobi preconditioner folded in, (M - cJ) D^{-1} = I + O D^{-1}
// (D the diagonal blocks, O the face-neighbour blocks; B_{e,f} = O_{e,f} D^{-1}_{nbr}
// precomputed per stage).  All read every matrix entry exactly once per call, which
// makes them the streaming (HBM / L2) core of each Krylov step of the stage solves.
//
// Design for sm_103a:
//  - persistent CTAs, grid = resident CTAs per SM x SM count, element e of CTA b is
//    b + i * gridDim.x;
//  - one producer warp: a single lane issues, per (element, block), two bulk copies (the
//    nb x nb block and the nb-vector it multiplies) into a ring of R shared-memory units,
//    each completing on the unit's "full" mbarrier;
//  - ceil(4 nb / 32) consumer warps: lane p owns the (row, column group) pair
//    (p mod nb, p / nb), so every lane is busy for nb = 24, 40 (and 94% at nb = 60);
//    a column group is one block (NBLK = 4) or nb/4 columns of the block (NBLK = 1);
//    the four partial rows meet in shared memory;
//  - consumers release a unit through its "empty" mbarrier; the producer refills it.
// Every mbarrier wait is bounded (about a second of clock cycles); on expiry the error is
// recorded in g_stream_error and the producer, or all consumers together, leave.  Copies start on 16-byte
// boundaries: nb is a multiple of 4, so every block and every element slice of x is
// 16-byte aligned whenever the base pointers are (checked by the launcher).
#include <cstdint>
#include <cstdlib>

#include "pp_internal.h"

namespace pp {

namespace {

__device__ int g_stream_error;

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the completion of the phase with the given parity; false after kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Barrier over the consumer warps that also returns the AND of v over them, so that a
// timeout seen by any consumer thread makes all of them leave together.
__device__ __forceinline__ bool consumer_all(bool v, int nthreads) {
  uint32_t out;
  asm volatile(
      "{\n"
      "  .reg .pred pi, po;\n"
      "  setp.ne.u32 pi, %1, 0;\n"
      "  bar.red.and.pred po, 1, %2, pi;\n"
      "  selp.u32 %0, 1, 0, po;\n"
      "}\n"
      : "=r"(out)
      : "r"((uint32_t)v), "r"(nthreads)
      : "memory");
  return out != 0;
}

}  // namespace

template <int NB, int NBLK, class S>
struct StreamShape {
  static constexpr int NG = NBLK == 3 ? 3 : 4;  // column groups per element
  static constexpr int CW = (NG * NB + 31) / 32;  // consumer warps
  static constexpr int THREADS = 32 * (CW + 1);
  static constexpr int UNIT = NB * NB + 2 * NB;  // block + input slice (+ own slice), elements of S
  static constexpr int UNIT_BYTES = UNIT * (int)sizeof(S);
  static constexpr int BUDGET = 100 * 1024;  // two CTAs per SM where the units fit (measured
                                             // faster than four smaller rings at nb = 40)
  static constexpr int R = (BUDGET / UNIT_BYTES) > NBLK + 1 ? (BUDGET / UNIT_BYTES) : NBLK + 1;
  static constexpr int RED_BYTES = NG * NB * (int)sizeof(S);
  static constexpr int SMEM = R * UNIT_BYTES + RED_BYTES + 2 * R * 8 + R * 4;
};

namespace {

template <int NB, int NBLK, class S>
__global__ void __launch_bounds__(StreamShape<NB, NBLK, S>::THREADS)
    k_stream_rows(DevMesh m, DevTables tb, const S* __restrict__ B, double alpha, double beta,
                  const S* __restrict__ x, S* __restrict__ y) {
  using Sh = StreamShape<NB, NBLK, S>;
  constexpr int R = Sh::R, UNIT = Sh::UNIT, CW = Sh::CW;
  constexpr int NP = NB / 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S* ring = reinterpret_cast<S*>(smem_raw);
  S* red = ring + (size_t)R * UNIT;  // [4][NB]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)R * Sh::UNIT_BYTES + Sh::RED_BYTES);
  uint64_t* empty = full + R;
  int* pres = reinterpret_cast<int*>(empty + R);  // block of the unit present (not a boundary face)

  const int tid = threadIdx.x, warp = tid >> 5;
  const int G = gridDim.x;
  const int nE = (m.ne - (int)blockIdx.x + G - 1) / G;  // elements of this CTA
  if (tid == 0) {
    for (int s = 0; s < R; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == CW) {
    // ---------------- producer
    if ((tid & 31) != 0) return;
    const int nunits = nE * NBLK;
    for (int u = 0; u < nunits; ++u) {
      const int slot = u % R;
      if (u >= R && !mbar_wait(&empty[slot], (uint32_t)((u / R) - 1) & 1u)) {
        atomicExch(&g_stream_error, 1);
        return;
      }
      const int li = u / NBLK, q = u - li * NBLK;
      const int e = (int)blockIdx.x + li * G;
      int src = e;
      if (NBLK == 4 && q > 0) src = m.nbr[3 * e + q - 1];
      if (NBLK == 3) src = m.nbr[3 * e + q];
      S* dst = ring + (size_t)slot * UNIT;
      const bool own = (NBLK == 3 && q == 0);  // the identity term needs the element's own slice
      const uint32_t bytes = (src >= 0 ? (uint32_t)((NB * NB + NB) * sizeof(S)) : 0u) +
                             (own ? (uint32_t)(NB * sizeof(S)) : 0u);
      pres[slot] = src >= 0 ? 1 : 0;
      if (bytes == 0) {
        mbar_arrive(&full[slot]);  // boundary face: nothing to load, the consumers skip it
      } else {
        mbar_arrive_expect_tx(&full[slot], bytes);
        if (src >= 0) {
          bulk_load(dst, B + ((size_t)e * NBLK + q) * NB * NB, (uint32_t)(NB * NB * sizeof(S)), &full[slot]);
          bulk_load(dst + NB * NB, x + (size_t)src * NB, (uint32_t)(NB * sizeof(S)), &full[slot]);
        }
        if (own) bulk_load(dst + NB * NB + NB, x + (size_t)e * NB, (uint32_t)(NB * sizeof(S)), &full[slot]);
      }
    }
    return;
  }

  // ---------------- consumers: lane p <-> (row, group)
  constexpr int NG = Sh::NG;
  const int p = tid;
  const int row = p % NB, g = p / NB;
  const bool active = p < NG * NB;
  for (int li = 0; li < nE; ++li) {
    const int e = (int)blockIdx.x + li * G;
    bool ok = true;
#pragma unroll
    for (int q = 0; q < NBLK; ++q) {
      const int u = li * NBLK + q;
      ok = ok && mbar_wait(&full[u % R], (uint32_t)(u / R) & 1u);
    }
    if (!consumer_all(ok, 32 * CW)) {
      // record the failure, give copies still in flight one more bounded wait, leave
      atomicExch(&g_stream_error, 1);
#pragma unroll
      for (int q = 0; q < NBLK; ++q) {
        const int u = li * NBLK + q;
        mbar_wait(&full[u % R], (uint32_t)(u / R) & 1u);
      }
      return;
    }
    if (active) {
      // eight independent accumulation chains (columns c mod 8) keep the FMA pipe fed
      S acc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = S(0);
      if (NBLK == 4 || NBLK == 3) {
        const int slot = (li * NBLK + g) % R;
        if (pres[slot]) {
          const S* Bs = ring + (size_t)slot * UNIT;
          const S* xs = Bs + NB * NB;
#pragma unroll
          for (int c = 0; c < NB; ++c) acc[c & 7] += Bs[c * NB + row] * xs[c];
        }
      } else {
        const S* Bs = ring + (size_t)(li % R) * UNIT;
        const S* xs = Bs + NB * NB;
        const int c0 = g * NP;
#pragma unroll
        for (int c = 0; c < NP; ++c) acc[c & 7] += Bs[(c0 + c) * NB + row] * xs[c0 + c];
      }
      red[g * NB + row] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    }
    consumer_sync(32 * CW);
    if (p < NB) {
      S s;
      if (NBLK == 3) {
        // y = beta x + B x: beta = 1 gives the folded operator I + B, beta = 0 the
        // shifted Krylov operator B
        const S bx = red[p] + red[NB + p] + red[2 * NB + p];
        s = beta != 0.0 ? ring[(size_t)((li * 3) % R) * UNIT + NB * NB + NB + p] + bx : bx;
      }
      else s = (red[p] + red[NB + p]) + (red[2 * NB + p] + red[3 * NB + p]);
      if (NBLK == 4) {
        s *= S(beta);
        if (alpha != 0.0) {
          const S* xe = ring + (size_t)((li * 4) % R) * UNIT + NB * NB;
          const int a = p / NP, i = p - a * NP;
          S mm = S(0);
          for (int jj = 0; jj < NP; ++jj) mm += S(tb.Mref[i * NP + jj]) * xe[a * NP + jj];
          s += S(alpha * m.detB[e]) * mm;
        }
      }
      y[(size_t)e * NB + p] = s;
    }
    consumer_sync(32 * CW);
    if (p == 0) {
#pragma unroll
      for (int q = 0; q < NBLK; ++q) mbar_arrive(&empty[(li * NBLK + q) % R]);
    }
  }
}

template <int NB, int NBLK, class S>
cudaError_t launch_rows(const DevMesh& m, const DevTables& tb, const S* B, double alpha, double beta, const S* x,
                        S* y, cudaStream_t st) {
  using Sh = StreamShape<NB, NBLK, S>;
  // resident CTAs per SM x SM count, set up once per process (thread-safe static
  // initialization; libpp serves one device per process, see pp_create)
  struct Setup {
    cudaError_t err;
    int grid;
  };
  static const Setup setup = [] {
    Setup r{cudaSuccess, 0};
    r.err = cudaFuncSetAttribute(k_stream_rows<NB, NBLK, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
    if (r.err != cudaSuccess) return r;
    int per_sm = 0, dev = 0, sms = 0;
    r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_rows<NB, NBLK, S>, Sh::THREADS, Sh::SMEM);
    if (r.err != cudaSuccess) return r;
    if ((r.err = cudaGetDevice(&dev)) != cudaSuccess) return r;
    if ((r.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
    if (per_sm < 1) r.err = cudaErrorInvalidConfiguration;
    r.grid = per_sm * sms;
    return r;
  }();
  if (setup.err != cudaSuccess) return setup.err;
  const int grid = setup.grid;
  const int g = m.ne < grid ? m.ne : grid;
  if (g < 1) return cudaSuccess;
  k_stream_rows<NB, NBLK, S><<<g, Sh::THREADS, Sh::SMEM, st>>>(m, tb, B, alpha, beta, x, y);
  return cudaGetLastError();
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

template <class S>
bool stream_rows_supported(int nb, const S* B, const S* x, const S* y) {
  static const bool enabled = [] {
    const char* v = std::getenv("PP_STREAM_ROWS");  // "0" selects the warp-per-block kernels
    return !(v && v[0] == '0');
  }();
  return enabled && (nb == 12 || nb == 24 || nb == 40 || nb == 60) && B && aligned16(B) && aligned16(x) &&
         aligned16(y);
}

template <class S>
cudaError_t launch_stream_rows(const DevMesh& m, const DevTables& tb, int nb, int nblk, const S* B, double alpha,
                               double beta, const S* x, S* y, cudaStream_t st) {
#define PP_ROWS(NBV)                                                                      \
  case NBV:                                                                               \
    return nblk == 4   ? launch_rows<NBV, 4, S>(m, tb, B, alpha, beta, x, y, st)          \
           : nblk == 3 ? launch_rows<NBV, 3, S>(m, tb, B, alpha, beta, x, y, st)          \
                       : launch_rows<NBV, 1, S>(m, tb, B, alpha, beta, x, y, st);
  switch (nb) {
    PP_ROWS(12)
    PP_ROWS(24)
    PP_ROWS(40)
    PP_ROWS(60)
    default:
      return cudaErrorInvalidValue;
  }
#undef PP_ROWS
}

cudaError_t stream_rows_error(int* flag, bool reset) {
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_stream_error, sizeof(int));
  if (e != cudaSuccess || !reset || *flag == 0) return e;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_stream_error, &zero, sizeof(int));
}

template bool stream_rows_supported<double>(int, const double*, const double*, const double*);
template bool stream_rows_supported<float>(int, const float*, const float*, const float*);
template cudaError_t launch_stream_rows<double>(const DevMesh&, const DevTables&, int, int, const double*, double,
                                                double, const double*, double*, cudaStream_t);
template cudaError_t launch_stream_rows<float>(const DevMesh&, const DevTables&, int, int, const float*, double,
                                               double, const float*, float*, cudaStream_t);

}  // namespace pp
