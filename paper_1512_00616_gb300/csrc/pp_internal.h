// Internal declarations of libpp: device-side views of the mesh and the
// reference tables, the forward-mode dual number used for exact derivatives,
// and the kernel launch wrappers shared by the host-side solvers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pp.h"

#define PP_HD __host__ __device__ __forceinline__

namespace pp {

constexpr int kMaxP = 4;
constexpr int kMaxNp = 15;   // (p+1)(p+2)/2 at p = 4
constexpr int kMaxNb = 60;   // 4 * kMaxNp
constexpr int kMaxQv = 36;   // (p+2)^2 volume points at p = 4
constexpr int kMaxQf = 6;    // p+2 face points at p = 4
constexpr int kStages = 3;

// ---------------------------------------------------------------- dual numbers
// Forward-mode derivative carrier: value v and one directional derivative d.
struct Dual {
  double v, d;
  PP_HD Dual() : v(0.0), d(0.0) {}
  PP_HD Dual(double a) : v(a), d(0.0) {}
  PP_HD Dual(double a, double b) : v(a), d(b) {}
};
PP_HD Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
PP_HD Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
PP_HD Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
PP_HD Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
PP_HD Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
PP_HD Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
PP_HD Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
PP_HD Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
PP_HD Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
PP_HD Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
PP_HD Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
PP_HD Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
PP_HD Dual operator/(double a, Dual b) {
  double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}
PP_HD Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
PP_HD Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
PP_HD Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }

PP_HD double val(double a) { return a; }
PP_HD double val(Dual a) { return a.v; }
PP_HD double der(double) { return 0.0; }
PP_HD double der(Dual a) { return a.d; }
__device__ __forceinline__ double sqrtT(double a) { return sqrt(a); }
__device__ __forceinline__ Dual sqrtT(Dual a) {
  double s = sqrt(a.v);
  return Dual(s, 0.5 * a.d / s);
}
// |a| with the branch taken on the value (exact derivative away from a = 0)
PP_HD double absT(double a) { return a >= 0.0 ? a : -a; }
PP_HD Dual absT(Dual a) { return a.v >= 0.0 ? a : -a; }

// ---------------------------------------------------------------- physics and motion
struct Phys {
  double gam, Pr, mu;   // mu: dynamic viscosity 1/Re
  double Uinf[4];
  double x0[2];         // pitching axis in the reference configuration
};

// Rigid-body frame of Eq. defmap at one time: Q (row-major), Q' and h'.
template <class T>
struct FrameT {
  T Q[4];
  T Qd[4];
  T hd;
};

// ---------------------------------------------------------------- device views
struct DevTables {
  int p, Np, nb, nqv, nqf;
  const double* phi_v;   // [nqv][Np]
  const double* dphi_v;  // [nqv][Np][2]  d/dxi, d/deta
  const double* w_v;     // [nqv], sum 1/2
  const double* xi_v;    // [nqv][2]
  const double* phi_f;   // [3][nqf][Np]
  const double* dphi_f;  // [3][nqf][Np][2]
  const double* xi_f;    // [3][nqf][2]
  const double* w_f;     // [nqf], sum 1
  const double* Mref;    // [Np][Np]
  // CDG liftings on the reference element: the scalar lifting l of a jump given at the
  // points of face f, l = sum_j phi_j (Mref^-1 c)_j with c_i = sum_q w_q phi_i(f, q) jump_q,
  // evaluated at the volume points (lift_v) and at the points of face f itself (lift_f)
  const double* lift_v;  // [3][nqv][nqf]
  const double* lift_f;  // [3][nqf][nqf]
};

struct DevMesh {
  int ne;
  const double* X0;      // [ne][2]
  const double* B;       // [ne][4]  row-major 2x2, columns = edge vectors
  const double* BinvT;   // [ne][4]  row-major
  const double* detB;    // [ne]
  const double* N;       // [ne][3][2] reference outward unit normals
  const double* L;       // [ne][3]   face lengths
  const double* s_own;   // [ne][3]   |f| / detB_e  (lifting scale of face f into e)
  const double* s_nbr;   // [ne][3]   |f| / detB of the neighbour (interior faces)
  const double* c11;     // [ne][3]   boundary penalty 10 mu |f| / detB_e (0 on interior faces)
  const int* side;       // [ne][3]   1: e lifts face f and supplies its viscous flux (boundary
                         //           faces, and interior faces whose neighbour has a larger index)
  const int* nbr;        // [ne][3]   neighbour or -1
  const int* nbrface;    // [ne][3]
  const int* tag;        // [ne][3]   0 interior, 1 wall, 2 far field
};

// ---------------------------------------------------------------- kernel wrappers
// All take the stream explicitly and return the launch error (cudaSuccess on success).
cudaError_t launch_residual(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<double>& fr,
                            const double* u, double* r, cudaStream_t st);
// derivative of r with respect to a frame seed (the frame carries the derivative)
cudaError_t launch_residual_dframe(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<Dual>& fr,
                                   const double* u, double* dr, cudaStream_t st);
cudaError_t launch_jacobian(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<double>& fr,
                            const double* u, double* J, cudaStream_t st);
// per-element (P^h, F_x^h) contributions [ne][2]
cudaError_t launch_qoi(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<double>& fr,
                       const double* u, double* per_elem, cudaStream_t st);
cudaError_t launch_qoi_dframe(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<Dual>& fr,
                              const double* u, double* per_elem, cudaStream_t st);
// g = d(w0 P^h + w1 F_x^h)/du  (DEVICE [N_u], zero away from the wall)
cudaError_t launch_qoi_du(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<double>& fr,
                          const double* u, double w0, double w1, double* g, cudaStream_t st);

// Linear-algebra wrappers, templated on the vector/matrix type S (double or float).
// Stage matrix A_e = detB_e Mref (x) I4 - c J_ee (J in FP64), inverted per element by
// Gauss-Jordan with partial pivoting in precision S; AinvT (nullable) receives the
// transposed inverse.
template <class S>
cudaError_t launch_block_inverse(const DevMesh& m, const DevTables& tb, const double* J, double c, S* Ainv, S* AinvT,
                                 int* status, cudaStream_t st);
// y = alpha M x + beta J x (trans = 0) or alpha M x + beta J^T x (trans = 1); J may be null if beta == 0
template <class S>
cudaError_t launch_stage_matvec(const DevMesh& m, const DevTables& tb, const S* J, double alpha, double beta,
                                const S* x, S* y, int trans, cudaStream_t st);
// y = Ainv x (trans = 0) or Ainv^T x (trans = 1), per element
template <class S>
cudaError_t launch_block_apply(const DevMesh& m, int nb, const S* Ainv, const S* x, S* y, int trans, cudaStream_t st);
// JT: per element the transposed blocks of its block-column of J (output type may be narrower)
template <class Si, class So>
cudaError_t launch_transpose_blocks(const DevMesh& m, int nb, const Si* J, So* JT, cudaStream_t st);
template <class Si, class So>
cudaError_t launch_cast(int64_t n, So* y, const Si* x, cudaStream_t st);

// vectors of length n
template <class S>
cudaError_t launch_lincomb(int64_t n, S* y, int nterms, const double* c, const S* const* x,
                           cudaStream_t st);  // y = sum c_k x_k (y may alias one x_k)
cudaError_t launch_scale(int64_t n, double* y, double a, const double* x, cudaStream_t st);  // y = a x
template <class S>
cudaError_t launch_scale_dev(int64_t n, S* y, const double* a, const S* x, cudaStream_t st);  // y = a[0] x
// device-side GMRES bookkeeping; stat = {res, tol, hn, 1/hn, beta, 1/beta, flag, j}
cudaError_t launch_gmres_init(const double* bb, double rtol, double atol, int first, int m, double* g, double* stat,
                              cudaStream_t st);
cudaError_t launch_gmres_backsolve(int ncols, int m, const double* H, const double* g, double* y, cudaStream_t st);
// out[j] = V_j . w for j < k, V contiguous with stride ldv; deterministic two-level reduction
template <class S>
cudaError_t launch_mdot(int64_t n, const S* V, int64_t ldv, int k, const S* w, double* out, double* partial,
                        unsigned* counter, cudaStream_t st);
// w -= V h[0:k]; then out[0:k] = V_j . w  (fused CGS second pass)
template <class S>
cudaError_t launch_update_mdot(int64_t n, const S* V, int64_t ldv, int k, const double* h, S* w, double* out,
                               double* partial, unsigned* counter, cudaStream_t st);
// w -= V h[0:k]; then out[0] = w . w
template <class S>
cudaError_t launch_update_norm2(int64_t n, const S* V, int64_t ldv, int k, const double* h, S* w, double* out,
                                double* partial, unsigned* counter, cudaStream_t st);
// w -= V h[0:k]; out[0] = w . w; then the GMRES Givens update of Hessenberg column j
// One Arnoldi orthogonalization step against V[0..k) with selective reorthogonalization
// (classical Gram-Schmidt, a second pass only when more than half of |w|^2 cancels),
// ending with the Givens update of Hessenberg column j: h1[0..k] <- (V^T w, |w|^2),
// h2 the second-pass coefficients (zero when skipped), nrm[0] = |w|^2 after.
// One fused Arnoldi step (cooperative launch, k <= 40): classical Gram-Schmidt with
// selective reorthogonalization, the Givens update, v_k = w / |w| and the convergence
// record (stat[0..8)) also written to host_stat (a device-visible pinned slot, or null).
// shift: the Krylov operator is A - shift I; H(j, j) gets shift back.
// arn_partial holds arnoldi_partial_words() doubles; arn_bar arnoldi_barrier_words() zeroed
// words (arrival count, release epoch, and an error word set when a barrier wait expired).
template <class S>
cudaError_t launch_arnoldi_step(int64_t n, const S* V, int64_t ldv, int k, S* w, S* vnext, double* h1, double* h2,
                                double* nrm, double* arn_partial, unsigned* arn_bar, double* host_stat, int j, int m,
                                double* H, double* cs, double* sn, double* g, double* stat, double shift,
                                cudaStream_t st);
size_t arnoldi_partial_words();
int arnoldi_barrier_words();       // size of arn_bar in 32-bit words
int arnoldi_barrier_error_word();  // index of the error word in arn_bar
constexpr int kArnoldiFusedMaxK = 40;
template <class S>
cudaError_t launch_arnoldi_ortho(int64_t n, const S* V, int64_t ldv, int k, S* w, double* h1, double* h2,
                                 double* nrm, double* partial, unsigned* counter, int j, int m, double* H, double* cs,
                                 double* sn, double* g, double* stat, double shift, cudaStream_t st);
template <class S>
cudaError_t launch_update_norm2_givens(int64_t n, const S* V, int64_t ldv, int k, const double* h, S* w, double* out,
                                       double* partial, unsigned* counter, int j, int m, const double* h1,
                                       const double* h2, double* H, double* cs, double* sn, double* g, double* stat,
                                       cudaStream_t st);
// out[0] = x . y
template <class S>
cudaError_t launch_dot(int64_t n, const S* x, const S* y, double* out, double* partial, unsigned* counter,
                       cudaStream_t st);
// out[j] = sum over elements of per_elem[e][j], j < k (k <= 8)
cudaError_t launch_colsum(int ne, int k, const double* per_elem, double* out, double* partial, unsigned* counter,
                          cudaStream_t st);

// TMA-staged block-row products (stream_kernels.cu): nblk = 4, the stage operator
// y = alpha M x + beta J x; nblk = 3, the folded operator y = x + B x (beta != 0) or its
// shifted form y = B x (beta = 0); nblk = 1, the block product y = A x.  Normal products only.
template <class S>
bool stream_rows_supported(int nb, const S* B, const S* x, const S* y);
template <class S>
cudaError_t launch_stream_rows(const DevMesh& m, const DevTables& tb, int nb, int nblk, const S* B, double alpha,
                               double beta, const S* x, S* y, cudaStream_t st);
cudaError_t stream_rows_error(int* flag, bool reset);  // bounded-wait expiry flag of those kernels
// BN = -c J_off Ainv_nbr and BT = (-c Ainv_nbr J_off,nbr)^T (3 blocks per element each; BT may
// be null): the block-Jacobi preconditioner folded into the stage operator.
template <class S>
cudaError_t launch_fold_blocks(const DevMesh& m, int nb, const S* J, const S* Ainv, double c, S* BN, S* BT,
                               cudaStream_t st);
int reduction_blocks();  // number of partial sums used by the reductions

}  // namespace pp
