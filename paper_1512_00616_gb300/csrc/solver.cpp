// Host-driven solvers of libpp; every vector lives in device memory and every
// arithmetic step runs in the kernels of dg_kernels.cu / linalg_kernels.cu.
// Only Krylov scalars (Hessenberg column, norms) cross to the host.
//
//  - gmres():          restarted, right-preconditioned GMRES with classical
//                      Gram-Schmidt and selective reorthogonalization (fused
//                      update + multi-dot kernels), Givens rotations on the
//                      device.  Used for the stage solves (on the operator with
//                      the block-Jacobi preconditioner folded in) and, without
//                      preconditioner, for the shooting system (Algorithm primal)
//                      and the periodic adjoint system (Algorithm dual).
//  - primal_sweep():   Eq. dirk2: DIRK3 steps, Newton per stage on
//                      R_i = M k_i - dt r(u_i); stores u_i, dr/du(u_i) and the
//                      block-Jacobi inverse at the converged stage.
//  - tangent_sweep():  Eq. dirk-sens-mvp, returns v - Phi v.
//  - adjoint_sweep():  Eq. uns-disc-adj-dirk2 (with QoI terms) or
//                      Eq. uns-disc-adj-dirk-sens-mvp (without), plus the
//                      gradient reconstruction of Eq. funcl-grad-nosens-dirk.
//  - shoot_nk(), periodic_adjoint(): Algorithms primal, dual and grad.
#include <chrono>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <functional>

#include "context.h"
#include "prof.h"
#include "../../include/pp_prof.h"

namespace pp {

namespace {

template <class S>
using OpT = std::function<int(const S* x, S* y)>;
using Op = OpT<double>;

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <class S>
int host_dot(pp_ctx* ctx, int64_t n, const S* x, const S* y, double* out) {
  PP_CK(launch_dot<S>(n, x, y, ctx->d_scalar, ctx->d_partial, ctx->d_counter, ctx->stream));
  PP_CK(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PP_CK(cudaStreamSynchronize(ctx->stream));
  *out = ctx->h_scalar[0];
  return PP_OK;
}

int host_norm(pp_ctx* ctx, int64_t n, const double* x, double* out) {
  double d;
  PP_TRY(host_dot<double>(ctx, n, x, x, &d));
  *out = std::sqrt(d);
  if (!std::isfinite(*out)) return set_error(ctx, PP_ENAN, "non-finite norm");
  return PP_OK;
}

// Bounded-wait expiry in the TMA-staged block-row kernels (checked at sweep ends).
int check_stream_kernels(pp_ctx* ctx) {
  int flag = 0;
  PP_CK(stream_rows_error(&flag, true));
  if (flag) return set_error(ctx, PP_ECUDA, "block-row kernel: shared-memory pipeline wait expired");
  unsigned err = 0u;
  PP_CK(cudaMemcpy(&err, ctx->d_arn_bar + arnoldi_barrier_error_word(), sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (err != 0u) {
    PP_CK(cudaMemset(ctx->d_arn_bar, 0, sizeof(unsigned) * arnoldi_barrier_words()));
    return set_error(ctx, PP_ECUDA, "Arnoldi step: grid barrier wait expired");
  }
  return PP_OK;
}

template <class S>
int lincomb(pp_ctx* ctx, int64_t n, S* y, std::initializer_list<double> c, std::initializer_list<const S*> x) {
  double cc[4];
  const S* xx[4];
  int k = 0;
  auto it = x.begin();
  for (double v : c) {
    cc[k] = v;
    xx[k] = *it++;
    ++k;
  }
  PP_CK(launch_lincomb<S>(n, y, k, cc, xx, ctx->stream));
  return PP_OK;
}

int lincomb(pp_ctx* ctx, int64_t n, double* y, std::initializer_list<double> c,
            std::initializer_list<const double*> x) {
  return lincomb<double>(ctx, n, y, c, x);
}

template <class S>
int copy(pp_ctx* ctx, int64_t n, S* y, const S* x) {
  if (y != x) PP_CK(cudaMemcpyAsync(y, x, sizeof(S) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  return PP_OK;
}

// Restarted GMRES for A x = b, x0 = 0, in vector type S.  Right-preconditioned
// (x = P(V y)) or, with K.Z set and flexible = true, flexible (z_j = P(v_j) stored,
// x = Z y) so that the preconditioner may change between iterations.  Stops when
// ||b - A x|| <= max(rtol ||b||, atol) (Arnoldi estimate) or after maxit Krylov steps.
//
// The Hessenberg column, Givens rotations and residual estimate are kept on the
// device; the host watches the convergence flag one Arnoldi step behind (event +
// pinned copy per step), so the GPU queue never drains for a round trip.  The step
// enqueued past convergence is simply not used (its column is beyond ncols).
template <class S>
int gmres(pp_ctx* ctx, KrylovT<S>& K, const OpT<S>& A, const OpT<S>& prec, const S* b, S* x, double rtol,
          double atol, int maxit, int* iters, double* res_out, bool flexible = false, bool warm = false,
          double shift = 0.0) {
  const int64_t n = K.n;
  const int m = K.m;
  double* d_h1 = K.d_h;
  double* d_h2 = K.d_h + (m + 2);
  double* d_nrm = K.d_h + 2 * (m + 2);
  const bool flex = flexible && K.Z && prec;
  bool first = true;
  if (warm) {
    // initial guess in x: the tolerance stays relative to |b| (set here), the first cycle
    // starts from r = b - A x
    PP_CK(launch_dot<S>(n, b, b, d_nrm, ctx->d_partial, ctx->d_counter, ctx->stream));
    PP_CK(launch_gmres_init(d_nrm, rtol, atol, 1, m, K.d_g, K.d_stat, ctx->stream));
    PP_TRY(A(x, K.w));
    if (shift != 0.0) PP_TRY(lincomb<S>(ctx, n, K.r, {1.0, -1.0, -shift}, {b, K.w, x}));
    else PP_TRY(lincomb<S>(ctx, n, K.r, {1.0, -1.0}, {b, K.w}));
    first = false;
  } else {
    PP_CK(cudaMemsetAsync(x, 0, sizeof(S) * n, ctx->stream));
    PP_TRY(copy<S>(ctx, n, K.r, b));
  }
  int total = 0;
  double res = 0.0;
  int status = PP_ENOCONV;
  for (;;) {
    PP_CK(launch_dot<S>(n, K.r, K.r, d_nrm, ctx->d_partial, ctx->d_counter, ctx->stream));
    PP_CK(launch_gmres_init(d_nrm, rtol, atol, first ? 1 : 0, m, K.d_g, K.d_stat, ctx->stream));
    PP_CK(launch_scale_dev<S>(n, K.V, K.d_stat + 5, K.r, ctx->stream));
    first = false;
    int ncols = 0;
    double flag = 0.0;
    for (int j = 0; j < m; ++j) {
      S* vj = K.V + (size_t)j * n;
      const S* z = vj;
      if (prec) {
        S* zj = flex ? K.Z + (size_t)j * n : K.t;
        PP_TRY(prec(vj, zj));
        z = zj;
      }
      PP_TRY(A(z, K.w));
      double* slot = K.h_h + 8 * (j % kRing);
      S* vnext = K.V + (size_t)(j + 1) * n;
      if (j + 1 <= kArnoldiFusedMaxK && K.h_h_dev) {
        // one cooperative launch: orthogonalization, Givens, scaling, record into the ring
        PP_CK(launch_arnoldi_step<S>(n, K.V, n, j + 1, K.w, vnext, d_h1, d_h2, d_nrm, ctx->d_arn, ctx->d_arn_bar,
                                     K.h_h_dev + 8 * (j % kRing), j, m, K.d_H, K.d_cs, K.d_sn, K.d_g, K.d_stat,
                                     shift, ctx->stream));
        PP_CK(cudaEventRecord(K.ev[j % kRing], ctx->stream));
      } else {
        PP_CK(launch_arnoldi_ortho<S>(n, K.V, n, j + 1, K.w, d_h1, d_h2, d_nrm, ctx->d_partial, ctx->d_counter, j,
                                      m, K.d_H, K.d_cs, K.d_sn, K.d_g, K.d_stat, shift, ctx->stream));
        PP_CK(cudaMemcpyAsync(slot, K.d_stat, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        PP_CK(cudaEventRecord(K.ev[j % kRing], ctx->stream));
        PP_CK(launch_scale_dev<S>(n, vnext, K.d_stat + 3, K.w, ctx->stream));
      }
      ++total;
      // look one step behind
      const int jl = (j == m - 1) ? j : j - 1;
      if (jl < 0) continue;
      PP_CK(cudaEventSynchronize(K.ev[jl % kRing]));
      const double* st = K.h_h + 8 * (jl % kRing);
      flag = st[6];
      res = st[0];
      if (flag >= 8.0) {
        PP_CK(cudaStreamSynchronize(ctx->stream));
        PP_CK(cudaMemsetAsync(ctx->d_arn_bar, 0, sizeof(unsigned) * arnoldi_barrier_words(), ctx->stream));
        PP_CK(cudaStreamSynchronize(ctx->stream));
        return set_error(ctx, PP_ECUDA, "GMRES: Arnoldi grid barrier wait expired");
      }
      if (flag >= 4.0) return set_error(ctx, PP_ENAN, "GMRES: non-finite Arnoldi quantity");
      if (flag > 0.0 || total - (j - jl) >= maxit || j == m - 1) {
        ncols = jl + 1;
        break;
      }
    }
    if (ncols == 0) ncols = 1;
    // x += P(V y)  or  x += Z y
    PP_CK(launch_gmres_backsolve(ncols, m, K.d_H, K.d_g, K.d_y, ctx->stream));
    PP_CK(cudaMemsetAsync(K.w, 0, sizeof(S) * n, ctx->stream));
    PP_CK(launch_update_norm2<S>(n, flex ? K.Z : K.V, n, ncols, K.d_y, K.w, d_nrm, ctx->d_partial, ctx->d_counter,
                                 ctx->stream));
    if (prec && !flex) {
      PP_TRY(prec(K.w, K.t));
      PP_TRY(lincomb<S>(ctx, n, x, {1.0, 1.0}, {x, K.t}));
    } else {
      PP_TRY(lincomb<S>(ctx, n, x, {1.0, 1.0}, {x, K.w}));
    }
    if (flag == 1.0 || flag == 2.0) {
      status = PP_OK;
      break;
    }
    if (total >= maxit) break;
    // restart from the true residual r = b - A x
    PP_TRY(A(x, K.w));
    if (shift != 0.0) PP_TRY(lincomb<S>(ctx, n, K.r, {1.0, -1.0, -shift}, {b, K.w, x}));
    else PP_TRY(lincomb<S>(ctx, n, K.r, {1.0, -1.0}, {b, K.w}));
  }
  if (iters) *iters = total;
  if (res_out) *res_out = res;
  return status;
}

struct StageView {
  const double* J;
  const double* Ainv;             // FP64 mode
  double c;                       // a_ii dt
  const double* JT = nullptr;     // transposed block-columns (optional)
  const double* AinvT = nullptr;  // transposed inverses (optional, FP64 mode)
  const float* J32 = nullptr;     // mixed mode FP32 copies
  const float* JT32 = nullptr;
  const float* A32 = nullptr;
  const float* AT32 = nullptr;
  const double* BN = nullptr;     // folded operator I + BN = (M - cJ) D^{-1} (optional, FP64 mode)
  const double* BT = nullptr;     // folded transposed operator I + BT = (M - cJ)^T D^{-T}
  const float* BN32 = nullptr;    // mixed mode: FP32 folded blocks of the inner solves
  const float* BT32 = nullptr;
};

// FP32 GMRES on the FP32 stage operator (block-Jacobi FP32 preconditioner), b and x FP32.
int stage_solve32(pp_ctx* ctx, const pp_mesh* mesh, const StageView& sv, int trans, const float* b, float* x,
                  double rtol, int maxit, int* iters) {
  const DevMesh& m = mesh->dev;
  const float* Bf = trans ? sv.BT32 : sv.BN32;
  if (Bf) {
    // folded operator: GMRES on (I + B) y = b, then x = D^{-1} y (D^{-T} y)
    float* yv = ctx->k32.t;
    // Krylov recurrence on B (Arnoldi adds the unit shift back to H): w = B v keeps most of
    // its norm after the projections, where w = (I + B) v cancels down to |B v|
    OpT<float> A = [&](const float* in, float* out) {
      ProfScope ps(PP_K_STAGE_OP32, ctx->stream);
      PP_CK(launch_stream_rows<float>(m, ctx->tb, ctx->tb.nb, 3, Bf, 0.0, 0.0, in, out, ctx->stream));
      return PP_OK;
    };
    int st = gmres<float>(ctx, ctx->k32, A, OpT<float>(), b, yv, rtol, 0.0, maxit, iters, nullptr, false, false,
                          1.0);
    if (st != PP_OK && st != PP_ENOCONV) return st;
    PP_CK(launch_block_apply<float>(m, ctx->tb.nb, trans ? sv.AT32 : sv.A32, yv, x, 0, ctx->stream));
    return PP_OK;  // an inexact inner / Newton solve is acceptable
  }
  const float* Jm = trans ? sv.JT32 : sv.J32;   // the transposed copies run through the normal kernels
  const float* Am = trans ? sv.AT32 : sv.A32;
  OpT<float> A = [&](const float* in, float* out) {
    PP_CK(launch_stage_matvec<float>(m, ctx->tb, Jm, 1.0, -sv.c, in, out, 0, ctx->stream));
    return PP_OK;
  };
  OpT<float> P = [&](const float* in, float* out) {
    PP_CK(launch_block_apply<float>(m, ctx->tb.nb, Am, in, out, 0, ctx->stream));
    return PP_OK;
  };
  int st = gmres<float>(ctx, ctx->k32, A, P, b, x, rtol, 0.0, maxit, iters, nullptr);
  return st == PP_ENOCONV ? PP_OK : st;  // an inexact inner / Newton solve is acceptable
}

// Stage solve (M - c J) x = b or its transpose.  exact = false (primal Newton steps)
// may be inexact; exact = true (tangent / adjoint) must reach rtol on the FP64 operator.
int stage_solve(pp_ctx* ctx, const pp_mesh* mesh, const StageView& sv, int trans, const double* b, double* x,
                double rtol, double atol, int* iters, bool exact, double* ywarm = nullptr, bool use_warm = false) {
  const DevMesh& m = mesh->dev;
  const int64_t n = ctx->ws_nu;
  if (ctx->cfg.precision == PP_PREC_MIXED) {
    float* b32 = ctx->d_vec32;
    float* x32 = ctx->d_vec32 + n;
    if (!exact) {
      PP_CK(launch_cast<double, float>(n, b32, b, ctx->stream));
      PP_TRY(stage_solve32(ctx, mesh, sv, trans, b32, x32, rtol, ctx->cfg.gmres_maxit, iters));
      PP_CK(launch_cast<float, double>(n, x, x32, ctx->stream));
      return PP_OK;
    }
    // FP64 flexible GMRES on the exact operator, FP32 GMRES as the preconditioner
    const bool useT = trans && sv.JT;
    const double* Jm = useT ? sv.JT : sv.J;
    const int tr = useT ? 0 : trans;
    int inner_total = 0;
    Op A = [&](const double* in, double* out) {
      PP_CK(launch_stage_matvec<double>(m, ctx->tb, Jm, 1.0, -sv.c, in, out, tr, ctx->stream));
      return PP_OK;
    };
    Op P = [&](const double* in, double* out) {
      int it = 0;
      PP_CK(launch_cast<double, float>(n, b32, in, ctx->stream));
      PP_TRY(stage_solve32(ctx, mesh, sv, trans, b32, x32, ctx->cfg.inner_rtol, ctx->cfg.inner_maxit, &it));
      PP_CK(launch_cast<float, double>(n, out, x32, ctx->stream));
      inner_total += it;
      return PP_OK;
    };
    int outer = 0;
    int st = gmres<double>(ctx, ctx->kin, A, P, b, x, rtol, atol, ctx->cfg.gmres_maxit, &outer, nullptr, true);
    if (iters) *iters = outer + inner_total;
    if (st == PP_ENOCONV) return set_error(ctx, PP_ENOCONV, "stage FGMRES hit gmres_maxit");
    return st;
  }
  // FP64 path with the folded operator: GMRES on (I + B) y = b, then x = D^{-1} y (D^{-T} y)
  const double* Bf = trans ? sv.BT : sv.BN;
  if (Bf) {
    double* yv = ctx->kin.t;  // unused by GMRES without a preconditioner
    // Krylov recurrence on B, shifted back in H (see stage_solve32)
    Op A = [&](const double* in, double* out) {
      ProfScope ps(PP_K_STAGE_OP, ctx->stream);
      PP_CK(launch_stream_rows<double>(m, ctx->tb, ctx->tb.nb, 3, Bf, 0.0, 0.0, in, out, ctx->stream));
      return PP_OK;
    };
    // warm start (linear sweeps): the same stage's y of the previous step is the initial guess
    if (ywarm && use_warm) PP_TRY(copy(ctx, n, yv, ywarm));
    int st = gmres<double>(ctx, ctx->kin, A, Op(), b, yv, rtol, atol, ctx->cfg.gmres_maxit, iters, nullptr, false,
                           ywarm && use_warm, 1.0);
    if (st != PP_OK && st != PP_ENOCONV) return st;
    if (ywarm) PP_TRY(copy(ctx, n, ywarm, yv));
    if (!trans) PP_CK(launch_block_apply<double>(m, ctx->tb.nb, sv.Ainv, yv, x, 0, ctx->stream));
    else if (sv.AinvT) PP_CK(launch_block_apply<double>(m, ctx->tb.nb, sv.AinvT, yv, x, 0, ctx->stream));
    else PP_CK(launch_block_apply<double>(m, ctx->tb.nb, sv.Ainv, yv, x, 1, ctx->stream));
    if (st == PP_ENOCONV && exact) return set_error(ctx, PP_ENOCONV, "stage GMRES hit gmres_maxit");
    return PP_OK;
  }
  // FP64 path: with stored transposes the transposed system uses the normal (row-streaming) kernels
  const bool useT = trans && sv.JT && sv.AinvT;
  const double* Jm = useT ? sv.JT : sv.J;
  const double* Am = useT ? sv.AinvT : sv.Ainv;
  const int tr = useT ? 0 : trans;
  Op A = [&](const double* in, double* out) {
    PP_CK(launch_stage_matvec<double>(m, ctx->tb, Jm, 1.0, -sv.c, in, out, tr, ctx->stream));
    return PP_OK;
  };
  Op P = [&](const double* in, double* out) {
    PP_CK(launch_block_apply<double>(m, ctx->tb.nb, Am, in, out, tr, ctx->stream));
    return PP_OK;
  };
  int st = gmres<double>(ctx, ctx->kin, A, P, b, x, rtol, atol, ctx->cfg.gmres_maxit, iters, nullptr);
  if (st == PP_ENOCONV) {
    if (!exact) return PP_OK;
    return set_error(ctx, PP_ENOCONV, "stage GMRES hit gmres_maxit");
  }
  return st;
}

size_t nb2(const pp_ctx* ctx) { return (size_t)ctx->tb.nb * ctx->tb.nb; }

StageView stage_view_slot(pp_ctx* ctx, size_t s, double c) {
  const size_t ne = ctx->lin_mesh->ne;
  StageView v{ctx->st_J + s * ne * 4 * nb2(ctx), ctx->st_Ainv ? ctx->st_Ainv + s * ne * nb2(ctx) : nullptr, c};
  if (ctx->st_JT) v.JT = ctx->st_JT + s * ne * 4 * nb2(ctx);
  if (ctx->st_AinvT) v.AinvT = ctx->st_AinvT + s * ne * nb2(ctx);
  if (ctx->st_BN) v.BN = ctx->st_BN + s * ne * 3 * nb2(ctx);
  if (ctx->st_BT) v.BT = ctx->st_BT + s * ne * 3 * nb2(ctx);
  if (ctx->st_BN32) v.BN32 = ctx->st_BN32 + s * ne * 3 * nb2(ctx);
  if (ctx->st_BT32) v.BT32 = ctx->st_BT32 + s * ne * 3 * nb2(ctx);
  if (ctx->st_J32) {
    v.J32 = ctx->st_J32 + s * ne * 4 * nb2(ctx);
    v.JT32 = ctx->st_JT32 + s * ne * 4 * nb2(ctx);
    v.A32 = ctx->st_A32 + s * ne * nb2(ctx);
    v.AT32 = ctx->st_AT32 + s * ne * nb2(ctx);
  }
  return v;
}

StageView stored_stage(pp_ctx* ctx, int n, int i) {
  return stage_view_slot(ctx, (size_t)(n - ctx->seg_base) * 3 + i, ctx->A[i][i] * ctx->cfg.T / ctx->lin_Nt);
}

const double* stored_u(pp_ctx* ctx, int n, int i) {
  return ctx->st_u + ((size_t)(n - ctx->seg_base) * 3 + i) * ctx->ws_nu;
}

// Everything a stage slot stores from the FP64 Jacobian in slot J (already assembled):
// preconditioner(s), transposed copies and FP32 copies, as the precision mode needs.
int finalize_stage_slot(pp_ctx* ctx, const pp_mesh* mesh, const StageView& sv, bool full) {
  const DevMesh& m = mesh->dev;
  const int nb = ctx->tb.nb;
  const size_t nJ = (size_t)mesh->ne * 4 * nb2(ctx);
  if (ctx->cfg.precision == PP_PREC_MIXED) {
    PP_CK(launch_cast<double, float>((int64_t)nJ, const_cast<float*>(sv.J32), sv.J, ctx->stream));
    PP_CK(launch_block_inverse<float>(m, ctx->tb, sv.J, sv.c, const_cast<float*>(sv.A32),
                                      full ? const_cast<float*>(sv.AT32) : nullptr, ctx->d_status, ctx->stream));
    if (full) {
      PP_CK(launch_transpose_blocks<double, float>(m, nb, sv.J, const_cast<float*>(sv.JT32), ctx->stream));
      if (sv.JT) PP_CK(launch_transpose_blocks<double, double>(m, nb, sv.J, const_cast<double*>(sv.JT), ctx->stream));
    }
    if (sv.BN32)
      PP_CK(launch_fold_blocks<float>(m, nb, sv.J32, sv.A32, sv.c, const_cast<float*>(sv.BN32),
                                      full && sv.BT32 ? const_cast<float*>(sv.BT32) : nullptr, ctx->stream));
    return PP_OK;
  }
  PP_CK(launch_block_inverse<double>(m, ctx->tb, sv.J, sv.c, const_cast<double*>(sv.Ainv),
                                     full ? const_cast<double*>(sv.AinvT) : nullptr, ctx->d_status, ctx->stream));
  if (full && sv.JT)
    PP_CK(launch_transpose_blocks<double, double>(m, nb, sv.J, const_cast<double*>(sv.JT), ctx->stream));
  if (sv.BN)
    PP_CK(launch_fold_blocks(m, nb, sv.J, sv.Ainv, sv.c, const_cast<double*>(sv.BN),
                             full && sv.BT ? const_cast<double*>(sv.BT) : nullptr, ctx->stream));
  return PP_OK;
}

}  // namespace

// --------------------------------------------------------------------------- primal sweep
namespace {

// DIRK steps [s0, s1) of a period of Nt steps from state u with Newton predictor kprev
// (both updated in place).  Stage slot of (step, i) is (step - ctx->seg_base)*3 + i.
// record: accumulate the QoI rates and write u_traj (off when a checkpointed segment is
// recomputed).  The chord-Newton matrix restarts at s0, so a recomputation from a
// checkpoint follows exactly the original iterates.
int run_steps(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double* u, double* kprev, int s0, int s1,
              int Nt, bool record, double* u_traj) {
  const DevMesh& m = mesh->dev;
  const int64_t n = ctx->ws_nu;
  const double dt = ctx->cfg.T / Nt;
  double* k[3] = {work_vec(ctx, 1), work_vec(ctx, 2), work_vec(ctx, 3)};
  double* base = work_vec(ctx, 4);
  double* r = work_vec(ctx, 5);
  double* R = work_vec(ctx, 6);
  double* dk = work_vec(ctx, 7);
  // chord Newton: all stages share a_ii = gamma, so the stored matrix of the previous
  // stage (exact at its converged state) is the Newton matrix until contraction slows
  StageView nview{};
  bool have_nview = false;
  for (int step = s0; step < s1; ++step) {
    const double t0 = step * dt;
    for (int i = 0; i < 3; ++i) {
      const double ti = t0 + ctx->c[i] * dt;
      const double c = ctx->A[i][i] * dt;
      Motion mo = motion(ctx, mu, n_mu, ti);
      FrameT<double> fr = frame_of(mo);
      // base = u + sum_{j<i} a_ij k_j
      if (i == 0) PP_TRY(copy(ctx, n, base, u));
      if (i == 1) PP_TRY(lincomb(ctx, n, base, {1.0, ctx->A[1][0]}, {u, k[0]}));
      if (i == 2) PP_TRY(lincomb(ctx, n, base, {1.0, ctx->A[2][0], ctx->A[2][1]}, {u, k[0], k[1]}));
      PP_TRY(copy(ctx, n, k[i], i == 0 ? kprev : k[i - 1]));
      const size_t slot = (size_t)(step - ctx->seg_base) * 3 + i;
      const size_t qslot = (size_t)step * 3 + i;
      const StageView sview = stage_view_slot(ctx, slot, c);
      double* Js = const_cast<double*>(sview.J);
      double* us = ctx->st_u + slot * n;
      double prev_res = INFINITY, alpha = 1.0;
      int backtracks = 0;
      bool converged = false, refresh = !have_nview;
      for (int it = 0; it <= ctx->cfg.newton_maxit; ++it) {
        PP_TRY(lincomb(ctx, n, us, {1.0, ctx->A[i][i]}, {base, k[i]}));
        PP_CK(launch_residual(m, ctx->tb, ctx->ph, fr, us, r, ctx->stream));
        PP_CK(launch_stage_matvec<double>(m, ctx->tb, nullptr, 1.0, 0.0, k[i], R, 0, ctx->stream));
        PP_TRY(lincomb(ctx, n, R, {1.0, -dt}, {R, r}));
        double rn2, mun;
        PP_TRY(host_dot<double>(ctx, n, R, R, &rn2));
        double rn = std::sqrt(rn2);
        // backtracking safeguard: a step that made the residual non-finite or larger is halved
        if (it > 0 && (!std::isfinite(rn) || rn > prev_res) && backtracks < 8) {
          alpha *= 0.5;
          ++backtracks;
          refresh = true;
          PP_TRY(lincomb(ctx, n, k[i], {1.0, alpha}, {k[i], dk}));
          continue;
        }
        if (!std::isfinite(rn)) return set_error(ctx, PP_ENAN, "non-finite stage residual");
        if (it > 0 && rn > 0.25 * prev_res) refresh = true;  // slow chord contraction
        alpha = 1.0;
        PP_CK(launch_stage_matvec<double>(m, ctx->tb, nullptr, 1.0, 0.0, us, dk, 0, ctx->stream));
        PP_TRY(host_norm(ctx, n, dk, &mun));
        const double tol = ctx->cfg.newton_tol * mun;
        if (rn <= tol || (it > 0 && rn <= 1e3 * tol && rn > 0.5 * prev_res)) {
          converged = true;
          break;
        }
        if (it == ctx->cfg.newton_maxit) break;
        if (refresh) {
          // Newton matrix at the current iterate (this stage's slot doubles as scratch)
          PP_CK(launch_jacobian(m, ctx->tb, ctx->ph, fr, us, Js, ctx->stream));
          PP_TRY(finalize_stage_slot(ctx, mesh, sview, false));
          nview = sview;
          have_nview = true;
          refresh = false;
        }
        prev_res = rn;
        int gits = 0;
        int st = stage_solve(ctx, mesh, nview, 0, R, dk, ctx->cfg.gmres_rtol, 0.0, &gits, false);
        if (st != PP_OK && st != PP_ENOCONV) return st;
        ctx->last_gmres_iters += gits;
        PP_TRY(lincomb(ctx, n, k[i], {1.0, -1.0}, {k[i], dk}));
        ctx->last_newton_iters++;
      }
      if (converged) {
        // exact Jacobian and preconditioner(s) at the converged stage: the stored linearization
        PP_CK(launch_jacobian(m, ctx->tb, ctx->ph, fr, us, Js, ctx->stream));
        PP_TRY(finalize_stage_slot(ctx, mesh, sview, true));
        nview = sview;
        have_nview = true;
      }
      if (!converged) return set_error(ctx, PP_ENOCONV, "stage Newton did not converge");
      int status = 0;
      PP_CK(cudaMemcpyAsync(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      PP_CK(cudaStreamSynchronize(ctx->stream));
      if (status) {
        PP_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
        return set_error(ctx, PP_ENAN, "singular or non-finite stage block");
      }
      if (!record) continue;
      // QoI rates at the converged stage
      PP_CK(launch_qoi(m, ctx->tb, ctx->ph, fr, us, ctx->d_elem, ctx->stream));
      PP_CK(launch_colsum(mesh->ne, 2, ctx->d_elem, ctx->d_scalar + 8, ctx->d_partial, ctx->d_counter, ctx->stream));
      PP_CK(cudaMemcpyAsync(ctx->h_scalar + 8, ctx->d_scalar + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream));
      PP_CK(cudaStreamSynchronize(ctx->stream));
      ctx->lin_qoi_rates[qslot * 2] = ctx->h_scalar[8];
      ctx->lin_qoi_rates[qslot * 2 + 1] = ctx->h_scalar[9];
    }
    PP_TRY(lincomb(ctx, n, u, {1.0, ctx->b[0], ctx->b[1], ctx->b[2]}, {u, k[0], k[1], k[2]}));
    PP_TRY(copy(ctx, n, kprev, k[2]));
    if (u_traj) PP_TRY(copy(ctx, n, u_traj + (size_t)(step + 1) * n, u));
  }
  return PP_OK;
}

// Makes the stage data of step `step` resident (checkpointed linearization: recompute
// its segment from the stored state and predictor at the segment start).
int ensure_segment(pp_ctx* ctx, int step) {
  const int K = ctx->cfg.checkpoint_stride;
  if (K <= 0) return PP_OK;
  const int seg = step / K;
  if (seg == ctx->seg_cur) return PP_OK;
  const int64_t n = ctx->ws_nu;
  double* u = work_vec(ctx, 0);
  double* kprev = work_vec(ctx, 8);
  PP_TRY(copy(ctx, n, u, ctx->ck_u + (size_t)seg * n));
  PP_TRY(copy(ctx, n, kprev, ctx->ck_k + (size_t)seg * n));
  ctx->seg_base = seg * K;
  const int s1 = std::min((seg + 1) * K, ctx->lin_Nt);
  PP_TRY(run_steps(ctx, ctx->lin_mesh, ctx->lin_mu.data(), (int)ctx->lin_mu.size(), u, kprev, seg * K, s1,
                   ctx->lin_Nt, false, nullptr));
  ctx->seg_cur = seg;
  ctx->recomputed_segments++;
  return PP_OK;
}

}  // namespace

int primal_sweep(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                 double* u_traj, double* u_final, double* qoi) {
  PP_TRY(ensure_store(ctx, mesh, Nt));
  ctx->lin_valid = false;
  ctx->lin_mesh = mesh;
  ctx->lin_mu.assign(mu, mu + n_mu);
  ctx->lin_Nt = Nt;
  const int64_t n = ctx->ws_nu;
  const double dt = ctx->cfg.T / Nt;
  double* u = work_vec(ctx, 0);
  double* kprev = work_vec(ctx, 8);
  PP_TRY(copy(ctx, n, u, u0));
  PP_CK(cudaMemsetAsync(kprev, 0, sizeof(double) * n, ctx->stream));
  if (u_traj) PP_TRY(copy(ctx, n, u_traj, u));
  ctx->lin_qoi_rates.assign((size_t)Nt * 6, 0.0);
  ctx->last_newton_iters = 0;
  ctx->last_gmres_iters = 0;
  const int K = ctx->cfg.checkpoint_stride;
  if (K <= 0) {
    ctx->seg_base = 0;
    PP_TRY(run_steps(ctx, mesh, mu, n_mu, u, kprev, 0, Nt, Nt, true, u_traj));
  } else {
    // store (u, predictor) at every K-th step; keep one segment of stage data resident
    const int nseg = (Nt + K - 1) / K;
    for (int seg = 0; seg < nseg; ++seg) {
      PP_TRY(copy(ctx, n, ctx->ck_u + (size_t)seg * n, u));
      PP_TRY(copy(ctx, n, ctx->ck_k + (size_t)seg * n, kprev));
      ctx->seg_base = seg * K;
      PP_TRY(run_steps(ctx, mesh, mu, n_mu, u, kprev, seg * K, std::min((seg + 1) * K, Nt), Nt, true, u_traj));
      ctx->seg_cur = seg;
    }
  }
  double W = 0.0, Jx = 0.0;
  for (int step = 0; step < Nt; ++step)
    for (int i = 0; i < 3; ++i) {
      W += dt * ctx->b[i] * ctx->lin_qoi_rates[((size_t)step * 3 + i) * 2];
      Jx += dt * ctx->b[i] * ctx->lin_qoi_rates[((size_t)step * 3 + i) * 2 + 1];
    }
  ctx->lin_W = W;
  ctx->lin_Jx = Jx;
  if (qoi) {
    qoi[0] = W;
    qoi[1] = Jx;
    qoi[2] = -W / ctx->cfg.T;
    qoi[3] = -Jx / ctx->cfg.T;
  }
  if (u_final) PP_TRY(copy(ctx, n, u_final, u));
  PP_CK(cudaStreamSynchronize(ctx->stream));
  PP_TRY(check_stream_kernels(ctx));
  ctx->lin_valid = true;
  return PP_OK;
}

// --------------------------------------------------------------------------- tangent sweep
int tangent_sweep(pp_ctx* ctx, const double* v, double* out) {
  const pp_mesh* mesh = ctx->lin_mesh;
  const DevMesh& m = mesh->dev;
  const int64_t n = ctx->ws_nu;
  const int Nt = ctx->lin_Nt;
  const double dt = ctx->cfg.T / Nt;
  double* du = work_vec(ctx, 9);
  double* dk[3] = {work_vec(ctx, 10), work_vec(ctx, 11), work_vec(ctx, 12)};
  double* w = work_vec(ctx, 13);
  double* rhs = work_vec(ctx, 14);
  double* v0 = work_vec(ctx, 15);
  PP_TRY(copy(ctx, n, v0, v));
  PP_TRY(copy(ctx, n, du, v));
  ctx->last_gmres_tangent = 0;
  for (int step = 0; step < Nt; ++step) {
    PP_TRY(ensure_segment(ctx, step));
    for (int i = 0; i < 3; ++i) {
      StageView sv = stored_stage(ctx, step, i);
      const double* win = du;
      if (i == 1) {
        PP_TRY(lincomb(ctx, n, w, {1.0, ctx->A[1][0]}, {du, dk[0]}));
        win = w;
      } else if (i == 2) {
        PP_TRY(lincomb(ctx, n, w, {1.0, ctx->A[2][0], ctx->A[2][1]}, {du, dk[0], dk[1]}));
        win = w;
      }
      PP_CK(launch_stage_matvec<double>(m, ctx->tb, sv.J, 0.0, dt, win, rhs, 0, ctx->stream));
      int gits = 0;
      PP_TRY(stage_solve(ctx, mesh, sv, 0, rhs, dk[i], ctx->cfg.lin_rtol, 0.0, &gits, true, work_vec(ctx, 27 + i),
                         step > 0));
      ctx->last_gmres_tangent += gits;
    }
    PP_TRY(lincomb(ctx, n, du, {1.0, ctx->b[0], ctx->b[1], ctx->b[2]}, {du, dk[0], dk[1], dk[2]}));
  }
  PP_TRY(lincomb(ctx, n, out, {1.0, -1.0}, {v0, du}));
  PP_CK(cudaStreamSynchronize(ctx->stream));
  PP_TRY(check_stream_kernels(ctx));
  return PP_OK;
}

// --------------------------------------------------------------------------- adjoint sweep
int adjoint_sweep(pp_ctx* ctx, const double* lam_Nt, const double* weights, double* lam0, double* dFdmu) {
  const pp_mesh* mesh = ctx->lin_mesh;
  const DevMesh& m = mesh->dev;
  const int64_t n = ctx->ws_nu;
  const int Nt = ctx->lin_Nt;
  const double dt = ctx->cfg.T / Nt;
  const int n_mu = (int)ctx->lin_mu.size();
  const double* mu = ctx->lin_mu.data();
  double* lam = work_vec(ctx, 16);
  double* kap = work_vec(ctx, 17);
  double* y[3] = {work_vec(ctx, 18), work_vec(ctx, 19), work_vec(ctx, 20)};
  double* g[3] = {work_vec(ctx, 21), work_vec(ctx, 22), work_vec(ctx, 23)};
  double* rhs = work_vec(ctx, 14);
  double* dr = work_vec(ctx, 15);
  const bool withF = weights != nullptr;
  const double w0 = withF ? weights[0] : 0.0, w1 = withF ? weights[1] : 0.0;
  std::vector<double> grad(n_mu, 0.0);
  // kappa_i . dr/ds and the two QoI-rate derivatives for the 3 motion seeds of every stage stay
  // on the device until the sweep ends: one read-back instead of one host sync per stage.
  const size_t n_st = (size_t)3 * Nt;
  std::vector<double> ds_host;
  if (withF && dFdmu) {
    if (ctx->gterm_cap < n_st) {
      PP_CK(cudaStreamSynchronize(ctx->stream));
      cudaFree(ctx->d_gterm);
      ctx->d_gterm = nullptr;
      ctx->gterm_cap = 0;
      PP_CK(cudaMalloc(&ctx->d_gterm, sizeof(double) * 9 * n_st));
      ctx->gterm_cap = n_st;
    }
    ds_host.assign(n_st * 3 * (size_t)n_mu, 0.0);
  }
  PP_TRY(copy(ctx, n, lam, lam_Nt));
  ctx->last_gmres_adjoint = 0;
  for (int step = Nt - 1; step >= 0; --step) {
    PP_TRY(ensure_segment(ctx, step));
    for (int i = 2; i >= 0; --i) {
      StageView sv = stored_stage(ctx, step, i);
      const double ti = step * dt + ctx->c[i] * dt;
      Motion mo = motion(ctx, mu, n_mu, ti);
      FrameT<double> fr = frame_of(mo);
      const double* ui = stored_u(ctx, step, i);
      // rhs = b_i lam + sum_{j>i} a_ji y_j  (+ dF/dk_i = dt sum_{l>=i} b_l a_li g_l)
      if (withF) PP_CK(launch_qoi_du(m, ctx->tb, ctx->ph, fr, ui, w0, w1, g[i], ctx->stream));
      if (i == 2) {
        PP_TRY(lincomb(ctx, n, rhs, {ctx->b[2]}, {lam}));
      } else if (i == 1) {
        PP_TRY(lincomb(ctx, n, rhs, {ctx->b[1], ctx->A[2][1]}, {lam, y[2]}));
      } else {
        PP_TRY(lincomb(ctx, n, rhs, {ctx->b[0], ctx->A[1][0], ctx->A[2][0]}, {lam, y[1], y[2]}));
      }
      if (withF) {
        if (i == 2) PP_TRY(lincomb(ctx, n, rhs, {1.0, dt * ctx->b[2] * ctx->A[2][2]}, {rhs, g[2]}));
        if (i == 1)
          PP_TRY(lincomb(ctx, n, rhs, {1.0, dt * ctx->b[1] * ctx->A[1][1], dt * ctx->b[2] * ctx->A[2][1]},
                         {rhs, g[1], g[2]}));
        if (i == 0)
          PP_TRY(lincomb(ctx, n, rhs,
                         {1.0, dt * ctx->b[0] * ctx->A[0][0], dt * ctx->b[1] * ctx->A[1][0],
                          dt * ctx->b[2] * ctx->A[2][0]},
                         {rhs, g[0], g[1], g[2]}));
      }
      int gits = 0;
      PP_TRY(stage_solve(ctx, mesh, sv, 1, rhs, kap, ctx->cfg.lin_rtol, 0.0, &gits, true, work_vec(ctx, 27 + i),
                         step < Nt - 1));
      ctx->last_gmres_adjoint += gits;
      if (sv.JT) PP_CK(launch_stage_matvec<double>(m, ctx->tb, sv.JT, 0.0, dt, kap, y[i], 0, ctx->stream));
      else PP_CK(launch_stage_matvec<double>(m, ctx->tb, sv.J, 0.0, dt, kap, y[i], 1, ctx->stream));
      if (withF && dFdmu) {
        // kappa_i . dr/ds and dQ/ds for the motion seeds s = theta, theta', h'
        const size_t st = (size_t)step * 3 + i;
        double* gt = ctx->d_gterm + 9 * st;
        for (int s = 0; s < 3; ++s) {
          FrameT<Dual> fd;
          double cth = std::cos(mo.th), sth = std::sin(mo.th);
          double dQ[4] = {-sth, cth, -cth, -sth};        // dQ/dtheta
          double d2Q[4] = {-cth, -sth, sth, -cth};        // d2Q/dtheta2
          for (int k2 = 0; k2 < 4; ++k2) {
            fd.Q[k2] = Dual(fr.Q[k2], s == 0 ? dQ[k2] : 0.0);
            fd.Qd[k2] = Dual(fr.Qd[k2], s == 0 ? mo.thd * d2Q[k2] : (s == 1 ? dQ[k2] : 0.0));
          }
          fd.hd = Dual(fr.hd, s == 2 ? 1.0 : 0.0);
          PP_CK(launch_residual_dframe(m, ctx->tb, ctx->ph, fd, ui, dr, ctx->stream));
          PP_CK(launch_dot<double>(n, kap, dr, gt + s, ctx->d_partial, ctx->d_counter, ctx->stream));
          PP_CK(launch_qoi_dframe(m, ctx->tb, ctx->ph, fd, ui, ctx->d_elem, ctx->stream));
          PP_CK(launch_colsum(mesh->ne, 2, ctx->d_elem, gt + 3 + 2 * s, ctx->d_partial, ctx->d_counter,
                              ctx->stream));
        }
        for (int j = 0; j < n_mu; ++j) {
          double* d = &ds_host[(st * n_mu + j) * 3];
          d[0] = mo.dth[j];
          d[1] = mo.dthd[j];
          d[2] = mo.dhd[j];
        }
      }
    }
    // lam <- lam + sum_i y_i (+ dF/du^(n-1) = dt sum_l b_l g_l)
    PP_TRY(lincomb(ctx, n, lam, {1.0, 1.0, 1.0, 1.0}, {lam, y[0], y[1], y[2]}));
    if (withF)
      PP_TRY(lincomb(ctx, n, lam, {1.0, dt * ctx->b[0], dt * ctx->b[1], dt * ctx->b[2]}, {lam, g[0], g[1], g[2]}));
  }
  PP_TRY(copy(ctx, n, lam0, lam));
  std::vector<double> gterm;
  if (withF && dFdmu) {
    gterm.resize(9 * n_st);
    PP_CK(cudaMemcpyAsync(gterm.data(), ctx->d_gterm, sizeof(double) * 9 * n_st, cudaMemcpyDeviceToHost,
                          ctx->stream));
  }
  PP_CK(cudaStreamSynchronize(ctx->stream));
  PP_TRY(check_stream_kernels(ctx));
  if (withF && dFdmu) {
    // the same sums, in the same order, as the sweep's stage order (step Nt-1 .. 0, stage 2 .. 0)
    for (int step = Nt - 1; step >= 0; --step)
      for (int i = 2; i >= 0; --i) {
        const size_t st = (size_t)step * 3 + i;
        const double* gt = &gterm[9 * st];
        double sr[3], sq[3];
        for (int s = 0; s < 3; ++s) {
          sr[s] = gt[s];
          sq[s] = w0 * gt[3 + 2 * s] + w1 * gt[4 + 2 * s];
        }
        for (int j = 0; j < n_mu; ++j) {
          const double* ds = &ds_host[(st * n_mu + j) * 3];
          for (int s = 0; s < 3; ++s) grad[j] += dt * sr[s] * ds[s] + dt * ctx->b[i] * sq[s] * ds[s];
        }
      }
  }
  if (dFdmu)
    for (int j = 0; j < n_mu; ++j) dFdmu[j] = withF ? grad[j] : 0.0;
  return PP_OK;
}

// --------------------------------------------------------------------------- steady state
// Pseudo-transient continuation for r(u; theta(0), mesh at rest) = 0: backward-Euler pseudo
// steps (M - dtau J) du = dtau r(u), dtau grown by the residual ratio (switched evolution
// relaxation) and cut on a rejected step.  FP64 block-Jacobi GMRES, work buffers of the
// context.  Starts from the free stream.
int steady_state(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double* u, double tol, int maxit,
                 int* steps, double* rel_res) {
  PP_TRY(ensure_workspace(ctx, mesh));
  const DevMesh& m = mesh->dev;
  const int64_t n = ctx->ws_nu;
  Motion mo = motion(ctx, mu, n_mu, 0.0);
  mo.thd = 0.0;
  mo.hd = 0.0;
  FrameT<double> fr = frame_of(mo);
  {
    std::vector<double> fs(n);
    const int nb = ctx->tb.nb, Np = ctx->tb.Np;
    for (int64_t e = 0; e < mesh->ne; ++e)
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < Np; ++i) fs[e * nb + a * Np + i] = ctx->ph.Uinf[a];
    PP_CK(cudaMemcpyAsync(u, fs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    PP_CK(cudaStreamSynchronize(ctx->stream));
  }
  double* r = work_vec(ctx, 0);
  double* rt = work_vec(ctx, 1);
  double* du = work_vec(ctx, 2);
  double* ut = work_vec(ctx, 3);
  double* rhs = work_vec(ctx, 4);
  PP_CK(launch_residual(m, ctx->tb, ctx->ph, fr, u, r, ctx->stream));
  double rn0, rn;
  PP_TRY(host_norm(ctx, n, r, &rn0));
  rn = rn0;
  double dtau = 0.1;
  const double dtau_max = 1e4;
  int it = 0;
  for (; it < maxit; ++it) {
    if (rn <= tol * rn0) break;
    PP_CK(launch_jacobian(m, ctx->tb, ctx->ph, fr, u, ctx->d_J, ctx->stream));
    PP_CK(launch_block_inverse<double>(m, ctx->tb, ctx->d_J, dtau, ctx->d_Ainv, nullptr, ctx->d_status, ctx->stream));
    PP_TRY(lincomb(ctx, n, rhs, {dtau}, {r}));
    Op A = [&](const double* in, double* out) {
      PP_CK(launch_stage_matvec<double>(m, ctx->tb, ctx->d_J, 1.0, -dtau, in, out, 0, ctx->stream));
      return PP_OK;
    };
    Op P = [&](const double* in, double* out) {
      PP_CK(launch_block_apply<double>(m, ctx->tb.nb, ctx->d_Ainv, in, out, 0, ctx->stream));
      return PP_OK;
    };
    int gits = 0;
    int st = gmres<double>(ctx, ctx->kin, A, P, rhs, du, 1e-4, 0.0, ctx->cfg.gmres_maxit, &gits, nullptr);
    if (st != PP_OK && st != PP_ENOCONV) return st;
    PP_TRY(lincomb(ctx, n, ut, {1.0, 1.0}, {u, du}));
    PP_CK(launch_residual(m, ctx->tb, ctx->ph, fr, ut, rt, ctx->stream));
    double d2;
    PP_TRY(host_dot<double>(ctx, n, rt, rt, &d2));
    const double rnt = std::sqrt(d2);
    if (std::isfinite(rnt) && rnt < 2.0 * rn) {
      dtau = std::fmin(dtau * std::fmin(std::fmax(rn / rnt, 0.5), 4.0), dtau_max);
      PP_TRY(copy(ctx, n, u, ut));
      PP_TRY(copy(ctx, n, r, rt));
      rn = rnt;
    } else {
      dtau *= 0.25;
    }
  }
  PP_CK(cudaStreamSynchronize(ctx->stream));
  if (steps) *steps = it;
  if (rel_res) *rel_res = rn / rn0;
  if (rn > tol * rn0) return set_error(ctx, PP_ENOCONV, "pseudo-transient continuation did not converge");
  return PP_OK;
}

// --------------------------------------------------------------------------- shooting
int shoot_nk(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0_guess, int Nt,
             double tol, double* u0_out, double* qoi, pp_shoot_stats* stats) {
  const double t_start = now_s();
  PP_TRY(ensure_store(ctx, mesh, Nt));
  const int64_t n = ctx->ws_nu;
  pp_shoot_stats st{};
  // u0 lives in u0_out; the outer Krylov level owns V, w, t, r
  if (u0_guess) {
    PP_TRY(copy(ctx, n, u0_out, u0_guess));
    st.cold_start = 0;
  } else {
    // cold start: the steady flow at the t = 0 pose (Sec. 6.1); free stream if that stalls
    int steps = 0;
    double rr = 0.0;
    int ss = steady_state(ctx, mesh, mu, n_mu, u0_out, 1e-8, 100, &steps, &rr);
    st.cold_start = ss == PP_OK ? 2 : 1;
    if (ss != PP_OK) {
      if (ss != PP_ENOCONV && ss != PP_ENAN) return ss;
      std::vector<double> fs(n);
      const int nb = ctx->tb.nb, Np = ctx->tb.Np;
      for (int64_t e = 0; e < mesh->ne; ++e)
        for (int a = 0; a < 4; ++a)
          for (int i = 0; i < Np; ++i) fs[e * nb + a * Np + i] = ctx->ph.Uinf[a];
      PP_CK(cudaMemcpyAsync(u0_out, fs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
      PP_CK(cudaStreamSynchronize(ctx->stream));
    }
  }
  // outer-level scratch: the last three outer Krylov vectors are free between GMRES calls
  Krylov& K = ctx->kout;
  double* uN = K.r;   // reused only outside gmres
  // nonlinear preconditioning (Sec. 6.1): m steps of Algorithm fixedpt, u0 <- u^(Nt)(u0)
  for (int it = 0; it < ctx->cfg.nk_fixed_point_pre; ++it) {
    PP_TRY(primal_sweep(ctx, mesh, mu, n_mu, u0_out, Nt, nullptr, uN, nullptr));
    st.primal_sweeps++;
    st.stage_newton_iters += ctx->last_newton_iters;
    PP_TRY(copy(ctx, n, u0_out, uN));
  }
  int status = PP_ENOCONV;
  for (int it = 0; it <= ctx->cfg.nk_max_newton; ++it) {
    PP_TRY(primal_sweep(ctx, mesh, mu, n_mu, u0_out, Nt, nullptr, uN, qoi));
    st.primal_sweeps++;
    st.stage_newton_iters += ctx->last_newton_iters;
    double* R = work_vec(ctx, 24);  // outer-level vectors (24..26) are never touched by the sweeps
    PP_TRY(lincomb(ctx, n, R, {1.0, -1.0}, {uN, u0_out}));
    double rn;
    PP_TRY(host_norm(ctx, n, R, &rn));
    if (it < 64) st.residual[it] = rn;
    st.newton_iters = it;
    if (rn <= tol) {
      status = PP_OK;
      break;
    }
    if (it == ctx->cfg.nk_max_newton) break;
    // (Phi - I) du = R with matvec (Phi - I) v = -(v - Phi v)
    double* Rsave = work_vec(ctx, 25);
    PP_TRY(copy(ctx, n, Rsave, R));
    double* du = work_vec(ctx, 26);
    Op A = [&](const double* in, double* out) {
      PP_TRY(tangent_sweep(ctx, in, out));
      PP_TRY(lincomb(ctx, n, out, {-1.0}, {out}));
      return PP_OK;
    };
    int kits = 0;
    int gs = gmres<double>(ctx, K, A, Op(), Rsave, du, ctx->cfg.nk_gmres_rtol, 0.0, ctx->cfg.nk_max_krylov, &kits,
                           nullptr);
    if (gs != PP_OK && gs != PP_ENOCONV) return gs;
    st.krylov_iters += kits;
    PP_TRY(lincomb(ctx, n, u0_out, {1.0, -1.0}, {u0_out, du}));
  }
  if (status == PP_OK) {
    // the stored linearization is that of the returned u0 (the last sweep started from it)
  }
  st.seconds = now_s() - t_start;
  if (stats) *stats = st;
  if (status != PP_OK) return set_error(ctx, PP_ENOCONV, "shooting did not reach the tolerance");
  return PP_OK;
}

// --------------------------------------------------------------------------- periodic adjoint
int periodic_adjoint(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                     const double* weights, double* F, double* dFdmu, double* lam_Nt, pp_adj_stats* stats) {
  const double t_start = now_s();
  if (u0) {
    PP_TRY(primal_sweep(ctx, mesh, mu, n_mu, u0, Nt, nullptr, nullptr, nullptr));
  } else if (!ctx->lin_valid || ctx->lin_mesh != mesh || ctx->lin_Nt != Nt) {
    return set_error(ctx, PP_ESTATE, "pp_periodic_adjoint: no matching stored linearization");
  }
  const int64_t n = ctx->ws_nu;
  Krylov& K = ctx->kout;
  double* d = work_vec(ctx, 24);  // outer-level vectors (24..26) are never touched by the sweeps
  double* x = work_vec(ctx, 25);
  double* z = work_vec(ctx, 26);
  PP_CK(cudaMemsetAsync(z, 0, sizeof(double) * n, ctx->stream));
  // d = lambda^(0)(0) with the QoI terms; solve (Phi^T - I) x = -d
  PP_TRY(adjoint_sweep(ctx, z, weights, d, nullptr));
  PP_TRY(lincomb(ctx, n, d, {-1.0}, {d}));
  Op A = [&](const double* in, double* out) {
    PP_TRY(adjoint_sweep(ctx, in, nullptr, out, nullptr));
    PP_TRY(lincomb(ctx, n, out, {1.0, -1.0}, {out, in}));
    return PP_OK;
  };
  int kits = 0;
  int gs = gmres<double>(ctx, K, A, Op(), d, x, 0.0, ctx->cfg.adj_tol, ctx->cfg.adj_maxit, &kits, nullptr);
  if (gs != PP_OK && gs != PP_ENOCONV) return gs;
  // final sweep with the periodic final condition: multipliers and gradient
  PP_TRY(adjoint_sweep(ctx, x, weights, z, dFdmu));
  double res;
  PP_TRY(lincomb(ctx, n, z, {1.0, -1.0}, {z, x}));
  PP_TRY(host_norm(ctx, n, z, &res));
  if (lam_Nt) PP_TRY(copy(ctx, n, lam_Nt, x));
  if (F) *F = weights[0] * ctx->lin_W + weights[1] * ctx->lin_Jx;
  PP_CK(cudaStreamSynchronize(ctx->stream));
  if (stats) {
    stats->krylov_iters = kits;
    stats->residual = res;
    stats->seconds = now_s() - t_start;
  }
  if (gs == PP_ENOCONV) return set_error(ctx, PP_ENOCONV, "periodic adjoint GMRES hit adj_maxit");
  return PP_OK;
}

// --------------------------------------------------------------------------- fixed points
// Algorithm fixedpt: u0 <- u^(Nt)(u0) until ||u^(Nt)(u0) - u0||_2 <= tol (Eq. fixedpt).  On
// return the stored linearization is that of the returned u0.
int shoot_fixed_point(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0_guess,
                      int Nt, double tol, int maxit, double* u0_out, double* qoi, pp_shoot_stats* stats) {
  const double t_start = now_s();
  PP_TRY(ensure_store(ctx, mesh, Nt));
  const int64_t n = ctx->ws_nu;
  pp_shoot_stats st{};
  PP_TRY(copy(ctx, n, u0_out, u0_guess));
  double* uN = ctx->kout.r;
  double* R = work_vec(ctx, 24);
  int status = PP_ENOCONV;
  for (int it = 0; it <= maxit; ++it) {
    PP_TRY(primal_sweep(ctx, mesh, mu, n_mu, u0_out, Nt, nullptr, uN, qoi));
    st.primal_sweeps++;
    st.stage_newton_iters += ctx->last_newton_iters;
    PP_TRY(lincomb(ctx, n, R, {1.0, -1.0}, {uN, u0_out}));
    double rn;
    PP_TRY(host_norm(ctx, n, R, &rn));
    if (it < 64) st.residual[it] = rn;
    st.newton_iters = it;
    if (!std::isfinite(rn)) return set_error(ctx, PP_ENAN, "fixed-point iteration: non-finite residual");
    if (rn <= tol) {
      status = PP_OK;
      break;
    }
    if (it == maxit) break;
    PP_TRY(copy(ctx, n, u0_out, uN));
  }
  st.seconds = now_s() - t_start;
  if (stats) *stats = st;
  if (status != PP_OK) return set_error(ctx, PP_ENOCONV, "fixed-point iteration did not reach the tolerance");
  return PP_OK;
}

// The periodic adjoint condition (Eq. fixedpt-dual; dF/du^(Nt) = 0 for stage-only QoIs) by
// fixed-point iteration x <- lambda^(0)(x) from x = 0, then the gradient of Algorithm grad
// with the converged multipliers.  Iterations and the final residual go to stats.
int periodic_adjoint_fixed_point(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0,
                                 int Nt, const double* weights, double tol, int maxit, double* F, double* dFdmu,
                                 double* lam_Nt, pp_adj_stats* stats) {
  const double t_start = now_s();
  if (u0) PP_TRY(primal_sweep(ctx, mesh, mu, n_mu, u0, Nt, nullptr, nullptr, nullptr));
  if (!ctx->lin_valid) return set_error(ctx, PP_ESTATE, "periodic adjoint: no stored primal sweep");
  const int64_t n = ctx->ws_nu;
  double* x = ctx->kout.V;
  double* y = ctx->kout.w;
  double* r = ctx->kout.t;
  PP_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
  double res = 0.0;
  int its = 0, status = PP_ENOCONV;
  for (;; ++its) {
    PP_TRY(adjoint_sweep(ctx, x, weights, y, nullptr));
    PP_TRY(lincomb(ctx, n, r, {1.0, -1.0}, {y, x}));
    PP_TRY(host_norm(ctx, n, r, &res));
    if (!std::isfinite(res)) return set_error(ctx, PP_ENAN, "dual fixed point: non-finite residual");
    if (res <= tol) {
      status = PP_OK;
      break;
    }
    if (its >= maxit) break;
    PP_TRY(copy(ctx, n, x, y));
  }
  // gradient and multipliers of the converged final condition
  PP_TRY(adjoint_sweep(ctx, x, weights, y, dFdmu));
  if (lam_Nt) PP_TRY(copy(ctx, n, lam_Nt, x));
  if (F) *F = weights[0] * ctx->lin_W + weights[1] * ctx->lin_Jx;
  PP_CK(cudaStreamSynchronize(ctx->stream));
  if (stats) {
    stats->krylov_iters = its + 1;
    stats->residual = res;
    stats->seconds = now_s() - t_start;
  }
  if (status != PP_OK) return set_error(ctx, PP_ENOCONV, "dual fixed point did not reach the tolerance");
  return PP_OK;
}

// --------------------------------------------------------------------------- multi-QoI adjoint
namespace {

// Least squares min ||E - H Y||_F for the (r x c) block Hessenberg H (row-major, r > c) and
// E (r x s) by Householder QR on the host; returns Y (c x s) and the residual norms of the
// s columns.
void small_lsq(int r, int c, int s, std::vector<double> H, std::vector<double> E, std::vector<double>& Y,
               std::vector<double>& res) {
  for (int k = 0; k < c; ++k) {
    double nrm = 0.0;
    for (int i = k; i < r; ++i) nrm += H[(size_t)i * c + k] * H[(size_t)i * c + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    const double alpha = H[(size_t)k * c + k] >= 0.0 ? -nrm : nrm;
    std::vector<double> v(r, 0.0);
    for (int i = k; i < r; ++i) v[i] = H[(size_t)i * c + k];
    v[k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < r; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int j = k; j < c; ++j) {
      double d = 0.0;
      for (int i = k; i < r; ++i) d += v[i] * H[(size_t)i * c + j];
      d *= 2.0 / vv;
      for (int i = k; i < r; ++i) H[(size_t)i * c + j] -= d * v[i];
    }
    for (int j = 0; j < s; ++j) {
      double d = 0.0;
      for (int i = k; i < r; ++i) d += v[i] * E[(size_t)i * s + j];
      d *= 2.0 / vv;
      for (int i = k; i < r; ++i) E[(size_t)i * s + j] -= d * v[i];
    }
  }
  Y.assign((size_t)c * s, 0.0);
  for (int j = 0; j < s; ++j) {
    for (int k = c - 1; k >= 0; --k) {
      double acc = E[(size_t)k * s + j];
      for (int l = k + 1; l < c; ++l) acc -= H[(size_t)k * c + l] * Y[(size_t)l * s + j];
      const double d = H[(size_t)k * c + k];
      Y[(size_t)k * s + j] = d != 0.0 ? acc / d : 0.0;
    }
  }
  res.assign(s, 0.0);
  for (int j = 0; j < s; ++j) {
    double acc = 0.0;
    for (int i = c; i < r; ++i) acc += E[(size_t)i * s + j] * E[(size_t)i * s + j];
    res[j] = std::sqrt(acc);
  }
}

}  // namespace

// The periodic adjoint problems of several QoIs, (Phi^T - I) x_q = -d_q with d_q =
// lambda^(0)(0) under weights q, by one restarted block GMRES: the operator is the same for
// every QoI (Sec. 4), so all right-hand sides share one block Krylov space.  The basis grows
// by the s images A v of the newest block, each orthogonalized against every earlier basis
// vector (two classical Gram-Schmidt passes), so A V_m = V_(m+1) H with H block upper
// Hessenberg; the s least-squares problems min ||E_1 S - H Y|| share H.  Then per QoI the
// final sweep with the QoI terms gives dF/dmu (Algorithm grad).
int periodic_adjoint_multi(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                           int n_qoi, const double* weights, double* F, double* dFdmu, double* lam_Nt,
                           pp_adj_stats* stats) {
  const double t_start = now_s();
  if (u0) PP_TRY(primal_sweep(ctx, mesh, mu, n_mu, u0, Nt, nullptr, nullptr, nullptr));
  if (!ctx->lin_valid) return set_error(ctx, PP_ESTATE, "periodic adjoint: no stored primal sweep");
  const int s = n_qoi;
  const int64_t n = ctx->ws_nu;
  Krylov& K = ctx->kout;
  const int mb = std::max(1, std::min(K.m, 64) / s - 1);  // block steps per restart: (mb + 1) s <= basis size
  const int nvec = (mb + 1) * s;
  if (nvec > K.m + 1) return set_error(ctx, PP_EINVAL, "multi-QoI adjoint: adj_restart too small for the QoI count");
  double* V = K.V;                          // [(mb+1) s][n] basis (the outer Krylov level's vectors)
  double* X = nullptr;                      // [s][n] solutions
  double* Bm = nullptr;                     // [s][n] right-hand sides -d_q
  if (cudaMalloc(&X, sizeof(double) * (size_t)s * n) != cudaSuccess ||
      cudaMalloc(&Bm, sizeof(double) * (size_t)s * n) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(X);
    return set_error(ctx, PP_ENOMEM, "multi-QoI adjoint: allocation failed");
  }
  struct Guard {
    double* a;
    double* b;
    ~Guard() {
      cudaFree(a);
      cudaFree(b);
    }
  } guard{X, Bm};
  double* w = work_vec(ctx, 24);
  double* zero = work_vec(ctx, 25);
  double* d_h = K.d_h;                      // scratch of >= 2 (64 + 2) doubles
  PP_CK(cudaMemsetAsync(zero, 0, sizeof(double) * n, ctx->stream));
  PP_CK(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)s * n, ctx->stream));
  int sweeps = 0;
  for (int q = 0; q < s; ++q) {
    PP_TRY(adjoint_sweep(ctx, zero, weights + 2 * q, Bm + (size_t)q * n, nullptr));
    ++sweeps;
    PP_TRY(lincomb(ctx, n, Bm + (size_t)q * n, {-1.0}, {Bm + (size_t)q * n}));
  }
  // A v = lambda^(0)(v) - v (sensitivity sweep without QoI terms)
  auto apply = [&](const double* in, double* out) -> int {
    PP_TRY(adjoint_sweep(ctx, in, nullptr, out, nullptr));
    ++sweeps;
    return lincomb(ctx, n, out, {1.0, -1.0}, {out, in});
  };
  // orthogonalize w against V[0..k) (two passes); returns the coefficients and |w|
  std::vector<double> hbuf(66);
  auto ortho = [&](int k, double* coef, double* nrm) -> int {
    for (int t = 0; t < k; ++t) coef[t] = 0.0;
    double n2 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      if (k > 0) {
        PP_CK(launch_mdot<double>(n, V, n, k, w, d_h, ctx->d_partial, ctx->d_counter, ctx->stream));
        PP_CK(launch_update_norm2<double>(n, V, n, k, d_h, w, d_h + 64, ctx->d_partial, ctx->d_counter, ctx->stream));
      } else {
        PP_CK(launch_dot<double>(n, w, w, d_h + 64, ctx->d_partial, ctx->d_counter, ctx->stream));
      }
      PP_CK(cudaMemcpyAsync(hbuf.data(), d_h, sizeof(double) * 65, cudaMemcpyDeviceToHost, ctx->stream));
      PP_CK(cudaStreamSynchronize(ctx->stream));
      for (int t = 0; t < k; ++t) coef[t] += hbuf[t];
      n2 = hbuf[64];
    }
    *nrm = std::sqrt(std::max(n2, 0.0));
    return PP_OK;
  };
  std::vector<double> res(s, 0.0), Y;
  int iters = 0, status = PP_ENOCONV;
  const double tol = ctx->cfg.adj_tol;
  for (int cycle = 0; cycle < 1000; ++cycle) {
    // residual block R = B - A X, its QR R = V_1 S
    std::vector<double> S((size_t)s * s, 0.0), coef(64);
    for (int q = 0; q < s; ++q) {
      if (cycle == 0) {
        PP_TRY(copy(ctx, n, w, Bm + (size_t)q * n));
      } else {
        PP_TRY(apply(X + (size_t)q * n, w));
        PP_TRY(lincomb(ctx, n, w, {1.0, -1.0}, {Bm + (size_t)q * n, w}));
      }
      double nr;
      PP_TRY(ortho(q, coef.data(), &nr));
      for (int t = 0; t < q; ++t) S[(size_t)t * s + q] = coef[t];
      S[(size_t)q * s + q] = nr;
      PP_CK(launch_scale(n, V + (size_t)q * n, nr > 0.0 ? 1.0 / nr : 0.0, w, ctx->stream));
    }
    // the true residual norms of this cycle's start
    bool done = true;
    for (int q = 0; q < s; ++q) {
      double r2 = 0.0;
      for (int t = 0; t <= q; ++t) r2 += S[(size_t)t * s + q] * S[(size_t)t * s + q];
      res[q] = std::sqrt(r2);
      if (!(res[q] <= tol)) done = false;
    }
    if (done) {
      status = PP_OK;
      break;
    }
    if (iters >= ctx->cfg.adj_maxit) break;
    std::vector<double> H((size_t)nvec * (mb * s), 0.0);
    int cols = 0;
    for (int j = 0; j < mb && iters < ctx->cfg.adj_maxit; ++j) {
      for (int i = 0; i < s; ++i) {
        const int c = j * s + i;   // new column: A applied to basis vector c
        PP_TRY(apply(V + (size_t)c * n, w));
        double nr;
        const int k = c + s;       // vectors present: the first block plus the new ones so far
        PP_TRY(ortho(k, coef.data(), &nr));
        for (int t = 0; t < k; ++t) H[(size_t)t * (mb * s) + c] = coef[t];
        H[(size_t)k * (mb * s) + c] = nr;
        PP_CK(launch_scale(n, V + (size_t)k * n, nr > 0.0 ? 1.0 / nr : 0.0, w, ctx->stream));
      }
      ++iters;
      cols = (j + 1) * s;
      const int rows = cols + s;
      std::vector<double> Hs((size_t)rows * cols), E((size_t)rows * s, 0.0);
      for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) Hs[(size_t)r * cols + c] = H[(size_t)r * (mb * s) + c];
      for (int r = 0; r < s; ++r)
        for (int q = 0; q < s; ++q) E[(size_t)r * s + q] = S[(size_t)r * s + q];
      small_lsq(rows, cols, s, Hs, E, Y, res);
      bool conv = true;
      for (int q = 0; q < s; ++q)
        if (!(res[q] <= tol)) conv = false;
      if (conv) break;
    }
    // X += V Y
    for (int q = 0; q < s; ++q)
      for (int c = 0; c < cols; ++c) {
        const double yc = Y[(size_t)c * s + q];
        if (yc != 0.0) PP_TRY(lincomb(ctx, n, X + (size_t)q * n, {1.0, yc}, {X + (size_t)q * n, V + (size_t)c * n}));
      }
  }
  // gradients with the converged multipliers (Algorithm grad), one final sweep per QoI
  double resmax = 0.0;
  for (int q = 0; q < s; ++q) {
    PP_TRY(adjoint_sweep(ctx, X + (size_t)q * n, weights + 2 * q, w, dFdmu + (size_t)q * n_mu));
    ++sweeps;
    PP_TRY(lincomb(ctx, n, w, {1.0, -1.0}, {w, X + (size_t)q * n}));
    double r;
    PP_TRY(host_norm(ctx, n, w, &r));
    resmax = std::max(resmax, r);
    if (lam_Nt) PP_TRY(copy(ctx, n, lam_Nt + (size_t)q * n, X + (size_t)q * n));
    if (F) F[q] = weights[2 * q] * ctx->lin_W + weights[2 * q + 1] * ctx->lin_Jx;
  }
  PP_CK(cudaStreamSynchronize(ctx->stream));
  if (stats) {
    stats->krylov_iters = sweeps;
    stats->residual = resmax;
    stats->seconds = now_s() - t_start;
  }
  if (status != PP_OK) return set_error(ctx, PP_ENOCONV, "multi-QoI adjoint: block GMRES hit adj_maxit");
  return PP_OK;
}

// --------------------------------------------------------------------------- stored operators
// Applies one operator of the stored linearization of step `step`, stage i (diagnostics):
//   kind 0: y = (M - c J) x,           trans: (M - c J)^T x
//   kind 1: y = D^{-1} x,              trans: D^{-T} x     (D = block diagonal of M - c J)
//   kind 2: y = (I + B) x = (M - c J) D^{-1} x,  trans: (M - c J)^T D^{-T} x
// with c = a_ii dt.  prec 1 applies the FP32 copies of the mixed-precision mode (x and y are
// cast through FP32 work vectors).  x, y: DEVICE FP64 [N_u], distinct.
int stage_apply(pp_ctx* ctx, int step, int i, int kind, int trans, int prec, const double* x, double* y) {
  if (!ctx->lin_valid || !ctx->lin_mesh) return set_error(ctx, PP_ESTATE, "pp_stage_apply: no stored linearization");
  if (step < 0 || step >= ctx->lin_Nt || i < 0 || i > 2 || kind < 0 || kind > 2 || trans < 0 || trans > 1 ||
      prec < 0 || prec > 1 || !x || !y || x == y)
    return set_error(ctx, PP_EINVAL, "pp_stage_apply: bad arguments");
  if (prec == 1 && ctx->cfg.precision != PP_PREC_MIXED)
    return set_error(ctx, PP_EINVAL, "pp_stage_apply: FP32 copies exist in PP_PREC_MIXED only");
  PP_TRY(ensure_segment(ctx, step));
  const pp_mesh* mesh = ctx->lin_mesh;
  const DevMesh& m = mesh->dev;
  const int64_t n = ctx->ws_nu;
  const int nb = ctx->tb.nb;
  StageView sv = stored_stage(ctx, step, i);
  if (prec == 0) {
    if (kind == 0) {
      if (trans && sv.JT) PP_CK(launch_stage_matvec<double>(m, ctx->tb, sv.JT, 1.0, -sv.c, x, y, 0, ctx->stream));
      else PP_CK(launch_stage_matvec<double>(m, ctx->tb, sv.J, 1.0, -sv.c, x, y, trans, ctx->stream));
    } else if (kind == 1) {
      if (!sv.Ainv) return set_error(ctx, PP_ESTATE, "pp_stage_apply: no FP64 block inverse stored");
      if (trans && sv.AinvT) PP_CK(launch_block_apply<double>(m, nb, sv.AinvT, x, y, 0, ctx->stream));
      else PP_CK(launch_block_apply<double>(m, nb, sv.Ainv, x, y, trans, ctx->stream));
    } else {
      const double* Bf = trans ? sv.BT : sv.BN;
      if (!Bf) return set_error(ctx, PP_ESTATE, "pp_stage_apply: no FP64 folded operator stored");
      PP_CK(launch_stream_rows<double>(m, ctx->tb, nb, 3, Bf, 0.0, 1.0, x, y, ctx->stream));
    }
  } else {
    if (!sv.J32) return set_error(ctx, PP_ESTATE, "pp_stage_apply: no FP32 copies stored");
    float* x32 = ctx->d_vec32 + 2 * n;
    float* y32 = ctx->d_vec32 + 3 * n;
    PP_CK(launch_cast<double, float>(n, x32, x, ctx->stream));
    if (kind == 0) {
      PP_CK(launch_stage_matvec<float>(m, ctx->tb, trans ? sv.JT32 : sv.J32, 1.0, -sv.c, x32, y32, 0, ctx->stream));
    } else if (kind == 1) {
      PP_CK(launch_block_apply<float>(m, nb, trans ? sv.AT32 : sv.A32, x32, y32, 0, ctx->stream));
    } else {
      const float* Bf = trans ? sv.BT32 : sv.BN32;
      if (!Bf) return set_error(ctx, PP_ESTATE, "pp_stage_apply: no FP32 folded operator stored");
      PP_CK(launch_stream_rows<float>(m, ctx->tb, nb, 3, Bf, 0.0, 1.0, x32, y32, ctx->stream));
    }
    PP_CK(launch_cast<float, double>(n, y, y32, ctx->stream));
  }
  PP_CK(cudaStreamSynchronize(ctx->stream));
  return check_stream_kernels(ctx);
}

}  // namespace pp
