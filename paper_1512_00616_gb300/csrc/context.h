// Host-side state of libpp: the context (stream, tables, workspace, stored
// linearization) and the device mesh.
#pragma once

#include <string>
#include <vector>

#include "pp_internal.h"

struct pp_mesh {
  pp_ctx* ctx = nullptr;
  int ne = 0;
  double* d_real = nullptr;  // one allocation for all FP64 geometry arrays
  int* d_int = nullptr;      // one allocation for nbr, nbrface, tag, side
  pp::DevMesh dev{};
};

namespace pp {

// Reference-element tables computed on the host (see host.cpp).
struct RefHost {
  int p = 0, Np = 0, nb = 0, nqv = 0, nqf = 0;
  std::vector<double> phi_v, dphi_v, w_v, xi_v, phi_f, dphi_f, xi_f, w_f, Mref, lift_v, lift_f;
};

// Krylov workspace of one GMRES level (stage solves and the outer shooting /
// periodic-adjoint solves each own one, because the latter call the former).  S is the
// vector type; Hessenberg data and scalars are FP64.  Z (flexible GMRES only) keeps the
// preconditioned directions.
template <class S>
struct KrylovT {
  int m = 0;
  int64_t n = 0;
  S* V = nullptr;        // [m+1][n]
  S* w = nullptr;        // [n]
  S* t = nullptr;        // [n]
  S* r = nullptr;        // [n]
  S* Z = nullptr;        // [m][n] or null
  double* d_h = nullptr; // device: h1 [m+2] | h2 [m+2] | norm2 | y | H [(m+1) m] | cs | sn | g | stat [8]
  double* h_h = nullptr; // pinned ring of stat copies [kRing][8]
  double* h_h_dev = nullptr; // device alias of h_h (null: copied by cudaMemcpyAsync)
  double* d_y = nullptr; // [m+1]
  double* d_H = nullptr;
  double* d_cs = nullptr;
  double* d_sn = nullptr;
  double* d_g = nullptr;
  double* d_stat = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};
using Krylov = KrylovT<double>;
constexpr int kRing = 4;

// Motion quantities at one time and their derivatives w.r.t. mu.
struct Motion {
  double th, thd, hd;
  double dth[8], dthd[8], dhd[8];
};

}  // namespace pp

struct pp_ctx {
  pp_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  pp::RefHost ref;
  double* d_tables = nullptr;
  pp::DevTables tb{};
  pp::Phys ph{};
  double A[3][3]{}, b[3]{}, c[3]{};

  // reductions
  double* d_partial = nullptr;
  unsigned* d_counter = nullptr;
  double* d_scalar = nullptr;  // [64]
  double* h_scalar = nullptr;  // pinned [64]
  int* d_status = nullptr;
  double* d_arn = nullptr;     // fused Arnoldi step: CTA partials
  unsigned* d_arn_bar = nullptr;  // fused Arnoldi step: arrival count, release epoch, error word
  double* d_gterm = nullptr;   // adjoint-sweep gradient terms, 9 per stage [3 * Nt][9]
  size_t gterm_cap = 0;        // capacity in stages

  // per-mesh-size workspace
  int64_t ws_nu = 0;
  int ws_ne = 0;
  double* d_J = nullptr;        // work Jacobian [ne*4*nb*nb]
  double* d_Ainv = nullptr;     // work inverse [ne*nb*nb]
  double* d_vec = nullptr;      // pool of work vectors
  int n_vec = 0;
  double* d_elem = nullptr;     // [ne*8] per-element partials
  pp::Krylov kin, kout;         // stage-solve and outer (shooting / periodic adjoint) GMRES levels
  pp::KrylovT<float> k32;       // inner FP32 level of the mixed-precision stage solves
  float* d_vec32 = nullptr;     // FP32 work vectors [4][nu]

  // stored linearization (the last primal sweep)
  const pp_mesh* lin_mesh = nullptr;
  std::vector<double> lin_mu;
  int lin_Nt = 0;
  bool lin_valid = false;
  size_t store_stages = 0;      // capacity in stages
  double* st_J = nullptr;       // [stages][ne*4*nb*nb]
  double* st_Ainv = nullptr;    // [stages][ne*nb*nb]
  double* st_u = nullptr;       // [stages][nu] stage states
  double* st_JT = nullptr;      // [stages][ne*4*nb*nb] transposed block-columns (optional)
  double* st_AinvT = nullptr;   // [stages][ne*nb*nb] transposed inverses (optional; FP64 mode)
  double* st_BN = nullptr;      // [stages][ne*3*nb*nb] folded operator blocks -c J_off D^-1 (optional; FP64 mode)
  double* st_BT = nullptr;      // [stages][ne*3*nb*nb] folded transposed blocks (optional; FP64 mode)
  float* st_BN32 = nullptr;     // mixed mode: FP32 folded blocks from the FP32 copies (optional)
  float* st_BT32 = nullptr;
  float* st_J32 = nullptr;      // mixed mode: FP32 copies of J, J^T-columns and the inverses
  float* st_JT32 = nullptr;
  float* st_A32 = nullptr;
  float* st_AT32 = nullptr;
  std::vector<double> lin_qoi_rates;  // [Nt*3][2]
  // checkpointed linearization (cfg.checkpoint_stride > 0): (u, predictor) at segment starts,
  // one segment of stage data resident, slot = (step - seg_base)*3 + i
  double* ck_u = nullptr;
  double* ck_k = nullptr;
  int seg_base = 0;
  int seg_cur = -1;
  size_t ck_segments = 0;
  int64_t recomputed_segments = 0;
  double lin_W = 0.0, lin_Jx = 0.0;
  int64_t last_newton_iters = 0;
  int64_t last_gmres_iters = 0;
  int64_t last_gmres_tangent = 0;
  int64_t last_gmres_adjoint = 0;
};

namespace pp {
// host.cpp
int set_error(pp_ctx* ctx, int code, const std::string& msg);
Motion motion(const pp_ctx* ctx, const double* mu, int n_mu, double t);
Motion motion_eval(int kin, double T, const double* mu, double t);  // no context needed
int kin_param_count(int kin);                                      // -1 for an unknown mode
FrameT<double> frame_of(const Motion& mo);
int check_mu(pp_ctx* ctx, int n_mu);
int ensure_workspace(pp_ctx* ctx, const pp_mesh* mesh);
int ensure_store(pp_ctx* ctx, const pp_mesh* mesh, int Nt);
double* work_vec(pp_ctx* ctx, int i);
int64_t mesh_nu(const pp_ctx* ctx, const pp_mesh* mesh);
// solver.cpp
int primal_sweep(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                 double* u_traj, double* u_final, double* qoi);
int tangent_sweep(pp_ctx* ctx, const double* v, double* out);
int adjoint_sweep(pp_ctx* ctx, const double* lam_Nt, const double* weights, double* lam0, double* dFdmu);
int steady_state(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double* u, double tol, int maxit,
                 int* steps, double* rel_res);
int shoot_nk(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0_guess, int Nt,
             double tol, double* u0_out, double* qoi, pp_shoot_stats* stats);
int periodic_adjoint(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                     const double* weights, double* F, double* dFdmu, double* lam_Nt, pp_adj_stats* stats);
int stage_apply(pp_ctx* ctx, int step, int i, int kind, int trans, int prec, const double* x, double* y);
int periodic_adjoint_multi(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                           int n_qoi, const double* weights, double* F, double* dFdmu, double* lam_Nt,
                           pp_adj_stats* stats);
int shoot_fixed_point(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0_guess,
                      int Nt, double tol, int maxit, double* u0_out, double* qoi, pp_shoot_stats* stats);
int periodic_adjoint_fixed_point(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0,
                                 int Nt, const double* weights, double tol, int maxit, double* F, double* dFdmu,
                                 double* lam_Nt, pp_adj_stats* stats);
}  // namespace pp

#define PP_CK(...)                                                                                   \
  do {                                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                                  \
    if (e_ != cudaSuccess)                                                                           \
      return pp::set_error(ctx, PP_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define PP_TRY(call)        \
  do {                      \
    int s_ = (call);        \
    if (s_ != PP_OK) return s_; \
  } while (0)
