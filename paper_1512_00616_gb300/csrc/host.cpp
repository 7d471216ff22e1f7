// libpp host side: reference-element tables, mesh upload, context and the
// C ABI entry points declared in include/pp.h.
//
// The reference tables are built here independently of any other component:
// Gauss-Legendre rules by Newton iteration on the Legendre recurrence, the
// triangle rule by the collapsed (Duffy) map, and the equispaced nodal Lagrange
// basis in closed (Silvester) product form in barycentric coordinates.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <utility>

#include "context.h"
#include "../../include/pp_prof.h"

namespace pp {

int set_error(pp_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

// ------------------------------------------------------------------ quadrature and basis
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pm = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  // exact symmetry of the rule (points come in +-pairs)
  for (int i = 0; i < n / 2; ++i) {
    double a = 0.5 * (std::fabs(x[i]) + std::fabs(x[n - 1 - i]));
    double ww = 0.5 * (w[i] + w[n - 1 - i]);
    double sgn = x[i] > 0 ? 1.0 : -1.0;
    x[i] = sgn * a;
    x[n - 1 - i] = -sgn * a;
    w[i] = w[n - 1 - i] = ww;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// R_m(l) = prod_{k<m} (p l - k)/(k+1) and its derivative
static void silvester(int p, int m, double l, double& R, double& dR) {
  R = 1.0;
  dR = 0.0;
  for (int k = 0; k < m; ++k) {
    double f = (p * l - k) / (k + 1.0);
    double df = p / (k + 1.0);
    dR = dR * f + R * df;
    R *= f;
  }
}

static void lagrange(int p, double xi, double eta, std::vector<double>& phi, std::vector<double>& dphi) {
  int Np = (p + 1) * (p + 2) / 2;
  phi.assign(Np, 0.0);
  dphi.assign(2 * Np, 0.0);
  double l1 = xi, l2 = eta, l0 = 1.0 - xi - eta;
  int idx = 0;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i <= p - j; ++i, ++idx) {
      int k = p - i - j;
      double Ri, dRi, Rj, dRj, Rk, dRk;
      silvester(p, i, l1, Ri, dRi);
      silvester(p, j, l2, Rj, dRj);
      silvester(p, k, l0, Rk, dRk);
      phi[idx] = Ri * Rj * Rk;
      dphi[2 * idx] = dRi * Rj * Rk - Ri * Rj * dRk;
      dphi[2 * idx + 1] = Ri * dRj * Rk - Ri * Rj * dRk;
    }
}

static RefHost build_tables(int p) {
  RefHost r;
  r.p = p;
  r.Np = (p + 1) * (p + 2) / 2;
  r.nb = 4 * r.Np;
  int n = p + 2;
  std::vector<double> gx, gw;
  gauss_legendre(n, gx, gw);
  std::vector<double> phi, dphi;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double xi = (1.0 + gx[a]) * (1.0 - gx[b]) / 4.0;
      double eta = (1.0 + gx[b]) / 2.0;
      r.xi_v.push_back(xi);
      r.xi_v.push_back(eta);
      r.w_v.push_back(gw[a] * gw[b] * (1.0 - gx[b]) / 8.0);
      lagrange(p, xi, eta, phi, dphi);
      r.phi_v.insert(r.phi_v.end(), phi.begin(), phi.end());
      r.dphi_v.insert(r.dphi_v.end(), dphi.begin(), dphi.end());
    }
  r.nqv = n * n;
  r.nqf = n;
  const double C[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
  for (int q = 0; q < n; ++q) r.w_f.push_back(0.5 * gw[q]);
  for (int f = 0; f < 3; ++f) {
    const double* A = C[f];
    const double* B = C[(f + 1) % 3];
    for (int q = 0; q < n; ++q) {
      double s = 0.5 * (gx[q] + 1.0);
      double xi = A[0] + s * (B[0] - A[0]), eta = A[1] + s * (B[1] - A[1]);
      r.xi_f.push_back(xi);
      r.xi_f.push_back(eta);
      lagrange(p, xi, eta, phi, dphi);
      r.phi_f.insert(r.phi_f.end(), phi.begin(), phi.end());
      r.dphi_f.insert(r.dphi_f.end(), dphi.begin(), dphi.end());
    }
  }
  r.Mref.assign(r.Np * r.Np, 0.0);
  for (int q = 0; q < r.nqv; ++q)
    for (int i = 0; i < r.Np; ++i)
      for (int j = 0; j < r.Np; ++j) r.Mref[i * r.Np + j] += r.w_v[q] * r.phi_v[q * r.Np + i] * r.phi_v[q * r.Np + j];
  // CDG lifting tables: Minv by Gauss-Jordan (the reference mass matrix is SPD), then
  // E_f[j][q] = sum_i Minv[j][i] phi_i(f, q) w_q, the nodal coefficients of the lifting of a
  // unit jump at face point q, evaluated at the volume and at the face-f points
  const int Np = r.Np, nqv = r.nqv, nqf = r.nqf;
  std::vector<double> A(r.Mref), Minv(Np * Np, 0.0);
  for (int i = 0; i < Np; ++i) Minv[i * Np + i] = 1.0;
  for (int k = 0; k < Np; ++k) {
    const double d = 1.0 / A[k * Np + k];
    for (int j = 0; j < Np; ++j) {
      A[k * Np + j] *= d;
      Minv[k * Np + j] *= d;
    }
    for (int i = 0; i < Np; ++i) {
      if (i == k) continue;
      const double f = A[i * Np + k];
      if (f == 0.0) continue;
      for (int j = 0; j < Np; ++j) {
        A[i * Np + j] -= f * A[k * Np + j];
        Minv[i * Np + j] -= f * Minv[k * Np + j];
      }
    }
  }
  r.lift_v.assign(3 * nqv * nqf, 0.0);
  r.lift_f.assign(3 * nqf * nqf, 0.0);
  std::vector<double> E(Np * nqf);
  for (int f = 0; f < 3; ++f) {
    for (int j = 0; j < Np; ++j)
      for (int q = 0; q < nqf; ++q) {
        double s = 0.0;
        for (int i = 0; i < Np; ++i) s += Minv[j * Np + i] * r.phi_f[(f * nqf + q) * Np + i];
        E[j * nqf + q] = s * r.w_f[q];
      }
    for (int qv = 0; qv < nqv; ++qv)
      for (int q = 0; q < nqf; ++q) {
        double s = 0.0;
        for (int j = 0; j < Np; ++j) s += r.phi_v[qv * Np + j] * E[j * nqf + q];
        r.lift_v[(f * nqv + qv) * nqf + q] = s;
      }
    for (int qf = 0; qf < nqf; ++qf)
      for (int q = 0; q < nqf; ++q) {
        double s = 0.0;
        for (int j = 0; j < Np; ++j) s += r.phi_f[(f * nqf + qf) * Np + j] * E[j * nqf + q];
        r.lift_f[(f * nqf + qf) * nqf + q] = s;
      }
  }
  return r;
}

// Alexander's 3-stage DIRK3: gamma is the root in (1/6, 1/2) of g^3 - 3g^2 + 3/2 g - 1/6
static void dirk3(double A[3][3], double b[3], double c[3]) {
  double g = 0.43;
  for (int it = 0; it < 100; ++it) {
    double f = ((g - 3.0) * g + 1.5) * g - 1.0 / 6.0;
    double df = (3.0 * g - 6.0) * g + 1.5;
    double d = f / df;
    g -= d;
    if (std::fabs(d) < 1e-17) break;
  }
  double b1 = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0;
  double b2 = (6.0 * g * g - 20.0 * g + 5.0) / 4.0;
  double AA[3][3] = {{g, 0, 0}, {(1.0 - g) / 2.0, g, 0}, {b1, b2, g}};
  std::memcpy(A, AA, sizeof(AA));
  b[0] = b1;
  b[1] = b2;
  b[2] = g;
  c[0] = g;
  c[1] = (1.0 + g) / 2.0;
  c[2] = 1.0;
}

// ------------------------------------------------------------------ motion (Eq. defmap with Sec. 6.1 kinematics)
namespace {

// Mirrored spline kinematics (Sec. 6.2, Eq. mirror): h and theta are periodic cubic splines
// through 8 equally spaced knots of the period whose second half repeats the first with the
// opposite sign, f(t + T/2) = -f(t); the free values are the 4 knots of the first half.  The
// spline is linear in the knot values, so it is a sum of 4 "mirrored cardinal" functions
// (knot data e_j - e_{j+4}).  Knot second derivatives: the cyclic system
// M[k-1] + 4 M[k] + M[k+1] = 6 (y[k+1] - 2 y[k] + y[k-1]) / d^2, d = T / 8, solved once for the
// unit right-hand sides (Gauss-Jordan on the 8 x 8 matrix; its inverse scaled by 6 / d^2 later).
constexpr int kKnots = 8;

struct CyclicInverse {
  double a[kKnots][kKnots];
};

const CyclicInverse& cyclic_inverse() {
  static const CyclicInverse inv = [] {
    CyclicInverse r{};
    double m[kKnots][2 * kKnots] = {};
    for (int k = 0; k < kKnots; ++k) {
      m[k][k] = 4.0;
      m[k][(k + 1) % kKnots] = 1.0;
      m[k][(k + kKnots - 1) % kKnots] = 1.0;
      m[k][kKnots + k] = 1.0;
    }
    // diagonally dominant: no pivoting needed
    for (int c = 0; c < kKnots; ++c) {
      const double piv = m[c][c];
      for (int q = 0; q < 2 * kKnots; ++q) m[c][q] /= piv;
      for (int r2 = 0; r2 < kKnots; ++r2) {
        if (r2 == c) continue;
        const double f = m[r2][c];
        for (int q = 0; q < 2 * kKnots; ++q) m[r2][q] -= f * m[c][q];
      }
    }
    for (int k = 0; k < kKnots; ++k)
      for (int q = 0; q < kKnots; ++q) r.a[k][q] = m[k][kKnots + q];
    return r;
  }();
  return inv;
}

// value and time derivative at t of the mirrored cardinal function of free knot j (0..3)
void mirrored_cardinal(int j, double T, double t, double* val, double* der) {
  const double d = T / kKnots;
  double y[kKnots] = {};
  y[j] = 1.0;
  y[j + kKnots / 2] = -1.0;
  double rhs[kKnots];
  for (int k = 0; k < kKnots; ++k)
    rhs[k] = 6.0 * (y[(k + 1) % kKnots] - 2.0 * y[k] + y[(k + kKnots - 1) % kKnots]) / (d * d);
  const CyclicInverse& inv = cyclic_inverse();
  double M[kKnots];
  for (int k = 0; k < kKnots; ++k) {
    double acc = 0.0;
    for (int q = 0; q < kKnots; ++q) acc += inv.a[k][q] * rhs[q];
    M[k] = acc;
  }
  double tau = std::fmod(t, T);
  if (tau < 0.0) tau += T;
  int k = (int)std::floor(tau / d);
  if (k > kKnots - 1) k = kKnots - 1;
  if (k < 0) k = 0;
  const double s = (tau - k * d) / d, r = 1.0 - s;
  const int k1 = (k + 1) % kKnots;
  *val = r * y[k] + s * y[k1] + d * d / 6.0 * ((r * r * r - r) * M[k] + (s * s * s - s) * M[k1]);
  *der = (y[k1] - y[k]) / d + d / 6.0 * (-(3.0 * r * r - 1.0) * M[k] + (3.0 * s * s - 1.0) * M[k1]);
}

}  // namespace

int kin_param_count(int kin) {
  switch (kin) {
    case PP_KIN_HEAVE_PITCH:
      return 3;
    case PP_KIN_FOURIER6:
      return 6;
    case PP_KIN_SPLINE8:
      return 8;
    default:
      return -1;
  }
}

Motion motion_eval(int kin, double T, const double* mu, double t) {
  Motion mo{};
  const double w = 2.0 * M_PI / T;
  if (kin == PP_KIN_HEAVE_PITCH) {
    double h0 = mu[0], th0 = mu[1], ph = mu[2];
    double cw = std::cos(w * t), sp = std::sin(w * t + ph), cp = std::cos(w * t + ph);
    mo.hd = h0 * w * cw;
    mo.th = th0 * sp;
    mo.thd = th0 * w * cp;
    mo.dhd[0] = w * cw;
    mo.dth[1] = sp;
    mo.dth[2] = th0 * cp;
    mo.dthd[1] = w * cp;
    mo.dthd[2] = -th0 * w * sp;
  } else if (kin == PP_KIN_SPLINE8) {
    // mu = (h knots at t = 0, T/8, T/4, 3T/8; theta knots at the same times)
    for (int j = 0; j < kKnots / 2; ++j) {
      double a, da;
      mirrored_cardinal(j, T, t, &a, &da);
      mo.hd += mu[j] * da;
      mo.th += mu[4 + j] * a;
      mo.thd += mu[4 + j] * da;
      mo.dhd[j] = da;
      mo.dth[4 + j] = a;
      mo.dthd[4 + j] = da;
    }
  } else {
    double s1 = std::sin(w * t), c1 = std::cos(w * t), s2 = std::sin(2 * w * t), c2 = std::cos(2 * w * t);
    mo.hd = mu[0] * w * c1 - mu[1] * w * s1 + mu[2] * 2 * w * c2;
    mo.th = mu[3] * s1 + mu[4] * c1 + mu[5] * s2;
    mo.thd = mu[3] * w * c1 - mu[4] * w * s1 + mu[5] * 2 * w * c2;
    mo.dhd[0] = w * c1;
    mo.dhd[1] = -w * s1;
    mo.dhd[2] = 2 * w * c2;
    mo.dth[3] = s1;
    mo.dth[4] = c1;
    mo.dth[5] = s2;
    mo.dthd[3] = w * c1;
    mo.dthd[4] = -w * s1;
    mo.dthd[5] = 2 * w * c2;
  }
  return mo;
}

Motion motion(const pp_ctx* ctx, const double* mu, int n_mu, double t) {
  (void)n_mu;
  return motion_eval(ctx->cfg.kin, ctx->cfg.T, mu, t);
}

FrameT<double> frame_of(const Motion& mo) {
  FrameT<double> f;
  double c = std::cos(mo.th), s = std::sin(mo.th);
  f.Q[0] = c;
  f.Q[1] = s;
  f.Q[2] = -s;
  f.Q[3] = c;
  f.Qd[0] = -s * mo.thd;
  f.Qd[1] = c * mo.thd;
  f.Qd[2] = -c * mo.thd;
  f.Qd[3] = -s * mo.thd;
  f.hd = mo.hd;
  return f;
}

int check_mu(pp_ctx* ctx, int n_mu) {
  const int need = kin_param_count(ctx->cfg.kin);
  if (n_mu != need) return set_error(ctx, PP_EINVAL, "n_mu does not match the kinematics mode");
  return PP_OK;
}

int64_t mesh_nu(const pp_ctx* ctx, const pp_mesh* mesh) { return (int64_t)mesh->ne * ctx->tb.nb; }

double* work_vec(pp_ctx* ctx, int i) { return ctx->d_vec + (size_t)i * ctx->ws_nu; }

template <class S>
static void free_krylov(KrylovT<S>& k) {
  cudaFree(k.V);
  cudaFree(k.Z);
  cudaFree(k.d_h);
  if (k.h_h) cudaFreeHost(k.h_h);
  k.V = k.Z = nullptr;
  k.d_h = k.h_h = k.h_h_dev = nullptr;
}

template <class S>
static int alloc_krylov(pp_ctx* ctx, KrylovT<S>& k, int m, int64_t n, bool flexible) {
  free_krylov(k);
  k.m = m;
  k.n = n;
  PP_CK(cudaMalloc(&k.V, sizeof(S) * (size_t)(m + 4) * n));
  k.w = k.V + (size_t)(m + 1) * n;
  k.t = k.w + n;
  k.r = k.t + n;
  if (flexible) PP_CK(cudaMalloc(&k.Z, sizeof(S) * (size_t)m * n));
  const size_t nh = 2 * (m + 2) + 4 + (m + 2) + (size_t)(m + 1) * m + 3 * (m + 2) + 16;
  PP_CK(cudaMalloc(&k.d_h, sizeof(double) * nh));
  PP_CK(cudaMemset(k.d_h, 0, sizeof(double) * nh));
  PP_CK(cudaMallocHost(&k.h_h, sizeof(double) * 8 * kRing + 64));
  // the fused Arnoldi step writes the convergence record straight into the ring
  void* dev_alias = nullptr;
  k.h_h_dev = cudaHostGetDevicePointer(&dev_alias, k.h_h, 0) == cudaSuccess ? (double*)dev_alias : nullptr;
  cudaGetLastError();
  k.d_y = k.d_h + 2 * (m + 2) + 4;
  k.d_H = k.d_y + (m + 2);
  k.d_cs = k.d_H + (size_t)(m + 1) * m;
  k.d_sn = k.d_cs + (m + 2);
  k.d_g = k.d_sn + (m + 2);
  k.d_stat = k.d_g + (m + 2);
  for (int i = 0; i < kRing; ++i)
    if (!k.ev[i]) PP_CK(cudaEventCreateWithFlags(&k.ev[i], cudaEventDisableTiming));
  return PP_OK;
}

int ensure_workspace(pp_ctx* ctx, const pp_mesh* mesh) {
  const int64_t nu = mesh_nu(ctx, mesh);
  if (ctx->ws_ne == mesh->ne && ctx->d_J) return PP_OK;
  cudaFree(ctx->d_J);
  cudaFree(ctx->d_Ainv);
  cudaFree(ctx->d_vec);
  cudaFree(ctx->d_elem);
  ctx->d_J = ctx->d_Ainv = ctx->d_vec = ctx->d_elem = nullptr;
  const size_t nb2 = (size_t)ctx->tb.nb * ctx->tb.nb;
  ctx->n_vec = 30;  // 0-8 primal, 9-15 tangent, 14-23 adjoint, 24-26 shooting / periodic adjoint,
                    // 27-29 warm starts of the linear stage solves
  if (cudaMalloc(&ctx->d_J, sizeof(double) * mesh->ne * 4 * nb2) != cudaSuccess ||
      cudaMalloc(&ctx->d_Ainv, sizeof(double) * mesh->ne * nb2) != cudaSuccess ||
      cudaMalloc(&ctx->d_vec, sizeof(double) * ctx->n_vec * nu) != cudaSuccess ||
      cudaMalloc(&ctx->d_elem, sizeof(double) * mesh->ne * 8) != cudaSuccess) {
    cudaGetLastError();
    ctx->ws_ne = 0;
    return set_error(ctx, PP_ENOMEM, "workspace allocation failed");
  }
  ctx->ws_ne = mesh->ne;
  ctx->ws_nu = nu;
  const bool mixed = ctx->cfg.precision == PP_PREC_MIXED;
  PP_TRY(alloc_krylov(ctx, ctx->kin, ctx->cfg.gmres_restart, nu, mixed));
  int mo = ctx->cfg.nk_restart > ctx->cfg.adj_restart ? ctx->cfg.nk_restart : ctx->cfg.adj_restart;
  PP_TRY(alloc_krylov(ctx, ctx->kout, mo, nu, false));
  if (mixed) {
    int mi = ctx->cfg.inner_maxit > ctx->cfg.gmres_restart ? ctx->cfg.inner_maxit : ctx->cfg.gmres_restart;
    PP_TRY(alloc_krylov(ctx, ctx->k32, mi, nu, false));
    cudaFree(ctx->d_vec32);
    PP_CK(cudaMalloc(&ctx->d_vec32, sizeof(float) * 4 * nu));
  }
  ctx->lin_valid = false;
  return PP_OK;
}

int ensure_store(pp_ctx* ctx, const pp_mesh* mesh, int Nt) {
  PP_TRY(ensure_workspace(ctx, mesh));
  const int K = ctx->cfg.checkpoint_stride;
  const size_t stages = (size_t)(K > 0 ? std::min(K, Nt) : Nt) * 3;
  ctx->seg_cur = -1;
  if (K > 0) {
    const size_t nseg = (size_t)(Nt + K - 1) / K;
    if (nseg > ctx->ck_segments || ctx->lin_mesh != mesh) {
      cudaFree(ctx->ck_u);
      cudaFree(ctx->ck_k);
      ctx->ck_u = ctx->ck_k = nullptr;
      ctx->ck_segments = 0;
      if (cudaMalloc(&ctx->ck_u, sizeof(double) * nseg * mesh_nu(ctx, mesh)) != cudaSuccess ||
          cudaMalloc(&ctx->ck_k, sizeof(double) * nseg * mesh_nu(ctx, mesh)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, PP_ENOMEM, "checkpoint storage does not fit in device memory");
      }
      ctx->ck_segments = nseg;
    }
  }
  if (ctx->store_stages >= stages && ctx->lin_mesh == mesh) return PP_OK;
  auto release = [&]() {
    for (double** p : {&ctx->st_J, &ctx->st_Ainv, &ctx->st_u, &ctx->st_JT, &ctx->st_AinvT, &ctx->st_BN, &ctx->st_BT}) {
      cudaFree(*p);
      *p = nullptr;
    }
    for (float** p : {&ctx->st_J32, &ctx->st_JT32, &ctx->st_A32, &ctx->st_AT32, &ctx->st_BN32, &ctx->st_BT32}) {
      cudaFree(*p);
      *p = nullptr;
    }
    ctx->store_stages = 0;
  };
  release();
  const bool mixed = ctx->cfg.precision == PP_PREC_MIXED;
  const size_t nb2 = (size_t)ctx->tb.nb * ctx->tb.nb;
  const size_t nJ = stages * mesh->ne * 4 * nb2, nA = stages * mesh->ne * nb2;
  bool ok = cudaMalloc(&ctx->st_J, sizeof(double) * nJ) == cudaSuccess &&
            cudaMalloc(&ctx->st_u, sizeof(double) * stages * mesh_nu(ctx, mesh)) == cudaSuccess;
  if (ok && !mixed) ok = cudaMalloc(&ctx->st_Ainv, sizeof(double) * nA) == cudaSuccess;
  if (ok && mixed)
    ok = cudaMalloc(&ctx->st_J32, sizeof(float) * nJ) == cudaSuccess &&
         cudaMalloc(&ctx->st_JT32, sizeof(float) * nJ) == cudaSuccess &&
         cudaMalloc(&ctx->st_A32, sizeof(float) * nA) == cudaSuccess &&
         cudaMalloc(&ctx->st_AT32, sizeof(float) * nA) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release();
    return set_error(ctx, PP_ENOMEM, "linearization store does not fit in device memory");
  }
  size_t fr = 0, tot = 0;
  // the block-Jacobi preconditioner folded into the stage operator (three neighbour blocks
  // per element, normal and transposed; FP64, or FP32 for the inner solves of the mixed
  // path), kept while 8 GB of device memory stay free
  {
    const size_t nB = stages * mesh->ne * 3 * nb2;
    const size_t word = mixed ? sizeof(float) : sizeof(double);
    cudaMemGetInfo(&fr, &tot);
    if (fr > word * 2 * nB + ((size_t)8 << 30)) {
      bool okB;
      if (!mixed)
        okB = cudaMalloc(&ctx->st_BN, sizeof(double) * nB) == cudaSuccess &&
              cudaMalloc(&ctx->st_BT, sizeof(double) * nB) == cudaSuccess;
      else
        okB = cudaMalloc(&ctx->st_BN32, sizeof(float) * nB) == cudaSuccess &&
              cudaMalloc(&ctx->st_BT32, sizeof(float) * nB) == cudaSuccess;
      if (!okB) {
        cudaGetLastError();
        cudaFree(ctx->st_BN);
        cudaFree(ctx->st_BT);
        cudaFree(ctx->st_BN32);
        cudaFree(ctx->st_BT32);
        ctx->st_BN = ctx->st_BT = nullptr;
        ctx->st_BN32 = ctx->st_BT32 = nullptr;
      }
    }
  }
  // FP64 transposed copies let the adjoint stream row-major blocks with the normal
  // kernels; they are kept only while at least 8 GB of device memory stay free
  cudaMemGetInfo(&fr, &tot);
  const size_t extra = sizeof(double) * (nJ + (mixed ? 0 : nA));
  if (fr > extra + ((size_t)8 << 30)) {
    bool okT = cudaMalloc(&ctx->st_JT, sizeof(double) * nJ) == cudaSuccess;
    if (okT && !mixed) okT = cudaMalloc(&ctx->st_AinvT, sizeof(double) * nA) == cudaSuccess;
    if (!okT) {
      cudaGetLastError();
      cudaFree(ctx->st_JT);
      cudaFree(ctx->st_AinvT);
      ctx->st_JT = ctx->st_AinvT = nullptr;
    }
  }
  ctx->store_stages = stages;
  return PP_OK;
}

}  // namespace pp

using namespace pp;

// ====================================================================== C ABI
extern "C" {

const char* pp_version(void) { return "libpp 0.1 (sm_103a, FP64)"; }

int pp_motion_eval(int kin, double T, const double* mu, int n_mu, double t, double* out) {
  const int need = kin_param_count(kin);
  if (need < 0 || n_mu != need || !(T > 0) || !mu || !out) return PP_EINVAL;
  const Motion mo = motion_eval(kin, T, mu, t);
  out[0] = mo.th;
  out[1] = mo.thd;
  out[2] = mo.hd;
  for (int j = 0; j < n_mu; ++j) {
    out[3 + 3 * j] = mo.dth[j];
    out[4 + 3 * j] = mo.dthd[j];
    out[5 + 3 * j] = mo.dhd[j];
  }
  return PP_OK;
}

void pp_config_default(pp_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->p = 3;
  c->gamma = 1.4;
  c->Pr = 0.72;
  c->Mach = 0.2;
  c->Re = 1000.0;
  c->T = 5.0;
  c->kin = PP_KIN_HEAVE_PITCH;
  c->device = 0;
  c->stream = nullptr;
  c->newton_tol = 1e-10;
  c->newton_maxit = 20;
  c->gmres_rtol = 1e-3;
  c->gmres_restart = 40;
  c->gmres_maxit = 400;
  c->lin_rtol = 1e-11;
  c->nk_gmres_rtol = 1e-3;
  c->nk_restart = 30;
  c->nk_max_newton = 30;
  c->nk_max_krylov = 60;
  c->adj_tol = 1e-10;
  c->adj_restart = 30;
  c->adj_maxit = 200;
  c->precision = PP_PREC_FP64;
  c->checkpoint_stride = 0;
  c->inner_maxit = 30;
  c->inner_rtol = 1e-2;
}

int pp_create(const pp_config* cfg, pp_ctx** out) {
  if (!cfg || !out) return PP_EINVAL;
  if (cfg->p < 1 || cfg->p > kMaxP || cfg->gmres_restart < 1 || cfg->gmres_restart > 60 || cfg->nk_restart < 1 ||
      cfg->nk_restart > 60 || cfg->adj_restart < 1 || cfg->adj_restart > 60 || !(cfg->T > 0) || !(cfg->Re > 0) ||
      !(cfg->Mach > 0) || kin_param_count(cfg->kin) < 0 ||
      (cfg->precision != PP_PREC_FP64 && cfg->precision != PP_PREC_MIXED) ||
      (cfg->precision == PP_PREC_MIXED && (cfg->inner_maxit < 1 || cfg->inner_maxit > 60)) ||
      cfg->checkpoint_stride < 0 || cfg->nk_fixed_point_pre < 0)
    return PP_EINVAL;
  {
    // the launch set-up cached by the kernels' host wrappers is per process: one device
    static std::atomic<int> process_device{-1};
    int expected = -1;
    if (!process_device.compare_exchange_strong(expected, cfg->device) && expected != cfg->device)
      return PP_EINVAL;
  }
  pp_ctx* ctx = new pp_ctx();
  ctx->cfg = *cfg;
  ctx->device = cfg->device;
  auto fail = [&](int code) {
    pp_destroy(ctx);
    return code;
  };
  if (cudaSetDevice(cfg->device) != cudaSuccess) return fail(PP_ECUDA);
  if (cfg->stream) {
    ctx->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(PP_ECUDA);
    ctx->own_stream = true;
  }
  ctx->ref = build_tables(cfg->p);
  const RefHost& r = ctx->ref;
  std::vector<double> all;
  auto put = [&](const std::vector<double>& v) {
    size_t off = all.size();
    all.insert(all.end(), v.begin(), v.end());
    while (all.size() % 4) all.push_back(0.0);
    return off;
  };
  size_t o_phv = put(r.phi_v), o_dphv = put(r.dphi_v), o_wv = put(r.w_v), o_xiv = put(r.xi_v), o_phf = put(r.phi_f),
         o_dphf = put(r.dphi_f), o_xif = put(r.xi_f), o_wf = put(r.w_f), o_M = put(r.Mref), o_lv = put(r.lift_v),
         o_lf = put(r.lift_f);
  if (cudaMalloc(&ctx->d_tables, sizeof(double) * all.size()) != cudaSuccess) return fail(PP_ENOMEM);
  if (cudaMemcpy(ctx->d_tables, all.data(), sizeof(double) * all.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(PP_ECUDA);
  DevTables& tb = ctx->tb;
  tb.p = r.p;
  tb.Np = r.Np;
  tb.nb = r.nb;
  tb.nqv = r.nqv;
  tb.nqf = r.nqf;
  tb.phi_v = ctx->d_tables + o_phv;
  tb.dphi_v = ctx->d_tables + o_dphv;
  tb.w_v = ctx->d_tables + o_wv;
  tb.xi_v = ctx->d_tables + o_xiv;
  tb.phi_f = ctx->d_tables + o_phf;
  tb.dphi_f = ctx->d_tables + o_dphf;
  tb.xi_f = ctx->d_tables + o_xif;
  tb.w_f = ctx->d_tables + o_wf;
  tb.Mref = ctx->d_tables + o_M;
  tb.lift_v = ctx->d_tables + o_lv;
  tb.lift_f = ctx->d_tables + o_lf;
  Phys& ph = ctx->ph;
  ph.gam = cfg->gamma;
  ph.Pr = cfg->Pr;
  ph.mu = 1.0 / cfg->Re;
  double pinf = 1.0 / (cfg->gamma * cfg->Mach * cfg->Mach);
  ph.Uinf[0] = 1.0;
  ph.Uinf[1] = 1.0;
  ph.Uinf[2] = 0.0;
  ph.Uinf[3] = pinf / (cfg->gamma - 1.0) + 0.5;
  ph.x0[0] = 1.0 / 3.0;
  ph.x0[1] = 0.0;
  dirk3(ctx->A, ctx->b, ctx->c);
  if (cudaMalloc(&ctx->d_partial, sizeof(double) * reduction_blocks() * 128) != cudaSuccess ||
      cudaMalloc(&ctx->d_counter, sizeof(unsigned) * 4) != cudaSuccess ||
      cudaMalloc(&ctx->d_scalar, sizeof(double) * 64) != cudaSuccess ||
      cudaMalloc(&ctx->d_status, sizeof(int) * 4) != cudaSuccess ||
      cudaMalloc(&ctx->d_arn, sizeof(double) * arnoldi_partial_words()) != cudaSuccess ||
      cudaMalloc(&ctx->d_arn_bar, sizeof(unsigned) * arnoldi_barrier_words()) != cudaSuccess ||
      cudaMallocHost(&ctx->h_scalar, sizeof(double) * 64) != cudaSuccess)
    return fail(PP_ENOMEM);
  if (cudaMemset(ctx->d_counter, 0, sizeof(unsigned) * 4) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(int) * 4) != cudaSuccess ||
      cudaMemset(ctx->d_arn_bar, 0, sizeof(unsigned) * arnoldi_barrier_words()) != cudaSuccess)
    return fail(PP_ECUDA);
  *out = ctx;
  return PP_OK;
}

int pp_destroy(pp_ctx* ctx) {
  if (!ctx) return PP_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->d_tables);
  cudaFree(ctx->d_partial);
  cudaFree(ctx->d_counter);
  cudaFree(ctx->d_scalar);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_gterm);
  cudaFree(ctx->d_arn);
  cudaFree(ctx->d_arn_bar);
  if (ctx->h_scalar) cudaFreeHost(ctx->h_scalar);
  cudaFree(ctx->d_J);
  cudaFree(ctx->d_Ainv);
  cudaFree(ctx->d_vec);
  cudaFree(ctx->d_vec32);
  cudaFree(ctx->d_elem);
  for (Krylov* k : {&ctx->kin, &ctx->kout}) {
    free_krylov(*k);
    for (int i = 0; i < kRing; ++i)
      if (k->ev[i]) cudaEventDestroy(k->ev[i]);
  }
  free_krylov(ctx->k32);
  for (int i = 0; i < kRing; ++i)
    if (ctx->k32.ev[i]) cudaEventDestroy(ctx->k32.ev[i]);
  cudaFree(ctx->st_J);
  cudaFree(ctx->st_Ainv);
  cudaFree(ctx->st_u);
  cudaFree(ctx->st_JT);
  cudaFree(ctx->st_AinvT);
  cudaFree(ctx->st_BN);
  cudaFree(ctx->st_BT);
  cudaFree(ctx->st_J32);
  cudaFree(ctx->st_JT32);
  cudaFree(ctx->st_A32);
  cudaFree(ctx->st_AT32);
  cudaFree(ctx->st_BN32);
  cudaFree(ctx->st_BT32);
  cudaFree(ctx->ck_u);
  cudaFree(ctx->ck_k);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return PP_OK;
}

const char* pp_last_error(const pp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int pp_mesh_create(pp_ctx* ctx, const double* verts, int nv, const int32_t* tris, const int32_t* ftag, int nt,
                   pp_mesh** out) {
  if (!ctx || !verts || !tris || !ftag || !out || nv < 3 || nt < 1)
    return set_error(ctx, PP_EINVAL, "pp_mesh_create: bad arguments");
  const int p = ctx->cfg.p;
  std::vector<int> nbr(3 * nt, -1), nbrface(3 * nt, -1), tag(3 * nt);
  std::map<std::pair<int, int>, std::pair<int, int>> open;
  for (int e = 0; e < nt; ++e)
    for (int f = 0; f < 3; ++f) {
      int a = tris[3 * e + f], b = tris[3 * e + (f + 1) % 3];
      if (a < 0 || a >= nv || b < 0 || b >= nv || a == b)
        return set_error(ctx, PP_EINVAL, "pp_mesh_create: vertex index out of range");
      tag[3 * e + f] = ftag[3 * e + f];
      auto key = std::make_pair(a < b ? a : b, a < b ? b : a);
      auto it = open.find(key);
      if (it != open.end()) {
        int e2 = it->second.first, f2 = it->second.second;
        nbr[3 * e + f] = e2;
        nbrface[3 * e + f] = f2;
        nbr[3 * e2 + f2] = e;
        nbrface[3 * e2 + f2] = f;
        open.erase(it);
      } else {
        open[key] = std::make_pair(e, f);
      }
    }
  for (int i = 0; i < 3 * nt; ++i) {
    bool interior = nbr[i] >= 0;
    if (interior != (tag[i] == 0) || tag[i] < 0 || tag[i] > 2)
      return set_error(ctx, PP_EINVAL, "pp_mesh_create: face tags inconsistent with connectivity");
  }
  // geometry
  std::vector<double> X0(2 * nt), B(4 * nt), BinvT(4 * nt), detB(nt), N(6 * nt), L(3 * nt), s_own(3 * nt),
      s_nbr(3 * nt), c11(3 * nt);
  std::vector<int> side(3 * nt);
  for (int e = 0; e < nt; ++e) {
    const double* v0 = verts + 2 * tris[3 * e];
    const double* v1 = verts + 2 * tris[3 * e + 1];
    const double* v2 = verts + 2 * tris[3 * e + 2];
    X0[2 * e] = v0[0];
    X0[2 * e + 1] = v0[1];
    double b00 = v1[0] - v0[0], b01 = v2[0] - v0[0], b10 = v1[1] - v0[1], b11 = v2[1] - v0[1];
    double det = b00 * b11 - b01 * b10;
    if (!(det > 0.0)) return set_error(ctx, PP_EINVAL, "pp_mesh_create: inverted or degenerate element");
    B[4 * e] = b00;
    B[4 * e + 1] = b01;
    B[4 * e + 2] = b10;
    B[4 * e + 3] = b11;
    detB[e] = det;
    // B^{-T} = (1/det) [[b11, -b10], [-b01, b00]]
    BinvT[4 * e] = b11 / det;
    BinvT[4 * e + 1] = -b10 / det;
    BinvT[4 * e + 2] = -b01 / det;
    BinvT[4 * e + 3] = b00 / det;
    for (int f = 0; f < 3; ++f) {
      const double* a = verts + 2 * tris[3 * e + f];
      const double* b = verts + 2 * tris[3 * e + (f + 1) % 3];
      double tx = b[0] - a[0], ty = b[1] - a[1];
      double len = std::sqrt(tx * tx + ty * ty);
      L[3 * e + f] = len;
      N[6 * e + 2 * f] = ty / len;
      N[6 * e + 2 * f + 1] = -tx / len;
    }
  }
  // CDG data: lifting scales, boundary penalty C11 = 10 mu / h (h = detB / |f|), and the side
  // that lifts each face (the element itself on the boundary, the lower index inside)
  const double mu = 1.0 / ctx->cfg.Re;
  for (int e = 0; e < nt; ++e)
    for (int f = 0; f < 3; ++f) {
      const int i = 3 * e + f, e2 = nbr[i];
      s_own[i] = L[i] / detB[e];
      s_nbr[i] = e2 >= 0 ? L[i] / detB[e2] : s_own[i];
      c11[i] = e2 >= 0 ? 0.0 : 10.0 * mu * L[i] / detB[e];
      side[i] = (e2 < 0 || e2 > e) ? 1 : 0;
    }
  (void)p;
  pp_mesh* m = new pp_mesh();
  m->ctx = ctx;
  m->ne = nt;
  std::vector<double> real;
  auto put = [&](const std::vector<double>& v) {
    size_t o = real.size();
    real.insert(real.end(), v.begin(), v.end());
    return o;
  };
  size_t oX0 = put(X0), oB = put(B), oBi = put(BinvT), od = put(detB), oN = put(N), oL = put(L), oso = put(s_own),
         osn = put(s_nbr), oc = put(c11);
  std::vector<int> ints;
  ints.insert(ints.end(), nbr.begin(), nbr.end());
  ints.insert(ints.end(), nbrface.begin(), nbrface.end());
  ints.insert(ints.end(), tag.begin(), tag.end());
  ints.insert(ints.end(), side.begin(), side.end());
  if (cudaSetDevice(ctx->device) != cudaSuccess ||
      cudaMalloc(&m->d_real, sizeof(double) * real.size()) != cudaSuccess ||
      cudaMalloc(&m->d_int, sizeof(int) * ints.size()) != cudaSuccess) {
    cudaGetLastError();
    pp_mesh_destroy(m);
    return set_error(ctx, PP_ENOMEM, "pp_mesh_create: device allocation failed");
  }
  if (cudaMemcpy(m->d_real, real.data(), sizeof(double) * real.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_int, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    pp_mesh_destroy(m);
    return set_error(ctx, PP_ECUDA, "pp_mesh_create: copy failed");
  }
  DevMesh& d = m->dev;
  d.ne = nt;
  d.X0 = m->d_real + oX0;
  d.B = m->d_real + oB;
  d.BinvT = m->d_real + oBi;
  d.detB = m->d_real + od;
  d.N = m->d_real + oN;
  d.L = m->d_real + oL;
  d.s_own = m->d_real + oso;
  d.s_nbr = m->d_real + osn;
  d.c11 = m->d_real + oc;
  d.nbr = m->d_int;
  d.nbrface = m->d_int + 3 * nt;
  d.tag = m->d_int + 6 * nt;
  d.side = m->d_int + 9 * nt;
  *out = m;
  return PP_OK;
}

int pp_sweep_counts(const pp_ctx* ctx, int64_t* newton, int64_t* gmres_primal, int64_t* gmres_tangent,
                    int64_t* gmres_adjoint) {
  if (!ctx) return PP_EINVAL;
  if (newton) *newton = ctx->last_newton_iters;
  if (gmres_primal) *gmres_primal = ctx->last_gmres_iters;
  if (gmres_tangent) *gmres_tangent = ctx->last_gmres_tangent;
  if (gmres_adjoint) *gmres_adjoint = ctx->last_gmres_adjoint;
  return PP_OK;
}

int pp_mesh_destroy(pp_mesh* m) {
  if (!m) return PP_OK;
  if (m->ctx && m->ctx->lin_mesh == m) {
    m->ctx->lin_mesh = nullptr;
    m->ctx->lin_valid = false;
  }
  cudaFree(m->d_real);
  cudaFree(m->d_int);
  delete m;
  return PP_OK;
}

int pp_mesh_info(const pp_mesh* m, int* ne, int* np, int64_t* nu) {
  if (!m) return PP_EINVAL;
  if (ne) *ne = m->ne;
  if (np) *np = m->ctx->tb.Np;
  if (nu) *nu = (int64_t)m->ne * m->ctx->tb.nb;
  return PP_OK;
}

int pp_residual(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double t, const double* u, double* r) {
  if (!ctx || !mesh || !mu || !u || !r) return set_error(ctx, PP_EINVAL, "pp_residual: null argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  FrameT<double> fr = frame_of(motion(ctx, mu, n_mu, t));
  PP_CK(launch_residual(mesh->dev, ctx->tb, ctx->ph, fr, u, r, ctx->stream));
  PP_CK(cudaStreamSynchronize(ctx->stream));
  return PP_OK;
}

int pp_jacobian_blocks(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double t, const double* u,
                       double* blocks) {
  if (!ctx || !mesh || !mu || !u || !blocks) return set_error(ctx, PP_EINVAL, "pp_jacobian_blocks: null argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  FrameT<double> fr = frame_of(motion(ctx, mu, n_mu, t));
  PP_CK(launch_jacobian(mesh->dev, ctx->tb, ctx->ph, fr, u, blocks, ctx->stream));
  PP_CK(cudaStreamSynchronize(ctx->stream));
  return PP_OK;
}

int pp_qoi_rate(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double t, const double* u,
                double* out) {
  if (!ctx || !mesh || !mu || !u || !out) return set_error(ctx, PP_EINVAL, "pp_qoi_rate: null argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  PP_TRY(ensure_workspace(ctx, mesh));
  FrameT<double> fr = frame_of(motion(ctx, mu, n_mu, t));
  PP_CK(launch_qoi(mesh->dev, ctx->tb, ctx->ph, fr, u, ctx->d_elem, ctx->stream));
  PP_CK(launch_colsum(mesh->ne, 2, ctx->d_elem, ctx->d_scalar, ctx->d_partial, ctx->d_counter, ctx->stream));
  PP_CK(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PP_CK(cudaStreamSynchronize(ctx->stream));
  out[0] = ctx->h_scalar[0];
  out[1] = ctx->h_scalar[1];
  return PP_OK;
}

int pp_primal_period(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                     double* u_traj, double* u_final, double* qoi) {
  if (!ctx || !mesh || !mu || !u0 || Nt < 1) return set_error(ctx, PP_EINVAL, "pp_primal_period: bad argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  return primal_sweep(ctx, mesh, mu, n_mu, u0, Nt, u_traj, u_final, qoi);
}

int pp_tangent_matvec(pp_ctx* ctx, const double* v, double* out) {
  if (!ctx || !v || !out) return set_error(ctx, PP_EINVAL, "pp_tangent_matvec: null argument");
  if (!ctx->lin_valid) return set_error(ctx, PP_ESTATE, "pp_tangent_matvec: no stored primal sweep");
  PP_CK(cudaSetDevice(ctx->device));
  return tangent_sweep(ctx, v, out);
}

int pp_adjoint_sweep(pp_ctx* ctx, const double* lam_Nt, const double* weights, double* lam0, double* dFdmu) {
  if (!ctx || !lam_Nt || !lam0) return set_error(ctx, PP_EINVAL, "pp_adjoint_sweep: null argument");
  if (!ctx->lin_valid) return set_error(ctx, PP_ESTATE, "pp_adjoint_sweep: no stored primal sweep");
  PP_CK(cudaSetDevice(ctx->device));
  return adjoint_sweep(ctx, lam_Nt, weights, lam0, dFdmu);
}

int pp_shoot_nk(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0_guess, int Nt,
                double tol, double* u0_out, double* qoi, pp_shoot_stats* stats) {
  if (!ctx || !mesh || !mu || !u0_out || Nt < 1 || !(tol > 0))
    return set_error(ctx, PP_EINVAL, "pp_shoot_nk: bad argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  return shoot_nk(ctx, mesh, mu, n_mu, u0_guess, Nt, tol, u0_out, qoi, stats);
}

int pp_steady_state(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double tol, int maxit, double* u,
                    int* steps, double* rel_res) {
  if (!ctx || !mesh || !mu || !u || !(tol > 0) || maxit < 1)
    return set_error(ctx, PP_EINVAL, "pp_steady_state: bad argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  return steady_state(ctx, mesh, mu, n_mu, u, tol, maxit, steps, rel_res);
}

int pp_periodic_adjoint(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                        const double* weights, double* F, double* dFdmu, double* lam_Nt, pp_adj_stats* stats) {
  if (!ctx || !mesh || !mu || !weights || !dFdmu || Nt < 1)
    return set_error(ctx, PP_EINVAL, "pp_periodic_adjoint: bad argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  return periodic_adjoint(ctx, mesh, mu, n_mu, u0, Nt, weights, F, dFdmu, lam_Nt, stats);
}

int pp_shoot_nk_batched(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, int n_batch,
                        const double* u0_guess, int Nt, double tol, double* u0_out, double* qoi, pp_shoot_stats* stats,
                        int* status) {
  if (!ctx || !mesh || !mu || !u0_out || n_batch < 1 || Nt < 1 || !(tol > 0))
    return set_error(ctx, PP_EINVAL, "pp_shoot_nk_batched: bad argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  const int64_t nu = mesh_nu(ctx, mesh);
  int first = PP_OK;
  for (int b = 0; b < n_batch; ++b) {
    const int st = shoot_nk(ctx, mesh, mu + (size_t)b * n_mu, n_mu, u0_guess ? u0_guess + (size_t)b * nu : nullptr, Nt,
                            tol, u0_out + (size_t)b * nu, qoi ? qoi + 4 * (size_t)b : nullptr,
                            stats ? stats + b : nullptr);
    if (status) status[b] = st;
    if (st != PP_OK && st != PP_ENOCONV) return st;
    if (st != PP_OK && first == PP_OK) first = st;
  }
  return first;
}

int pp_periodic_adjoint_batched(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, int n_batch,
                                const double* u0, int Nt, const double* weights, double* F, double* dFdmu,
                                double* lam_Nt, pp_adj_stats* stats) {
  if (!ctx || !mesh || !mu || !u0 || !weights || !dFdmu || n_batch < 1 || Nt < 1)
    return set_error(ctx, PP_EINVAL, "pp_periodic_adjoint_batched: bad argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  const int64_t nu = mesh_nu(ctx, mesh);
  for (int b = 0; b < n_batch; ++b)
    PP_TRY(periodic_adjoint(ctx, mesh, mu + (size_t)b * n_mu, n_mu, u0 + (size_t)b * nu, Nt, weights + 2 * (size_t)b,
                            F ? F + b : nullptr, dFdmu + (size_t)b * n_mu, lam_Nt ? lam_Nt + (size_t)b * nu : nullptr,
                            stats ? stats + b : nullptr));
  return PP_OK;
}

int pp_periodic_adjoint_multi(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                              int n_qoi, const double* weights, double* F, double* dFdmu, double* lam_Nt,
                              pp_adj_stats* stats) {
  if (!ctx || !mesh || !mu || !weights || !dFdmu || Nt < 1 || n_qoi < 1 || n_qoi > 4)
    return set_error(ctx, PP_EINVAL, "pp_periodic_adjoint_multi: bad argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  return periodic_adjoint_multi(ctx, mesh, mu, n_mu, u0, Nt, n_qoi, weights, F, dFdmu, lam_Nt, stats);
}

int pp_shoot_fixed_point(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0_guess,
                         int Nt, double tol, int maxit, double* u0_out, double* qoi, pp_shoot_stats* stats) {
  if (!ctx || !mesh || !mu || !u0_guess || !u0_out || Nt < 1 || !(tol > 0) || maxit < 0)
    return set_error(ctx, PP_EINVAL, "pp_shoot_fixed_point: bad argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  return shoot_fixed_point(ctx, mesh, mu, n_mu, u0_guess, Nt, tol, maxit, u0_out, qoi, stats);
}

int pp_periodic_adjoint_fixed_point(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0,
                                    int Nt, const double* weights, double tol, int maxit, double* F, double* dFdmu,
                                    double* lam_Nt, pp_adj_stats* stats) {
  if (!ctx || !mesh || !mu || !weights || !dFdmu || Nt < 1 || !(tol > 0) || maxit < 0)
    return set_error(ctx, PP_EINVAL, "pp_periodic_adjoint_fixed_point: bad argument");
  PP_TRY(check_mu(ctx, n_mu));
  PP_CK(cudaSetDevice(ctx->device));
  return periodic_adjoint_fixed_point(ctx, mesh, mu, n_mu, u0, Nt, weights, tol, maxit, F, dFdmu, lam_Nt, stats);
}

int pp_stage_apply(pp_ctx* ctx, int step, int stage, int kind, int trans, int prec, const double* x, double* y) {
  if (!ctx) return PP_EINVAL;
  PP_CK(cudaSetDevice(ctx->device));
  return stage_apply(ctx, step, stage, kind, trans, prec, x, y);
}

}  // extern "C"
