// Element-local quadrature kernels of the ALE DG discretization (Sec. 6):
//  - k_residual     r(u, mu, t) of M du/dt = r (Eq. semidisc) with the CDG viscous
//                   terms (liftings of the face jumps); with a dual-valued
//                   frame it gives dr/ds for a motion seed s (theta, theta', h'),
//                   the building block of dr/dmu in Eq. funcl-grad-nosens-dirk;
//  - k_jacobian     element block Jacobian dr/du (diagonal + 3 face-neighbour
//                   blocks): exact flux derivatives at every quadrature point by
//                   forward-mode dual numbers, contracted with the basis;
//  - k_qoi*         instantaneous power and x-force on the wall (Eq. qoi) and
//                   their exact derivatives with respect to u and the frame.
//
// Layouts: u[e][a][i] (nb = 4 Np doubles per element, contiguous); Jacobian
// blocks [e][slot][col][row] (column-major nb x nb).
#include <mutex>

#include "flux.cuh"
#include "prof.h"
#include "../../include/pp_prof.h"

namespace pp {

namespace {

constexpr int RES_WARPS = 4;
constexpr int JAC_THREADS = 128;
constexpr int NSV = 12;  // volume seeds: U (4) + grad U (8)
constexpr int NSF = 24;  // face seeds: U-, grad U-, U+, grad U+

template <class T>
__device__ __forceinline__ void frame_P(const FrameT<T>& fr, const double* BinvT, T P[4]) {
  // grad_x phi = Q grad_X phi = Q B^{-T} grad_xi phi  =>  P = Q B^{-T}
  P[0] = fr.Q[0] * BinvT[0] + fr.Q[1] * BinvT[2];
  P[1] = fr.Q[0] * BinvT[1] + fr.Q[1] * BinvT[3];
  P[2] = fr.Q[2] * BinvT[0] + fr.Q[3] * BinvT[2];
  P[3] = fr.Q[2] * BinvT[1] + fr.Q[3] * BinvT[3];
}

template <class T>
__device__ __forceinline__ void mesh_velocity(const FrameT<T>& fr, const Phys& ph, double X, double Y, T vG[2]) {
  double dx = X - ph.x0[0], dy = Y - ph.x0[1];
  vG[0] = fr.Qd[0] * dx + fr.Qd[1] * dy;
  vG[1] = fr.Qd[2] * dx + fr.Qd[3] * dy + fr.hd;
}

__device__ __forceinline__ void ref_to_X(const DevMesh& m, int e, double xi, double eta, double& X, double& Y) {
  const double* B = m.B + 4 * e;
  X = m.X0[2 * e] + B[0] * xi + B[1] * eta;
  Y = m.X0[2 * e + 1] + B[2] * xi + B[3] * eta;
}

// state and physical gradient at a point from nodal values ue[a*Np + i]
template <class T>
__device__ __forceinline__ void interp(const double* ue, int Np, const double* phi, const double* dphi,
                                       const T P[4], T U[4], T dU[4][2]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double s = 0.0, s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < Np; ++i) {
      double c = ue[a * Np + i];
      s += phi[i] * c;
      s0 += dphi[2 * i] * c;
      s1 += dphi[2 * i + 1] * c;
    }
    U[a] = T(s);
    dU[a][0] = P[0] * s0 + P[1] * s1;
    dU[a][1] = P[2] * s0 + P[3] * s1;
  }
}

template <class T>
__device__ __forceinline__ void rotate_normal(const FrameT<T>& fr, const double* N, T n[2]) {
  n[0] = fr.Q[0] * N[0] + fr.Q[1] * N[1];
  n[1] = fr.Q[2] * N[0] + fr.Q[3] * N[1];
}

// value of U at a point from nodal values ue[a*Np + i]
__device__ __forceinline__ void interp_val(const double* ue, int Np, const double* phi, double U[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double s = 0.0;
    for (int i = 0; i < Np; ++i) s += phi[i] * ue[a * Np + i];
    U[a] = s;
  }
}

// CDG lifting of face jumps into a gradient at one point: dU[a][d] += s n[d] sum_p A[p*step] J[p][a]
// (A: one row of a reference lifting table, read forwards (step 1) or in reverse (step -1)
// for a neighbour's face whose points are matched in reverse order).
template <class T, class TJ>
__device__ __forceinline__ void lift_add(T dU[4][2], const T n[2], double s, const double* A, int step,
                                         const TJ* J, int nqf) {
  TJ l[4] = {TJ(0.0), TJ(0.0), TJ(0.0), TJ(0.0)};
  for (int p = 0; p < nqf; ++p) {
    const double c = A[p * step];
#pragma unroll
    for (int a = 0; a < 4; ++a) l[a] += c * J[p * 4 + a];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    dU[a][0] += s * (l[a] * n[0]);
    dU[a][1] += s * (l[a] * n[1]);
  }
}

// lifting-table row of face f at point q of this element, for the side that lifts it
// (side 1: the element's own face f; side 0: the neighbour's face g, points reversed)
__device__ __forceinline__ const double* lift_row(const DevTables& tb, int side, int f, int g, int q, int& step) {
  const int nqf = tb.nqf;
  if (side) {
    step = 1;
    return tb.lift_f + (f * nqf + q) * nqf;
  }
  step = -1;
  return tb.lift_f + (g * nqf + nqf - 1 - q) * nqf + nqf - 1;
}

// ------------------------------------------------------------------------ residual
// Warp per element.  Phase A: the jumps U_hat - U- at every face point (both traces).
// Phase B: volume points, gradient lifted by the element's own face liftings.  Phase C:
// face points, with the lifted gradient of the side that supplies the viscous flux.
// Phase D: projection on the test functions.
template <class T>
__global__ void __launch_bounds__(RES_WARPS * 32)
    k_residual(DevMesh m, DevTables tb, Phys ph, FrameT<T> fr, const double* __restrict__ u,
               double* __restrict__ rval, double* __restrict__ rder) {
  constexpr int W = sizeof(T) / sizeof(double);
  __shared__ double s_u[RES_WARPS][4 * kMaxNb];
  __shared__ double s_G[RES_WARPS][kMaxQv * 8 * W];
  __shared__ double s_H[RES_WARPS][3 * kMaxQf * 4 * W];
  __shared__ double s_J[RES_WARPS][3 * kMaxQf * 4 * W];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * RES_WARPS + warp;
  if (e >= m.ne) return;
  const int Np = tb.Np, nb = tb.nb, nqv = tb.nqv, nqf = tb.nqf;
  double* su = s_u[warp];
  T* G = reinterpret_cast<T*>(s_G[warp]);
  T* Hs = reinterpret_cast<T*>(s_H[warp]);
  T* Js = reinterpret_cast<T*>(s_J[warp]);

  for (int idx = lane; idx < 4 * nb; idx += 32) {
    int slot = idx / nb, k = idx - slot * nb;
    int src = e;
    if (slot > 0) {
      int nn = m.nbr[3 * e + slot - 1];
      src = nn >= 0 ? nn : e;
    }
    su[idx] = u[(size_t)src * nb + k];
  }
  __syncwarp();

  T P[4];
  frame_P(fr, m.BinvT + 4 * e, P);
  const double detB = m.detB[e];
  T nf[3][2];
#pragma unroll
  for (int f = 0; f < 3; ++f) rotate_normal(fr, m.N + 6 * e + 2 * f, nf[f]);

  // phase A: jumps
  for (int idx = lane; idx < 3 * nqf; idx += 32) {
    const int f = idx / nqf, q = idx - f * nqf;
    const int tag = m.tag[3 * e + f];
    double um[4], up[4];
    interp_val(su, Np, tb.phi_f + (f * nqf + q) * Np, um);
    if (tag == 0) {
      const int g = m.nbrface[3 * e + f], qq = nqf - 1 - q;
      interp_val(su + (1 + f) * nb, Np, tb.phi_f + (g * nqf + qq) * Np, up);
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a) up[a] = um[a];
    }
    T Um[4], Up[4], vG[2], Uh[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      Um[a] = T(um[a]);
      Up[a] = T(up[a]);
    }
    double X, Y;
    ref_to_X(m, e, tb.xi_f[2 * (f * nqf + q)], tb.xi_f[2 * (f * nqf + q) + 1], X, Y);
    mesh_velocity(fr, ph, X, Y, vG);
    face_value(tag, Um, Up, vG, ph, Uh);
#pragma unroll
    for (int a = 0; a < 4; ++a) Js[(f * kMaxQf + q) * 4 + a] = Uh[a] - Um[a];
  }
  __syncwarp();

  // phase B: volume points
  for (int q = lane; q < nqv; q += 32) {
    T U[4], dU[4][2], vG[2], F[4][2];
    interp(su, Np, tb.phi_v + q * Np, tb.dphi_v + 2 * q * Np, P, U, dU);
#pragma unroll
    for (int f = 0; f < 3; ++f)
      if (m.side[3 * e + f])
        lift_add(dU, nf[f], m.s_own[3 * e + f], tb.lift_v + (f * nqv + q) * nqf, 1, Js + f * kMaxQf * 4, nqf);
    double X, Y;
    ref_to_X(m, e, tb.xi_v[2 * q], tb.xi_v[2 * q + 1], X, Y);
    mesh_velocity(fr, ph, X, Y, vG);
    volume_flux(U, dU, vG, ph, F);
    double wq = tb.w_v[q] * detB;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      G[(q * 4 + a) * 2 + 0] = wq * (P[0] * F[a][0] + P[2] * F[a][1]);
      G[(q * 4 + a) * 2 + 1] = wq * (P[1] * F[a][0] + P[3] * F[a][1]);
    }
  }
  // phase C: face points
  for (int idx = lane; idx < 3 * nqf; idx += 32) {
    const int f = idx / nqf, q = idx - f * nqf;
    const int tag = m.tag[3 * e + f], side = m.side[3 * e + f];
    T Um[4], dUm[4][2], Up[4], dUp[4][2], vG[2], H[4];
    interp(su, Np, tb.phi_f + (f * nqf + q) * Np, tb.dphi_f + 2 * (f * nqf + q) * Np, P, Um, dUm);
    int g = 0;
    if (tag == 0) {
      const int e2 = m.nbr[3 * e + f], qq = nqf - 1 - q;
      g = m.nbrface[3 * e + f];
      T P2[4];
      frame_P(fr, m.BinvT + 4 * e2, P2);
      interp(su + (1 + f) * nb, Np, tb.phi_f + (g * nqf + qq) * Np, tb.dphi_f + 2 * (g * nqf + qq) * Np, P2, Up,
             dUp);
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        Up[a] = Um[a];
        dUp[a][0] = dUm[a][0];
        dUp[a][1] = dUm[a][1];
      }
    }
    T QS[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      QS[a][0] = side ? dUm[a][0] : dUp[a][0];
      QS[a][1] = side ? dUm[a][1] : dUp[a][1];
    }
    int step;
    const double* A = lift_row(tb, side, f, g, q, step);
    lift_add(QS, nf[f], side ? m.s_own[3 * e + f] : m.s_nbr[3 * e + f], A, step, Js + f * kMaxQf * 4, nqf);
    double X, Y;
    ref_to_X(m, e, tb.xi_f[2 * (f * nqf + q)], tb.xi_f[2 * (f * nqf + q) + 1], X, Y);
    mesh_velocity(fr, ph, X, Y, vG);
    face_flux(tag, side, Um, Up, QS, nf[f], vG, m.c11[3 * e + f], ph, H);
    double wl = tb.w_f[q] * m.L[3 * e + f];
#pragma unroll
    for (int a = 0; a < 4; ++a) Hs[(f * kMaxQf + q) * 4 + a] = wl * H[a];
  }
  __syncwarp();
  for (int o = lane; o < nb; o += 32) {
    int a = o / Np, i = o - a * Np;
    T acc(0.0);
    for (int q = 0; q < nqv; ++q) {
      const double* d = tb.dphi_v + 2 * (q * Np + i);
      acc += d[0] * G[(q * 4 + a) * 2] + d[1] * G[(q * 4 + a) * 2 + 1];
    }
    for (int f = 0; f < 3; ++f)
      for (int q = 0; q < nqf; ++q) acc -= tb.phi_f[(f * nqf + q) * Np + i] * Hs[(f * kMaxQf + q) * 4 + a];
    if (rval) rval[(size_t)e * nb + o] = val(acc);
    if (rder) rder[(size_t)e * nb + o] = der(acc);
  }
}

// ------------------------------------------------------------------------ Jacobian
// Shared-memory carve-up of k_jacobian (doubles), sized from the runtime degree.
struct JacSmem {
  int su, SV, SF, Cv, Cf, Tv, Tf, Tn, Wv, Wf, Wn, Js, Gb, cv, cf, Y, Lam, LamW, total;
  __host__ __device__ JacSmem(int nb, int Np, int nqv) {
    su = 0;
    SV = su + 4 * nb;                 // [q][12]: U, lifted grad U at the volume points
    SF = SV + nqv * 12;               // [side][f][q][12]: both traces (flux side: lifted gradient)
    Cv = SF + 2 * 3 * kMaxQf * 12;
    Cf = Cv + nqv * 4 * 2 * NSV;
    Tv = Cf + 3 * kMaxQf * 4 * NSF;
    Tf = Tv + nqv * 3 * Np;
    Tn = Tf + 3 * kMaxQf * 3 * Np;
    Wv = Tn + 3 * kMaxQf * 3 * Np;
    Wf = Wv + nqv * 2 * Np;
    Wn = Wf + 3 * kMaxQf * Np;
    Js = Wn + 3 * kMaxQf * Np;        // [f][q][4] jumps U_hat - U-
    Gb = Js + 3 * kMaxQf * 4;         // [f][q][4][4] d U_wall / d U- at wall points
    cv = Gb + 3 * kMaxQf * 16;        // [f][q][k] per pair: volume gradient coefficients along n_f
    cf = cv + 3 * nqv * 2;            // [f][q]    per pair: face gradient coefficients along n_f
    Y = cf + 3 * kMaxQf;              // [f][i][q] per pair: cv contracted with the test gradients
    Lam = Y + 3 * Np * nqv;           // [f][i][p] per pair: d r_(a,i) / d jump_(f,b)(p)
    LamW = Lam + 3 * Np * kMaxQf;     // [f][b][i][p] Lam of wall faces for every b of the row a
    total = LamW + 3 * 4 * Np * kMaxQf;
  }
};

// Element block Jacobian.  Phase 0: U and grad U at every point (both traces on faces), the
// face jumps U_hat - U- and, at wall points, d U_wall / d U-; then the CDG liftings: the
// volume gradients and the flux side's face gradients become the lifted ones.  Phase 1:
// exact derivatives of the quadrature-point fluxes with respect to (U, lifted grad U) by
// dual numbers (state seeds) and by linearity (gradient seeds: the viscous flux is linear
// in the gradient at fixed U), weighted and projected on the reference test gradients (C).
// Phase 2, per variable pair (a, b): W = C T over the trial tables, J_ab = D W, plus the
// liftings' chain: Lam = d r_a / d jump_b at the face points (through the volume and the
// face gradients), contracted with d jump / d u (-phi of this element, +phi of the
// neighbour; at wall points d U_wall / d U- couples b to every variable, added per row a).
__global__ void __launch_bounds__(JAC_THREADS)
    k_jacobian(DevMesh m, DevTables tb, Phys ph, FrameT<double> fr, const double* __restrict__ u,
               double* __restrict__ J) {
  extern __shared__ double smem[];
  const int e = blockIdx.x;
  const int tid = threadIdx.x;
  const int Np = tb.Np, nb = tb.nb, nqv = tb.nqv, nqf = tb.nqf;
  const JacSmem L(nb, Np, nqv);
  double* su = smem + L.su;
  double* Cv = smem + L.Cv;
  double* Cf = smem + L.Cf;
  double* Tv = smem + L.Tv;  // [q][t][j]
  double* Tf = smem + L.Tf;  // [f][q][t][j] (own trace)
  double* Tn = smem + L.Tn;  // [f][q][t][j] (neighbour trace at the matched point)
  double* Wv = smem + L.Wv;  // [q][k][j]
  double* Wf = smem + L.Wf;  // [f][q][j]
  double* Wn = smem + L.Wn;  // [f][q][j]
  double* Js = smem + L.Js;
  double* Gb = smem + L.Gb;
  double* cvv = smem + L.cv;
  double* cff = smem + L.cf;
  double* Yv = smem + L.Y;
  double* Lam = smem + L.Lam;
  double* LamW = smem + L.LamW;
  for (int idx = tid; idx < 4 * nb; idx += JAC_THREADS) {
    int slot = idx / nb, k = idx - slot * nb;
    int src = e;
    if (slot > 0) {
      int nn = m.nbr[3 * e + slot - 1];
      src = nn >= 0 ? nn : e;
    }
    su[idx] = u[(size_t)src * nb + k];
  }
  __syncthreads();
  double P[4];
  frame_P(fr, m.BinvT + 4 * e, P);
  const double detB = m.detB[e];
  FrameT<Dual> frd;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    frd.Q[k] = Dual(fr.Q[k]);
    frd.Qd[k] = Dual(fr.Qd[k]);
  }
  frd.hd = Dual(fr.hd);
  double nf[3][2];
  int sidef[3], tagf[3], gf[3];
  double s_lift[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    rotate_normal(fr, m.N + 6 * e + 2 * f, nf[f]);
    sidef[f] = m.side[3 * e + f];
    tagf[f] = m.tag[3 * e + f];
    gf[f] = tagf[f] == 0 ? m.nbrface[3 * e + f] : 0;
    s_lift[f] = sidef[f] ? m.s_own[3 * e + f] : m.s_nbr[3 * e + f];
  }
  const bool has_wall = tagf[0] == 1 || tagf[1] == 1 || tagf[2] == 1;

  double* SV = smem + L.SV;
  double* SF = smem + L.SF;
  // phase 0a: U and grad U at every quadrature point, once (both traces on faces)
  for (int task = tid; task < nqv + 6 * nqf; task += JAC_THREADS) {
    double U0[4], dU0[4][2];
    double* dst;
    if (task < nqv) {
      interp(su, Np, tb.phi_v + task * Np, tb.dphi_v + 2 * task * Np, P, U0, dU0);
      dst = SV + task * 12;
    } else {
      const int t2 = task - nqv, side = t2 / (3 * nqf), r2 = t2 - side * 3 * nqf, f = r2 / nqf, q = r2 - f * nqf;
      dst = SF + ((side * 3 + f) * kMaxQf + q) * 12;
      if (side == 0 || tagf[f] != 0) {
        interp(su, Np, tb.phi_f + (f * nqf + q) * Np, tb.dphi_f + 2 * (f * nqf + q) * Np, P, U0, dU0);
      } else {
        const int e2 = m.nbr[3 * e + f], g = gf[f], qq = nqf - 1 - q;
        double P2[4];
        frame_P(fr, m.BinvT + 4 * e2, P2);
        interp(su + (1 + f) * nb, Np, tb.phi_f + (g * nqf + qq) * Np, tb.dphi_f + 2 * (g * nqf + qq) * Np, P2, U0,
               dU0);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      dst[a] = U0[a];
      dst[4 + 2 * a] = dU0[a][0];
      dst[5 + 2 * a] = dU0[a][1];
    }
  }
  __syncthreads();
  // phase 0b: jumps, and d U_wall / d U- at wall points (4 dual seeds)
  for (int idx = tid; idx < 3 * nqf; idx += JAC_THREADS) {
    const int f = idx / nqf, q = idx - f * nqf;
    const double* Sm = SF + ((0 * 3 + f) * kMaxQf + q) * 12;
    const double* Sp = SF + ((1 * 3 + f) * kMaxQf + q) * 12;
    double X, Y, vG[2], Uh[4];
    ref_to_X(m, e, tb.xi_f[2 * (f * nqf + q)], tb.xi_f[2 * (f * nqf + q) + 1], X, Y);
    mesh_velocity(fr, ph, X, Y, vG);
    face_value(tagf[f], Sm, Sp, vG, ph, Uh);
#pragma unroll
    for (int a = 0; a < 4; ++a) Js[(f * kMaxQf + q) * 4 + a] = Uh[a] - Sm[a];
    if (tagf[f] == 1) {
      Dual vd[2] = {Dual(vG[0]), Dual(vG[1])};
      for (int c = 0; c < 4; ++c) {
        Dual Ud[4], Ub[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) Ud[a] = Dual(Sm[a], a == c ? 1.0 : 0.0);
        wall_state(Ud, vd, Ub);
#pragma unroll
        for (int b = 0; b < 4; ++b) Gb[((f * kMaxQf + q) * 4 + b) * 4 + c] = Ub[b].d;
      }
    }
  }
  __syncthreads();
  // phase 0c: lifted gradients (volume points; the flux side's trace on each face)
  for (int task = tid; task < nqv + 3 * nqf; task += JAC_THREADS) {
    double dU[4][2];
    double* dst;
    if (task < nqv) {
      dst = SV + task * 12;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        dU[a][0] = 0.0;
        dU[a][1] = 0.0;
      }
      for (int f = 0; f < 3; ++f)
        if (sidef[f]) lift_add(dU, nf[f], s_lift[f], tb.lift_v + (f * nqv + task) * nqf, 1, Js + f * kMaxQf * 4, nqf);
    } else {
      const int t2 = task - nqv, f = t2 / nqf, q = t2 - f * nqf;
      dst = SF + (((sidef[f] ? 0 : 1) * 3 + f) * kMaxQf + q) * 12;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        dU[a][0] = 0.0;
        dU[a][1] = 0.0;
      }
      int step;
      const double* A = lift_row(tb, sidef[f], f, gf[f], q, step);
      lift_add(dU, nf[f], s_lift[f], A, step, Js + f * kMaxQf * 4, nqf);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      dst[4 + 2 * a] += dU[a][0];
      dst[5 + 2 * a] += dU[a][1];
    }
  }
  __syncthreads();

  // phase 1a: volume seeds.  The state seeds (4 per point) run the flux in dual numbers;
  // the viscous flux is linear in grad U at fixed U, so the derivative for gradient seed
  // (b, d) is the viscous flux of the unit gradient (8 per point, plain FP64).
  for (int task = tid; task < nqv * NSV; task += JAC_THREADS) {
    const bool dual = task < 4 * nqv;
    const int q = dual ? task >> 2 : (task - 4 * nqv) >> 3;
    const int s = dual ? (task & 3) : 4 + ((task - 4 * nqv) & 7);
    const double* Sq = SV + q * 12;
    double Fd[4][2];
    if (dual) {
      Dual U[4], dU[4][2], vG[2], F[4][2];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        U[a] = Dual(Sq[a], s == a ? 1.0 : 0.0);
        dU[a][0] = Dual(Sq[4 + 2 * a]);
        dU[a][1] = Dual(Sq[5 + 2 * a]);
      }
      double X, Y;
      ref_to_X(m, e, tb.xi_v[2 * q], tb.xi_v[2 * q + 1], X, Y);
      mesh_velocity(frd, ph, X, Y, vG);
      volume_flux(U, dU, vG, ph, F);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        Fd[a][0] = F[a][0].d;
        Fd[a][1] = F[a][1].d;
      }
    } else {
      double U[4], E[4][2], Fv[4][2];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        U[a] = Sq[a];
        E[a][0] = (s == 4 + 2 * a) ? 1.0 : 0.0;
        E[a][1] = (s == 5 + 2 * a) ? 1.0 : 0.0;
      }
      viscous_flux(U, E, ph, false, Fv);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        Fd[a][0] = -Fv[a][0];
        Fd[a][1] = -Fv[a][1];
      }
    }
    const double wq = tb.w_v[q] * detB;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      Cv[((q * 4 + a) * 2 + 0) * NSV + s] = wq * (P[0] * Fd[a][0] + P[2] * Fd[a][1]);
      Cv[((q * 4 + a) * 2 + 1) * NSV + s] = wq * (P[1] * Fd[a][0] + P[3] * Fd[a][1]);
    }
  }
  // phase 1b: face seeds: both traces' states in dual numbers (U- 0..3, U+ 12..15) with the
  // lifted gradient held fixed; the flux side's gradient by linearity (grad U- 4..11 when
  // this element supplies the viscous flux, grad U+ 16..23 when the neighbour does)
  for (int task = tid; task < 3 * nqf * NSF; task += JAC_THREADS) {
    const bool dual = task < 3 * nqf * 8;
    int f, q, s;
    if (dual) {
      f = task / (nqf * 8);
      const int rem = task - f * nqf * 8;
      q = rem >> 3;
      const int j = rem & 7;
      s = j < 4 ? j : 8 + j;  // 0..3 (U-), 12..15 (U+)
    } else {
      const int t2 = task - 3 * nqf * 8;
      f = t2 / (nqf * 16);
      const int rem = t2 - f * nqf * 16;
      q = rem >> 4;
      const int j = rem & 15;
      s = j < 8 ? 4 + j : 8 + j;  // 4..11 (grad U-), 16..23 (grad U+)
    }
    const int tag = tagf[f], side = sidef[f];
    double* out = Cf + ((f * kMaxQf + q) * 4) * NSF + s;
    const bool grad_seed = !dual;
    const bool plus = s >= 12;
    if ((tag != 0 && plus) || (grad_seed && (plus ? side == 1 : side == 0))) {
#pragma unroll
      for (int a = 0; a < 4; ++a) out[a * NSF] = 0.0;
      continue;
    }
    const double* Sm = SF + ((0 * 3 + f) * kMaxQf + q) * 12;
    const double* Sp = SF + ((1 * 3 + f) * kMaxQf + q) * 12;
    const double* SS = side ? Sm : Sp;
    const double wl = tb.w_f[q] * m.L[3 * e + f];
    const double c11 = m.c11[3 * e + f];
    if (dual) {
      Dual Um[4], Up[4], QS[4][2], n[2], vG[2], H[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        Um[a] = Dual(Sm[a], s == a ? 1.0 : 0.0);
        Up[a] = Dual(Sp[a], s == 12 + a ? 1.0 : 0.0);
        QS[a][0] = Dual(SS[4 + 2 * a]);
        QS[a][1] = Dual(SS[5 + 2 * a]);
      }
      rotate_normal(frd, m.N + 6 * e + 2 * f, n);
      double X, Y;
      ref_to_X(m, e, tb.xi_f[2 * (f * nqf + q)], tb.xi_f[2 * (f * nqf + q) + 1], X, Y);
      mesh_velocity(frd, ph, X, Y, vG);
      face_flux(tag, side, Um, Up, QS, n, vG, c11, ph, H);
#pragma unroll
      for (int a = 0; a < 4; ++a) out[a * NSF] = wl * H[a].d;
    } else {
      const int sg = plus ? s - 16 : s - 4;
      const int b = sg >> 1, d = sg & 1;
      double U[4], E[4][2], Fv[4][2];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        U[a] = SS[a];
        E[a][0] = (a == b && d == 0) ? 1.0 : 0.0;
        E[a][1] = (a == b && d == 1) ? 1.0 : 0.0;
      }
      if (tag == 1) {
        // wall: the viscous flux is evaluated at the wall state (interior density and
        // internal energy, wall velocity), adiabatic
        double X, Y, vG[2], Ub[4];
        ref_to_X(m, e, tb.xi_f[2 * (f * nqf + q)], tb.xi_f[2 * (f * nqf + q) + 1], X, Y);
        mesh_velocity(fr, ph, X, Y, vG);
        wall_state(U, vG, Ub);
        viscous_flux(Ub, E, ph, true, Fv);
      } else {
        viscous_flux(U, E, ph, false, Fv);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) out[a * NSF] = -wl * (Fv[a][0] * nf[f][0] + Fv[a][1] * nf[f][1]);
    }
  }
  // trial tables: basis values and physical gradients at the volume / face points
  for (int idx = tid; idx < nqv * Np; idx += JAC_THREADS) {
    const int q = idx / Np, j = idx - q * Np;
    const double* dj = tb.dphi_v + 2 * (q * Np + j);
    Tv[(q * 3 + 0) * Np + j] = tb.phi_v[q * Np + j];
    Tv[(q * 3 + 1) * Np + j] = P[0] * dj[0] + P[1] * dj[1];
    Tv[(q * 3 + 2) * Np + j] = P[2] * dj[0] + P[3] * dj[1];
  }
  for (int idx = tid; idx < 3 * nqf * Np; idx += JAC_THREADS) {
    const int f = idx / (nqf * Np), rem = idx - f * nqf * Np, q = rem / Np, j = rem - q * Np;
    const double* dj = tb.dphi_f + 2 * ((f * nqf + q) * Np + j);
    double* to = Tf + ((f * kMaxQf + q) * 3) * Np + j;
    to[0] = tb.phi_f[(f * nqf + q) * Np + j];
    to[Np] = P[0] * dj[0] + P[1] * dj[1];
    to[2 * Np] = P[2] * dj[0] + P[3] * dj[1];
    double* tn = Tn + ((f * kMaxQf + q) * 3) * Np + j;
    if (tagf[f] == 0) {
      const int e2 = m.nbr[3 * e + f], g = gf[f], qq = nqf - 1 - q;
      double P2[4];
      frame_P(fr, m.BinvT + 4 * e2, P2);
      const double* dn = tb.dphi_f + 2 * ((g * nqf + qq) * Np + j);
      tn[0] = tb.phi_f[(g * nqf + qq) * Np + j];
      tn[Np] = P2[0] * dn[0] + P2[1] * dn[1];
      tn[2 * Np] = P2[2] * dn[0] + P2[3] * dn[1];
    } else {
      tn[0] = tn[Np] = tn[2 * Np] = 0.0;
    }
  }
  __syncthreads();

  // phase 2: per variable pair (a, b)
  const size_t nb2 = (size_t)nb * nb;
  double* Jd = J + (size_t)e * 4 * nb2;
  const int nW = nqv * 2 * Np, nWf = 3 * nqf * Np;
  for (int ab = 0; ab < 16; ++ab) {
    const int a = ab >> 2, b = ab & 3;
    const int sb[3] = {b, 4 + 2 * b, 5 + 2 * b};
    // W = C T, and the gradient coefficients along each face normal for the liftings
    for (int idx = tid; idx < nW + 2 * nWf + 3 * nqv * 2 + 3 * nqf; idx += JAC_THREADS) {
      if (idx < nW) {
        const int q = idx / (2 * Np), rem = idx - q * 2 * Np, k = rem / Np, j = rem - k * Np;
        const double* C = Cv + ((q * 4 + a) * 2 + k) * NSV;
        const double* T = Tv + (q * 3) * Np + j;
        Wv[idx] = C[sb[0]] * T[0] + C[sb[1]] * T[Np] + C[sb[2]] * T[2 * Np];
      } else if (idx < nW + 2 * nWf) {
        const int id2 = idx - nW;
        const int side = id2 >= nWf;  // 0 own trace, 1 neighbour trace
        const int id3 = side ? id2 - nWf : id2;
        const int f = id3 / (nqf * Np), rem = id3 - f * nqf * Np, q = rem / Np, j = rem - q * Np;
        const double* C = Cf + ((f * kMaxQf + q) * 4 + a) * NSF + (side ? 12 : 0);
        const double* T = (side ? Tn : Tf) + ((f * kMaxQf + q) * 3) * Np + j;
        const double w = C[sb[0]] * T[0] + C[sb[1]] * T[Np] + C[sb[2]] * T[2 * Np];
        (side ? Wn : Wf)[(f * kMaxQf + q) * Np + j] = w;
      } else if (idx < nW + 2 * nWf + 3 * nqv * 2) {
        // cv[f][q][k] = s_f sum_d C_v(q, a, k; grad_d U_b) n_f[d] (faces this element lifts)
        const int id2 = idx - nW - 2 * nWf, f = id2 / (nqv * 2), rem = id2 - f * nqv * 2, q = rem >> 1, k = rem & 1;
        const double* C = Cv + ((q * 4 + a) * 2 + k) * NSV;
        cvv[id2] = sidef[f] ? s_lift[f] * (C[sb[1]] * nf[f][0] + C[sb[2]] * nf[f][1]) : 0.0;
      } else {
        // cf[f][q] = s_S sum_d C_f(f, q, a; grad_d U_b of the flux side) n_f[d]
        const int id2 = idx - nW - 2 * nWf - 3 * nqv * 2, f = id2 / nqf, q = id2 - f * nqf;
        const double* C = Cf + ((f * kMaxQf + q) * 4 + a) * NSF + (sidef[f] ? 0 : 12);
        cff[f * kMaxQf + q] = s_lift[f] * (C[sb[1]] * nf[f][0] + C[sb[2]] * nf[f][1]);
      }
    }
    __syncthreads();
    // Y[f][i][q] = sum_k dphi_k,i(q) cv[f][q][k]
    for (int idx = tid; idx < 3 * Np * nqv; idx += JAC_THREADS) {
      const int f = idx / (Np * nqv), rem = idx - f * Np * nqv, i = rem / nqv, q = rem - i * nqv;
      const double* di = tb.dphi_v + 2 * (q * Np + i);
      const double* c = cvv + (f * nqv + q) * 2;
      Yv[idx] = di[0] * c[0] + di[1] * c[1];
    }
    __syncthreads();
    // Lam[f][i][p] = d r_(a,i) / d jump_(f,b)(p): volume part (faces this element lifts)
    // minus the face part (test function phi_i on face f, the flux side's lifting row)
    for (int idx = tid; idx < 3 * Np * nqf; idx += JAC_THREADS) {
      const int f = idx / (Np * nqf), rem = idx - f * Np * nqf, i = rem / nqf, p = rem - i * nqf;
      double acc = 0.0;
      if (sidef[f]) {
        const double* y = Yv + (f * Np + i) * nqv;
        const double* lv = tb.lift_v + f * nqv * nqf + p;
        for (int q = 0; q < nqv; ++q) acc += y[q] * lv[q * nqf];
      }
      for (int q = 0; q < nqf; ++q) {
        int step;
        const double* A = lift_row(tb, sidef[f], f, gf[f], q, step);
        acc -= tb.phi_f[(f * nqf + q) * Np + i] * cff[f * kMaxQf + q] * A[p * step];
      }
      Lam[(f * Np + i) * kMaxQf + p] = acc;
      if (tagf[f] == 1) LamW[((f * 4 + b) * Np + i) * kMaxQf + p] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < 4 * Np * Np; idx += JAC_THREADS) {
      const int slot = idx / (Np * Np), rem = idx - slot * Np * Np, j = rem / Np, i = rem - j * Np;
      double acc = 0.0;
      if (slot == 0) {
        for (int q = 0; q < nqv; ++q) {
          const double* di = tb.dphi_v + 2 * (q * Np + i);
          acc += di[0] * Wv[(q * 2 + 0) * Np + j] + di[1] * Wv[(q * 2 + 1) * Np + j];
        }
        for (int f = 0; f < 3; ++f) {
          for (int q = 0; q < nqf; ++q)
            acc -= tb.phi_f[(f * nqf + q) * Np + i] * Wf[(f * kMaxQf + q) * Np + j];
          // d jump / d u_e = -phi_j (the wall state's own dependence is added below)
          for (int p = 0; p < nqf; ++p)
            acc -= Lam[(f * Np + i) * kMaxQf + p] * Tf[((f * kMaxQf + p) * 3) * Np + j];
        }
      } else {
        const int f = slot - 1;
        for (int q = 0; q < nqf; ++q) acc -= tb.phi_f[(f * nqf + q) * Np + i] * Wn[(f * kMaxQf + q) * Np + j];
        // d jump / d u_nbr = +phi_j of the neighbour at the matched point (zero off interior faces)
        for (int p = 0; p < nqf; ++p) acc += Lam[(f * Np + i) * kMaxQf + p] * Tn[((f * kMaxQf + p) * 3) * Np + j];
      }
      Jd[(size_t)slot * nb2 + (size_t)(b * Np + j) * nb + a * Np + i] = acc;
    }
    __syncthreads();
    if (has_wall && b == 3) {
      // wall points: the jump U_wall(U-) - U- also depends on U- through the wall state:
      // J_(a,c) += sum_b sum_p Lam_(a,b)[i][p] dU_wall,b/dU-_c phi_j(p)
      for (int idx = tid; idx < 4 * Np * Np; idx += JAC_THREADS) {
        const int c = idx / (Np * Np), rem = idx - c * Np * Np, j = rem / Np, i = rem - j * Np;
        double acc = 0.0;
        for (int f = 0; f < 3; ++f) {
          if (tagf[f] != 1) continue;
          for (int p = 0; p < nqf; ++p) {
            const double phij = Tf[((f * kMaxQf + p) * 3) * Np + j];
            const double* G = Gb + (f * kMaxQf + p) * 16;
            double s = 0.0;
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) s += LamW[((f * 4 + bb) * Np + i) * kMaxQf + p] * G[bb * 4 + c];
            acc += s * phij;
          }
        }
        Jd[(size_t)(c * Np + j) * nb + a * Np + i] += acc;
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------ QoI
// Per element: sum over its wall faces of w L (f . v_G, f_x), f = momentum part of the wall
// flux (with the CDG lifting of the wall jump; the wall faces are always lifted by the element).
template <class T>
__global__ void __launch_bounds__(RES_WARPS * 32)
    k_qoi(DevMesh m, DevTables tb, Phys ph, FrameT<T> fr, const double* __restrict__ u, double* __restrict__ out,
          int want_der) {
  constexpr int W = sizeof(T) / sizeof(double);
  __shared__ double s_J[RES_WARPS][3 * kMaxQf * 4 * W];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * RES_WARPS + warp;
  if (e >= m.ne) return;
  const int Np = tb.Np, nb = tb.nb, nqf = tb.nqf;
  const double* ue = u + (size_t)e * nb;
  T* Js = reinterpret_cast<T*>(s_J[warp]);
  T P[4];
  frame_P(fr, m.BinvT + 4 * e, P);
  for (int idx = lane; idx < 3 * nqf; idx += 32) {
    int f = idx / nqf, q = idx - f * nqf;
    if (m.tag[3 * e + f] != 1) continue;
    double um[4];
    interp_val(ue, Np, tb.phi_f + (f * nqf + q) * Np, um);
    T Um[4], vG[2], Ub[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) Um[a] = T(um[a]);
    double X, Y;
    ref_to_X(m, e, tb.xi_f[2 * (f * nqf + q)], tb.xi_f[2 * (f * nqf + q) + 1], X, Y);
    mesh_velocity(fr, ph, X, Y, vG);
    wall_state(Um, vG, Ub);
#pragma unroll
    for (int a = 0; a < 4; ++a) Js[(f * kMaxQf + q) * 4 + a] = Ub[a] - Um[a];
  }
  __syncwarp();
  T pw(0.0), fx(0.0);
  for (int idx = lane; idx < 3 * nqf; idx += 32) {
    int f = idx / nqf, q = idx - f * nqf;
    if (m.tag[3 * e + f] != 1) continue;
    T Um[4], dUm[4][2], n[2], vG[2], H[4];
    interp(ue, Np, tb.phi_f + (f * nqf + q) * Np, tb.dphi_f + 2 * (f * nqf + q) * Np, P, Um, dUm);
    rotate_normal(fr, m.N + 6 * e + 2 * f, n);
    lift_add(dUm, n, m.s_own[3 * e + f], tb.lift_f + (f * nqf + q) * nqf, 1, Js + f * kMaxQf * 4, nqf);
    double X, Y;
    ref_to_X(m, e, tb.xi_f[2 * (f * nqf + q)], tb.xi_f[2 * (f * nqf + q) + 1], X, Y);
    mesh_velocity(fr, ph, X, Y, vG);
    face_flux(1, 1, Um, Um, dUm, n, vG, m.c11[3 * e + f], ph, H);
    double wl = tb.w_f[q] * m.L[3 * e + f];
    pw += wl * (H[1] * vG[0] + H[2] * vG[1]);
    fx += wl * H[1];
  }
  double a0 = want_der ? der(pw) : val(pw);
  double a1 = want_der ? der(fx) : val(fx);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
  }
  if (lane == 0) {
    out[2 * e] = a0;
    out[2 * e + 1] = a1;
  }
}

// g_e = d(w0 P^h + w1 F_x^h)/du_e on wall elements (zero elsewhere).  Seeds at each wall
// point: U- (4) and the lifted gradient Q (8); the lifting adds the chain through the
// jumps U_wall(U-) - U- at every point p of the face: Lam_b(p) = sum_q sum_d C_Q(q)_(b,d)
// n_d s lift_f[q][p], folded into the state seeds as Lam(p) (dU_wall/dU- - I).
__global__ void __launch_bounds__(RES_WARPS * 32)
    k_qoi_du(DevMesh m, DevTables tb, Phys ph, FrameT<double> fr, const double* __restrict__ u, double w0, double w1,
             double* __restrict__ g) {
  __shared__ double s_C[RES_WARPS][3 * kMaxQf * NSV];
  __shared__ double s_J[RES_WARPS][3 * kMaxQf * 4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * RES_WARPS + warp;
  if (e >= m.ne) return;
  const int Np = tb.Np, nb = tb.nb, nqf = tb.nqf;
  const bool wall = m.tag[3 * e] == 1 || m.tag[3 * e + 1] == 1 || m.tag[3 * e + 2] == 1;
  if (!wall) {
    for (int o = lane; o < nb; o += 32) g[(size_t)e * nb + o] = 0.0;
    return;
  }
  double* C = s_C[warp];
  double* Js = s_J[warp];
  const double* ue = u + (size_t)e * nb;
  double P[4];
  frame_P(fr, m.BinvT + 4 * e, P);
  FrameT<Dual> frd;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    frd.Q[k] = Dual(fr.Q[k]);
    frd.Qd[k] = Dual(fr.Qd[k]);
  }
  frd.hd = Dual(fr.hd);
  for (int idx = lane; idx < 3 * nqf; idx += 32) {
    int f = idx / nqf, q = idx - f * nqf;
    if (m.tag[3 * e + f] != 1) continue;
    double Um[4], vG[2], Ub[4], X, Y;
    interp_val(ue, Np, tb.phi_f + (f * nqf + q) * Np, Um);
    ref_to_X(m, e, tb.xi_f[2 * (f * nqf + q)], tb.xi_f[2 * (f * nqf + q) + 1], X, Y);
    mesh_velocity(fr, ph, X, Y, vG);
    wall_state(Um, vG, Ub);
#pragma unroll
    for (int a = 0; a < 4; ++a) Js[(f * kMaxQf + q) * 4 + a] = Ub[a] - Um[a];
  }
  __syncwarp();
  for (int task = lane; task < 3 * nqf * NSV; task += 32) {
    int f = task / (nqf * NSV);
    int rem = task - f * nqf * NSV;
    int q = rem / NSV, s = rem - q * NSV;
    if (m.tag[3 * e + f] != 1) {
      C[(f * kMaxQf + q) * NSV + s] = 0.0;
      continue;
    }
    double U0[4], dU0[4][2], n0[2];
    interp(ue, Np, tb.phi_f + (f * nqf + q) * Np, tb.dphi_f + 2 * (f * nqf + q) * Np, P, U0, dU0);
    rotate_normal(fr, m.N + 6 * e + 2 * f, n0);
    lift_add(dU0, n0, m.s_own[3 * e + f], tb.lift_f + (f * nqf + q) * nqf, 1, Js + f * kMaxQf * 4, nqf);
    Dual Um[4], dUm[4][2], n[2], vG[2], H[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      Um[a] = Dual(U0[a], s == a ? 1.0 : 0.0);
      dUm[a][0] = Dual(dU0[a][0], s == 4 + 2 * a ? 1.0 : 0.0);
      dUm[a][1] = Dual(dU0[a][1], s == 5 + 2 * a ? 1.0 : 0.0);
    }
    rotate_normal(frd, m.N + 6 * e + 2 * f, n);
    double X, Y;
    ref_to_X(m, e, tb.xi_f[2 * (f * nqf + q)], tb.xi_f[2 * (f * nqf + q) + 1], X, Y);
    mesh_velocity(frd, ph, X, Y, vG);
    face_flux(1, 1, Um, Um, dUm, n, vG, m.c11[3 * e + f], ph, H);
    double wl = tb.w_f[q] * m.L[3 * e + f];
    Dual val = w0 * (H[1] * vG[0] + H[2] * vG[1]) + w1 * H[1];
    C[(f * kMaxQf + q) * NSV + s] = wl * val.d;
  }
  __syncwarp();
  // fold the lifting chain into the state seeds (reads gradient seeds, writes state seeds)
  double add[4] = {0.0, 0.0, 0.0, 0.0};
  int fp = -1;
  if (lane < 3 * nqf) {
    const int f = lane / nqf, p = lane - f * nqf;
    if (m.tag[3 * e + f] == 1) {
      fp = lane;
      double n0[2];
      rotate_normal(fr, m.N + 6 * e + 2 * f, n0);
      const double s = m.s_own[3 * e + f];
      double lam[4] = {0.0, 0.0, 0.0, 0.0};
      for (int q = 0; q < nqf; ++q) {
        const double A = tb.lift_f[(f * nqf + q) * nqf + p] * s;
        const double* Cq = C + (f * kMaxQf + q) * NSV;
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) lam[bb] += A * (Cq[4 + 2 * bb] * n0[0] + Cq[5 + 2 * bb] * n0[1]);
      }
      double Um[4], vG[2], X, Y;
      interp_val(ue, Np, tb.phi_f + (f * nqf + p) * Np, Um);
      ref_to_X(m, e, tb.xi_f[2 * (f * nqf + p)], tb.xi_f[2 * (f * nqf + p) + 1], X, Y);
      mesh_velocity(fr, ph, X, Y, vG);
      Dual vd[2] = {Dual(vG[0]), Dual(vG[1])};
      for (int c = 0; c < 4; ++c) {
        Dual Ud[4], Ub[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) Ud[a] = Dual(Um[a], a == c ? 1.0 : 0.0);
        wall_state(Ud, vd, Ub);
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) add[c] += lam[bb] * (Ub[bb].d - (bb == c ? 1.0 : 0.0));
      }
    }
  }
  __syncwarp();
  if (fp >= 0) {
    const int f = fp / nqf, p = fp - f * nqf;
#pragma unroll
    for (int c = 0; c < 4; ++c) C[(f * kMaxQf + p) * NSV + c] += add[c];
  }
  __syncwarp();
  for (int o = lane; o < nb; o += 32) {
    int b = o / Np, j = o - b * Np;
    double acc = 0.0;
    for (int f = 0; f < 3; ++f) {
      if (m.tag[3 * e + f] != 1) continue;
      for (int q = 0; q < nqf; ++q) {
        const double* dj = tb.dphi_f + 2 * ((f * nqf + q) * Np + j);
        double phij = tb.phi_f[(f * nqf + q) * Np + j];
        double g0 = P[0] * dj[0] + P[1] * dj[1];
        double g1 = P[2] * dj[0] + P[3] * dj[1];
        const double* Cq = C + (f * kMaxQf + q) * NSV;
        acc += Cq[b] * phij + Cq[4 + 2 * b] * g0 + Cq[5 + 2 * b] * g1;
      }
    }
    g[(size_t)e * nb + o] = acc;
  }
}

}  // namespace

static int res_blocks(int ne) { return (ne + RES_WARPS - 1) / RES_WARPS; }

cudaError_t launch_residual(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<double>& fr,
                            const double* u, double* r, cudaStream_t st) {
  ProfScope ps(PP_K_RESIDUAL, st);
  k_residual<double><<<res_blocks(m.ne), RES_WARPS * 32, 0, st>>>(m, tb, ph, fr, u, r, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_residual_dframe(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<Dual>& fr,
                                   const double* u, double* dr, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_residual<Dual><<<res_blocks(m.ne), RES_WARPS * 32, 0, st>>>(m, tb, ph, fr, u, nullptr, dr);
  return cudaGetLastError();
}

cudaError_t launch_jacobian(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<double>& fr,
                            const double* u, double* J, cudaStream_t st) {
  ProfScope ps(PP_K_JACOBIAN, st);
  const size_t bytes = sizeof(double) * JacSmem(tb.nb, tb.Np, tb.nqv).total;
  {
    // largest dynamic shared memory requested so far (contexts of several degrees may share
    // the process; one device per process, see pp_create)
    static std::mutex mu;
    static size_t configured = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (bytes > configured) {
      cudaError_t e = cudaFuncSetAttribute(k_jacobian, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      configured = bytes;
    }
  }
  k_jacobian<<<m.ne, JAC_THREADS, bytes, st>>>(m, tb, ph, fr, u, J);
  return cudaGetLastError();
}

cudaError_t launch_qoi(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<double>& fr,
                       const double* u, double* per_elem, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_qoi<double><<<res_blocks(m.ne), RES_WARPS * 32, 0, st>>>(m, tb, ph, fr, u, per_elem, 0);
  return cudaGetLastError();
}

cudaError_t launch_qoi_dframe(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<Dual>& fr,
                              const double* u, double* per_elem, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_qoi<Dual><<<res_blocks(m.ne), RES_WARPS * 32, 0, st>>>(m, tb, ph, fr, u, per_elem, 1);
  return cudaGetLastError();
}

cudaError_t launch_qoi_du(const DevMesh& m, const DevTables& tb, const Phys& ph, const FrameT<double>& fr,
                          const double* u, double w0, double w1, double* g, cudaStream_t st) {
  ProfScope ps(PP_K_OTHER, st);
  k_qoi_du<<<res_blocks(m.ne), RES_WARPS * 32, 0, st>>>(m, tb, ph, fr, u, w0, w1, g);
  return cudaGetLastError();
}

}  // namespace pp
