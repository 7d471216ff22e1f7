// Pointwise fluxes of the ALE compressible Navier-Stokes discretization
// (Sec. 6: Eqs. ns1-ns5 and the ALE transformation of Eqs. ns-cons-ref,
// transform2-nogcl specialised to the rigid-body map of Eq. defmap, where
// G = Q, g = 1 and the transformed flux is the physical flux minus U (x) v_G
// evaluated with physical gradients and normals).
//
// Numerical fluxes (the paper defers them to its references; readings):
//  - inviscid: Roe's approximate Riemann solver applied to the ALE normal flux
//    F(U).n - (v_G.n) U, Harten entropy fix with delta = 0.1 c;
//  - viscous: the compact discontinuous Galerkin (CDG) scheme of Sec. 6: liftings of
//    the face jumps U_hat - U- into the element (the lifted gradients are formed by the
//    kernels from the reference lifting tables); on an interior face the element with
//    the smaller index supplies the viscous flux F_vis(U_S, grad U_S + r_f) . n with the
//    lifting of that face only; boundary faces add the penalty c11 (U_hat - U-);
//  - wall: no-slip, adiabatic; wall state with the mesh velocity; exact
//    no-penetration inviscid flux;  far field: free-stream state.
//
// Every function is templated on the scalar type so that the same code gives
// values (double) and exact directional derivatives (Dual).
#pragma once

#include "pp_internal.h"

namespace pp {

template <class T>
__device__ __forceinline__ T pressure(const T U[4], double gam) {
  return (gam - 1.0) * (U[3] - 0.5 * (U[1] * U[1] + U[2] * U[2]) / U[0]);
}

// F[a][d]: inviscid flux of variable a in direction d
template <class T>
__device__ __forceinline__ void inviscid_flux(const T U[4], double gam, T F[4][2]) {
  T r = U[0];
  T u = U[1] / r, v = U[2] / r;
  T p = pressure(U, gam);
  F[0][0] = U[1];
  F[1][0] = U[1] * u + p;
  F[2][0] = U[2] * u;
  F[3][0] = (U[3] + p) * u;
  F[0][1] = U[2];
  F[1][1] = U[1] * v;
  F[2][1] = U[2] * v + p;
  F[3][1] = (U[3] + p) * v;
}

// viscous flux from the state and its physical gradient dU[a][d];
// q = -(mu/Pr) grad(E + p/rho - |u|^2/2) = -(mu gamma/Pr) grad(e)
template <class T>
__device__ __forceinline__ void viscous_flux(const T U[4], const T dU[4][2], const Phys& ph, bool adiabatic,
                                             T F[4][2]) {
  T r = U[0];
  T ir = 1.0 / r;
  T u = U[1] * ir, v = U[2] * ir, E = U[3] * ir;
  T du[2], dv[2], dE[2];
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    du[d] = (dU[1][d] - u * dU[0][d]) * ir;
    dv[d] = (dU[2][d] - v * dU[0][d]) * ir;
    dE[d] = (dU[3][d] - E * dU[0][d]) * ir;
  }
  T div = du[0] + dv[1];
  T txx = ph.mu * (2.0 * du[0] - (2.0 / 3.0) * div);
  T tyy = ph.mu * (2.0 * dv[1] - (2.0 / 3.0) * div);
  T txy = ph.mu * (du[1] + dv[0]);
  double kq = adiabatic ? 0.0 : ph.mu * ph.gam / ph.Pr;
  T qx = -kq * (dE[0] - u * du[0] - v * dv[0]);
  T qy = -kq * (dE[1] - u * du[1] - v * dv[1]);
  F[0][0] = T(0.0);
  F[1][0] = txx;
  F[2][0] = txy;
  F[3][0] = u * txx + v * txy - qx;
  F[0][1] = T(0.0);
  F[1][1] = txy;
  F[2][1] = tyy;
  F[3][1] = u * txy + v * tyy - qy;
}

// total ALE volume flux F_inv - U (x) v_G - F_vis
template <class T>
__device__ __forceinline__ void volume_flux(const T U[4], const T dU[4][2], const T vG[2], const Phys& ph,
                                            T F[4][2]) {
  T Fi[4][2], Fv[4][2];
  inviscid_flux(U, ph.gam, Fi);
  viscous_flux(U, dU, ph, false, Fv);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int d = 0; d < 2; ++d) F[a][d] = Fi[a][d] - U[a] * vG[d] - Fv[a][d];
}

template <class T>
__device__ __forceinline__ void normal_flux(const T U[4], const T n[2], const T& vn, double gam, T out[4]) {
  T F[4][2];
  inviscid_flux(U, gam, F);
#pragma unroll
  for (int a = 0; a < 4; ++a) out[a] = F[a][0] * n[0] + F[a][1] * n[1] - vn * U[a];
}

template <class T>
__device__ __forceinline__ T entropy_fix(T l, T delta) {
  T al = absT(l);
  if (val(al) < val(delta)) return (l * l + delta * delta) / (2.0 * delta);
  return al;
}

// Roe flux of the ALE normal flux; |A - vn I| (UR - UL) written with the two
// wave-strength scalars of the acoustic pair.
template <class T>
__device__ __forceinline__ void roe_flux(const T UL[4], const T UR[4], const T n[2], const T& vn, double gam,
                                         T out[4]) {
  T rL = UL[0], rR = UR[0];
  T uL = UL[1] / rL, vL = UL[2] / rL, uR = UR[1] / rR, vR = UR[2] / rR;
  T pL = pressure(UL, gam), pR = pressure(UR, gam);
  T HL = (UL[3] + pL) / rL, HR = (UR[3] + pR) / rR;
  T sL = sqrtT(rL), sR = sqrtT(rR);
  T isum = 1.0 / (sL + sR);
  T ut = (sL * uL + sR * uR) * isum;
  T vt = (sL * vL + sR * vR) * isum;
  T Ht = (sL * HL + sR * HR) * isum;
  T q2 = ut * ut + vt * vt;
  T c2 = (gam - 1.0) * (Ht - 0.5 * q2);
  T c = sqrtT(c2);
  T un = ut * n[0] + vt * n[1];
  T lu = un - vn;
  T delta = 0.1 * c;
  T l1 = entropy_fix(lu + c, delta);
  T l2 = entropy_fix(lu - c, delta);
  T l3 = entropy_fix(lu, delta);
  T D[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) D[a] = UR[a] - UL[a];
  T dp = (gam - 1.0) * (0.5 * q2 * D[0] - ut * D[1] - vt * D[2] + D[3]);
  T dUn = D[1] * n[0] + D[2] * n[1] - un * D[0];
  T s1 = 0.5 * (l1 + l2) - l3;
  T s2 = (l1 - l2) / (2.0 * c);
  T G1 = s1 * dp / c2 + s2 * dUn;
  T G2 = s2 * dp + s1 * dUn;
  T FL[4], FR[4];
  normal_flux(UL, n, vn, gam, FL);
  normal_flux(UR, n, vn, gam, FR);
  T ev1[4] = {T(1.0), ut, vt, Ht};
  T ev2[4] = {T(0.0), n[0], n[1], un};
#pragma unroll
  for (int a = 0; a < 4; ++a) out[a] = 0.5 * (FL[a] + FR[a]) - 0.5 * (l3 * D[a] + G1 * ev1[a] + G2 * ev2[a]);
}

// No-slip wall state: the interior density and internal energy, moving with the wall.
template <class T>
__device__ __forceinline__ void wall_state(const T Um[4], const T vG[2], T Ub[4]) {
  T r = Um[0];
  T eint = Um[3] / r - 0.5 * (Um[1] * Um[1] + Um[2] * Um[2]) / (r * r);
  Ub[0] = r;
  Ub[1] = r * vG[0];
  Ub[2] = r * vG[1];
  Ub[3] = r * (eint + 0.5 * (vG[0] * vG[0] + vG[1] * vG[1]));
}

// Face value U_hat of U at one face point: the neighbour trace (tag 0), the wall state
// (tag 1) or the free stream (tag 2).
template <class T>
__device__ __forceinline__ void face_value(int tag, const T Um[4], const T Up[4], const T vG[2], const Phys& ph,
                                           T Uh[4]) {
  if (tag == 1) {
    wall_state(Um, vG, Uh);
  } else if (tag == 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a) Uh[a] = Up[a];
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a) Uh[a] = T(ph.Uinf[a]);
  }
}

// CDG numerical flux H (outward from the "-" element, per unit length) at one face point:
//   H = H_inv(U-, U+) - F_vis(U_S, Q_S) . n - c11 (U_hat - U-)
// with H_inv Roe's flux (interior, far field) or the exact wall flux, and Q_S the lifted
// gradient of the side S that supplies the viscous flux (side = 1: this element, whose
// viscous state is U- or, on the wall, the wall state; side = 0: the neighbour, U+).
// The wall flux is adiabatic (zero heat flux); c11 is zero on interior faces.
template <class T>
__device__ __forceinline__ void face_flux(int tag, int side, const T Um[4], const T Up[4], const T QS[4][2],
                                          const T n[2], const T vG[2], double c11, const Phys& ph, T H[4]) {
  T vn = vG[0] * n[0] + vG[1] * n[1];
  T Hi[4], Uh[4], Fv[4][2];
  face_value(tag, Um, Up, vG, ph, Uh);
  if (tag == 1) {
    normal_flux(Uh, n, vn, ph.gam, Hi);
    viscous_flux(Uh, QS, ph, true, Fv);
  } else {
    roe_flux(Um, Uh, n, vn, ph.gam, Hi);
    viscous_flux(side ? Um : Up, QS, ph, false, Fv);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) H[a] = Hi[a] - (Fv[a][0] * n[0] + Fv[a][1] * n[1] + c11 * (Uh[a] - Um[a]));
}

}  // namespace pp
