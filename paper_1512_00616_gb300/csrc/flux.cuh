// Pointwise fluxes of the ALE compressible Navier-Stokes discretization
// (Sec. 6: Eqs. ns1-ns5 and the ALE transformation of Eqs. ns-cons-ref,
// transform2-nogcl specialised to the rigid-body map of Eq. defmap, where
// G = Q, g = 1 and the transformed flux is the physical flux minus U (x) v_G
// evaluated with physical gradients and normals).
//
// Numerical fluxes (the paper defers them to its references; readings):
//  - inviscid: Roe's approximate Riemann solver applied to the ALE normal flux
//    F(U).n - (v_G.n) U, Harten entropy fix with delta = 0.1 c;
//  - viscous: interior penalty {F_vis}.n + sigma (U+ - U-);
//  - wall: no-slip, adiabatic; ghost state with the mesh velocity; exact
//    no-penetration inviscid flux;  far field: free-stream ghost state.
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

// Numerical flux H (outward from the "-" element, per unit length) at one face point.
// tag 0 interior (Up, dUp used), 1 wall, 2 far field.
template <class T>
__device__ __forceinline__ void face_flux(int tag, const T Um[4], const T dUm[4][2], const T Up[4],
                                          const T dUp[4][2], const T n[2], const T vG[2], double sigma,
                                          const Phys& ph, T H[4]) {
  T vn = vG[0] * n[0] + vG[1] * n[1];
  T Fvm[4][2];
  if (tag == 1) {
    // no-slip adiabatic wall: ghost shares density and internal energy, moves with the wall
    T r = Um[0];
    T eint = Um[3] / r - 0.5 * (Um[1] * Um[1] + Um[2] * Um[2]) / (r * r);
    T Ub[4] = {r, r * vG[0], r * vG[1], r * (eint + 0.5 * (vG[0] * vG[0] + vG[1] * vG[1]))};
    T Fn[4];
    normal_flux(Ub, n, vn, ph.gam, Fn);
    viscous_flux(Ub, dUm, ph, true, Fvm);
#pragma unroll
    for (int a = 0; a < 4; ++a)
      H[a] = Fn[a] - (Fvm[a][0] * n[0] + Fvm[a][1] * n[1] + sigma * (Ub[a] - Um[a]));
    return;
  }
  viscous_flux(Um, dUm, ph, false, Fvm);
  if (tag == 0) {
    T Fvp[4][2];
    viscous_flux(Up, dUp, ph, false, Fvp);
    T R[4];
    roe_flux(Um, Up, n, vn, ph.gam, R);
#pragma unroll
    for (int a = 0; a < 4; ++a)
      H[a] = R[a] - (0.5 * ((Fvm[a][0] + Fvp[a][0]) * n[0] + (Fvm[a][1] + Fvp[a][1]) * n[1]) +
                     sigma * (Up[a] - Um[a]));
  } else {
    T Ui[4] = {T(ph.Uinf[0]), T(ph.Uinf[1]), T(ph.Uinf[2]), T(ph.Uinf[3])};
    T R[4];
    roe_flux(Um, Ui, n, vn, ph.gam, R);
#pragma unroll
    for (int a = 0; a < 4; ++a)
      H[a] = R[a] - (Fvm[a][0] * n[0] + Fvm[a][1] * n[1] + sigma * (Ui[a] - Um[a]));
  }
}

}  // namespace pp
