"""ALE discontinuous Galerkin semi-discretization M du/dt = r(u, mu, t) (oracle).

Restates Sec. 6 of the paper (compressible Navier-Stokes, Eqs. ns1-ns5; ALE
map to a fixed reference domain, Eqs. ns-cons-ref, transform1-nogcl,
transform2-nogcl; rigid-body map, Eq. defmap; QoIs, Eq. qoi) together with the
readings the paper leaves open (it defers spatial details to other papers):

* four conservative variables U = (rho, rho u, rho v, rho E) (full NS with
  energy); nondimensional with chord 1, rho_inf = 1, |u_inf| = 1 along +x,
  p_inf = 1/(gamma M^2), constant viscosity mu_visc = 1/Re;
* rigid-body map x = v(t) + Q(t)(X - x0) + x0 (Eq. defmap), x0 = (1/3, 0),
  so G = Q, g = 1, v_G = (0, h') + Q'(X - x0) and the mass matrix is constant;
  physical gradients are grad_x = Q grad_X, physical normals n = Q N;
* inviscid interface flux: Roe's flux of F(U).n - (v_G.n) U with Harten's
  entropy fix (delta = 0.1 c);
* viscous terms: the compact discontinuous Galerkin (CDG) scheme the paper
  names in Sec. 6, written from Peraire and Persson's definition.  With U_hat
  the face value of U (the other side's trace on an interior face, the boundary
  state on a boundary face), the lifting of face f into element K is the
  degree-p field r_f with  int_K r_f . tau = int_f (U_hat - U_K) tau . n_K  for
  all tau; on straight faces r_f = n_f s_f l_f with s_f = |f| / (2 |K|) and l_f
  the scalar lifting of the jump on the reference element.  Volume term:
  F_vis(U, grad U + sum_f r_f) over the faces K lifts.  Face flux: on an
  interior face the element with the smaller index supplies the viscous flux
  F_vis(U_S, grad U_S + r_f^S) . n with the lifting of that face alone, and U_hat
  is the other side's trace (the C12 switch of LDG, so the stencil is the
  element and its face neighbours); on boundary faces the element itself lifts
  the jump to the boundary state and a penalty C11 (U_b - U) with
  C11 = 10 mu_visc |f| / (2 |K|) (10 mu / h) is added;
* wall (no-slip, adiabatic): boundary state U_b = (rho-, rho- v_G,
  rho-(e- + |v_G|^2/2)), exact ALE wall flux F(U_b).n - (v_G.n) U_b, viscous
  flux F_vis(U_b, grad U + r_f) with zero heat flux;
* far field: Roe flux against the free stream (or a prescribed boundary state,
  for manufactured solutions), viscous flux F_vis(U, grad U + r_f) with the
  lifting of the jump to that state;
* force on the airfoil: the momentum components of the wall numerical flux
  (the momentum leaving the fluid through the wall), so that the power is
  P^h = int f . x' dS and the x-force F_x^h = int f . e1 dS (Eq. qoi).

Every function is generic in the scalar type, so complex inputs give
complex-step derivatives (exact to round-off) of r and of the QoIs.

Layout: u[e, a, i] (element, conservative variable, node), flattened in C
order.  Jacobian block [e, 0] = d r_e / d u_e; [e, 1+f] = d r_e / d u_nbr(e,f).
"""
import numpy as np
import scipy.sparse as sp

from . import refelem

KIN_HEAVE_PITCH = 0
KIN_FOURIER6 = 1
KIN_SPLINE8 = 2   # Sec. 6.2, Eq. mirror: knots of h and theta, 4 each
CS_STEP = 1e-30
C11_ETA = 10.0   # boundary penalty C11 = C11_ETA mu_visc / h with h = 2 |K| / |f|


def cabs(x):
    """|x| for real or complex-step arguments (sign taken from the real part)."""
    return np.where(np.real(x) >= 0, x, -x)


def pressure(U, gam):
    return (gam - 1.0) * (U[..., 3] - 0.5 * (U[..., 1] ** 2 + U[..., 2] ** 2) / U[..., 0])


def inviscid_flux(U, gam):
    """F_inv(U), shape [..., 4, 2] (Eqs. ns1-ns3, ns5)."""
    rho = U[..., 0]
    u = U[..., 1] / rho
    v = U[..., 2] / rho
    p = pressure(U, gam)
    Fx = np.stack([U[..., 1], U[..., 1] * u + p, U[..., 2] * u, (U[..., 3] + p) * u], -1)
    Fy = np.stack([U[..., 2], U[..., 1] * v, U[..., 2] * v + p, (U[..., 3] + p) * v], -1)
    return np.stack([Fx, Fy], -1)


def viscous_flux(U, dU, mu, Pr, gam, adiabatic=False):
    """F_vis(U, grad U), shape [..., 4, 2] (stress and heat flux of Sec. 6).

    q = -(mu/Pr) grad(E + p/rho - |u|^2/2) = -(mu/Pr) gamma grad(e).
    """
    rho = U[..., 0]
    u = U[..., 1] / rho
    v = U[..., 2] / rho
    E = U[..., 3] / rho
    drho = dU[..., 0, :]
    du = (dU[..., 1, :] - u[..., None] * drho) / rho[..., None]
    dv = (dU[..., 2, :] - v[..., None] * drho) / rho[..., None]
    dE = (dU[..., 3, :] - E[..., None] * drho) / rho[..., None]
    ux, uy = du[..., 0], du[..., 1]
    vx, vy = dv[..., 0], dv[..., 1]
    div = ux + vy
    txx = mu * (2.0 * ux - 2.0 / 3.0 * div)
    tyy = mu * (2.0 * vy - 2.0 / 3.0 * div)
    txy = mu * (uy + vx)
    de = dE - u[..., None] * du - v[..., None] * dv
    kq = 0.0 if adiabatic else mu / Pr * gam
    qx = -kq * de[..., 0]
    qy = -kq * de[..., 1]
    zero = 0.0 * txx
    Fx = np.stack([zero, txx, txy, u * txx + v * txy - qx], -1)
    Fy = np.stack([zero, txy, tyy, u * txy + v * tyy - qy], -1)
    return np.stack([Fx, Fy], -1)


def normal_flux(U, n, vn, gam):
    """F_inv(U).n - (v_G.n) U."""
    F = inviscid_flux(U, gam)
    return F[..., 0] * n[..., None, 0] + F[..., 1] * n[..., None, 1] - vn[..., None] * U


def roe_flux(UL, UR, n, vn, gam):
    """Roe flux for the ALE normal flux F.n - vn U (eigenvalues shifted by -vn)."""
    rL, rR = UL[..., 0], UR[..., 0]
    uL, vL = UL[..., 1] / rL, UL[..., 2] / rL
    uR, vR = UR[..., 1] / rR, UR[..., 2] / rR
    pL, pR = pressure(UL, gam), pressure(UR, gam)
    HL = (UL[..., 3] + pL) / rL
    HR = (UR[..., 3] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    ut = (sL * uL + sR * uR) / (sL + sR)
    vt = (sL * vL + sR * vR) / (sL + sR)
    Ht = (sL * HL + sR * HR) / (sL + sR)
    q2 = ut * ut + vt * vt
    c2 = (gam - 1.0) * (Ht - 0.5 * q2)
    c = np.sqrt(c2)
    nx, ny = n[..., 0], n[..., 1]
    un = ut * nx + vt * ny
    lu = un - vn
    delta = 0.1 * c

    def fix(l):
        al = cabs(l)
        return np.where(np.real(al) < np.real(delta), (l * l + delta * delta) / (2.0 * delta), al)

    l1 = fix(lu + c)
    l2 = fix(lu - c)
    l3 = fix(lu)
    D = UR - UL
    dp = (gam - 1.0) * (0.5 * q2 * D[..., 0] - ut * D[..., 1] - vt * D[..., 2] + D[..., 3])
    dUn = D[..., 1] * nx + D[..., 2] * ny - un * D[..., 0]
    s1 = 0.5 * (l1 + l2) - l3
    s2 = (l1 - l2) / (2.0 * c)
    G1 = s1 * dp / c2 + s2 * dUn
    G2 = s2 * dp + s1 * dUn
    AD = l3[..., None] * D + G1[..., None] * np.stack([1.0 + 0.0 * ut, ut, vt, Ht], -1) \
        + G2[..., None] * np.stack([0.0 * ut, nx + 0.0 * ut, ny + 0.0 * ut, un], -1)
    return 0.5 * (normal_flux(UL, n, vn, gam) + normal_flux(UR, n, vn, gam)) - 0.5 * AD


def dot_n(F, n):
    return F[..., 0] * n[..., None, 0] + F[..., 1] * n[..., None, 1]


def periodic_cubic_spline(y, T, t):
    """Value and first derivative at time t of the periodic cubic spline (period T) through
    the m equally spaced knots (k T / m, y[k]).  Textbook construction: with d = T / m the
    knot second derivatives M solve the cyclic system
        M[k-1] + 4 M[k] + M[k+1] = 6 (y[k+1] - 2 y[k] + y[k-1]) / d^2,
    and on [k d, (k+1) d] with s = (t - k d) / d
        S = (1-s) y[k] + s y[k+1] + d^2/6 (((1-s)^3 - (1-s)) M[k] + (s^3 - s) M[k+1]).
    y may be complex (complex-step derivatives with respect to the knot values)."""
    y = np.asarray(y)
    m = len(y)
    d = T / m
    A = 4.0 * np.eye(m) + np.roll(np.eye(m), 1, axis=1) + np.roll(np.eye(m), -1, axis=1)
    rhs = 6.0 * (np.roll(y, -1) - 2.0 * y + np.roll(y, 1)) / d ** 2
    M = np.linalg.solve(A, rhs)
    tau = float(np.real(t)) % T
    k = min(int(np.floor(tau / d)), m - 1)
    s = (tau - k * d) / d
    k1 = (k + 1) % m
    val = (1 - s) * y[k] + s * y[k1] + d ** 2 / 6.0 * (((1 - s) ** 3 - (1 - s)) * M[k] + (s ** 3 - s) * M[k1])
    der = (y[k1] - y[k]) / d + d / 6.0 * (-(3 * (1 - s) ** 2 - 1) * M[k] + (3 * s ** 2 - 1) * M[k1])
    return val, der


def mirrored_knots(half):
    """Knot values over the whole period from the four free knots of the first half: the
    mirror condition of Eq. mirror, f(t + T/2) = -f(t), fixes the second half (and the knot at
    T/2, -f(0)), so the 8 equally spaced knots carry (f0, f1, f2, f3, -f0, -f1, -f2, -f3)."""
    half = np.asarray(half)
    return np.concatenate([half, -half])


class DG:
    """The semi-discretization on a given mesh; see module docstring."""

    NV = 4   # conservative variables (rho, rho u, rho v, rho E)

    def __init__(self, mesh, p, gamma=1.4, Pr=0.72, Mach=0.2, Re=1000.0, kin=KIN_HEAVE_PITCH, T=5.0,
                 farfield=None):
        """farfield: optional boundary state U_b(X) [..., 2] -> [..., 4] of the far-field faces
        (default: the uniform free stream); used by manufactured-solution tests."""
        self.mesh = mesh
        self.farfield = farfield
        self.p = p
        self.gam, self.Pr, self.Mach, self.Re = gamma, Pr, Mach, Re
        self.mu_visc = 1.0 / Re
        self.kin = kin
        self.T = T
        self.omega = 2.0 * np.pi / T
        self.x0 = np.array([1.0 / 3.0, 0.0])
        self.nv = self.NV
        self.Uinf = self.free_stream()

        self.basis = refelem.Basis(p)
        Np = self.Np = self.basis.np
        self.nb = self.nv * Np
        tris = mesh.tris.astype(np.int64)
        V = mesh.verts
        Ne = self.Ne = tris.shape[0]
        self.Nu = Ne * self.nv * Np

        # connectivity: local face f = edge (v_f, v_{f+1})
        edge = {}
        self.nbr = -np.ones((Ne, 3), dtype=np.int64)
        self.nbr_face = -np.ones((Ne, 3), dtype=np.int64)
        for e in range(Ne):
            for f in range(3):
                a, b = tris[e, f], tris[e, (f + 1) % 3]
                key = (min(a, b), max(a, b))
                if key in edge:
                    e2, f2 = edge.pop(key)
                    self.nbr[e, f], self.nbr_face[e, f] = e2, f2
                    self.nbr[e2, f2], self.nbr_face[e2, f2] = e, f
                else:
                    edge[key] = (e, f)
        self.tag = mesh.ftag.astype(np.int64)
        interior = self.nbr >= 0
        if np.any(interior != (self.tag == 0)):
            raise ValueError("face tags inconsistent with connectivity")

        # affine element maps X = X0 + B xi
        X0 = V[tris[:, 0]]
        B = np.stack([V[tris[:, 1]] - X0, V[tris[:, 2]] - X0], axis=2)  # B[e, :, k] = edge k
        self.X0, self.B = X0, B
        self.detB = B[:, 0, 0] * B[:, 1, 1] - B[:, 0, 1] * B[:, 1, 0]
        if np.any(self.detB <= 0):
            raise ValueError("mesh has inverted elements")
        self.area = 0.5 * self.detB
        self.BinvT = np.transpose(np.linalg.inv(B), (0, 2, 1))

        # faces: outward unit normals and lengths in the reference configuration
        self.L = np.zeros((Ne, 3))
        self.N = np.zeros((Ne, 3, 2))
        for f in range(3):
            t = V[tris[:, (f + 1) % 3]] - V[tris[:, f]]
            Lf = np.hypot(t[:, 0], t[:, 1])
            self.L[:, f] = Lf
            self.N[:, f, 0] = t[:, 1] / Lf
            self.N[:, f, 1] = -t[:, 0] / Lf

        nq = p + 2
        self.xi_v, self.w_v = refelem.triangle_rule(nq)
        self.phi_v = self.basis.phi(self.xi_v)            # [nqv, Np]
        self.dphi_v = self.basis.dphi(self.xi_v)          # [nqv, Np, 2]
        self.Xq_v = X0[:, None, :] + np.einsum("edk,qk->eqd", B, self.xi_v)
        self.s_f, self.w_f = refelem.gauss_legendre_01(nq)
        self.phi_f = np.stack([self.basis.phi(refelem.face_points(f, self.s_f)) for f in range(3)])
        self.dphi_f = np.stack([self.basis.dphi(refelem.face_points(f, self.s_f)) for f in range(3)])
        self.Xq_f = np.stack([X0[:, None, :] + np.einsum("edk,qk->eqd", B, refelem.face_points(f, self.s_f))
                              for f in range(3)], axis=1)  # [Ne, 3, nqf, 2]

        # neighbour basis at matched face points (parameter 1 - s on its face)
        nqf = len(self.s_f)
        self.phiN = np.zeros((Ne, 3, nqf, Np))
        self.dphiN = np.zeros((Ne, 3, nqf, Np, 2))
        for e in range(Ne):
            for f in range(3):
                e2, g = self.nbr[e, f], self.nbr_face[e, f]
                if e2 >= 0:
                    xi2 = refelem.face_points(g, 1.0 - self.s_f)
                    self.phiN[e, f] = self.basis.phi(xi2)
                    self.dphiN[e, f] = self.basis.dphi(xi2)
                    Xm = X0[e2] + xi2 @ B[e2].T
                    assert np.allclose(Xm, self.Xq_f[e, f], atol=1e-12)
                else:  # boundary: placeholder values (the interior branch is masked out)
                    self.phiN[e, f] = self.phi_f[f]
                    self.dphiN[e, f] = self.dphi_f[f]
        self.nbr_safe = np.where(self.nbr >= 0, self.nbr, np.arange(Ne)[:, None])
        self.BinvT_nbr = self.BinvT[self.nbr_safe]                      # [Ne, 3, 2, 2]

        # mass matrix: M_e = detB * int phi_i phi_j over the reference triangle
        self.Mref = np.einsum("q,qi,qj->ij", self.w_v, self.phi_v, self.phi_v)

        # CDG liftings.  The scalar lifting of a jump j given at the points of face f is
        # l = sum_j phi_j (Mref^-1 c)_j with c_i = sum_q w_q phi_i(face point q) j_q, so that
        # int_K r_f . tau = int_f j tau . n holds for r_f = n_f (|f| / detB) l (affine K).
        # lift_v[f]: l at the volume points per unit jump at face point q; lift_f[f]: l at
        # the points of face f itself.
        Minv = np.linalg.inv(self.Mref)
        self.lift_v = np.stack([self.phi_v @ Minv @ (self.phi_f[f].T * self.w_f[None, :]) for f in range(3)])
        self.lift_f = np.stack([self.phi_f[f] @ Minv @ (self.phi_f[f].T * self.w_f[None, :]) for f in range(3)])
        # the element that supplies the viscous flux of a face and lifts its jump: the
        # element itself on boundary faces, the one with the smaller index on interior faces
        self.flux_side = (self.nbr < 0) | (self.nbr > np.arange(Ne)[:, None])
        self.s_own = self.L / self.detB[:, None]
        self.s_nbr = self.L / self.detB[self.nbr_safe]
        # the neighbour's lifting of its own face, in this element's point order (the face
        # points are matched in reverse)
        self.lift_fN = self.lift_f[np.where(self.nbr >= 0, self.nbr_face, 0)][:, :, ::-1, ::-1].copy()
        self.c11 = np.where(self.nbr < 0, C11_ETA * self.mu_visc * self.L / self.detB[:, None], 0.0)

    # ------------------------------------------------------------------ physics (Sec. 6)
    def free_stream(self):
        """Free-stream state: density 1, velocity (1, 0), Mach number Mach."""
        pinf = 1.0 / (self.gam * self.Mach * self.Mach)
        return np.array([1.0, 1.0, 0.0, pinf / (self.gam - 1.0) + 0.5])

    def flux_inv(self, U):
        return inviscid_flux(U, self.gam)

    def flux_vis(self, U, dU, adiabatic=False):
        return viscous_flux(U, dU, self.mu_visc, self.Pr, self.gam, adiabatic)

    def flux_normal(self, U, n, vn):
        return normal_flux(U, n, vn, self.gam)

    def flux_roe(self, UL, UR, n, vn):
        return roe_flux(UL, UR, n, vn, self.gam)

    def wall_state(self, Um, vG):
        """No-slip wall state: interior density and internal energy, wall velocity."""
        rho = Um[..., 0]
        e_int = Um[..., 3] / rho - 0.5 * (Um[..., 1] ** 2 + Um[..., 2] ** 2) / rho**2
        vGb = vG + 0.0 * rho[..., None]
        return np.stack([rho, rho * vGb[..., 0], rho * vGb[..., 1],
                         rho * (e_int + 0.5 * (vGb[..., 0] ** 2 + vGb[..., 1] ** 2))], -1)

    # ------------------------------------------------------------------ kinematics
    def motion(self, mu, t):
        """(theta, theta', h') of the prescribed motion at time t (Eq. nominal form)."""
        w = self.omega
        if self.kin == KIN_HEAVE_PITCH:
            h0, th0, ph = mu[0], mu[1], mu[2]
            hdot = h0 * w * np.cos(w * t)
            th = th0 * np.sin(w * t + ph)
            thdot = th0 * w * np.cos(w * t + ph)
        elif self.kin == KIN_SPLINE8:
            # mu = (h knots at t = 0, T/8, T/4, 3T/8; theta knots at the same times)
            _, hdot = periodic_cubic_spline(mirrored_knots(mu[0:4]), self.T, t)
            th, thdot = periodic_cubic_spline(mirrored_knots(mu[4:8]), self.T, t)
        else:
            a1, b1, a2, al1, be1, al2 = mu[0], mu[1], mu[2], mu[3], mu[4], mu[5]
            hdot = a1 * w * np.cos(w * t) - b1 * w * np.sin(w * t) + a2 * 2 * w * np.cos(2 * w * t)
            th = al1 * np.sin(w * t) + be1 * np.cos(w * t) + al2 * np.sin(2 * w * t)
            thdot = al1 * w * np.cos(w * t) - be1 * w * np.sin(w * t) + al2 * 2 * w * np.cos(2 * w * t)
        return th, thdot, hdot

    def frame(self, mu, t):
        if t is None:  # frozen pose of t = 0 with the mesh at rest (steady-state problem)
            th, _, _ = self.motion(mu, 0.0)
            thd, hd = 0.0 * th, 0.0 * th
        else:
            th, thd, hd = self.motion(mu, t)
        c, s = np.cos(th), np.sin(th)
        Q = np.array([[c, s], [-s, c]])
        Qd = thd * np.array([[-s, c], [-c, -s]])
        return Q, Qd, hd

    def mesh_velocity(self, X, Qd, hd):
        """v_G at reference points X [..., 2]: (0, h') + Q'(X - x0)."""
        d = X - self.x0
        vx = Qd[0, 0] * d[..., 0] + Qd[0, 1] * d[..., 1]
        vy = Qd[1, 0] * d[..., 0] + Qd[1, 1] * d[..., 1] + hd
        return np.stack([vx, vy], -1)

    # ------------------------------------------------------------------ residual
    def _traces(self, uS, uN, f, Q, Qd, hd, P):
        """Both traces of U and their physical gradients at the points of local face f, the
        physical outward normal, the mesh velocity and the face value U_hat of U (the
        neighbour trace, the wall state or the far-field state by tag)."""
        Um = np.einsum("...eai,qi->...eqa", uS, self.phi_f[f])
        gm = np.einsum("edk,qik->eqid", P, self.dphi_f[f])
        dUm = np.einsum("...eai,eqid->...eqad", uS, gm)
        Up = np.einsum("...eai,eqi->...eqa", uN[..., f, :, :], self.phiN[:, f])
        Pn = np.einsum("dk,ekl->edl", Q, self.BinvT_nbr[:, f])
        gp = np.einsum("edk,eqik->eqid", Pn, self.dphiN[:, f])
        dUp = np.einsum("...eai,eqid->...eqad", uN[..., f, :, :], gp)
        n = np.einsum("dk,ek->ed", Q, self.N[:, f])[:, None, :]        # [Ne, 1, 2]
        vG = self.mesh_velocity(self.Xq_f[:, f], Qd, hd)                 # [Ne, nqf, 2]
        vn = vG[..., 0] * n[..., 0] + vG[..., 1] * n[..., 1]
        Ub = self.wall_state(Um, vG)
        if self.farfield is None:
            Uf = np.broadcast_to(self.Uinf, Um.shape) + 0.0 * Um
        else:
            Uf = np.broadcast_to(self.farfield(self.Xq_f[:, f]), Um.shape) + 0.0 * Um
        tag = self.tag[:, f][:, None, None]
        Uhat = np.where(tag == 0, Up, np.where(tag == 1, Ub, Uf))
        return Um, dUm, Up, dUp, n, vG, vn, Ub, Uf, Uhat

    def _face_flux(self, uS, uN, f, Q, Qd, hd, P):
        """Numerical flux H (outward, per unit length) at the quadrature points of local face f."""
        Um, dUm, Up, dUp, n, vG, vn, Ub, Uf, Uhat = self._traces(uS, uN, f, Q, Qd, hd, P)
        nf = n[:, 0, :]                                                  # [Ne, 2]
        # lifted gradient of the side that supplies the viscous flux (this face's lifting only)
        l_own = np.einsum("qp,...epa->...eqa", self.lift_f[f], Uhat - Um) * self.s_own[:, f][:, None, None]
        Q_own = dUm + l_own[..., None] * nf[:, None, None, :]
        l_nbr = np.einsum("eqp,...epa->...eqa", self.lift_fN[:, f], Up - Um) * self.s_nbr[:, f][:, None, None]
        Q_nbr = dUp + l_nbr[..., None] * nf[:, None, None, :]
        side = self.flux_side[:, f][:, None, None]
        tag = self.tag[:, f][:, None, None]
        US = np.where(side, np.where(tag == 1, Ub, Um), Up)
        QS = np.where(side[..., None], Q_own, Q_nbr)
        FvS_int = self.flux_vis(US, QS)
        FvS_wall = self.flux_vis(US, QS, adiabatic=True)
        FvS = np.where(tag[..., None] == 1, FvS_wall, FvS_int)
        pen = self.c11[:, f][:, None, None] * (Uhat - Um)
        inv_int = self.flux_roe(Um, Up, n, vn)
        inv_far = self.flux_roe(Um, Uf, n, vn)
        inv_wall = self.flux_normal(Ub, n, vn)
        Hinv = np.where(tag == 0, inv_int, np.where(tag == 1, inv_wall, inv_far))
        H = Hinv - (dot_n(FvS, n) + pen)
        return H, vG

    def _volume_lifting(self, uS, uN, Q, Qd, hd, P):
        """sum over the faces this element lifts of r_f at the volume points [.., Ne, nqv, 4, 2]."""
        out = 0.0
        for f in range(3):
            Um, _, _, _, n, _, _, _, _, Uhat = self._traces(uS, uN, f, Q, Qd, hd, P)
            w = (self.s_own[:, f] * self.flux_side[:, f])[:, None, None]
            l = np.einsum("qp,...epa->...eqa", self.lift_v[f], Uhat - Um) * w
            out = out + l[..., None] * n[:, 0, None, None, :]
        return out

    def residual_local(self, uS, uN, mu, t):
        """r_e from the element's own state uS [..., Ne, 4, Np] and face-neighbour states
        uN [..., Ne, 3, 4, Np] (boundary slots ignored).  t = None: the airfoil frozen at
        its t = 0 pose with the mesh at rest (the steady-state problem)."""
        Q, Qd, hd = self.frame(mu, t)
        P = np.einsum("dk,ekl->edl", Q, self.BinvT)                      # grad_x = P grad_xi
        # volume term: int grad_x phi_i . (F_inv - U v_G - F_vis) dX
        U = np.einsum("...eai,qi->...eqa", uS, self.phi_v)
        gphys = np.einsum("edk,qik->eqid", P, self.dphi_v)
        dU = np.einsum("...eai,eqid->...eqad", uS, gphys) + self._volume_lifting(uS, uN, Q, Qd, hd, P)
        vG = self.mesh_velocity(self.Xq_v, Qd, hd)
        Ftot = self.flux_inv(U) - U[..., None] * vG[..., None, :] - self.flux_vis(U, dU)
        wq = self.w_v[None, :] * self.detB[:, None]
        r = np.einsum("eq,eqid,...eqad->...eai", wq, gphys, Ftot)
        # face terms: - int_f phi_i H dS
        for f in range(3):
            H, _ = self._face_flux(uS, uN, f, Q, Qd, hd, P)
            r = r - np.einsum("q,e,qi,...eqa->...eai", self.w_f, self.L[:, f], self.phi_f[f], H)
        return r

    def subset(self, elems):
        """A view restricted to the rows of the given elements (for sampled checks on
        large meshes): residual_local on it takes uS = u[elems], uN = u[nbr_safe[elems]]."""
        import copy
        sub = copy.copy(self)
        elems = np.asarray(elems)
        for name in ("X0", "B", "detB", "area", "BinvT", "L", "N", "Xq_v", "Xq_f", "phiN", "dphiN", "flux_side",
                     "s_own", "s_nbr", "lift_fN", "c11", "tag", "nbr", "nbr_face", "nbr_safe", "BinvT_nbr"):
            setattr(sub, name, getattr(self, name)[elems])
        sub.Ne = len(elems)
        sub.Nu = sub.Ne * self.nv * self.Np
        return sub

    def jac_blocks_subset(self, u, mu, t, elems):
        """Block rows of the element Jacobian for the given elements only."""
        sub = self.subset(elems)
        nb, Np = self.nb, self.Np
        nv = self.nv
        us = np.asarray(u, dtype=np.float64).reshape(self.Ne, nv, Np)
        uS = us[np.asarray(elems)]
        uN = us[sub.nbr_safe]
        E = np.eye(nb).reshape(nb, 1, nv, Np)
        n = sub.Ne
        out = np.zeros((n, 4, nb, nb))
        rS = sub.residual_local(uS[None] + 1j * CS_STEP * E, uN[None] + 0j, mu, t)
        out[:, 0] = np.transpose(np.imag(rS).reshape(nb, n, nb), (1, 2, 0)) / CS_STEP
        for f in range(3):
            dN = np.zeros((nb, 1, 3, nv, Np))
            dN[:, :, f] = E
            rN = sub.residual_local(uS[None] + 0j, uN[None] + 1j * CS_STEP * dN, mu, t)
            blk = np.transpose(np.imag(rN).reshape(nb, n, nb), (1, 2, 0)) / CS_STEP
            blk[sub.nbr[:, f] < 0] = 0.0
            out[:, 1 + f] = blk
        return out

    def residual_subset(self, u, mu, t, elems):
        sub = self.subset(elems)
        us = np.asarray(u, dtype=np.float64).reshape(self.Ne, self.nv, self.Np)
        return sub.residual_local(us[np.asarray(elems)], us[sub.nbr_safe], mu, t)

    def gather(self, u):
        u = u.reshape(u.shape[:-1] + (self.Ne, self.nv, self.Np)) if u.shape[-1] == self.Nu else u
        return u[..., self.nbr_safe, :, :]

    def residual(self, u, mu, t):
        us = np.asarray(u).reshape(np.shape(u)[:-1] + (self.Ne, self.nv, self.Np))
        return self.residual_local(us, us[..., self.nbr_safe, :, :], mu, t).reshape(np.shape(u))

    # ------------------------------------------------------------------ QoI (Eq. qoi)
    def qoi_rate(self, u, mu, t):
        """Instantaneous power P^h and x-force F_x^h the fluid exerts on the airfoil."""
        us = np.asarray(u).reshape(np.shape(u)[:-1] + (self.Ne, self.nv, self.Np))
        uN = us[..., self.nbr_safe, :, :]
        Q, Qd, hd = self.frame(mu, t)
        P = np.einsum("dk,ekl->edl", Q, self.BinvT)
        Pw = 0.0
        Fx = 0.0
        for f in range(3):
            H, vG = self._face_flux(us, uN, f, Q, Qd, hd, P)
            wall = (self.tag[:, f] == 1).astype(np.float64)
            wl = self.w_f[None, :] * (self.L[:, f] * wall)[:, None]
            force = H[..., 1:3]
            Pw = Pw + np.einsum("eq,...eq->...", wl, force[..., 0] * vG[..., 0] + force[..., 1] * vG[..., 1])
            Fx = Fx + np.einsum("eq,...eq->...", wl, force[..., 0])
        return Pw, Fx

    # ------------------------------------------------------------------ exact derivatives
    def jac_blocks(self, u, mu, t):
        """Element block Jacobian by complex step: [Ne, 4 slots, nb, nb] (rows (a,i), cols (b,j))."""
        nb, Ne, Np = self.nb, self.Ne, self.Np
        nv = self.nv
        us = np.asarray(u, dtype=np.float64).reshape(Ne, nv, Np)
        uN = us[self.nbr_safe]
        E = np.eye(nb).reshape(nb, 1, nv, Np)
        out = np.zeros((Ne, 4, nb, nb))
        rS = self.residual_local(us[None] + 1j * CS_STEP * E, uN[None] + 0j, mu, t)
        out[:, 0] = np.transpose(np.imag(rS).reshape(nb, Ne, nb), (1, 2, 0)) / CS_STEP
        for f in range(3):
            dN = np.zeros((nb, 1, 3, nv, Np))
            dN[:, :, f] = E
            rN = self.residual_local(us[None] + 0j, uN[None] + 1j * CS_STEP * dN, mu, t)
            blk = np.transpose(np.imag(rN).reshape(nb, Ne, nb), (1, 2, 0)) / CS_STEP
            blk[self.nbr[:, f] < 0] = 0.0
            out[:, 1 + f] = blk
        return out

    def blocks_to_sparse(self, blocks):
        Ne, nb = self.Ne, self.nb
        rows, cols, vals = [], [], []
        ii, jj = np.meshgrid(np.arange(nb), np.arange(nb), indexing="ij")
        for e in range(Ne):
            for slot in range(4):
                c = e if slot == 0 else self.nbr[e, slot - 1]
                if c < 0:
                    continue
                rows.append((e * nb + ii).ravel())
                cols.append((c * nb + jj).ravel())
                vals.append(blocks[e, slot].ravel())
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.Nu, self.Nu))

    def jacobian(self, u, mu, t):
        return self.blocks_to_sparse(self.jac_blocks(u, mu, t))

    def mass(self):
        blocks = [sp.coo_matrix(self.detB[e] * self.Mref) for e in range(self.Ne) for _ in range(self.nv)]
        return sp.block_diag(blocks, format="csr")

    def dr_dmu(self, u, mu, t):
        """d r / d mu [Nu, n_mu] by complex step in the motion parameters."""
        mu = np.asarray(mu, dtype=np.float64)
        cols = []
        for j in range(len(mu)):
            m = mu + 0j
            m[j] += 1j * CS_STEP
            cols.append(np.imag(self.residual(np.asarray(u) + 0j, m, t)) / CS_STEP)
        return np.stack(cols, 1)

    def dqoi_du(self, u, mu, t):
        """d(P^h, F_x^h)/du [2, Nu]: the QoI is face-local to wall elements, so one
        complex perturbation of local dof (a, i) in every element at once is exact."""
        nb, Ne, Np = self.nb, self.Ne, self.Np
        us = np.asarray(u, dtype=np.float64).reshape(Ne, self.nv, Np)
        Q, Qd, hd = self.frame(mu, t)
        P = np.einsum("dk,ekl->edl", Q, self.BinvT)
        E = np.eye(nb).reshape(nb, 1, self.nv, Np)
        uS = us[None] + 1j * CS_STEP * E
        uN = us[self.nbr_safe][None] + 0j
        out = np.zeros((2, Ne, nb))
        for f in range(3):
            H, vG = self._face_flux(uS, uN, f, Q, Qd, hd, P)
            wall = (self.tag[:, f] == 1).astype(np.float64)
            wl = self.w_f[None, :] * (self.L[:, f] * wall)[:, None]
            force = H[..., 1:3]
            pw = np.einsum("eq,deq->de", wl, force[..., 0] * vG[..., 0] + force[..., 1] * vG[..., 1])
            fx = np.einsum("eq,deq->de", wl, force[..., 0])
            out[0] += np.imag(pw).T / CS_STEP
            out[1] += np.imag(fx).T / CS_STEP
        return out.reshape(2, self.Nu)

    def dqoi_dmu(self, u, mu, t):
        mu = np.asarray(mu, dtype=np.float64)
        out = np.zeros((2, len(mu)))
        for j in range(len(mu)):
            m = mu + 0j
            m[j] += 1j * CS_STEP
            pw, fx = self.qoi_rate(np.asarray(u) + 0j, m, t)
            out[0, j] = np.imag(pw) / CS_STEP
            out[1, j] = np.imag(fx) / CS_STEP
        return out
