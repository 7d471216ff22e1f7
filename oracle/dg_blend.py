"""ALE DG residual for the rigid-plus-blended mesh motion with a discrete geometric
conservation law (oracle; test infrastructure only).

The map x(X, t) of oracle/blend.py is interpolated nodally in each element's degree-p
space (x_h, v_h), so that the cofactor matrix C = g_h G_h^{-1} of G_h = grad_X x_h is a
polynomial and C N is continuous across faces (the interpolant is conforming).  The
unknown is U_X = gbar U on the reference domain, with

    M dU_X/dt = r(U_X) = int grad_X phi . C (F(U, grad_x U) - U (x) v_h) dX
                         - sum_faces int phi |C^T N| H(U-, U+, n, v_h . n) dS_X,

U = U_X / gbar, grad_x U = G_h^{-T} grad_X U, n = C^T N / |C^T N| (Nanson), and the
numerical flux H of the rigid oracle.  gbar is the discrete GCL field,

    M dgbar/dt = -D[C v_h],   D[f] = int grad_X phi . f dX - sum_faces int phi f . N dS_X,

integrated by the same DIRK as the flow.  Because D[C] = 0 exactly (Piola identity of
the polynomial map, integrated exactly), r(gbar U_inf) = -U_inf D[C v_h] for any gbar,
so a uniform flow stays uniform through every DIRK stage.  With b = 1 everywhere the
residual is the rigid one (G = Q, g = 1, gbar = 1).

Readings kept from the rigid oracle: fluxes, boundary states, the CDG viscous terms
(liftings and the boundary penalty on the reference element and reference face length,
where the elements are affine; the lifted reference gradient is mapped by G^-T of its
side), mass matrix of the reference element.
"""
import numpy as np

from . import blend
from .dg import (CS_STEP, DG, KIN_HEAVE_PITCH, KIN_SPLINE8, inviscid_flux, mirrored_knots, normal_flux,
                 periodic_cubic_spline, roe_flux, viscous_flux)


class BlendedDG(DG):
    def __init__(self, mesh, p, r1=2.0, r2=8.0, **kw):
        super().__init__(mesh, p, **kw)
        self.r1, self.r2 = r1, r2
        xi_n = self.basis.nodes                                              # [Np, 2]
        self.Xn = self.X0[:, None, :] + np.einsum("edk,jk->ejd", self.B, xi_n)   # [Ne, Np, 2]
        self.Minv_ref = np.linalg.inv(self.Mref)

    # ------------------------------------------------------------------ kinematics
    def heave(self, mu, t):
        w = self.omega
        if self.kin == KIN_HEAVE_PITCH:
            return mu[0] * np.sin(w * t)
        if self.kin == KIN_SPLINE8:
            return periodic_cubic_spline(mirrored_knots(mu[0:4]), self.T, t)[0]
        return mu[0] * np.sin(w * t) + mu[1] * np.cos(w * t) + mu[2] * np.sin(2 * w * t)

    def nodal_map(self, mu, t):
        """x and v_X of the blended map at the element nodes, [Ne, Np, 2] each.  t = None:
        the t = 0 pose with the mesh at rest (the steady-state problem)."""
        if t is None:
            th, _, _ = self.motion(mu, 0.0)
            x, _, _, _, v = blend.blended_map(self.Xn, self.heave(mu, 0.0), th, 0.0 * th, 0.0 * th,
                                              self.r1, self.r2)
            return x, 0.0 * v
        th, thd, hd = self.motion(mu, t)
        x, _, _, _, v = blend.blended_map(self.Xn, self.heave(mu, t), th, hd, thd, self.r1, self.r2)
        return x, v

    def _geom(self, xn, vn, phi, dphi):
        """G_h, cofactor C = g G^{-1}, G^{-T} and v_h at points with basis values phi
        [nq, Np] and reference gradients dphi [nq, Np, 2] (per element)."""
        gradX = np.einsum("ekl,qjl->eqjk", self.BinvT, dphi)                # grad_X phi_j [Ne, nq, Np, 2]
        return self._geom_pts(xn, vn, np.broadcast_to(phi, (self.Ne,) + phi.shape), gradX)

    @staticmethod
    def _geom_pts(xn, vn, phi, gradX):
        """As _geom with per-element basis values phi [Ne, nq, Np] and gradients gradX."""
        G = np.einsum("eji,eqjk->eqik", xn, gradX)                          # dx_i / dX_k
        g = G[..., 0, 0] * G[..., 1, 1] - G[..., 0, 1] * G[..., 1, 0]
        C = np.stack([np.stack([G[..., 1, 1], -G[..., 0, 1]], -1),
                      np.stack([-G[..., 1, 0], G[..., 0, 0]], -1)], -2)     # g G^{-1}
        GinvT = np.swapaxes(C, -1, -2) / g[..., None, None]
        v = np.einsum("eqj,eji->eqi", phi, vn)
        return G, g, C, GinvT, v, gradX

    # ------------------------------------------------------------------ GCL
    def gcl_rhs(self, mu, t):
        """-D[C v_h] per element node [Ne, Np] (right-hand side of M dgbar/dt)."""
        xn, vn = self.nodal_map(mu, t)
        _, _, C, _, v, gradX = self._geom(xn, vn, self.phi_v, self.dphi_v)
        Cv = np.einsum("eqJi,eqi->eqJ", C, v)
        wq = self.w_v[None, :] * self.detB[:, None]
        D = np.einsum("eq,eqjJ,eqJ->ej", wq, gradX, Cv)
        for f in range(3):
            _, _, Cf, _, vf, _ = self._geom(xn, vn, self.phi_f[f], self.dphi_f[f])
            CvN = np.einsum("eqJi,eqi,eJ->eq", Cf, vf, self.N[:, f])
            D = D - np.einsum("q,e,qj,eq->ej", self.w_f, self.L[:, f], self.phi_f[f], CvN)
        return -D

    def gcl_rate(self, mu, t):
        """dgbar/dt = M^{-1}(-D[C v_h]) per element [Ne, Np]."""
        return np.einsum("ij,ej->ei", self.Minv_ref, self.gcl_rhs(mu, t)) / self.detB[:, None]

    def geometric_g(self, mu, t):
        """g_h of the interpolated map at the element nodes [Ne, Np] (the initial gbar);
        t = None: the frozen t = 0 pose."""
        xn, vn = self.nodal_map(mu, t)
        return self._geom(xn, vn, np.eye(self.Np), self.basis.dphi(self.basis.nodes))[1]

    # ------------------------------------------------------------------ residual
    def residual_blended(self, uX, mu, t, gbar):
        """r(U_X) [.., Ne, 4, Np] for nodal U_X [.., Ne, 4, Np] and gbar [Ne, Np]."""
        return self.residual_blended_local(uX, uX[..., self.nbr_safe, :, :], mu, t, gbar)

    def residual_blended_local(self, uX, uN, mu, t, gbar):
        """As residual_blended with the face-neighbour states uN [.., Ne, 3, 4, Np] given
        separately (for block Jacobians by the complex step)."""
        gam, mu_v, Pr = self.gam, self.mu_visc, self.Pr
        xn, vn = self.nodal_map(mu, t)
        gN = gbar[self.nbr_safe]

        # volume
        G, g, C, GinvT, v, gradX = self._geom(xn, vn, self.phi_v, self.dphi_v)
        phi_e = np.broadcast_to(self.phi_v, (self.Ne,) + self.phi_v.shape)
        U, dUX = self._state(uX, gbar, phi_e, gradX)
        dUX = dUX + self.volume_lifting_blended(uX, uN, gbar, gN, xn, vn)      # lifted grad_X U
        dU = np.einsum("eqik,...eqak->...eqai", GinvT, dUX)                    # grad_x U
        Ftot = inviscid_flux(U, gam) - U[..., None] * v[..., None, :] - viscous_flux(U, dU, mu_v, Pr, gam)
        FX = np.einsum("eqJi,...eqai->...eqaJ", C, Ftot)
        wq = self.w_v[None, :] * self.detB[:, None]
        r = np.einsum("eq,eqjJ,...eqaJ->...eaj", wq, gradX, FX)
        # faces
        for f in range(3):
            H = self.face_flux_blended(uX, uN, gbar, gN, f, xn, vn)
            r = r - np.einsum("q,e,qj,...eqa->...eaj", self.w_f, self.L[:, f], self.phi_f[f], H)
        return r

    @staticmethod
    def _state(u, gb, phi, gradX):
        """U = U_X / gbar and its reference gradient grad_X U at points."""
        UX = np.einsum("...eai,eqi->...eqa", u, phi)
        gq = np.einsum("ei,eqi->eq", gb, phi)
        dUX = np.einsum("...eai,eqid->...eqad", u, gradX)
        dg = np.einsum("ei,eqid->eqd", gb, gradX)
        U = UX / gq[..., None]
        return U, (dUX - U[..., None] * dg[..., None, :]) / gq[..., None, None]

    def _traces_blended(self, uX, uN, gbar, gN, f, xn, vn):
        """Both traces of U with their reference gradients at the points of local face f,
        the geometry there (G^-T of both sides, C^T N, the physical normal n, v_h) and the
        face value U_hat of U (neighbour trace, wall state or far-field state by tag)."""
        Gf, gf, Cf, GinvTf, vf, gradXf = self._geom(xn, vn, self.phi_f[f], self.dphi_f[f])
        phi_m = np.broadcast_to(self.phi_f[f], (self.Ne,) + self.phi_f[f].shape)
        Um, dUXm = self._state(uX, gbar, phi_m, gradXf)
        # neighbour trace at the matched points, with the neighbour's own map (the
        # interpolated map is continuous across the face, its gradient is not)
        gradXn = np.einsum("ekl,eqjl->eqjk", self.BinvT_nbr[:, f], self.dphiN[:, f])
        nb = self.nbr_safe[:, f]
        GinvTp = self._geom_pts(xn[nb], vn[nb], self.phiN[:, f], gradXn)[3]
        Up, dUXp = self._state(uN[..., f, :, :], gN[:, f], self.phiN[:, f], gradXn)
        nt = np.einsum("eqJi,eJ->eqi", Cf, self.N[:, f])                      # C^T N
        ln = np.sqrt(nt[..., 0] ** 2 + nt[..., 1] ** 2)
        n = nt / ln[..., None]
        vnrm = vf[..., 0] * n[..., 0] + vf[..., 1] * n[..., 1]
        rho = Um[..., 0]
        e_int = Um[..., 3] / rho - 0.5 * (Um[..., 1] ** 2 + Um[..., 2] ** 2) / rho**2
        vb = vf + 0.0 * rho[..., None]
        Ub = np.stack([rho, rho * vb[..., 0], rho * vb[..., 1],
                       rho * (e_int + 0.5 * (vb[..., 0] ** 2 + vb[..., 1] ** 2))], -1)
        Uinf = np.broadcast_to(self.Uinf, Um.shape) + 0.0 * Um
        tag = self.tag[:, f][:, None, None]
        Uhat = np.where(tag == 0, Up, np.where(tag == 1, Ub, Uinf))
        return dict(Um=Um, dUXm=dUXm, Up=Up, dUXp=dUXp, GinvTm=GinvTf, GinvTp=GinvTp, n=n, ln=ln, vf=vf,
                    vn=vnrm, Ub=Ub, Uinf=Uinf, Uhat=Uhat)

    def volume_lifting_blended(self, uX, uN, gbar, gN, xn, vn):
        """sum over the faces this element lifts of the reference lifting N_f s_f l_f at the
        volume points [.., Ne, nqv, 4, 2] (CDG in the reference coordinates, where the
        elements are affine)."""
        out = 0.0
        for f in range(3):
            tr = self._traces_blended(uX, uN, gbar, gN, f, xn, vn)
            w = (self.s_own[:, f] * self.flux_side[:, f])[:, None, None]
            l = np.einsum("qp,...epa->...eqa", self.lift_v[f], tr["Uhat"] - tr["Um"]) * w
            out = out + l[..., None] * self.N[:, f][:, None, None, :]
        return out

    def face_flux_blended(self, uX, uN, gbar, gN, f, xn, vn):
        """Reference-face numerical flux |C^T N| H at the points of local face f
        [.., Ne, nqf, 4] (outward from the element, per unit reference length).  The CDG
        viscous flux of the rigid oracle, with the liftings taken in the reference
        coordinates and the lifted reference gradient mapped by G^-T of its side."""
        gam, mu_v, Pr = self.gam, self.mu_visc, self.Pr
        tr = self._traces_blended(uX, uN, gbar, gN, f, xn, vn)
        Um, Up, Uhat, n, ln = tr["Um"], tr["Up"], tr["Uhat"], tr["n"], tr["ln"]
        Nf = self.N[:, f][:, None, None, :]
        l_own = np.einsum("qp,...epa->...eqa", self.lift_f[f], Uhat - Um) * self.s_own[:, f][:, None, None]
        Q_own = np.einsum("eqik,...eqak->...eqai", tr["GinvTm"], tr["dUXm"] + l_own[..., None] * Nf)
        l_nbr = np.einsum("eqp,...epa->...eqa", self.lift_fN[:, f], Up - Um) * self.s_nbr[:, f][:, None, None]
        Q_nbr = np.einsum("eqik,...eqak->...eqai", tr["GinvTp"], tr["dUXp"] + l_nbr[..., None] * Nf)
        side = self.flux_side[:, f][:, None, None]
        tag = self.tag[:, f][:, None, None]
        US = np.where(side, np.where(tag == 1, tr["Ub"], Um), Up)
        QS = np.where(side[..., None], Q_own, Q_nbr)
        FvS = np.where(tag[..., None] == 1, viscous_flux(US, QS, mu_v, Pr, gam, adiabatic=True),
                       viscous_flux(US, QS, mu_v, Pr, gam))

        def dn(F):
            return F[..., 0] * n[..., None, 0] + F[..., 1] * n[..., None, 1]

        pen = self.c11[:, f][:, None, None] * (Uhat - Um)
        Hinv = np.where(tag == 0, roe_flux(Um, Up, n, tr["vn"], gam),
                        np.where(tag == 1, normal_flux(tr["Ub"], n, tr["vn"], gam),
                                 roe_flux(Um, tr["Uinf"], n, tr["vn"], gam)))
        return (Hinv - (dn(FvS) + pen)) * ln[..., None]

    # ------------------------------------------------------------------ period grid
    def set_period_steps(self, Nt):
        """Equal DIRK steps of dt = T / Nt from t = 0: the stage times at which gbar is
        tabulated (gbar(0) = g_h at t = 0, the map's own Jacobian)."""
        from . import dirk
        self.Nt_grid = Nt
        self._tab = dirk.tableau()
        self._gcache = {}

    def gbar_at(self, mu, t):
        """gbar at a stage time of the period grid (or the frozen pose for t = None).  The
        table is built once per mu by the DIRK of the GCL; complex mu is allowed, so that
        complex-step derivatives in mu include d gbar / d mu."""
        if t is None:
            return self.geometric_g(mu, None)
        key = tuple(np.asarray(mu).ravel().tolist())
        tab = self._gcache.get(key)
        if tab is None:
            A, b, c = self._tab
            dt = self.T / self.Nt_grid
            g = self.geometric_g(mu, 0.0)
            tab = {round(0.0, 10): g}
            for n in range(self.Nt_grid):
                t0 = n * dt
                stages, g = self.gbar_dirk(mu, t0, dt, g, self._tab)
                for i in range(len(b)):
                    tab[round(t0 + c[i] * dt, 10)] = stages[i]   # the sweeps' own stage times
            self._gcache[key] = tab
        k = round(float(np.real(t)), 10)
        if k not in tab:
            raise KeyError(f"t = {t} is not a stage time of the period grid")
        return tab[k]

    # ------------------------------------------------------------------ DG interface
    def residual_local(self, uS, uN, mu, t):
        """The base-class interface (used by residual, block Jacobians, dr/dmu and the
        sweeps): the blended residual with gbar from the period grid."""
        return self.residual_blended_local(uS, uN, mu, t, self.gbar_at(mu, t))

    def qoi_rate(self, u, mu, t):
        """Power and x-force on the airfoil from the wall numerical flux (per unit physical
        length: the reference flux carries the factor |C^T N|)."""
        us = np.asarray(u).reshape(np.shape(u)[:-1] + (self.Ne, 4, self.Np))
        uN = us[..., self.nbr_safe, :, :]
        gbar = self.gbar_at(mu, t)
        xn, vn = self.nodal_map(mu, t)
        Pw, Fx = 0.0, 0.0
        for f in range(3):
            H = self.face_flux_blended(us, uN, gbar, gbar[self.nbr_safe], f, xn, vn)
            vf = self._geom(xn, vn, self.phi_f[f], self.dphi_f[f])[4]
            wall = (self.tag[:, f] == 1).astype(np.float64)
            wl = self.w_f[None, :] * (self.L[:, f] * wall)[:, None]
            force = H[..., 1:3]
            Pw = Pw + np.einsum("eq,...eq->...", wl, force[..., 0] * vf[..., 0] + force[..., 1] * vf[..., 1])
            Fx = Fx + np.einsum("eq,...eq->...", wl, force[..., 0])
        return Pw, Fx

    def dqoi_du(self, u, mu, t):
        """d(P^h, F_x^h)/du [2, Nu] (face-local to wall elements: one complex perturbation
        of local dof (a, i) in every element at once is exact)."""
        nb, Ne, Np = self.nb, self.Ne, self.Np
        us = np.asarray(u, dtype=np.float64).reshape(Ne, 4, Np)
        gbar = self.gbar_at(mu, t)
        xn, vn = self.nodal_map(mu, t)
        E = np.eye(nb).reshape(nb, 1, 4, Np)
        uS = us[None] + 1j * CS_STEP * E
        uN = us[self.nbr_safe][None] + 0j
        out = np.zeros((2, Ne, nb))
        for f in range(3):
            H = self.face_flux_blended(uS, uN, gbar, gbar[self.nbr_safe], f, xn, vn)
            vf = self._geom(xn, vn, self.phi_f[f], self.dphi_f[f])[4]
            wall = (self.tag[:, f] == 1).astype(np.float64)
            wl = self.w_f[None, :] * (self.L[:, f] * wall)[:, None]
            force = H[..., 1:3]
            pw = np.einsum("eq,deq->de", wl, force[..., 0] * vf[..., 0] + force[..., 1] * vf[..., 1])
            fx = np.einsum("eq,deq->de", wl, force[..., 0])
            out[0] += np.imag(pw).T / CS_STEP
            out[1] += np.imag(fx).T / CS_STEP
        return out.reshape(2, self.Nu)

    def gbar_dirk(self, mu, t0, dt, g0, tableau):
        """gbar at the stages and at the end of one DIRK step from gbar(t0) = g0: the GCL
        rate does not depend on gbar, so every stage value is explicit."""
        A, b, c = tableau
        k = [self.gcl_rate(mu, t0 + c[i] * dt) for i in range(len(b))]
        stages = [g0 + dt * sum(A[i][j] * k[j] for j in range(i + 1)) for i in range(len(b))]
        return stages, g0 + dt * sum(b[i] * k[i] for i in range(len(b)))
