"""Oracle: the isentropic variant of the semi-discretization (Sec. 6, Eq. entropy).

Test infrastructure only (imported by tests); nothing in the product imports it.

With the entropy s = p / rho^gamma constant, the pressure is a function of the density,
p = s rho^gamma, and the energy equation drops out: the state is (rho, rho u, rho v), the
momentum equations keep the viscous stress of Sec. 6 and there is no heat flux.  s is the
free stream's, s = p_inf / rho_inf^gamma = 1 / (gamma Mach^2) (rho_inf = 1, |u_inf| = 1).

Everything else -- the ALE form, the CDG liftings and one-sided viscous face fluxes, the
boundary penalty, the quadrature, the element Jacobian by complex step, the QoIs -- is the
4-variable oracle's (`DG` with NV = 3 and these physics hooks).

Inviscid face flux (a reading, the paper names Roe's flux for its compressible solver):
Roe-type, F_hat = (F.n(UL) + F.n(UR)) / 2 - |A~ - v_G.n I| (UR - UL) / 2, with A~ the normal
flux Jacobian at the sqrt(rho)-weighted velocity and the sound speed of the geometric-mean
density, c~^2 = gamma s (sqrt(rho_L rho_R))^(gamma - 1), and the Harten entropy fix
delta = 0.1 c~ on the three waves.  It is consistent, conservative and upwind; it is not an
exact Roe linearization (that would need c~^2 = (pR - pL) / (rhoR - rhoL)).
"""
import numpy as np

from .dg import DG, cabs


def isentropic_pressure(rho, s, gam):
    return s * rho ** gam


def inviscid_flux_isen(U, s, gam):
    """F_inv(U), shape [..., 3, 2] (Eqs. ns1-ns2 with p = s rho^gamma)."""
    rho = U[..., 0]
    u = U[..., 1] / rho
    v = U[..., 2] / rho
    p = isentropic_pressure(rho, s, gam)
    Fx = np.stack([U[..., 1], U[..., 1] * u + p, U[..., 2] * u], -1)
    Fy = np.stack([U[..., 2], U[..., 1] * v, U[..., 2] * v + p], -1)
    return np.stack([Fx, Fy], -1)


def viscous_flux_isen(U, dU, mu):
    """F_vis(U, grad U), shape [..., 3, 2]: the stress tensor of Sec. 6, no heat flux."""
    rho = U[..., 0]
    u = U[..., 1] / rho
    v = U[..., 2] / rho
    drho = dU[..., 0, :]
    du = (dU[..., 1, :] - u[..., None] * drho) / rho[..., None]
    dv = (dU[..., 2, :] - v[..., None] * drho) / rho[..., None]
    ux, uy = du[..., 0], du[..., 1]
    vx, vy = dv[..., 0], dv[..., 1]
    div = ux + vy
    txx = mu * (2.0 * ux - 2.0 / 3.0 * div)
    tyy = mu * (2.0 * vy - 2.0 / 3.0 * div)
    txy = mu * (uy + vx)
    zero = 0.0 * txx
    Fx = np.stack([zero, txx, txy], -1)
    Fy = np.stack([zero, txy, tyy], -1)
    return np.stack([Fx, Fy], -1)


def normal_flux_isen(U, n, vn, s, gam):
    """F_inv(U).n - (v_G.n) U."""
    F = inviscid_flux_isen(U, s, gam)
    return F[..., 0] * n[..., None, 0] + F[..., 1] * n[..., None, 1] - vn[..., None] * U


def roe_flux_isen(UL, UR, n, vn, s, gam):
    """Roe-type flux of the ALE normal flux (see the module docstring).  Waves of the normal
    Jacobian at (u~, v~, c~), eigenvalues shifted by -v_G.n:
        un - c~:  (1, u~ - c~ nx, v~ - c~ ny)
        un:       (0, -ny, nx)
        un + c~:  (1, u~ + c~ nx, v~ + c~ ny)
    with strengths from drho, the normal and the tangential momentum jumps."""
    rL, rR = UL[..., 0], UR[..., 0]
    uL, vL = UL[..., 1] / rL, UL[..., 2] / rL
    uR, vR = UR[..., 1] / rR, UR[..., 2] / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    ut = (sL * uL + sR * uR) / (sL + sR)
    vt = (sL * vL + sR * vR) / (sL + sR)
    c2 = gam * s * (sL * sR) ** (gam - 1.0)
    c = np.sqrt(c2)
    nx, ny = n[..., 0], n[..., 1]
    un = ut * nx + vt * ny
    tn = -ut * ny + vt * nx
    lu = un - vn
    delta = 0.1 * c

    def fix(l):
        al = cabs(l)
        return np.where(np.real(al) < np.real(delta), (l * l + delta * delta) / (2.0 * delta), al)

    lm, l0, lp = fix(lu - c), fix(lu), fix(lu + c)
    D = UR - UL
    dmn = D[..., 1] * nx + D[..., 2] * ny
    dmt = -D[..., 1] * ny + D[..., 2] * nx
    ac = (dmn - un * D[..., 0]) / c
    am = 0.5 * (D[..., 0] - ac)
    ap = 0.5 * (D[..., 0] + ac)
    a0 = dmt - tn * D[..., 0]
    one = 1.0 + 0.0 * ut
    rm = np.stack([one, ut - c * nx, vt - c * ny], -1)
    r0 = np.stack([0.0 * ut, -ny + 0.0 * ut, nx + 0.0 * ut], -1)
    rp = np.stack([one, ut + c * nx, vt + c * ny], -1)
    AD = (lm * am)[..., None] * rm + (l0 * a0)[..., None] * r0 + (lp * ap)[..., None] * rp
    return 0.5 * (normal_flux_isen(UL, n, vn, s, gam) + normal_flux_isen(UR, n, vn, s, gam)) - 0.5 * AD


class IsentropicDG(DG):
    """The isentropic semi-discretization: state (rho, rho u, rho v), p = s rho^gamma."""

    NV = 3

    @property
    def s_entropy(self):
        return 1.0 / (self.gam * self.Mach * self.Mach)

    def free_stream(self):
        return np.array([1.0, 1.0, 0.0])

    def flux_inv(self, U):
        return inviscid_flux_isen(U, self.s_entropy, self.gam)

    def flux_vis(self, U, dU, adiabatic=False):
        return viscous_flux_isen(U, dU, self.mu_visc)

    def flux_normal(self, U, n, vn):
        return normal_flux_isen(U, n, vn, self.s_entropy, self.gam)

    def flux_roe(self, UL, UR, n, vn):
        return roe_flux_isen(UL, UR, n, vn, self.s_entropy, self.gam)

    def wall_state(self, Um, vG):
        """No-slip wall state: interior density, wall velocity."""
        rho = Um[..., 0]
        vGb = vG + 0.0 * rho[..., None]
        return np.stack([rho, rho * vGb[..., 0], rho * vGb[..., 1]], -1)
