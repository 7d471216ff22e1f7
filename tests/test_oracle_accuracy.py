"""Accuracy pin of the oracle's spatial discretization: steady manufactured solutions.

A smooth state U_ex(x) is made an exact steady solution of the Navier-Stokes
equations by the source S = div(F_inv(U_ex) - F_vis(U_ex, grad U_ex)), and the
discrete steady problem r(u) + int phi S = 0 is solved by Newton on refined meshes
of the unit square with U_ex as the far-field boundary state.  A consistent,
stable DG discretization of degree p converges in L2 at order p + 1 for smooth
solutions; the test asks for an observed order of at least p + 0.5 between the last
two meshes of three.  Two cases isolate the two parts of the residual:

* inviscid (viscosity 0): Roe flux, boundary states, quadrature, geometry;
* viscous-dominated (Re = 10): the CDG liftings, the one-sided viscous face flux,
  the boundary penalty.  A wrong sign or factor on the viscous face flux or on a
  lifting makes the scheme inconsistent, and the observed order drops to 1 or less.

The source uses the oracle's pointwise flux functions (they are pinned separately
against closed forms); its divergence is taken by a fourth-order central difference
of width 1e-3 around each quadrature point, with the state gradient inside the flux
exact by complex step, so the source error (~1e-11) stays far below the
discretization errors measured here.  Meshes: the unit square cut into n x n quads,
two triangles each, interior vertices moved by a smooth map that vanishes on the
boundary (so the meshes refine consistently and no edge is axis-aligned inside).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.dg import DG, KIN_HEAVE_PITCH, inviscid_flux, viscous_flux
from pp_inputs import box

GAM, PR, MACH = 1.4, 0.72, 0.5
PINF = 1.0 / (GAM * MACH * MACH)


def u_exact(X):
    """Smooth manufactured state (conservative variables) at points X [..., 2]."""
    x, y = X[..., 0], X[..., 1]
    rho = 1.0 + 0.1 * np.sin(np.pi * x) * np.cos(np.pi * y)
    u = 0.5 + 0.1 * np.cos(np.pi * x) * np.sin(np.pi * y)
    v = 0.1 * np.sin(np.pi * x) * np.sin(np.pi * y) - 0.05
    p = PINF * (1.0 + 0.1 * np.cos(np.pi * x) * np.sin(2.0 * np.pi * y))
    E = p / (GAM - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], -1)


def grad_exact(X):
    """d U_ex / dx_d by complex step, [..., 4, 2]."""
    h = 1e-30
    cols = []
    for d in range(2):
        Xc = X + 0j
        Xc[..., d] += 1j * h
        cols.append(np.imag(u_exact(Xc)) / h)
    return np.stack(cols, -1)


def total_flux(X, mu_visc):
    U = u_exact(X)
    F = inviscid_flux(U, GAM)
    if mu_visc > 0:
        F = F - viscous_flux(U, grad_exact(X), mu_visc, PR, GAM)
    return F                                                  # [..., 4, 2]


def source(X, mu_visc, h=1e-3):
    """S = sum_d d/dx_d F_d(U_ex) by fourth-order central differences."""
    S = 0.0
    for d in range(2):
        e = np.zeros(2)
        e[d] = h
        fp1, fm1 = total_flux(X + e, mu_visc)[..., d], total_flux(X - e, mu_visc)[..., d]
        fp2, fm2 = total_flux(X + 2 * e, mu_visc)[..., d], total_flux(X - 2 * e, mu_visc)[..., d]
        S = S + (8.0 * (fp1 - fm1) - (fp2 - fm2)) / (12.0 * h)
    return S                                                  # [..., 4]


def square_mesh(n):
    m = box(n, n, seed=0, x0=0.0, x1=1.0, y0=0.0, y1=1.0, jitter=0.0)
    x, y = m.verts[:, 0].copy(), m.verts[:, 1].copy()
    m.verts[:, 0] = x + 0.04 * np.sin(np.pi * x) * np.sin(2 * np.pi * y)
    m.verts[:, 1] = y + 0.04 * np.sin(2 * np.pi * x) * np.sin(np.pi * y)
    return m


def steady_error(n, p, Re):
    dg = DG(square_mesh(n), p, gamma=GAM, Pr=PR, Mach=MACH, Re=Re, kin=KIN_HEAVE_PITCH, farfield=u_exact)
    mu = np.zeros(3)                      # no motion: the frozen pose is the reference configuration
    wq = dg.w_v[None, :] * dg.detB[:, None]
    s = np.einsum("eq,qi,eqa->eai", wq, dg.phi_v, source(dg.Xq_v, dg.mu_visc)).reshape(-1)
    Xn = dg.X0[:, None, :] + np.einsum("edk,jk->ejd", dg.B, dg.basis.nodes)
    u = np.transpose(u_exact(Xn), (0, 2, 1)).reshape(-1)   # nodal interpolant as the first guess
    for _ in range(20):
        R = dg.residual(u, mu, None) + s
        du = spla.splu(dg.jacobian(u, mu, None).tocsc()).solve(R)
        u = u - du
        if np.max(np.abs(du)) <= 1e-12 * np.max(np.abs(u)):
            break
    else:
        raise RuntimeError("manufactured steady state did not converge")
    assert np.max(np.abs(dg.residual(u, mu, None) + s)) <= 1e-8 * np.max(np.abs(s))
    uq = np.einsum("qi,eai->eqa", dg.phi_v, u.reshape(dg.Ne, 4, dg.Np))
    scale = np.array([1.0, 1.0, 1.0, 1.0 / PINF])
    err = (uq - u_exact(dg.Xq_v)) * scale
    return float(np.sqrt(np.einsum("eq,eqa->", wq, err * err)))


CASES = {  # p -> mesh sizes n (n x n quads)
    1: (4, 8, 16),
    2: (3, 6, 12),
    3: (2, 4, 8),
}


@pytest.mark.parametrize("Re", [np.inf, 10.0], ids=["inviscid", "viscous_Re10"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_manufactured_solution_converges_at_order_p_plus_1(p, Re):
    ns = CASES[p]
    errs = [steady_error(n, p, Re) for n in ns]
    orders = [np.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    print(f"p={p} Re={Re}: errors {errs}, observed orders {orders}")
    assert errs[-1] < errs[0]
    assert orders[-1] >= p + 0.5, (errs, orders)
