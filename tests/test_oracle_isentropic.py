"""Pins for the oracle's isentropic variant (Sec. 6, Eq. entropy: p = s rho^gamma, no energy
equation; state (rho, rho u, rho v)).

Checks against something other than the oracle itself: closed-form fluxes; the Roe-type
flux's consistency and conservation, and its small-jump limit against |A - v_G.n I| formed
by a library eigendecomposition of the flux Jacobian; free-stream preservation on a moving
mesh; the no-slip wall (no mass flux through the moving wall, momentum flux p n); the
element Jacobian against central differences of the residual; and order-of-accuracy p + 1
for steady manufactured solutions, inviscid and viscous (Re = 10), the source built from the
pointwise fluxes pinned here."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import isentropic as I
from oracle.dg import KIN_HEAVE_PITCH
from pp_inputs import MU_C0, box

G = 1.4
MACH = 0.2
S = 1.0 / (G * MACH * MACH)


def _state(rho, u, v):
    return np.array([rho, rho * u, rho * v])


def test_free_stream_and_pressure_law():
    dg = I.IsentropicDG(box(2, 2, seed=0), 1, Mach=MACH)
    assert dg.nv == 3 and dg.nb == 3 * dg.Np and dg.Nu == dg.Ne * 3 * dg.Np
    assert np.array_equal(dg.Uinf, [1.0, 1.0, 0.0])
    assert abs(I.isentropic_pressure(1.0, dg.s_entropy, G) - 1.0 / (G * MACH ** 2)) < 1e-14
    # s = p / rho^gamma is the same at any density
    for rho in (0.5, 1.0, 2.3):
        assert abs(I.isentropic_pressure(rho, S, G) / rho ** G - S) < 1e-12


def test_fluxes_closed_form():
    rho, u, v = 1.3, 0.5, -0.25
    U = _state(rho, u, v)
    p = S * rho ** G
    F = I.inviscid_flux_isen(U, S, G)
    assert np.allclose(F[:, 0], [rho * u, rho * u * u + p, rho * u * v], atol=1e-13)
    assert np.allclose(F[:, 1], [rho * v, rho * u * v, rho * v * v + p], atol=1e-13)
    # Couette: u_y = 2 gives tau_xy = 2 mu and nothing in the mass row
    mu = 1e-3
    dU = np.zeros((3, 2))
    dU[1, 1] = 2.0
    Fv = I.viscous_flux_isen(_state(1.0, 0.0, 0.0), dU, mu)
    assert np.allclose(Fv[:, 0], [0, 0, 2 * mu], atol=1e-15)
    assert np.allclose(Fv[:, 1], [0, 2 * mu, 0], atol=1e-15)


def test_roe_type_flux_consistency_conservation_and_dissipation():
    n = np.array([0.6, 0.8])
    for vn in (0.0, 0.3, -0.7):
        U = _state(1.2, 0.3, -0.2)
        assert np.allclose(I.roe_flux_isen(U, U, n, np.array(vn), S, G),
                           I.normal_flux_isen(U, n, np.array(vn), S, G), atol=1e-13)
    UL, UR = _state(1.0, 0.4, 0.1), _state(0.9, 0.2, -0.3)
    assert np.allclose(I.roe_flux_isen(UL, UR, n, np.array(0.2), S, G),
                       -I.roe_flux_isen(UR, UL, -n, np.array(-0.2), S, G), atol=1e-13)
    # small jumps: the dissipation is |A - vn I| dU, A the Jacobian of F.n at the state
    # (waves un - c = -4.1, un = 0.9 - vn, un + c = 5.9 with c = 5 are outside the entropy fix)
    U = _state(1.0, 0.9, 0.3)
    nn = np.array([1.0, 0.0])
    vn = np.array(0.2)
    Jac = np.zeros((3, 3))
    for b in range(3):
        Uc = U + 0j
        Uc[b] += 1e-30j
        Jac[:, b] = np.imag(I.normal_flux_isen(Uc, nn, vn + 0j, S, G)) / 1e-30
    lam, R = np.linalg.eig(Jac)
    absA = np.real(R @ np.diag(np.abs(lam)) @ np.linalg.inv(R))
    d = np.array([0.3, -0.2, 0.5])
    eps = 1e-7
    UR = U + eps * d
    diss = (I.normal_flux_isen(U, nn, vn, S, G) + I.normal_flux_isen(UR, nn, vn, S, G)
            - 2.0 * I.roe_flux_isen(U, UR, nn, vn, S, G)) / eps
    assert np.allclose(diss, absA @ d, rtol=1e-5, atol=1e-5)


def test_no_slip_wall_flux():
    dg = I.IsentropicDG(box(2, 2, seed=0), 1, Mach=MACH)
    rng = np.random.default_rng(8)
    Um = np.stack([1.0 + 0.2 * rng.random(5), rng.standard_normal(5), rng.standard_normal(5)], -1)
    vG = rng.standard_normal((5, 2))
    th = rng.uniform(0, 2 * np.pi, 5)
    n = np.stack([np.cos(th), np.sin(th)], -1)
    vn = np.sum(vG * n, -1)
    Ub = dg.wall_state(Um, vG)
    assert np.allclose(Ub[:, 0], Um[:, 0]) and np.allclose(Ub[:, 1:] / Ub[:, :1], vG)
    F = dg.flux_normal(Ub, n, vn)
    p = I.isentropic_pressure(Um[:, 0], dg.s_entropy, G)
    assert np.max(np.abs(F[:, 0])) < 1e-14
    assert np.allclose(F[:, 1:], p[:, None] * n, atol=1e-12)


def _uniform(dg):
    return np.broadcast_to(dg.Uinf[None, :, None], (dg.Ne, 3, dg.Np)).reshape(-1).copy()


@pytest.mark.parametrize("p", [1, 3])
def test_free_stream_preserved_on_moving_mesh(p):
    dg = I.IsentropicDG(box(4, 3, seed=1), p, Mach=MACH)
    u = _uniform(dg)
    for t in (0.0, 0.37, 1.9):
        assert np.max(np.abs(dg.residual(u, MU_C0, t))) < 2e-13


def test_jacobian_blocks_match_central_differences():
    from pp_inputs import ogrid
    dg = I.IsentropicDG(ogrid(8, 2, seed=0), 2, Mach=MACH)
    rng = np.random.default_rng(7)
    u = _uniform(dg) + 1e-2 * rng.standard_normal(dg.Nu)
    J = dg.jacobian(u, MU_C0, 0.41)
    v = rng.standard_normal(dg.Nu)
    h = 1e-6
    fd = (dg.residual(u + h * v, MU_C0, 0.41) - dg.residual(u - h * v, MU_C0, 0.41)) / (2 * h)
    assert np.max(np.abs(J @ v - fd)) <= 1e-7 * np.max(np.abs(fd))


# ---------------------------------------------------------------------- manufactured solutions
MACH_MMS = 0.5
S_MMS = 1.0 / (G * MACH_MMS * MACH_MMS)


def u_exact(X):
    """Smooth manufactured state (rho, rho u, rho v) at points X [..., 2]."""
    x, y = X[..., 0], X[..., 1]
    rho = 1.0 + 0.1 * np.sin(np.pi * x) * np.cos(np.pi * y)
    u = 0.5 + 0.1 * np.cos(np.pi * x) * np.sin(np.pi * y)
    v = 0.1 * np.sin(np.pi * x) * np.sin(np.pi * y) - 0.05
    return np.stack([rho, rho * u, rho * v], -1)


def _grad_exact(X):
    cols = []
    for d in range(2):
        Xc = X + 0j
        Xc[..., d] += 1e-30j
        cols.append(np.imag(u_exact(Xc)) / 1e-30)
    return np.stack(cols, -1)


def _total_flux(X, mu_visc):
    U = u_exact(X)
    F = I.inviscid_flux_isen(U, S_MMS, G)
    if mu_visc > 0:
        F = F - I.viscous_flux_isen(U, _grad_exact(X), mu_visc)
    return F


def _source(X, mu_visc, h=1e-3):
    S = 0.0
    for d in range(2):
        e = np.zeros(2)
        e[d] = h
        fp1, fm1 = _total_flux(X + e, mu_visc)[..., d], _total_flux(X - e, mu_visc)[..., d]
        fp2, fm2 = _total_flux(X + 2 * e, mu_visc)[..., d], _total_flux(X - 2 * e, mu_visc)[..., d]
        S = S + (8.0 * (fp1 - fm1) - (fp2 - fm2)) / (12.0 * h)
    return S


def _square(n):
    m = box(n, n, seed=0, x0=0.0, x1=1.0, y0=0.0, y1=1.0, jitter=0.0)
    x, y = m.verts[:, 0].copy(), m.verts[:, 1].copy()
    m.verts[:, 0] = x + 0.04 * np.sin(np.pi * x) * np.sin(2 * np.pi * y)
    m.verts[:, 1] = y + 0.04 * np.sin(2 * np.pi * x) * np.sin(np.pi * y)
    return m


def _steady_error(n, p, Re):
    dg = I.IsentropicDG(_square(n), p, gamma=G, Mach=MACH_MMS, Re=Re, kin=KIN_HEAVE_PITCH, farfield=u_exact)
    mu = np.zeros(3)
    wq = dg.w_v[None, :] * dg.detB[:, None]
    s = np.einsum("eq,qi,eqa->eai", wq, dg.phi_v, _source(dg.Xq_v, dg.mu_visc)).reshape(-1)
    Xn = dg.X0[:, None, :] + np.einsum("edk,jk->ejd", dg.B, dg.basis.nodes)
    u = np.transpose(u_exact(Xn), (0, 2, 1)).reshape(-1)
    for _ in range(20):
        R = dg.residual(u, mu, None) + s
        du = spla.splu(dg.jacobian(u, mu, None).tocsc()).solve(R)
        u = u - du
        if np.max(np.abs(du)) <= 1e-12 * np.max(np.abs(u)):
            break
    else:
        raise RuntimeError("manufactured steady state did not converge")
    uq = np.einsum("qi,eai->eqa", dg.phi_v, u.reshape(dg.Ne, 3, dg.Np))
    err = uq - u_exact(dg.Xq_v)
    return float(np.sqrt(np.einsum("eq,eqa->", wq, err * err)))


@pytest.mark.parametrize("p,Re,ns", [(1, np.inf, (4, 8, 16)), (2, np.inf, (3, 6, 12)), (2, 10.0, (3, 6, 12))],
                         ids=["p1-inviscid", "p2-inviscid", "p2-viscous_Re10"])
def test_manufactured_solution_converges_at_order_p_plus_1(p, Re, ns):
    errs = [_steady_error(n, p, Re) for n in ns]
    orders = [np.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    print(f"isentropic p={p} Re={Re}: errors {errs}, observed orders {orders}")
    assert orders[-1] >= p + 0.5, (errs, orders)
