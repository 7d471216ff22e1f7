"""Pins for the oracle's ALE DG residual, fluxes, QoIs and exact derivatives.

Each test checks the oracle against something other than itself: closed-form
flux identities, free-stream preservation (the paper's GCL requirement, Sec. 6),
discrete conservation, rotational invariance of the Navier-Stokes equations,
and central finite differences for the complex-step derivatives."""
import numpy as np
import pytest

from oracle import dg as D
from pp_inputs import box, ogrid, free_stream_state, state_perturbation, MU_C0, fourier6_samples

G = 1.4


def _state(rho, u, v, p):
    return np.array([rho, rho * u, rho * v, p / (G - 1) + 0.5 * rho * (u * u + v * v)])


def test_roe_consistency_and_supersonic_upwinding():
    rng = np.random.default_rng(0)
    n = np.array([0.6, 0.8])
    for vn in (0.0, 0.3, -0.7):
        U = _state(1.2, 0.3, -0.2, 2.0)
        assert np.allclose(D.roe_flux(U, U, n, np.array(vn), G), D.normal_flux(U, n, np.array(vn), G), atol=1e-13)
    # all eigenvalues of the relative normal flux positive => Roe = left flux exactly
    for _ in range(5):
        UL = _state(1 + 0.1 * rng.random(), 3.0 + 0.2 * rng.random(), 0.1, 1.0 + 0.1 * rng.random())
        UR = _state(1 + 0.1 * rng.random(), 3.1 + 0.2 * rng.random(), -0.1, 1.0 + 0.1 * rng.random())
        vn = np.array(-0.5)
        FL = D.normal_flux(UL, n, vn, G)
        assert np.allclose(D.roe_flux(UL, UR, n, vn, G), FL, rtol=1e-12, atol=1e-12)
    # conservation: H(L, R, n) = -H(R, L, -n)
    UL, UR = _state(1.0, 0.4, 0.1, 1.5), _state(0.9, 0.2, -0.3, 1.3)
    assert np.allclose(D.roe_flux(UL, UR, n, np.array(0.2), G), -D.roe_flux(UR, UL, -n, np.array(-0.2), G), atol=1e-13)


def test_inviscid_flux_closed_form_and_rotation():
    U = _state(1.3, 0.5, -0.25, 2.0)
    F = D.inviscid_flux(U, G)
    rho, u, v, p = 1.3, 0.5, -0.25, 2.0
    E = U[3]
    assert np.allclose(F[:, 0], [rho * u, rho * u * u + p, rho * u * v, (E + p) * u], atol=1e-14)
    assert np.allclose(F[:, 1], [rho * v, rho * u * v, rho * v * v + p, (E + p) * v], atol=1e-14)
    th = 0.7
    n = np.array([np.cos(th), np.sin(th)])
    R = np.array([[1, 0, 0, 0], [0, np.cos(th), np.sin(th), 0], [0, -np.sin(th), np.cos(th), 0], [0, 0, 0, 1.0]])
    assert np.allclose(F @ n, R.T @ D.inviscid_flux(R @ U, G)[:, 0], atol=1e-13)


def test_viscous_flux_couette_and_heat_conduction():
    mu, Pr = 1e-3, 0.72
    rho, p = 1.0, 10.0
    U = _state(rho, 0.0, 0.0, p)
    dU = np.zeros((4, 2))
    dU[1, 1] = 2.0                         # d(rho u)/dy = 2 with rho = 1: u_y = 2
    F = D.viscous_flux(U, dU, mu, Pr, G)
    assert np.allclose(F[:, 0], [0, 0, 2 * mu, 0], atol=1e-15)
    assert np.allclose(F[:, 1], [0, 2 * mu, 0, 0], atol=1e-15)
    # pure conduction: d(rho E)/dx = 1 at rest, rho const: e_x = 1, q_x = -(mu/Pr) gamma e_x
    dU = np.zeros((4, 2))
    dU[3, 0] = 1.0
    F = D.viscous_flux(U, dU, mu, Pr, G)
    assert abs(F[3, 0] - mu / Pr * G) < 1e-15
    assert abs(D.viscous_flux(U, dU, mu, Pr, G, adiabatic=True)[3, 0]) < 1e-15


@pytest.mark.parametrize("p", [1, 2, 3])
def test_free_stream_preserved_on_moving_mesh(p):
    dg = D.DG(box(4, 3, seed=1), p)
    u = free_stream_state(dg.Ne, p).reshape(-1)
    for t in (0.0, 0.37, 1.9, 3.3):
        r = dg.residual(u, MU_C0, t)
        assert np.max(np.abs(r)) < 2e-13


def test_global_conservation_and_wall_force():
    """Interior numerical fluxes cancel (discrete conservation), so with free stream
    in the far-field ring the summed mass residual vanishes and the summed momentum
    residual equals minus the force on the wall (Eq. qoi, instantaneous form)."""
    mesh = ogrid(16, 4, seed=3)
    dg = D.DG(mesh, 2)
    u = free_stream_state(dg.Ne, 2) + state_perturbation(dg.Ne, 2, 7, amp=3e-2)
    far = np.any(dg.tag == 2, axis=1)
    near_far = far | np.any(far[dg.nbr_safe] & (dg.nbr >= 0), axis=1)
    u[near_far] = free_stream_state(int(near_far.sum()), 2)
    for t in (0.3, 2.2):
        r = dg.residual(u.reshape(-1), MU_C0, t).reshape(dg.Ne, 4, dg.Np)
        tot = r.sum(axis=(0, 2))
        assert abs(tot[0]) < 1e-12
        _, fx = dg.qoi_rate(u.reshape(-1), MU_C0, t)
        assert abs(tot[1] + fx) < 1e-11 * max(1.0, abs(fx))


def test_rotation_invariance_of_interior_residual():
    """With the pitch held (theta' = h' = 0) the mesh is the reference mesh rotated by
    Q; the Navier-Stokes equations are rotation invariant, so on elements away from
    the boundary r_Q(U) = R^T r_0(R U) with R rotating momentum by Q^T."""
    mesh = box(5, 4, seed=2)
    dg = D.DG(mesh, 2, kin=D.KIN_FOURIER6)
    th = 0.3
    mu_rot = np.array([0, 0, 0, 0, th, 0.0])       # theta = beta1 cos(wt) -> th at t = 0, theta' = 0
    mu_0 = np.zeros(6)
    u = free_stream_state(dg.Ne, 2) + state_perturbation(dg.Ne, 2, 3, amp=5e-2)
    Q = np.array([[np.cos(th), np.sin(th)], [-np.sin(th), np.cos(th)]])
    uR = u.copy()
    uR[:, 1:3, :] = np.einsum("dk,ekn->edn", Q.T, u[:, 1:3, :])
    r_rot = dg.residual(u.reshape(-1), mu_rot, 0.0).reshape(u.shape)
    r_0 = dg.residual(uR.reshape(-1), mu_0, 0.0).reshape(u.shape)
    back = r_0.copy()
    back[:, 1:3, :] = np.einsum("dk,ekn->edn", Q, r_0[:, 1:3, :])
    interior = np.all(dg.tag == 0, axis=1)
    assert np.allclose(r_rot[interior], back[interior], atol=1e-12, rtol=1e-12)


def test_jacobian_blocks_match_central_differences():
    mesh = ogrid(8, 2, seed=0)
    dg = D.DG(mesh, 2)
    u = (free_stream_state(dg.Ne, 2) + state_perturbation(dg.Ne, 2, 11, amp=1e-2)).reshape(-1)
    J = dg.jacobian(u, MU_C0, 0.8)
    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal(dg.Nu)
        h = 1e-6
        fd = (dg.residual(u + h * v, MU_C0, 0.8) - dg.residual(u - h * v, MU_C0, 0.8)) / (2 * h)
        assert np.linalg.norm(J @ v - fd) <= 1e-7 * np.linalg.norm(fd)


def test_mu_and_qoi_derivatives_match_central_differences():
    mesh = ogrid(8, 2, seed=0)
    dg = D.DG(mesh, 1, kin=D.KIN_FOURIER6)
    mu = fourier6_samples(1, 5)[0]
    u = (free_stream_state(dg.Ne, 1) + state_perturbation(dg.Ne, 1, 12, amp=1e-2)).reshape(-1)
    t = 1.3
    drdmu = dg.dr_dmu(u, mu, t)
    dq_du = dg.dqoi_du(u, mu, t)
    dq_dmu = dg.dqoi_dmu(u, mu, t)
    h = 1e-6
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        fd = (dg.residual(u, mu + e, t) - dg.residual(u, mu - e, t)) / (2 * h)
        assert np.linalg.norm(drdmu[:, j] - fd) <= 1e-6 * max(np.linalg.norm(fd), 1e-8)
        qp = np.array(dg.qoi_rate(u, mu + e, t))
        qm = np.array(dg.qoi_rate(u, mu - e, t))
        assert np.allclose(dq_dmu[:, j], (qp - qm) / (2 * h), rtol=1e-6, atol=1e-9)
    v = np.random.default_rng(1).standard_normal(dg.Nu)
    qp = np.array(dg.qoi_rate(u + h * v, mu, t))
    qm = np.array(dg.qoi_rate(u - h * v, mu, t))
    assert np.allclose(dq_du @ v, (qp - qm) / (2 * h), rtol=1e-6, atol=1e-9)


def test_fluid_at_rest_exerts_no_net_force():
    dg = D.DG(ogrid(16, 2, seed=0), 2)
    U = _state(1.0, 0.0, 0.0, 1.0 / (G * 0.04))
    u = np.broadcast_to(U[None, :, None], (dg.Ne, 4, dg.Np)).reshape(-1).copy()
    pw, fx = dg.qoi_rate(u, np.zeros(3), 0.0)
    assert abs(fx) < 1e-12 and abs(pw) < 1e-12


def test_steady_state_is_a_root_of_the_frozen_residual():
    """The cold start of Sec. 6.1 is the steady flow at the t = 0 pose with the mesh at
    rest: a root of r(u; theta(0), v_G = 0).  PTC must reach it from the free stream."""
    from oracle import periodic as P
    dg = D.DG(ogrid(12, 2, seed=0), 1)
    u_inf = free_stream_state(dg.Ne, 1).reshape(-1)
    u, it, rr = P.steady_state(dg, MU_C0, u_inf)
    assert rr <= 1e-12 and it < 100
    r = dg.residual(u, MU_C0, None)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(dg.residual(u_inf, MU_C0, None))
    # the frozen pose is the t = 0 pose: same residual as the moving problem with zero velocities
    mu0 = np.array([0.0, MU_C0[1], MU_C0[2]])     # h0 = 0: no heave velocity
    assert np.allclose(dg.residual(u, mu0, None), r, atol=1e-15)
