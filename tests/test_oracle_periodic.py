"""Pins for the oracle's sweeps, shooting and periodic adjoint on the tiny
O-grid (32 triangles, p = 1, 8 DIRK3 steps): tangent sweep vs finite
differences of the period map, tangent/adjoint duality (App. A), quadratic
Newton-Krylov convergence (Algorithm primal), the periodic adjoint vs a dense
solve with brute-force Phi^T, Floquet stability of the orbit (Sec. 3.3), and the
periodic gradient vs central differences of re-shot periodic QoIs (Sec. 6.2
protocol)."""
import numpy as np
import pytest

from oracle import periodic as P
from pp_inputs import CONFIGS, MU_C0, free_stream_state

NT = CONFIGS["tiny"]["Nt"]


@pytest.fixture(scope="module")
def periodic(tiny_dg):
    u0 = free_stream_state(tiny_dg.Ne, tiny_dg.p).reshape(-1)
    u0p, tr, hist = P.shoot_nk(tiny_dg, MU_C0, u0, NT, tol=1e-12)
    return u0p, tr, hist


def test_tangent_sweep_matches_central_differences(tiny_dg, periodic):
    u0p, tr, _ = periodic
    v = np.random.default_rng(1).standard_normal(tiny_dg.Nu)
    eps = 1e-5
    up = P.primal_sweep(tiny_dg, MU_C0, u0p + eps * v, NT, store=False, newton_tol=1e-15).u[-1]
    um = P.primal_sweep(tiny_dg, MU_C0, u0p - eps * v, NT, store=False, newton_tol=1e-15).u[-1]
    fd = (up - um) / (2 * eps)
    assert np.linalg.norm(P.tangent_sweep(tiny_dg, tr, v) - fd) <= 1e-6 * np.linalg.norm(fd)


def test_tangent_adjoint_duality(tiny_dg, periodic):
    _, tr, _ = periodic
    rng = np.random.default_rng(2)
    for _ in range(3):
        v, w = rng.standard_normal(tiny_dg.Nu), rng.standard_normal(tiny_dg.Nu)
        a = w @ P.tangent_sweep(tiny_dg, tr, v)
        b = P.adjoint_sweep(tiny_dg, tr, w)[0] @ v
        assert abs(a - b) <= 1e-12 * abs(a)


def test_shooting_converges_quadratically(periodic):
    u0p, tr, hist = periodic
    assert hist[-1] <= 1e-12
    assert np.linalg.norm(tr.u[-1] - u0p) <= 1e-12
    # quadratic contraction r_{k+1} <= C r_k^2 before the round-off floor is reached
    r = hist
    assert len(r) >= 3
    assert r[-2] <= 1.0 * r[-3] ** 2


def test_periodic_adjoint_matches_dense_solve_and_orbit_is_stable(tiny_dg, periodic):
    _, tr, _ = periodic
    Phi = P.dense_phi(tiny_dg, tr)
    PhiT = P.dense_phi_T(tiny_dg, tr)
    assert np.allclose(PhiT, Phi.T, atol=1e-12 * np.abs(Phi).max())
    w = np.array([1.0, 0.3])
    lam = P.periodic_adjoint(tiny_dg, tr, w, tol=1e-13)
    d, _ = P.adjoint_sweep(tiny_dg, tr, np.zeros(tiny_dg.Nu), w)
    lam_dense = np.linalg.solve(Phi.T - np.eye(tiny_dg.Nu), -d)
    assert np.linalg.norm(lam - lam_dense) <= 1e-9 * np.linalg.norm(lam_dense)
    # periodic adjoint condition lambda^(0)(lambda_Nt) = lambda_Nt
    lam0, _ = P.adjoint_sweep(tiny_dg, tr, lam, w)
    assert np.linalg.norm(lam0 - lam) <= 1e-10 * np.linalg.norm(lam)
    # Floquet multipliers of the periodic orbit inside the unit circle (Sec. 3.3)
    assert np.max(np.abs(np.linalg.eigvals(Phi))) < 1.0


@pytest.mark.slow
def test_periodic_gradient_matches_finite_differences(tiny_dg, periodic):
    u0p, tr, _ = periodic
    w = np.array([1.0, 0.5])
    F, grad, _ = P.periodic_gradient(tiny_dg, tr, w, tol=1e-13)
    tau = 1e-4
    fd = np.zeros(3)
    for j in range(3):
        e = np.zeros(3)
        e[j] = tau
        vals = []
        for sgn in (1, -1):
            _, trj, _ = P.shoot_nk(tiny_dg, MU_C0 + sgn * e, u0p, NT, tol=1e-12)
            vals.append(w[0] * trj.W + w[1] * trj.Jx)
        fd[j] = (vals[0] - vals[1]) / (2 * tau)
    assert np.linalg.norm(grad - fd) <= 1e-6 * np.linalg.norm(fd)
