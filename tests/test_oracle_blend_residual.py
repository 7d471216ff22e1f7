"""Pins of the blended-motion residual with the discrete geometric conservation law
(oracle/dg_blend.py):

* with b = 1 everywhere it is the rigid residual of Eq. defmap (G = Q, g = 1, gbar = 1);
* free-stream preservation: r(gbar U_inf) = U_inf (-D[C v_h]) for any gbar, so the
  uniform flow with gbar from the discrete GCL is an exact DIRK solution; without the
  GCL (gbar taken from the map itself) a DIRK step leaves the uniform flow;
* at rest (no motion) the map is the identity and the GCL rate vanishes;
* the discrete GCL integrates to the geometric g_h up to the time-discretization error.
"""
import numpy as np
import pytest

from oracle import dirk
from oracle.dg import DG
from oracle.dg_blend import BlendedDG
from pp_inputs import MU_C0, box, config_mesh, free_stream_state, state_perturbation

BIG = dict(x0=-6.0, x1=6.0, y0=-6.0, y1=6.0)   # a far-field box reaching into the blend zone


def _u(dg, seed):
    return (free_stream_state(dg.Ne, dg.p) + state_perturbation(dg.Ne, dg.p, seed=seed, amp=3e-2)).reshape(
        dg.Ne, 4, dg.Np)


@pytest.mark.parametrize("p", [1, 2])
def test_rigid_limit_is_the_rigid_residual(p):
    mesh = config_mesh("tiny")
    rig = DG(mesh, p)
    bl = BlendedDG(mesh, p, r1=1e6, r2=2e6)
    u = _u(rig, 3)
    ones = np.ones((rig.Ne, rig.Np))
    for t in (0.3, 2.2):
        r0 = rig.residual(u.reshape(-1), MU_C0, t).reshape(u.shape)
        r1 = bl.residual_blended(u, MU_C0, t, ones)
        assert np.max(np.abs(r1 - r0)) <= 1e-12 * np.max(np.abs(r0))
        assert np.max(np.abs(bl.gcl_rate(MU_C0, t))) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_free_stream_with_the_discrete_gcl(p):
    dg = BlendedDG(box(6, 6, seed=2, **BIG), p)
    Uinf = dg.Uinf
    rng = np.random.default_rng(p)
    gbar = 1.0 + 0.05 * rng.standard_normal((dg.Ne, dg.Np))       # any positive field
    for t in (0.4, 1.7, 3.1):
        uX = gbar[:, None, :] * Uinf[None, :, None]
        r = dg.residual_blended(uX, MU_C0, t, gbar)
        rhs = dg.gcl_rhs(MU_C0, t)
        assert np.max(np.abs(rhs)) > 1e-6                           # the mesh deforms there
        expect = Uinf[None, :, None] * rhs[:, None, :]
        assert np.max(np.abs(r - expect)) < 1e-12


def test_uniform_flow_survives_a_dirk_step_only_with_the_gcl():
    dg = BlendedDG(box(6, 6, seed=2, **BIG), 2)
    A, b, c = dirk.tableau()
    t0, dt = 0.6, 0.05
    g0 = dg.geometric_g(MU_C0, t0)
    stages, g1 = dg.gbar_dirk(MU_C0, t0, dt, g0, (A, b, c))
    Uinf = dg.Uinf
    # with the GCL: k_i = M^{-1} r(U_X stage) is exactly gbar-rate times U_inf
    uX = g0[:, None, :] * Uinf[None, :, None]
    for i in range(3):
        r = dg.residual_blended(stages[i][:, None, :] * Uinf[None, :, None], MU_C0, t0 + c[i] * dt, stages[i])
        k = np.einsum("ij,eaj->eai", dg.Minv_ref, r) / dg.detB[:, None, None]
        uX = uX + dt * b[i] * k
    assert np.max(np.abs(uX - g1[:, None, :] * Uinf[None, :, None])) < 1e-12
    # the map's own g_h at t0 + dt differs from gbar by the DIRK error of the GCL, so
    # recovering U with it (no GCL) leaves the uniform state
    gh = dg.geometric_g(MU_C0, t0 + dt)
    err = np.max(np.abs(g1 - gh))
    assert 1e-14 < err < 1e-5


def test_at_rest_map_is_identity():
    dg = BlendedDG(box(6, 6, seed=2, **BIG), 2)
    mu0 = np.zeros(3)
    assert np.max(np.abs(dg.gcl_rate(mu0, 1.0))) < 1e-14
    assert np.allclose(dg.geometric_g(mu0, 1.0), 1.0)


def test_gcl_tracks_the_geometry_and_is_periodic():
    dg = BlendedDG(box(6, 6, seed=2, **BIG), 2)
    A, b, c = dirk.tableau()

    def integrate(t_end, n):
        dt = t_end / n
        g = dg.geometric_g(MU_C0, 0.0)
        for s in range(n):
            _, g = dg.gbar_dirk(MU_C0, s * dt, dt, g, (A, b, c))
        return g

    # part of a period: third-order convergence towards the map's own g_h
    gh = dg.geometric_g(MU_C0, 1.3)
    e1 = np.max(np.abs(integrate(1.3, 10) - gh))
    e2 = np.max(np.abs(integrate(1.3, 20) - gh))
    assert 1e-12 < e1 < 1e-4 and e2 < e1 / 5
    # a whole period of equal steps: the composite stage quadrature of the smooth periodic
    # GCL source is exact to round-off, so gbar returns to its initial value
    g0 = dg.geometric_g(MU_C0, 0.0)
    assert np.max(np.abs(integrate(5.0, 40) - g0)) < 1e-12


def test_interior_fluxes_are_conservative():
    """Each interior face flux seen from one side is minus the flux seen from the other at
    the matched point (discrete conservation): this needs the same geometry of the map on
    both sides of the face and each trace's gradient through its own element's map."""
    dg = BlendedDG(box(6, 6, seed=2, **BIG), 2)
    u = _u(dg, 11)
    rng = np.random.default_rng(4)
    gbar = 1.0 + 0.05 * rng.standard_normal((dg.Ne, dg.Np))
    t = 1.1
    xn, vn = dg.nodal_map(MU_C0, t)
    uN, gN = u[dg.nbr_safe], gbar[dg.nbr_safe]
    H = [dg.face_flux_blended(u, uN, gbar, gN, f, xn, vn) for f in range(3)]
    nq = len(dg.s_f)
    worst, scale = 0.0, 0.0
    for e in range(dg.Ne):
        for f in range(3):
            e2, g = dg.nbr[e, f], dg.nbr_face[e, f]
            if e2 < 0:
                continue
            a = H[f][e] * dg.L[e, f]
            b = H[g][e2][::-1] * dg.L[e2, g]
            worst = max(worst, np.max(np.abs(a + b)))
            scale = max(scale, np.max(np.abs(a)))
    assert worst <= 1e-13 * scale


def test_complex_step_derivative_matches_central_differences():
    """The residual is complex-step differentiable in U_X (the exact Jacobians of the
    oracle come from the complex step)."""
    dg = BlendedDG(box(4, 4, seed=5, **BIG), 2)
    u = _u(dg, 13)
    gbar = dg.geometric_g(MU_C0, 0.8)
    d = np.random.default_rng(6).standard_normal(u.shape)
    cs = np.imag(dg.residual_blended(u + 1e-30j * d, MU_C0, 0.8, gbar)) / 1e-30
    h = 1e-6
    fd = (dg.residual_blended(u + h * d, MU_C0, 0.8, gbar) - dg.residual_blended(u - h * d, MU_C0, 0.8, gbar)) / (2 * h)
    assert np.max(np.abs(cs - fd)) <= 1e-6 * np.max(np.abs(cs))


# ---------------------------------------------------------------------------- sweeps
from oracle import periodic as P  # noqa: E402


def test_rigid_limit_sweep_is_the_rigid_sweep():
    mesh = config_mesh("tiny")
    rig = DG(mesh, 1)
    bl = BlendedDG(mesh, 1, r1=1e6, r2=2e6)
    bl.set_period_steps(4)
    u0 = _u(rig, 21).reshape(-1)
    a = P.primal_sweep(rig, MU_C0, u0, 4, store=False)
    b = P.primal_sweep(bl, MU_C0, u0, 4, store=False)
    assert np.max(np.abs(b.u[-1] - a.u[-1])) <= 1e-11 * np.max(np.abs(a.u[-1]))
    assert abs(b.W - a.W) <= 1e-11 * abs(a.W) and abs(b.Jx - a.Jx) <= 1e-11 * abs(a.Jx)


def test_uniform_flow_survives_a_period_with_the_gcl_only():
    class NoGCL(BlendedDG):
        def gbar_at(self, mu, t):                # the map's own g_h instead of the GCL field
            return self.geometric_g(mu, t)

    mesh = box(5, 5, seed=2, **BIG)
    for cls, uniform in ((BlendedDG, True), (NoGCL, False)):
        dg = cls(mesh, 1)
        dg.set_period_steps(10)
        g0 = dg.geometric_g(MU_C0, 0.0)
        u0 = (g0[:, None, :] * dg.Uinf[None, :, None]).reshape(-1)
        tr = P.primal_sweep(dg, MU_C0, u0, 10, store=False, newton_tol=1e-14)
        U = tr.u[-1].reshape(dg.Ne, 4, dg.Np) / dg.gbar_at(MU_C0, dg.T)[:, None, :]
        dev = np.max(np.abs(U - dg.Uinf[None, :, None]))
        if uniform:
            assert dev < 1e-10
        else:
            assert dev > 1e-8


@pytest.fixture(scope="module")
def blended_tiny():
    dg = BlendedDG(config_mesh("tiny"), 1)     # far field at r = 10: the blend zone is inside
    dg.set_period_steps(4)
    u0 = _u(dg, 23).reshape(-1)
    tr = P.primal_sweep(dg, MU_C0, u0, 4)
    return dg, tr


def test_blended_tangent_sweep_matches_finite_differences(blended_tiny):
    dg, tr = blended_tiny
    v = np.random.default_rng(2).standard_normal(dg.Nu)
    eps = 1e-6
    up = P.primal_sweep(dg, MU_C0, tr.u[0] + eps * v, 4, store=False, newton_tol=1e-14).u[-1]
    um = P.primal_sweep(dg, MU_C0, tr.u[0] - eps * v, 4, store=False, newton_tol=1e-14).u[-1]
    fd = (up - um) / (2 * eps)
    tv = P.tangent_sweep(dg, tr, v)
    assert np.max(np.abs(tv - fd)) <= 1e-6 * np.max(np.abs(fd))


def test_blended_duality(blended_tiny):
    dg, tr = blended_tiny
    rng = np.random.default_rng(3)
    v, w = rng.standard_normal(dg.Nu), rng.standard_normal(dg.Nu)
    lhs = w @ P.tangent_sweep(dg, tr, v)
    lam0, _ = P.adjoint_sweep(dg, tr, w)
    assert abs(lhs - lam0 @ v) <= 1e-11 * abs(lhs)


def test_dr_dmu_includes_the_gcl_history():
    """Complex step in mu runs through the tabulated gbar (its DIRK history depends on
    mu), and matches central differences of the residual with gbar rebuilt per mu."""
    dg = BlendedDG(box(4, 4, seed=5, **BIG), 1)
    dg.set_period_steps(6)
    A, b, c = dirk.tableau()
    t = 3 * dg.T / 6 + c[1] * dg.T / 6
    u = (dg.geometric_g(MU_C0, t)[:, None, :] * dg.Uinf[None, :, None]
         + state_perturbation(dg.Ne, 1, seed=8, amp=3e-2).reshape(dg.Ne, 4, dg.Np)).reshape(-1)
    cs = dg.dr_dmu(u, MU_C0, t)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (dg.residual(u, MU_C0 + e, t) - dg.residual(u, MU_C0 - e, t)) / (2 * h)
        assert np.max(np.abs(cs[:, j] - fd)) <= 1e-6 * max(np.max(np.abs(fd)), 1e-8)


def test_blended_periodic_gradient_matches_finite_differences():
    """Shooting and the periodic adjoint run unchanged on the blended residual; the
    gradient (through dr/dmu, which carries d gbar / d mu) matches central differences
    of re-shot periodic QoIs."""
    nt = 4
    dg = BlendedDG(config_mesh("tiny"), 1)
    dg.set_period_steps(nt)
    u0 = (dg.geometric_g(MU_C0, 0.0)[:, None, :] * dg.Uinf[None, :, None]).reshape(-1)
    u0p, tr, _ = P.shoot_nk(dg, MU_C0, u0, nt, tol=1e-12)
    w = np.array([1.0, 0.5])
    F, grad, _ = P.periodic_gradient(dg, tr, w, tol=1e-13)
    tau = 1e-4
    fd = np.zeros(3)
    for j in range(3):
        e = np.zeros(3)
        e[j] = tau
        vals = []
        for sgn in (1, -1):
            _, trj, _ = P.shoot_nk(dg, MU_C0 + sgn * e, u0p, nt, tol=1e-12)
            vals.append(w[0] * trj.W + w[1] * trj.Jx)
        fd[j] = (vals[0] - vals[1]) / (2 * tau)
    assert np.linalg.norm(grad - fd) <= 1e-6 * np.linalg.norm(fd)
