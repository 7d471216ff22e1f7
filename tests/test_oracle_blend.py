"""Pins of the blended-motion geometry (oracle/blend.py): the rigid map of Eq. defmap
inside r1, rest outside r2, G and v_X against finite differences of x, the Piola
identity div_X(g G^{-1}) = 0 and the geometric conservation law
dg/dt = div_X(g G^{-1} v_X) (Euler's expansion formula), and g > 0 for the motion
amplitudes of the workloads."""
import numpy as np

from oracle import blend as B

H0, TH0, PHI, OMEGA = 0.1, np.radians(5.0), np.pi / 2, 2 * np.pi / 5.0


def motion(t, scale=1.0):
    h = scale * H0 * np.sin(OMEGA * t)
    th = scale * TH0 * np.sin(OMEGA * t + PHI)
    return h, th, scale * H0 * OMEGA * np.cos(OMEGA * t), scale * TH0 * OMEGA * np.cos(OMEGA * t + PHI)


def points(n=400, seed=0, rmax=9.0):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.05, rmax, n)
    a = rng.uniform(0, 2 * np.pi, n)
    return B.X0 + np.stack([r * np.cos(a), r * np.sin(a)], -1)


def test_weight_is_a_c2_step():
    b, db = B.blend_weight(np.array([0.0, 2.0, 8.0, 9.0]))
    assert np.allclose(b, [1, 1, 0, 0]) and np.allclose(db, 0)
    r = np.linspace(1.5, 8.5, 7001)
    bb, dbb = B.blend_weight(r)
    h = r[1] - r[0]
    assert np.max(np.abs(np.gradient(bb, h) - dbb)) < 1e-4          # slope is the derivative
    d2 = np.diff(dbb) / h
    assert np.max(np.abs(np.diff(d2))) < 1e-3                          # curvature continuous


def test_rigid_inside_and_at_rest_outside():
    h, th, hd, thd = motion(0.7)
    Q, Qd = B.rotation(th), B.rotation_rate(th, thd)
    X = points(rmax=1.9)
    x, G, g, cof, vX = B.blended_map(X, h, th, hd, thd)
    assert np.allclose(x, np.array([0, h]) + (X - B.X0) @ Q.T + B.X0, atol=1e-14)
    assert np.allclose(G, Q, atol=1e-14) and np.allclose(g, 1.0, atol=1e-14)
    assert np.allclose(vX, np.array([0, hd]) + (X - B.X0) @ Qd.T, atol=1e-14)
    Xo = B.X0 + np.array([[8.5, 0.0], [0.0, -9.0], [-6.0, 6.0]])
    x, G, g, cof, vX = B.blended_map(Xo, h, th, hd, thd)
    assert np.allclose(x, Xo) and np.allclose(G, np.eye(2)) and np.allclose(vX, 0.0)


def test_jacobian_and_velocity_match_finite_differences():
    X = points(seed=1)
    t, e, dt = 1.3, 1e-6, 1e-6
    h, th, hd, thd = motion(t)
    x, G, g, cof, vX = B.blended_map(X, h, th, hd, thd)
    for k in range(2):
        dX = np.zeros(2)
        dX[k] = e
        xp = B.blended_map(X + dX, h, th, hd, thd)[0]
        xm = B.blended_map(X - dX, h, th, hd, thd)[0]
        assert np.max(np.abs((xp - xm) / (2 * e) - G[..., :, k])) < 1e-8
    xp = B.blended_map(X, *motion(t + dt)[:2], hd, thd)[0]
    xm = B.blended_map(X, *motion(t - dt)[:2], hd, thd)[0]
    assert np.max(np.abs((xp - xm) / (2 * dt) - vX)) < 1e-8
    assert np.allclose(np.einsum("...ij,...jk->...ik", cof, G), g[..., None, None] * np.eye(2), atol=1e-13)


def _div(f, X, e=1e-5):
    """Row-wise divergence of a field f(X) [..., m, 2] (or [..., 2]) by central differences."""
    out = 0.0
    for k in range(2):
        dX = np.zeros(2)
        dX[k] = e
        out = out + (f(X + dX)[..., k] - f(X - dX)[..., k]) / (2 * e)
    return out


def test_piola_identity_and_geometric_conservation_law():
    X = points(seed=2)
    X = X[np.abs(np.hypot(*(X - B.X0).T) - 2.0) > 1e-3]   # away from the C^2 junctions
    X = X[np.abs(np.hypot(*(X - B.X0).T) - 8.0) > 1e-3]
    t, dt = 2.1, 1e-5
    m = motion(t)
    # sum_J d/dX_J (g G^{-1})_{J i} = 0 for each i (divergence over the first index)
    piola = _div(lambda Y: np.swapaxes(B.blended_map(Y, *m)[3], -1, -2), X)
    assert np.max(np.abs(piola)) < 1e-6
    gcl_rhs = _div(lambda Y: np.einsum("...ij,...j->...i", *B.blended_map(Y, *m)[3:5]), X)
    gp = B.blended_map(X, *motion(t + dt))[2]
    gm = B.blended_map(X, *motion(t - dt))[2]
    assert np.max(np.abs((gp - gm) / (2 * dt) - gcl_rhs)) < 1e-6
    assert np.max(np.abs(gcl_rhs)) > 1e-4     # g really varies: the law is not trivially 0 = 0


def test_positive_jacobian_for_the_workload_amplitudes():
    X = points(n=4000, seed=3, rmax=10.0)
    for t in np.linspace(0, 5.0, 11):
        g = B.blended_map(X, *motion(t, scale=1.2))[2]    # +20% of the c0 amplitudes
        assert g.min() > 0.9
