"""Geometry of the rigid-plus-blended mesh motion (oracle; test infrastructure only).

The paper moves the whole mesh rigidly with the airfoil (Eq. defmap).  The blended
variant keeps that motion near the airfoil and lets it decay to rest towards the far
field:

    x(X, t) = X + b(r) d(X, t),   d = v(t) + (Q(t) - I)(X - x0),   r = |X - x0|,

with v = (0, h) the heave, Q the pitch rotation about x0 = (1/3, 0), and b a C^2 step
(b = 1 for r <= r1, b = 0 for r >= r2, the quintic smoothstep in between).  Inside r1
it is exactly the rigid map of Eq. defmap.  For the ALE form of the equations on the
reference domain the solver needs, at any reference point,

    G = grad_X x = I + d (grad_X b)^T + b (Q - I),   g = det G,
    g G^{-1} (the cofactor matrix, polynomial in G),  v_X = dx/dt|_X = b (v' + Q' (X - x0)).

Unlike the rigid map, g is not 1 and varies in space and time, so a discretization
must satisfy the geometric conservation law dg/dt = div_X(g G^{-1} v_X) discretely to
keep a uniform flow uniform.  The functions here are the exact geometry (no
discretization), checked against finite differences, the Piola identity and that law.
"""
import numpy as np

X0 = np.array([1.0 / 3.0, 0.0])


def blend_weight(r, r1=2.0, r2=8.0):
    """b(r) and db/dr: 1 inside r1, 0 outside r2, 1 - s^3 (10 - 15 s + 6 s^2) between,
    s = (r - r1) / (r2 - r1) (value, slope and curvature continuous at both ends)."""
    s = np.clip((np.asarray(r, dtype=float) - r1) / (r2 - r1), 0.0, 1.0)
    b = 1.0 - s**3 * (10.0 - 15.0 * s + 6.0 * s * s)
    db = -30.0 * s * s * (1.0 - s) ** 2 / (r2 - r1)
    return b, db


def rotation(theta):
    """Q(theta) in the convention of the oracle's rigid frame."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, s], [-s, c]])


def rotation_rate(theta, thetadot):
    c, s = np.cos(theta), np.sin(theta)
    return thetadot * np.array([[-s, c], [-c, -s]])


def blended_map(X, h, theta, hdot, thetadot, r1=2.0, r2=8.0):
    """x, G, g, g G^{-1}, v_X at reference points X [..., 2] for heave h, pitch theta
    and their rates."""
    X = np.asarray(X, dtype=float)
    Q, Qd = rotation(theta), rotation_rate(theta, thetadot)
    y = X - X0
    r = np.hypot(y[..., 0], y[..., 1])
    b, db = blend_weight(r, r1, r2)
    v = np.array([0.0, h])
    d = v + np.einsum("ij,...j->...i", Q - np.eye(2), y)
    x = X + b[..., None] * d
    with np.errstate(invalid="ignore", divide="ignore"):
        gradb = np.where(r[..., None] > 0, db[..., None] * y / r[..., None], 0.0)
    G = np.eye(2) + d[..., :, None] * gradb[..., None, :] + b[..., None, None] * (Q - np.eye(2))
    g = G[..., 0, 0] * G[..., 1, 1] - G[..., 0, 1] * G[..., 1, 0]
    cof = np.stack([np.stack([G[..., 1, 1], -G[..., 0, 1]], -1),
                    np.stack([-G[..., 1, 0], G[..., 0, 0]], -1)], -2)   # g G^{-1}
    vX = b[..., None] * (np.array([0.0, hdot]) + np.einsum("ij,...j->...i", Qd, y))
    return x, G, g, cof, vX
