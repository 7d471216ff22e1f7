"""Three-stage, third-order, L-stable DIRK scheme (oracle).

The paper uses "a third-order diagonally implicit Runge-Kutta" scheme without
printing its tableau (Sec. 6.1).  Reading adopted: Alexander's (1977)
stiffly accurate 3-stage scheme.  gamma is the root in (1/6, 1/2) of
gamma^3 - 3 gamma^2 + (3/2) gamma - 1/6 = 0; c = (gamma, (1+gamma)/2, 1);
a21 = (1-gamma)/2; a31 = b1 = -(6 gamma^2 - 16 gamma + 1)/4;
a32 = b2 = (6 gamma^2 - 20 gamma + 5)/4; a33 = b3 = gamma.

The stepping rule follows Eqs. dirk / dirk-stage:
u^(n) = u^(n-1) + sum_i b_i k_i,  M k_i = dt r(u_i, t_{n-1} + c_i dt),
u_i = u^(n-1) + sum_{j<=i} a_ij k_j.
"""
import numpy as np


def alexander_gamma():
    roots = np.roots([1.0, -3.0, 1.5, -1.0 / 6.0])
    real = [r.real for r in roots if abs(r.imag) < 1e-12 and 1.0 / 6.0 < r.real < 0.5]
    assert len(real) == 1
    return float(real[0])


def tableau():
    g = alexander_gamma()
    b1 = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0
    b2 = (6.0 * g * g - 20.0 * g + 5.0) / 4.0
    A = np.array([[g, 0.0, 0.0],
                  [(1.0 - g) / 2.0, g, 0.0],
                  [b1, b2, g]])
    b = np.array([b1, b2, g])
    c = np.array([g, (1.0 + g) / 2.0, 1.0])
    return A, b, c


def dirk_step_scalar(f, dfdy, y, t, dt, A=None, b=None, c=None, newton_tol=1e-15):
    """One DIRK step of the scalar ODE y' = f(y, t) (M = 1), Newton per stage."""
    if A is None:
        A, b, c = tableau()
    s = len(b)
    k = np.zeros(s)
    for i in range(s):
        base = y + sum(A[i, j] * k[j] for j in range(i))
        ki = k[i - 1] if i > 0 else dt * f(y, t)
        for _ in range(50):
            yi = base + A[i, i] * ki
            R = ki - dt * f(yi, t + c[i] * dt)
            dR = 1.0 - A[i, i] * dt * dfdy(yi, t + c[i] * dt)
            d = R / dR
            ki -= d
            if abs(d) <= newton_tol * max(1.0, abs(ki)):
                break
        k[i] = ki
    return y + float(np.dot(b, k))
