"""Sweeps, shooting and the periodic adjoint on top of the DG oracle.

Plain, step-by-step statements of Sec. 3-4 of the paper:

* ``primal_sweep``   -- u^(Nt)(u0; mu) by DIRK with exact Newton per stage and a
                        sparse direct solve (Eq. dirk2); stores the stage states
                        and the stage matrices M - a_ii dt dr/du at the converged
                        stages, and accumulates the discrete QoIs
                        W = sum_n dt sum_i b_i P^h(u_i^(n)), J_x likewise
                        (solver-consistent, Eq. qoi-disc).
* ``tangent_sweep``  -- (du^(Nt)/du0) v (Eq. dirk-sens-mvp).
* ``adjoint_sweep``  -- lambda^(0)(lambda_Nt) of Eq. uns-disc-adj-dirk2 with or
                        without the QoI terms; with them it also accumulates
                        dF/dmu of Eq. funcl-grad-nosens-dirk.
* ``shoot_nk``       -- Newton-Krylov shooting (Algorithm primal, with the
                        linear system (du^(Nt)/du0 - I) du = R, the reading of
                        Eq. jac-prim).
* ``periodic_adjoint`` / ``periodic_gradient`` -- Algorithm dual / Algorithm grad.
* ``shoot_fixed_point`` -- Algorithm fixedpt; ``shoot_nk(m_pre=m)`` -- Newton-Krylov
                        after m fixed-point steps (the nonlinear preconditioning of
                        Sec. 6.1); ``periodic_adjoint_fixed_point`` -- the dual fixed
                        point on Eq. fixedpt-dual.

The QoI functional is F = w_W W + w_x J_x for weights (w_W, w_x).  F depends
on the stages only, so dF/du^(Nt) = 0 and the periodic adjoint condition
lambda^(Nt) = lambda^(0) + dF/du^(Nt) reads lambda^(0)(lambda_Nt) = lambda_Nt.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .dirk import tableau


@dataclass
class Trajectory:
    mu: np.ndarray
    Nt: int
    dt: float
    u: list = field(default_factory=list)        # u^(0..Nt)
    ustage: list = field(default_factory=list)   # [n][i] stage states u_i^(n)
    tstage: list = field(default_factory=list)
    J: list = field(default_factory=list)        # [n][i] dr/du at the converged stage
    lu: list = field(default_factory=list)       # [n][i] factorization of M - a_ii dt J
    W: float = 0.0
    Jx: float = 0.0
    newton_its: list = field(default_factory=list)


def _stage_newton(dg, M, base, k, aii, dt, mu, t, tol, maxit):
    """Newton on R(k) = M k - dt r(base + a_ii k) = 0.  The Jacobian is refreshed
    every third iteration (the converged k does not depend on this)."""
    its = 0
    lu = None
    prev = np.inf
    for its in range(1, maxit + 1):
        ui = base + aii * k
        R = M @ k - dt * dg.residual(ui, mu, t)
        if lu is None or its % 3 == 0:
            lu = spla.splu((M - aii * dt * dg.jacobian(ui, mu, t)).tocsc())
        dk = lu.solve(R)
        k = k - dk
        scale = max(1.0, np.max(np.abs(ui)))
        step = np.max(np.abs(dk))
        if step <= tol * scale:
            break
        if step <= 1e-11 * scale and step >= 0.5 * prev:  # stagnated at round-off
            break
        prev = step
    else:
        raise RuntimeError("oracle stage Newton did not converge")
    return k, its


def primal_sweep(dg, mu, u0, Nt, store=True, newton_tol=1e-13, newton_maxit=30):
    A, b, c = tableau()
    s = len(b)
    dt = dg.T / Nt
    M = dg.mass()
    tr = Trajectory(mu=np.asarray(mu, dtype=np.float64), Nt=Nt, dt=dt)
    u = np.array(u0, dtype=np.float64).reshape(-1)
    tr.u.append(u.copy())
    k_prev = np.zeros_like(u)
    for n in range(1, Nt + 1):
        t0 = (n - 1) * dt
        ks, us, ts, Js, lus = [], [], [], [], []
        for i in range(s):
            ti = t0 + c[i] * dt
            base = u + sum(A[i, j] * ks[j] for j in range(i))
            k0 = ks[i - 1] if i > 0 else k_prev
            k, its = _stage_newton(dg, M, base, k0.copy(), A[i, i], dt, mu, ti, newton_tol, newton_maxit)
            tr.newton_its.append(its)
            ui = base + A[i, i] * k
            ks.append(k)
            us.append(ui)
            ts.append(ti)
            pw, fx = dg.qoi_rate(ui, mu, ti)
            tr.W += dt * b[i] * float(pw)
            tr.Jx += dt * b[i] * float(fx)
            if store:
                Ji = dg.jacobian(ui, mu, ti)
                Js.append(Ji)
                lus.append(spla.splu((M - A[i, i] * dt * Ji).tocsc()))
        u = u + sum(b[i] * ks[i] for i in range(s))
        k_prev = ks[-1]
        tr.u.append(u.copy())
        tr.ustage.append(us)
        tr.tstage.append(ts)
        if store:
            tr.J.append(Js)
            tr.lu.append(lus)
    return tr


def tangent_sweep(dg, tr, v):
    """(du^(Nt)/du0) v by the linear evolution of Eq. dirk-sens-mvp."""
    A, b, c = tableau()
    s = len(b)
    dt = tr.dt
    du = np.array(v, dtype=np.float64).reshape(-1)
    for n in range(tr.Nt):
        dks = []
        for i in range(s):
            w = du + sum(A[i, j] * dks[j] for j in range(i))
            dks.append(tr.lu[n][i].solve(dt * (tr.J[n][i] @ w)))
        du = du + sum(b[i] * dks[i] for i in range(s))
    return du


def _qoi_terms(dg, tr, n, weights):
    """g_l = w . d(P^h, F_x^h)/du at the stages of step n (row vectors as arrays)."""
    return [weights @ dg.dqoi_du(tr.ustage[n][i], tr.mu, tr.tstage[n][i]) for i in range(len(tr.ustage[n]))]


def adjoint_sweep(dg, tr, lam_Nt, weights=None):
    """lambda^(0)(lambda_Nt) of Eq. uns-disc-adj-dirk2.

    weights=None gives the adjoint sensitivity sweep (Eq.
    uns-disc-adj-dirk-sens-mvp, no QoI terms).  With weights, the QoI terms are
    included and dF/dmu (Eq. funcl-grad-nosens-dirk) is returned as well.
    """
    A, b, c = tableau()
    s = len(b)
    dt = tr.dt
    lam = np.array(lam_Nt, dtype=np.float64).reshape(-1)
    grad = None
    if weights is not None:
        weights = np.asarray(weights, dtype=np.float64)
        grad = np.zeros(len(tr.mu))
    for n in range(tr.Nt - 1, -1, -1):
        g = _qoi_terms(dg, tr, n, weights) if weights is not None else None
        kap = [None] * s
        for i in range(s - 1, -1, -1):
            rhs = b[i] * lam
            for j in range(i + 1, s):
                rhs = rhs + A[j, i] * dt * (tr.J[n][j].T @ kap[j])
            if g is not None:
                # dF/dk_i = dt sum_{l>=i} b_l a_li g_l
                rhs = rhs + dt * sum(b[l] * A[l, i] * g[l] for l in range(i, s))
            kap[i] = tr.lu[n][i].solve(rhs, trans="T")
        lam_prev = lam + sum(dt * (tr.J[n][i].T @ kap[i]) for i in range(s))
        if g is not None:
            lam_prev = lam_prev + dt * sum(b[l] * g[l] for l in range(s))  # dF/du^(n-1)
            for i in range(s):
                grad += dt * (kap[i] @ dg.dr_dmu(tr.ustage[n][i], tr.mu, tr.tstage[n][i]))
                grad += dt * b[i] * (weights @ dg.dqoi_dmu(tr.ustage[n][i], tr.mu, tr.tstage[n][i]))
        lam = lam_prev
    return lam, grad


def gmres(matvec, rhs, x0=None, tol=1e-10, restart=50, maxit=1000):
    """Restarted GMRES with modified Gram-Schmidt Arnoldi (Algorithm dual), absolute
    tolerance on ||rhs - A x||_2.  Returns (x, number of matvecs, residual history)."""
    n = len(rhs)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    hist = []
    nmv = 0
    while True:
        r = rhs - matvec(x) if np.any(x) else rhs.copy()
        nmv += int(np.any(x))
        beta = np.linalg.norm(r)
        hist.append(beta)
        if beta <= tol or nmv >= maxit:
            return x, nmv, hist
        V = [r / beta]
        H = np.zeros((restart + 1, restart))
        for j in range(restart):
            w = matvec(V[j])
            nmv += 1
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)
            hist.append(res)
            if res <= tol or H[j + 1, j] == 0.0 or nmv >= maxit:
                break
            V.append(w / H[j + 1, j])
        x = x + np.stack(V[:len(y)], 1) @ y
        if res <= tol or nmv >= maxit:
            return x, nmv, hist


def shoot_fixed_point(dg, mu, u0, Nt, tol=1e-10, maxit=500):
    """Algorithm fixedpt: u0 <- u^(Nt)(u0) until ||u^(Nt)(u0) - u0||_2 <= tol (Eq. fixedpt).
    Returns (u0, trajectory from u0, residual history)."""
    u0 = np.array(u0, dtype=np.float64).reshape(-1)
    history = []
    for _ in range(maxit + 1):
        tr = primal_sweep(dg, mu, u0, Nt)
        rn = np.linalg.norm(tr.u[-1] - u0)
        history.append(rn)
        if rn <= tol:
            return u0, tr, history
        u0 = tr.u[-1].copy()
    raise RuntimeError("oracle fixed-point iteration did not converge")


def shoot_nk(dg, mu, u0, Nt, tol=1e-10, gmres_rtol=1e-8, max_newton=30, m_pre=0):
    """Algorithm primal: Newton on R(u0) = u^(Nt)(u0) - u0 with matrix-free GMRES.  m_pre > 0
    first takes m_pre steps of Algorithm fixedpt (u0 <- u^(Nt)(u0)), the nonlinear
    preconditioning of Sec. 6.1."""
    u0 = np.array(u0, dtype=np.float64).reshape(-1)
    for _ in range(m_pre):
        u0 = primal_sweep(dg, mu, u0, Nt, store=False).u[-1].copy()
    history = []
    for _ in range(max_newton + 1):
        tr = primal_sweep(dg, mu, u0, Nt)
        R = tr.u[-1] - u0
        rn = np.linalg.norm(R)
        history.append(rn)
        if rn <= tol:
            return u0, tr, history
        du, _, _ = gmres(lambda v: tangent_sweep(dg, tr, v) - v, R, tol=gmres_rtol * rn)
        u0 = u0 - du
    raise RuntimeError("oracle Newton-Krylov shooting did not converge")


def periodic_adjoint(dg, tr, weights, tol=1e-12):
    """Algorithm dual: solve lambda^(0)(lambda_Nt) = lambda_Nt for lambda_Nt.

    lambda^(0)(x) = Phi^T x + d with d = lambda^(0)(0) (QoI terms on), so the
    system is (Phi^T - I) x = -d, solved by GMRES with adjoint sensitivity sweeps.
    """
    d, _ = adjoint_sweep(dg, tr, np.zeros(dg.Nu), weights)
    x, _, _ = gmres(lambda v: adjoint_sweep(dg, tr, v)[0] - v, -d, tol=tol)
    return x


def periodic_adjoint_fixed_point(dg, tr, weights, tol=1e-12, maxit=2000):
    """The periodic adjoint condition (Eq. fixedpt-dual, with dF/du^(Nt) = 0 here) solved by
    fixed-point iteration x <- lambda^(0)(x), from x = 0.  Returns (x, residual history)."""
    x = np.zeros(dg.Nu)
    history = []
    for _ in range(maxit + 1):
        y, _ = adjoint_sweep(dg, tr, x, weights)
        rn = np.linalg.norm(y - x)
        history.append(rn)
        if rn <= tol:
            return x, history
        x = y
    raise RuntimeError("oracle dual fixed-point iteration did not converge")


def periodic_gradient(dg, tr, weights, tol=1e-12):
    """Algorithm grad on an already periodic trajectory: returns (F, dF/dmu, lambda_Nt)."""
    w = np.asarray(weights, dtype=np.float64)
    lam = periodic_adjoint(dg, tr, w, tol)
    _, grad = adjoint_sweep(dg, tr, lam, w)
    F = w[0] * tr.W + w[1] * tr.Jx
    return F, grad, lam


def dense_phi(dg, tr):
    """Brute force du^(Nt)/du0, one tangent sweep per column (tiny meshes only)."""
    n = dg.Nu
    return np.stack([tangent_sweep(dg, tr, np.eye(n)[:, j]) for j in range(n)], 1)


def dense_phi_T(dg, tr):
    """Brute force d lambda^(0)/d lambda_Nt, one adjoint sensitivity sweep per column."""
    n = dg.Nu
    return np.stack([adjoint_sweep(dg, tr, np.eye(n)[:, j])[0] for j in range(n)], 1)


def steady_state(dg, mu, u0, tol=1e-12, maxit=200, dtau0=0.1, dtau_max=1e4):
    """Steady flow at the t = 0 pose with the mesh at rest (the paper's cold start, Sec. 6.1),
    by pseudo-transient continuation: backward-Euler pseudo steps (M - dtau J) du = dtau r(u)
    with the pseudo step grown by the residual ratio (switched evolution relaxation) and cut
    on a rejected step.  Stops when ||r|| <= tol ||r(u0)||."""
    M = dg.mass()
    u = np.array(u0, dtype=np.float64).reshape(-1)
    r = dg.residual(u, mu, None)
    rn0 = rn = np.linalg.norm(r)
    dtau = dtau0
    for it in range(maxit):
        if rn <= tol * rn0:
            return u, it, rn / rn0
        A = (M - dtau * dg.jacobian(u, mu, None)).tocsc()
        du = spla.splu(A).solve(dtau * r)
        ut = u + du
        rt = dg.residual(ut, mu, None)
        rnt = np.linalg.norm(rt)
        if np.isfinite(rnt) and rnt < 2.0 * rn:
            dtau = min(dtau * min(max(rn / rnt, 0.5), 4.0), dtau_max)
            u, r, rn = ut, rt, rnt
        else:
            dtau *= 0.25
    raise RuntimeError("oracle pseudo-transient continuation did not converge")
