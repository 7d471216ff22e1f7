"""GPU parity at the degrees the benchmark runs: p = 3 (nb = 40) and p = 4 (nb = 60).

The p = 1 tests of test_gpu_parity.py exercise the nb = 12 instantiations only.  Here
the block-row kernels, the block inverse and the folded stage operator at nb = 40 and
nb = 60 are compared with the FP64 oracle on the same seeded inputs:

* the primal trajectory, W and J_x over three steps of the config-1 step size;
* the tangent sweep and the adjoint sweep with and without QoI terms (lambda and dF/dmu);
* every stored stage operator applied to seeded vectors against dense products of the
  oracle's own matrices at its own converged stage (M - cJ, D^-1, (M - cJ) D^-1, and
  their transposes; Eqs. dirk-sens-mvp, uns-disc-adj-dirk2), in FP64 and, in the
  mixed-precision mode, the FP32 copies;
* the checkpointed linearization (stride 1 and stride 0);
* NK shooting and the periodic gradient at p = 3.

Bar: 1e-10 relative (FP64); products through an explicit block inverse add the
inverse's own rounding, of order nb u cond(D) |D^-1| |x| (u = 2^-53).  FP32 copies: the error of an FP32 product of n terms is
at most n u |A| |x| (u = 2^-24), and that of an FP32 Gauss-Jordan inverse of a block
is of order nb u cond(D) |D^-1|; the tests hold the FP32 operators to those bounds with
a factor 4 of slack, computed from the oracle's blocks.
"""
import numpy as np
import pytest

from gpu_common import PARITY_TOL, TIGHT, make, perturbed_state, rel_err, to_dev, to_host
from oracle import periodic as OP
from oracle.dg import DG
from oracle.dirk import tableau
from pp_inputs import (CONFIGS, KIN_FOURIER6, KIN_HEAVE_PITCH, MU_C0, config_mesh, config_mu, free_stream_state,
                       ogrid)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24
U64 = 2.0 ** -53
NT = 3
DT = 0.05            # the config-1 step size (T = 5, 100 steps)
T = NT * DT


def _mu():
    # motion amplitudes scaled with the period so that wall velocities stay those of config 1
    return config_mu("c1") * (T / 5.0)


@pytest.fixture(scope="module", params=[3, 4])
def sweep(request):
    p = request.param
    mesh = ogrid(12, 3, seed=6)
    mu = _mu()
    dg = DG(mesh, p, kin=KIN_FOURIER6, T=T)
    u0 = perturbed_state(dg.Ne, p, seed=60 + p, amp=1e-2)
    tr = OP.primal_sweep(dg, mu, u0, NT, newton_tol=1e-14)
    return dict(p=p, mesh=mesh, mu=mu, dg=dg, u0=u0, tr=tr)


def _ctx(s, **kw):
    return make(s["p"], KIN_FOURIER6, s["mesh"], T=T, **dict(TIGHT, **kw))


def test_primal_tangent_adjoint_parity_highp(sweep):
    s = sweep
    dg, tr = s["dg"], s["tr"]
    A, ctx, m = _ctx(s)
    try:
        traj = torch.zeros((NT + 1) * dg.Nu, dtype=torch.float64, device="cuda")
        qoi = A.pp_primal_period(ctx, m, s["mu"], to_dev(s["u0"]), NT, u_traj=traj)
        traj = to_host(traj).reshape(NT + 1, -1)
        for n in range(NT + 1):
            assert rel_err(traj[n], tr.u[n]) <= PARITY_TOL
        assert abs(qoi[0] - tr.W) <= PARITY_TOL * abs(tr.W)
        assert abs(qoi[1] - tr.Jx) <= PARITY_TOL * abs(tr.Jx)

        rng = np.random.default_rng(70 + s["p"])
        v = rng.standard_normal(dg.Nu)
        out = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        A.pp_tangent_matvec(ctx, to_dev(v), out)
        assert rel_err(to_host(out), v - OP.tangent_sweep(dg, tr, v)) <= PARITY_TOL

        lam = rng.standard_normal(dg.Nu)
        A.pp_adjoint_sweep(ctx, to_dev(lam), out)
        assert rel_err(to_host(out), OP.adjoint_sweep(dg, tr, lam)[0]) <= PARITY_TOL
        w = np.array([1.0, 0.5])
        g = A.pp_adjoint_sweep(ctx, to_dev(lam), out, weights=w, n_mu=6)
        ref_lam, ref_g = OP.adjoint_sweep(dg, tr, lam, w)
        assert rel_err(to_host(out), ref_lam) <= PARITY_TOL
        assert rel_err(g, ref_g) <= PARITY_TOL
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def _oracle_ops(dg, tr, step, i):
    """Dense M - cJ and its block diagonal D at the oracle's converged stage (step, i)."""
    Amat, _, _ = tableau()
    c = Amat[i, i] * tr.dt
    S = (dg.mass() - c * tr.J[step][i]).toarray()
    nb = dg.nb
    D = np.zeros_like(S)
    Dinv = np.zeros_like(S)
    conds = []
    for e in range(dg.Ne):
        sl = slice(e * nb, (e + 1) * nb)
        D[sl, sl] = S[sl, sl]
        Dinv[sl, sl] = np.linalg.inv(S[sl, sl])
        conds.append(np.linalg.cond(S[sl, sl]))
    return S, D, Dinv, max(conds)


def _apply_all(A, ctx, nu, step, i, x, prec):
    out = {}
    xd = to_dev(x)
    for kind in (0, 1, 2):
        for trans in (False, True):
            y = torch.zeros(nu, dtype=torch.float64, device="cuda")
            A.pp_stage_apply(ctx, step, i, kind, xd, y, trans=trans, prec=prec)
            out[kind, trans] = to_host(y)
    return out


def _dense_refs(S, Dinv, x):
    return {(0, False): S @ x, (0, True): S.T @ x, (1, False): Dinv @ x, (1, True): Dinv.T @ x,
            (2, False): S @ (Dinv @ x), (2, True): S.T @ (Dinv.T @ x)}


@pytest.mark.parametrize("stride", [0, 1])
def test_stored_stage_operators_fp64(sweep, stride):
    s = sweep
    dg, tr = s["dg"], s["tr"]
    A, ctx, m = _ctx(s, checkpoint_stride=stride)
    try:
        A.pp_primal_period(ctx, m, s["mu"], to_dev(s["u0"]), NT)
        x = np.random.default_rng(80 + s["p"]).standard_normal(dg.Nu)
        ax = np.abs(x)
        for step, i in ((0, 0), (1, 1), (2, 2)):
            S, _, Dinv, cond = _oracle_ops(dg, tr, step, i)
            got = _apply_all(A, ctx, dg.Nu, step, i, x, 0)
            ref = _dense_refs(S, Dinv, x)
            # explicit FP64 inverses (Gauss-Jordan on the GPU, LAPACK in the oracle) each carry
            # an error of order nb u64 cond(D) |D^-1| on top of the 1e-10 parity of the states
            e_inv = 8 * dg.nb * U64 * cond
            slack = {0: 0.0,
                     1: e_inv * max(np.max(np.abs(Dinv) @ ax), np.max(np.abs(Dinv.T) @ ax)),
                     2: e_inv * max(np.max(np.abs(S) @ (np.abs(Dinv) @ ax)),
                                    np.max(np.abs(S.T) @ (np.abs(Dinv.T) @ ax)))}
            for key in ref:
                err = np.max(np.abs(got[key] - ref[key]))
                assert err <= PARITY_TOL * np.max(np.abs(ref[key])) + slack[key[0]], (step, i, key)
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def test_stored_stage_operators_fp32_copies(sweep):
    s = sweep
    dg, tr = s["dg"], s["tr"]
    A, ctx, m = _ctx(s, precision=1)  # PP_PREC_MIXED
    try:
        A.pp_primal_period(ctx, m, s["mu"], to_dev(s["u0"]), NT)
        x = np.random.default_rng(90 + s["p"]).standard_normal(dg.Nu)
        nb = dg.nb
        for step, i in ((0, 0), (2, 2)):
            S, D, Dinv, cond = _oracle_ops(dg, tr, step, i)
            got = _apply_all(A, ctx, dg.Nu, step, i, x, 1)
            ref = _dense_refs(S, Dinv, x)
            ax = np.abs(x)
            # FP32 products: 4 nb terms per row of M - cJ (x rounded to FP32 as well)
            b0 = 4 * (4 * nb + 1) * U32 * np.max(np.abs(S) @ ax)
            b0t = 4 * (4 * nb + 1) * U32 * np.max(np.abs(S.T) @ ax)
            assert np.max(np.abs(got[0, False] - ref[0, False])) <= b0
            assert np.max(np.abs(got[0, True] - ref[0, True])) <= b0t
            # FP32 inverse: nb u cond(D) |D^-1| |x| per block, then the FP32 product
            e_inv = 4 * nb * U32 * cond
            b1 = e_inv * np.max(np.abs(Dinv) @ ax) + 4 * (nb + 1) * U32 * np.max(np.abs(Dinv) @ ax)
            assert np.max(np.abs(got[1, False] - ref[1, False])) <= b1
            assert np.max(np.abs(got[1, True] - ref[1, True])) <= b1
            # folded: (I + O D^-1) x with O D^-1 formed from the FP32 copies
            O = S - D
            b2 = (e_inv + 4 * (5 * nb + 2) * U32) * np.max(np.abs(O) @ (np.abs(Dinv) @ ax)) + 4 * U32 * np.max(ax)
            b2t = (e_inv + 4 * (5 * nb + 2) * U32) * np.max(np.abs(O.T) @ (np.abs(Dinv.T) @ ax)) \
                + 4 * U32 * np.max(ax)
            assert np.max(np.abs(got[2, False] - ref[2, False])) <= b2
            assert np.max(np.abs(got[2, True] - ref[2, True])) <= b2t
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def test_checkpointed_sweeps_match_stored_highp(sweep):
    """Stride 1 recomputes each step's stage data from its checkpoint with the same
    operations, so tangent and adjoint sweeps agree with the stored linearization to the
    last bit; both match the oracle."""
    s = sweep
    dg, tr = s["dg"], s["tr"]
    v = np.random.default_rng(100 + s["p"]).standard_normal(dg.Nu)
    res = {}
    for stride in (0, 1):
        A, ctx, m = _ctx(s, checkpoint_stride=stride)
        try:
            A.pp_primal_period(ctx, m, s["mu"], to_dev(s["u0"]), NT)
            t = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
            a = torch.zeros_like(t)
            A.pp_tangent_matvec(ctx, to_dev(v), t)
            g = A.pp_adjoint_sweep(ctx, to_dev(v), a, weights=[1.0, 0.5], n_mu=6)
            res[stride] = (to_host(t), to_host(a), np.asarray(g))
        finally:
            A.pp_mesh_destroy(m)
            A.pp_destroy(ctx)
    for k in range(3):
        assert np.array_equal(res[0][k], res[1][k])
    assert rel_err(res[1][0], v - OP.tangent_sweep(dg, tr, v)) <= PARITY_TOL
    ref_lam, ref_g = OP.adjoint_sweep(dg, tr, v, np.array([1.0, 0.5]))
    assert rel_err(res[1][1], ref_lam) <= PARITY_TOL
    assert rel_err(res[1][2], ref_g) <= PARITY_TOL


def test_shooting_and_periodic_gradient_parity_p3():
    """Algorithm primal and Algorithms dual / grad at p = 3 (nb = 40) on the 32-triangle
    O-grid, 8 steps per period, against the oracle's NK shooting and periodic gradient."""
    c = CONFIGS["tiny"]
    mesh = config_mesh("tiny")
    p = 3
    dg = DG(mesh, p, kin=KIN_HEAVE_PITCH)
    u0p, tr, _ = OP.shoot_nk(dg, MU_C0, free_stream_state(dg.Ne, p).reshape(-1), c["Nt"], tol=1e-12)
    w = np.array([1.0, 0.5])
    F, grad, lam = OP.periodic_gradient(dg, tr, w, tol=1e-13)
    A, ctx, m = make(p, KIN_HEAVE_PITCH, mesh, **TIGHT)
    try:
        u0 = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        qoi, st = A.pp_shoot_nk(ctx, m, MU_C0, c["Nt"], 1e-12, u0, u0_guess=to_dev(free_stream_state(dg.Ne, p)))
        assert st["residual"][-1] <= 1e-12
        assert rel_err(to_host(u0), u0p) <= PARITY_TOL
        lt = torch.zeros_like(u0)
        Fg, g, ast = A.pp_periodic_adjoint(ctx, m, MU_C0, c["Nt"], w, lam_Nt=lt)
        assert abs(Fg - F) <= PARITY_TOL * abs(F)
        assert rel_err(g, grad) <= 1e-9
        assert rel_err(to_host(lt), lam) <= 1e-9
        assert ast["residual"] <= 1e-11
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
