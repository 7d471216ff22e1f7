"""GPU parity of the fixed-point solvers against the oracle on the 32-triangle O-grid (p = 1,
one period T = 5 in 4 DIRK3 steps): Algorithm fixedpt (same iterates from the free stream:
residual history and final state), Newton-Krylov shooting with m = 5 fixed-point steps of
nonlinear preconditioning (Sec. 6.1), and the dual fixed point on Eq. fixedpt-dual with the
gradient of Algorithm grad."""
import numpy as np
import pytest

from gpu_common import PARITY_TOL, TIGHT, make, rel_err, to_dev, to_host
from oracle import periodic as OP
from oracle.dg import DG
from pp_inputs import CONFIGS, MU_C0, config_mesh, free_stream_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NT = 4


@pytest.fixture(scope="module")
def ref():
    c = CONFIGS["tiny"]
    dg = DG(config_mesh("tiny"), c["p"], kin=c["kin"])
    u0 = free_stream_state(dg.Ne, c["p"]).reshape(-1)
    uf, trf, hf = OP.shoot_fixed_point(dg, MU_C0, u0, NT, tol=1e-9)
    un, trn, hn = OP.shoot_nk(dg, MU_C0, u0, NT, tol=1e-12)
    w = np.array([1.0, 0.5])
    F, grad, lam = OP.periodic_gradient(dg, trn, w, tol=1e-13)
    return dict(c=c, dg=dg, u0=u0, uf=uf, hf=hf, un=un, hn=hn, w=w, F=F, grad=grad, lam=lam)


def test_fixed_point_iteration_parity(ref):
    c, dg = ref["c"], ref["dg"]
    A, ctx, m = make(c["p"], c["kin"], config_mesh("tiny"), **TIGHT)
    try:
        u = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        qoi, st = A.pp_shoot_fixed_point(ctx, m, MU_C0, NT, 1e-9, 200, to_dev(ref["u0"]), u)
        assert st["iterations"] + 1 == len(ref["hf"])
        # each residual ||u^(Nt) - u0|| is a difference of states that match the oracle to the
        # parity bar, so the histories agree to that bar times the size of the state
        h, hr = np.array(st["residual"]), np.array(ref["hf"])
        assert np.max(np.abs(h - hr)) <= PARITY_TOL * np.linalg.norm(ref["uf"])
        assert rel_err(to_host(u), ref["uf"]) <= PARITY_TOL
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def test_newton_krylov_with_fixed_point_preconditioning(ref):
    c, dg = ref["c"], ref["dg"]
    its = {}
    for mpre in (0, 5):
        A, ctx, m = make(c["p"], c["kin"], config_mesh("tiny"), nk_fixed_point_pre=mpre, **TIGHT)
        try:
            u = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
            _, st = A.pp_shoot_nk(ctx, m, MU_C0, NT, 1e-12, u, u0_guess=to_dev(ref["u0"]))
            assert st["residual"][-1] <= 1e-12
            assert rel_err(to_host(u), ref["un"]) <= PARITY_TOL
            its[mpre] = st["newton_iters"]
        finally:
            A.pp_mesh_destroy(m)
            A.pp_destroy(ctx)
    assert its[5] < its[0]


def test_dual_fixed_point_parity(ref):
    c, dg = ref["c"], ref["dg"]
    A, ctx, m = make(c["p"], c["kin"], config_mesh("tiny"), **TIGHT)
    try:
        u = to_dev(ref["un"])
        lam = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        F, g, st = A.pp_periodic_adjoint_fixed_point(ctx, m, MU_C0, NT, ref["w"], 1e-13, 500, u0=u, lam_Nt=lam)
        assert st["residual"] <= 1e-13
        assert abs(F - ref["F"]) <= PARITY_TOL * abs(ref["F"])
        assert rel_err(to_host(lam), ref["lam"]) <= 1e-9
        assert rel_err(g, ref["grad"]) <= 1e-9
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def test_batched_shooting_and_adjoint_match_single_calls(ref):
    """pp_shoot_nk_batched / pp_periodic_adjoint_batched on two motion vectors give the
    single-call results entry by entry (same operations, same order)."""
    c, dg = ref["c"], ref["dg"]
    mus = np.stack([MU_C0, MU_C0 * np.array([1.1, 0.9, 1.0])])
    A, ctx, m = make(c["p"], c["kin"], config_mesh("tiny"), **TIGHT)
    try:
        guess = to_dev(np.tile(ref["u0"], 2))
        ub = torch.zeros(2 * dg.Nu, dtype=torch.float64, device="cuda")
        qb, status, _ = A.pp_shoot_nk_batched(ctx, m, mus, NT, 1e-12, ub, u0_guess=guess)
        assert list(status) == [0, 0]
        w = np.array([[1.0, 0.5], [-0.2, 1.0]])
        Fb, gb = A.pp_periodic_adjoint_batched(ctx, m, mus, NT, w, ub)
        for b in range(2):
            us = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
            qs, _ = A.pp_shoot_nk(ctx, m, mus[b], NT, 1e-12, us, u0_guess=to_dev(ref["u0"]))
            assert np.array_equal(to_host(us), to_host(ub[b * dg.Nu:(b + 1) * dg.Nu]))
            assert np.array_equal(qs, qb[b])
            Fs, gs, _ = A.pp_periodic_adjoint(ctx, m, mus[b], NT, w[b], u0=us)
            assert Fs == Fb[b] and np.array_equal(gs, gb[b])
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
