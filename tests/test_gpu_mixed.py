"""Mixed-precision path (FP32 Jacobian copies, FP32 block-Jacobi inverses, FP32 inner
GMRES inside FP64 flexible GMRES; FP64 Newton residual, Arnoldi, periodicity residual
and gradient accumulation) against the FP64 oracle.  Because every outer quantity is
FP64 and the outer operator is the exact FP64 Jacobian, the bar is the same FP64
parity bar as the plain path; the measured errors are also reported."""
import numpy as np
import pytest

from gpu_common import PARITY_TOL, TIGHT, make, perturbed_state, rel_err, to_dev, to_host
from oracle import periodic as OP
from oracle.dg import DG
from pp_inputs import CONFIGS, MU_C0, config_mesh, config_mu, free_stream_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MIXED = dict(TIGHT, precision=1, inner_maxit=30, inner_rtol=1e-3)


@pytest.fixture(scope="module")
def c0_mixed():
    c = CONFIGS["c0"]
    mesh = config_mesh("c0")
    dg = DG(mesh, c["p"], kin=c["kin"])
    u0 = perturbed_state(dg.Ne, c["p"], seed=41, amp=1e-2)
    tr = OP.primal_sweep(dg, MU_C0, u0, c["Nt"], newton_tol=1e-14)
    A, ctx, m = make(c["p"], c["kin"], mesh, **MIXED)
    uN = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
    qoi = A.pp_primal_period(ctx, m, MU_C0, to_dev(u0), c["Nt"], u_final=uN)
    yield dict(A=A, ctx=ctx, m=m, dg=dg, tr=tr, uN=to_host(uN), qoi=qoi)
    A.pp_mesh_destroy(m)
    A.pp_destroy(ctx)


def test_mixed_primal_parity(c0_mixed):
    s = c0_mixed
    err_u = rel_err(s["uN"], s["tr"].u[-1])
    err_W = abs(s["qoi"][0] - s["tr"].W) / abs(s["tr"].W)
    print(f"mixed primal: u^(Nt) rel err {err_u:.2e}, W rel err {err_W:.2e}")
    assert err_u <= PARITY_TOL and err_W <= PARITY_TOL


def test_mixed_tangent_and_adjoint_parity(c0_mixed):
    s = c0_mixed
    A, ctx, dg, tr = s["A"], s["ctx"], s["dg"], s["tr"]
    v = np.random.default_rng(7).standard_normal(dg.Nu)
    out = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
    A.pp_tangent_matvec(ctx, to_dev(v), out)
    err_t = rel_err(to_host(out), v - OP.tangent_sweep(dg, tr, v))
    w = np.array([1.0, 0.5])
    g = A.pp_adjoint_sweep(ctx, to_dev(v), out, weights=w, n_mu=3)
    lam_ref, g_ref = OP.adjoint_sweep(dg, tr, v, w)
    err_l, err_g = rel_err(to_host(out), lam_ref), rel_err(g, g_ref)
    print(f"mixed tangent {err_t:.2e}, adjoint lambda {err_l:.2e}, dF/dmu {err_g:.2e}")
    assert err_t <= PARITY_TOL and err_l <= PARITY_TOL and err_g <= PARITY_TOL


def test_mixed_shooting_and_gradient_parity():
    c = CONFIGS["tiny"]
    mesh = config_mesh("tiny")
    dg = DG(mesh, c["p"], kin=c["kin"])
    u0 = free_stream_state(dg.Ne, c["p"]).reshape(-1)
    u0p, tr, _ = OP.shoot_nk(dg, MU_C0, u0, c["Nt"], tol=1e-12)
    w = np.array([1.0, 0.5])
    F, grad, _ = OP.periodic_gradient(dg, tr, w, tol=1e-13)
    A, ctx, m = make(c["p"], c["kin"], mesh, **MIXED)
    try:
        u = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        qoi, st = A.pp_shoot_nk(ctx, m, MU_C0, c["Nt"], 1e-12, u)
        Fg, g, ast = A.pp_periodic_adjoint(ctx, m, MU_C0, c["Nt"], w)
        err_u, err_F, err_g = rel_err(to_host(u), u0p), abs(Fg - F) / abs(F), rel_err(g, grad)
        print(f"mixed shooting: periodicity {st['residual'][-1]:.1e}, u0 {err_u:.2e}, F {err_F:.2e}, "
              f"dF/dmu {err_g:.2e}")
        assert st["residual"][-1] <= 1e-12
        assert err_u <= PARITY_TOL and err_F <= PARITY_TOL and err_g <= 1e-9
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def test_mixed_duality_full_config1():
    c = CONFIGS["c1"]
    mesh = config_mesh("c1")
    mu = config_mu("c1") / 50.0
    A, ctx, m = make(c["p"], c["kin"], mesh, T=0.1, **MIXED)
    try:
        u0 = to_dev(perturbed_state(mesh.nt, c["p"], seed=51, amp=1e-3))
        A.pp_primal_period(ctx, m, mu, u0, 2)
        rng = np.random.default_rng(8)
        v = to_dev(rng.standard_normal(u0.numel()))
        w = to_dev(rng.standard_normal(u0.numel()))
        tv, aw = torch.zeros_like(v), torch.zeros_like(v)
        A.pp_tangent_matvec(ctx, v, tv)
        A.pp_adjoint_sweep(ctx, w, aw)
        lhs, rhs = float(torch.dot(w, v - tv)), float(torch.dot(aw, v))
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
