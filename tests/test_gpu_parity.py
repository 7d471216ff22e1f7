"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs.  Bar: max|gpu - oracle| <= 1e-10 max|oracle| (FP64 residuals,
Jacobian blocks, trajectories, sensitivities and gradients).

Sizes: small meshes that span several blocks and every polynomial degree, the
64-element config-0 workload for the sweeps, and the full 2048-element p = 3
workload for the residual and (sampled) Jacobian rows."""
import numpy as np
import pytest

from gpu_common import PARITY_TOL, TIGHT, make, perturbed_state, rel_err, to_dev, to_host
from oracle import periodic as OP
from oracle.dg import DG
from pp_inputs import (CONFIGS, KIN_FOURIER6, KIN_HEAVE_PITCH, MU_C0, box, config_mesh, config_mu,
                       fourier6_samples, free_stream_state, ogrid)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("kin", [KIN_HEAVE_PITCH, KIN_FOURIER6])
def test_residual_parity_all_degrees(p, kin):
    mesh = ogrid(12, 3, seed=4)
    mu = MU_C0 if kin == KIN_HEAVE_PITCH else fourier6_samples(1, 3)[0]
    A, ctx, m = make(p, kin, mesh)
    try:
        dg = DG(mesh, p, kin=kin)
        u = perturbed_state(dg.Ne, p, seed=10 + p, amp=3e-2)
        for t in (0.0, 0.61, 3.7):
            r = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
            A.pp_residual(ctx, m, mu, t, to_dev(u), r)
            ref = dg.residual(u, mu, t)
            assert rel_err(to_host(r), ref) <= PARITY_TOL
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def test_residual_parity_full_config1():
    c = CONFIGS["c1"]
    mesh = config_mesh("c1")
    mu = config_mu("c1")
    A, ctx, m = make(c["p"], c["kin"], mesh)
    try:
        dg = DG(mesh, c["p"], kin=c["kin"])
        u = perturbed_state(dg.Ne, c["p"], seed=21)
        r = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        A.pp_residual(ctx, m, mu, 1.234, to_dev(u), r)
        assert rel_err(to_host(r), dg.residual(u, mu, 1.234)) <= PARITY_TOL
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_free_stream_preserved_on_gpu(p):
    mesh = box(6, 4, seed=2)
    A, ctx, m = make(p, KIN_HEAVE_PITCH, mesh)
    try:
        nt = mesh.nt
        u = to_dev(free_stream_state(nt, p))
        r = torch.zeros_like(u)
        for t in (0.2, 2.9):
            A.pp_residual(ctx, m, MU_C0, t, u, r)
            assert float(r.abs().max()) < 2e-13
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_jacobian_block_parity(p):
    mesh = ogrid(8, 2, seed=0)
    A, ctx, m = make(p, KIN_FOURIER6, mesh)
    mu = fourier6_samples(1, 7)[0]
    try:
        dg = DG(mesh, p, kin=KIN_FOURIER6)
        u = perturbed_state(dg.Ne, p, seed=30 + p)
        nb = dg.nb
        blk = torch.zeros(dg.Ne * 4 * nb * nb, dtype=torch.float64, device="cuda")
        A.pp_jacobian_blocks(ctx, m, mu, 0.9, to_dev(u), blk)
        gpu = to_host(blk).reshape(dg.Ne, 4, nb, nb).transpose(0, 1, 3, 2)  # column-major -> [row, col]
        ref = dg.jac_blocks(u, mu, 0.9)
        assert rel_err(gpu, ref) <= PARITY_TOL
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def test_jacobian_rows_full_config1_sampled():
    c = CONFIGS["c1"]
    mesh = config_mesh("c1")
    mu = config_mu("c1")
    A, ctx, m = make(c["p"], c["kin"], mesh)
    try:
        dg = DG(mesh, c["p"], kin=c["kin"])
        u = perturbed_state(dg.Ne, c["p"], seed=22)
        nb = dg.nb
        blk = torch.zeros(dg.Ne * 4 * nb * nb, dtype=torch.float64, device="cuda")
        A.pp_jacobian_blocks(ctx, m, mu, 2.5, to_dev(u), blk)
        elems = np.unique(np.concatenate([np.arange(0, dg.Ne, 61), [0, dg.Ne - 1],
                                          np.nonzero(np.any(dg.tag == 1, 1))[0][:8],
                                          np.nonzero(np.any(dg.tag == 2, 1))[0][:8]]))
        gpu = to_host(blk).reshape(dg.Ne, 4, nb, nb)[elems].transpose(0, 1, 3, 2)
        ref = dg.jac_blocks_subset(u, mu, 2.5, elems)
        assert rel_err(gpu, ref) <= PARITY_TOL
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def test_qoi_rate_parity():
    mesh = config_mesh("c0")
    A, ctx, m = make(1, KIN_HEAVE_PITCH, mesh)
    try:
        dg = DG(mesh, 1)
        u = perturbed_state(dg.Ne, 1, seed=5, amp=5e-2)
        for t in (0.3, 4.1):
            got = A.pp_qoi_rate(ctx, m, MU_C0, t, to_dev(u))
            ref = np.array(dg.qoi_rate(u, MU_C0, t))
            assert rel_err(got, ref) <= PARITY_TOL
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


@pytest.fixture(scope="module")
def c0_sweep():
    """Primal sweep on the config-0 workload (64 triangles, p = 1, 20 DIRK3 steps) from a
    seeded perturbation of the free stream, on the oracle and on the GPU."""
    c = CONFIGS["c0"]
    mesh = config_mesh("c0")
    dg = DG(mesh, c["p"], kin=c["kin"])
    u0 = perturbed_state(dg.Ne, c["p"], seed=40, amp=1e-2)
    tr = OP.primal_sweep(dg, MU_C0, u0, c["Nt"], newton_tol=1e-14)
    A, ctx, m = make(c["p"], c["kin"], mesh, **TIGHT)
    traj = torch.zeros((c["Nt"] + 1) * dg.Nu, dtype=torch.float64, device="cuda")
    qoi = A.pp_primal_period(ctx, m, MU_C0, to_dev(u0), c["Nt"], u_traj=traj)
    yield dict(A=A, ctx=ctx, m=m, dg=dg, tr=tr, u0=u0, traj=to_host(traj).reshape(c["Nt"] + 1, -1), qoi=qoi)
    A.pp_mesh_destroy(m)
    A.pp_destroy(ctx)


def test_primal_sweep_parity_config0(c0_sweep):
    s = c0_sweep
    tr = s["tr"]
    for n in range(0, tr.Nt + 1, 5):
        assert rel_err(s["traj"][n], tr.u[n]) <= PARITY_TOL
    assert rel_err(s["traj"][-1], tr.u[-1]) <= PARITY_TOL
    assert abs(s["qoi"][0] - tr.W) <= PARITY_TOL * abs(tr.W)
    assert abs(s["qoi"][1] - tr.Jx) <= PARITY_TOL * abs(tr.Jx)
    assert abs(s["qoi"][2] + tr.W / 5.0) <= PARITY_TOL * abs(tr.W)


def test_tangent_matvec_parity_config0(c0_sweep):
    s = c0_sweep
    A, ctx, dg, tr = s["A"], s["ctx"], s["dg"], s["tr"]
    v = np.random.default_rng(3).standard_normal(dg.Nu)
    out = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
    A.pp_tangent_matvec(ctx, to_dev(v), out)
    ref = v - OP.tangent_sweep(dg, tr, v)
    assert rel_err(to_host(out), ref) <= PARITY_TOL


def test_adjoint_sweep_parity_config0(c0_sweep):
    s = c0_sweep
    A, ctx, dg, tr = s["A"], s["ctx"], s["dg"], s["tr"]
    lam = np.random.default_rng(4).standard_normal(dg.Nu)
    out = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
    A.pp_adjoint_sweep(ctx, to_dev(lam), out)
    assert rel_err(to_host(out), OP.adjoint_sweep(dg, tr, lam)[0]) <= PARITY_TOL
    w = np.array([1.0, 0.5])
    g = A.pp_adjoint_sweep(ctx, to_dev(lam), out, weights=w, n_mu=3)
    ref_lam, ref_g = OP.adjoint_sweep(dg, tr, lam, w)
    assert rel_err(to_host(out), ref_lam) <= PARITY_TOL
    assert rel_err(g, ref_g) <= PARITY_TOL


def test_tangent_adjoint_duality_full_config1():
    """Property at full size: <w, Phi v> = <Phi^T w, v> on the 2048-element p = 3 mesh
    (two DIRK3 steps of the period, so the check stays short)."""
    c = CONFIGS["c1"]
    mesh = config_mesh("c1")
    # a period of T = 0.1 in two steps keeps the config-1 step size dt = 0.05; the motion
    # amplitudes are scaled by the same factor 1/50 so that wall velocities are unchanged
    mu = config_mu("c1") / 50.0
    A, ctx, m = make(c["p"], c["kin"], mesh, T=0.1, **TIGHT)
    try:
        nt = mesh.nt
        u0 = to_dev(perturbed_state(nt, c["p"], seed=50, amp=1e-3))
        A.pp_primal_period(ctx, m, mu, u0, 2)
        rng = np.random.default_rng(5)
        v = to_dev(rng.standard_normal(u0.numel()))
        w = to_dev(rng.standard_normal(u0.numel()))
        tv = torch.zeros_like(v)
        aw = torch.zeros_like(v)
        A.pp_tangent_matvec(ctx, v, tv)
        A.pp_adjoint_sweep(ctx, w, aw)
        lhs = float(torch.dot(w, v - tv))
        rhs = float(torch.dot(aw, v))
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


@pytest.fixture(scope="module")
def tiny_periodic():
    c = CONFIGS["tiny"]
    mesh = config_mesh("tiny")
    dg = DG(mesh, c["p"], kin=c["kin"])
    u0 = free_stream_state(dg.Ne, c["p"]).reshape(-1)
    u0p, tr, hist = OP.shoot_nk(dg, MU_C0, u0, c["Nt"], tol=1e-12)
    w = np.array([1.0, 0.5])
    F, grad, lam = OP.periodic_gradient(dg, tr, w, tol=1e-13)
    return dict(dg=dg, u0p=u0p, tr=tr, F=F, grad=grad, lam=lam, w=w, mesh=mesh, c=c)


def test_shooting_and_periodic_gradient_parity(tiny_periodic):
    s = tiny_periodic
    c, dg = s["c"], s["dg"]
    A, ctx, m = make(c["p"], c["kin"], s["mesh"], **TIGHT)
    try:
        u0 = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        qoi, st = A.pp_shoot_nk(ctx, m, MU_C0, c["Nt"], 1e-12, u0)
        assert st["residual"][-1] <= 1e-12
        assert rel_err(to_host(u0), s["u0p"]) <= PARITY_TOL
        lam = torch.zeros_like(u0)
        F, g, ast = A.pp_periodic_adjoint(ctx, m, MU_C0, c["Nt"], s["w"], lam_Nt=lam)
        assert abs(F - s["F"]) <= PARITY_TOL * abs(s["F"])
        assert rel_err(g, s["grad"]) <= 1e-9
        assert rel_err(to_host(lam), s["lam"]) <= 1e-9
        assert ast["residual"] <= 1e-11
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


def test_error_codes():
    from gpu_common import api
    A = api()
    mesh = ogrid(8, 2, seed=0)
    ctx = A.pp_create(A.pp_config_default(p=1))
    try:
        bad = mesh.ftag.copy()
        bad[0, 0] = 1 if bad[0, 0] == 0 else 0
        with pytest.raises(A.PPError) as ei:
            A.pp_mesh_create(ctx, mesh.verts, mesh.tris, bad)
        assert ei.value.code == A.PP_EINVAL
        m = A.pp_mesh_create(ctx, mesh.verts, mesh.tris, mesh.ftag)
        v = torch.zeros(mesh.nt * 12, dtype=torch.float64, device="cuda")
        with pytest.raises(A.PPError) as ei:
            A.pp_tangent_matvec(ctx, v, v)
        assert ei.value.code == A.PP_ESTATE
        with pytest.raises(A.PPError) as ei:
            A.pp_residual(ctx, m, np.zeros(6), 0.0, v, v)   # heave-pitch mode wants 3 parameters
        assert ei.value.code == A.PP_EINVAL
        with pytest.raises(A.PPError) as ei:
            A.pp_primal_period(ctx, m, MU_C0, v, 2)          # zero density state
        assert ei.value.code in (A.PP_ENAN, A.PP_ENOCONV)
        A.pp_mesh_destroy(m)
    finally:
        A.pp_destroy(ctx)


def test_steady_state_parity_and_cold_start():
    c = CONFIGS["c0"]
    mesh = config_mesh("c0")
    dg = DG(mesh, c["p"], kin=c["kin"])
    u_ref, _, _ = OP.steady_state(dg, MU_C0, free_stream_state(dg.Ne, c["p"]).reshape(-1), tol=1e-12)
    A, ctx, m = make(c["p"], c["kin"], mesh, **TIGHT)
    try:
        u = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        steps, rel = A.pp_steady_state(ctx, m, MU_C0, u, tol=1e-12, maxit=100)
        assert rel <= 1e-12
        assert rel_err(to_host(u), u_ref) <= PARITY_TOL
        u0 = torch.zeros_like(u)
        qoi, st = A.pp_shoot_nk(ctx, m, MU_C0, c["Nt"], 1e-10, u0)
        assert st["cold_start"] == 2 and st["residual"][-1] <= 1e-10
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
