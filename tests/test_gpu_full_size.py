"""Full-size checks on the largest workload: 32,768 triangles at p = 4 (60 DOF per
element, 1,966,080 DOF).  The oracle evaluates sampled elements (residual and Jacobian
rows one element at a time); the sweeps are checked by the tangent/adjoint duality
property, with the stored and with the checkpointed linearization (stage data
recomputed from a state checkpoint every step)."""
import numpy as np
import pytest

from gpu_common import PARITY_TOL, TIGHT, make, perturbed_state, rel_err, to_dev, to_host
from oracle.dg import DG
from pp_inputs import CONFIGS, config_mesh, config_mu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def c3():
    c = CONFIGS["c3"]
    mesh = config_mesh("c3")
    dg = DG(mesh, c["p"], kin=c["kin"])
    return dict(c=c, mesh=mesh, dg=dg)


def _sample(dg):
    return np.unique(np.concatenate([np.arange(0, dg.Ne, 997), [0, dg.Ne - 1],
                                     np.nonzero(np.any(dg.tag == 1, 1))[0][:6],
                                     np.nonzero(np.any(dg.tag == 2, 1))[0][:6]]))


def test_residual_and_jacobian_rows_config3_sampled(c3):
    c, mesh, dg = c3["c"], c3["mesh"], c3["dg"]
    mu = config_mu("c3")
    A, ctx, m = make(c["p"], c["kin"], mesh)
    try:
        u = perturbed_state(dg.Ne, c["p"], seed=23)
        elems = _sample(dg)
        r = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        A.pp_residual(ctx, m, mu, 0.77, to_dev(u), r)
        gpu_r = to_host(r).reshape(dg.Ne, -1)[elems]
        ref_r = dg.residual_subset(u, mu, 0.77, elems).reshape(len(elems), -1)
        assert rel_err(gpu_r, ref_r) <= PARITY_TOL
        nb = dg.nb
        blk = torch.zeros(dg.Ne * 4 * nb * nb, dtype=torch.float64, device="cuda")
        A.pp_jacobian_blocks(ctx, m, mu, 0.77, to_dev(u), blk)
        gpu_j = to_host(blk).reshape(dg.Ne, 4, nb, nb)[elems].transpose(0, 1, 3, 2)
        ref_j = dg.jac_blocks_subset(u, mu, 0.77, elems)
        assert rel_err(gpu_j, ref_j) <= PARITY_TOL
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)


@pytest.mark.parametrize("stride", [0, 1])
def test_duality_config3_checkpointed(c3, stride):
    """<w, Phi v> = <Phi^T w, v> over two steps of dt = 2.5e-4 on the c3 mesh at p = 4, with
    the whole linearization stored (stride 0) and with a checkpoint stride of one step (the
    stage data of the first step is recomputed from its checkpoint for the tangent and the
    adjoint sweep).  Duality holds for the stored linearization at any step size.  The
    initial state is the free stream (plus a 1e-5 perturbation), an impulsive start at
    the no-slip wall; at the c3 step (dt = 0.025), and still at dt = 0.0025, the stage
    Newton iterations of that start on this wall resolution contract slowly (about 0.1 per
    iteration with the exact Jacobian and 1e-8 linear solves) and can use up their
    backtracking, so the check runs at dt = 2.5e-4, where the same kernels (nb = 60 blocks,
    folds, transposes, recomputation) run with short solves.  Each of the 2 x 6 stage solves
    of the two sweeps contributes an error of about lin_rtol |w| |v| to the two inner
    products, so the bar is 1e-9 |w| |v| for lin_rtol = 1e-10: a wrong transpose, fold or
    recomputation gives differences of the order of |w| |v|."""
    c, mesh = c3["c"], c3["mesh"]
    mu = config_mu("c3") * (5e-4 / 5.0)  # period 5e-4 in two steps, motion scaled alike
    # duality holds for the stored linearization whatever the Newton tolerance
    cfg = dict(TIGHT, newton_tol=1e-10, lin_rtol=1e-10, gmres_maxit=20000)
    A, ctx, m = make(c["p"], c["kin"], mesh, T=5e-4, checkpoint_stride=stride, **cfg)
    try:
        u0 = to_dev(perturbed_state(mesh.nt, c["p"], seed=52, amp=1e-5))
        A.pp_primal_period(ctx, m, mu, u0, 2)
        rng = np.random.default_rng(9)
        v = to_dev(rng.standard_normal(u0.numel()))
        w = to_dev(rng.standard_normal(u0.numel()))
        tv, aw = torch.zeros_like(v), torch.zeros_like(v)
        A.pp_tangent_matvec(ctx, v, tv)
        A.pp_adjoint_sweep(ctx, w, aw)
        lhs, rhs = float(torch.dot(w, v - tv)), float(torch.dot(aw, v))
        print(f"c3 duality (stride {stride}): {lhs:.12e} vs {rhs:.12e}")
        scale = float(torch.linalg.norm(w) * torch.linalg.norm(v))
        assert abs(lhs - rhs) <= 1e-9 * scale
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
