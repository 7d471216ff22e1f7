"""torch.autograd.Function mu -> (J_E, J_T) through shooting and the periodic adjoint:
gradients against the FP64 oracle, against central finite differences of re-shot
periodic QoIs (step 1e-5), and the checkpointed linearization against the stored one."""
import numpy as np
import pytest

from gpu_common import TIGHT
from oracle import periodic as OP
from oracle.dg import DG
from pp_inputs import CONFIGS, MU_C0, config_mesh, free_stream_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solver(**kw):
    from paper_1512_00616_gb300.autograd import PeriodicSolver
    c = CONFIGS["tiny"]
    cfg = dict(TIGHT)
    cfg.update(kw)
    return PeriodicSolver(config_mesh("tiny"), c["p"], c["kin"], c["Nt"], tol=1e-12, **cfg)


def test_autograd_gradient_matches_oracle_and_checkpointing():
    from paper_1512_00616_gb300.autograd import PeriodicQoI
    c = CONFIGS["tiny"]
    mus = np.stack([MU_C0, MU_C0 * np.array([1.1, 0.9, 1.0])])
    gE, gT = 1.0, 0.5
    grads = {}
    for stride in (0, 3):
        s = _solver(checkpoint_stride=stride)
        try:
            mu = torch.tensor(mus, dtype=torch.float64, requires_grad=True)
            J = PeriodicQoI.apply(mu, s)
            (gE * J[:, 0] + gT * J[:, 1]).sum().backward()
            grads[stride] = (J.detach().numpy(), mu.grad.numpy().copy())
        finally:
            s.close()
    # checkpointed recomputation follows the same iterates
    assert np.max(np.abs(grads[3][1] - grads[0][1])) <= 1e-12 * np.max(np.abs(grads[0][1]))
    # oracle: F = gE J_E + gT J_T = w . (W, J_x) with w = (-gE/T, -gT/T)
    dg = DG(config_mesh("tiny"), c["p"], kin=c["kin"])
    w = np.array([-gE / 5.0, -gT / 5.0])
    for b, m in enumerate(mus):
        _, tr, _ = OP.shoot_nk(dg, m, free_stream_state(dg.Ne, c["p"]).reshape(-1), c["Nt"], tol=1e-12)
        F, g, _ = OP.periodic_gradient(dg, tr, w, tol=1e-13)
        assert abs(grads[0][0][b, 0] + tr.W / 5.0) <= 1e-10 * abs(tr.W / 5.0)
        assert np.max(np.abs(grads[0][1][b] - g)) <= 1e-9 * np.max(np.abs(g))


def test_autograd_gradient_matches_central_differences():
    from paper_1512_00616_gb300.autograd import PeriodicQoI
    s = _solver()
    try:
        mu = torch.tensor(MU_C0[None, :], dtype=torch.float64, requires_grad=True)
        J = PeriodicQoI.apply(mu, s)
        J[0, 0].backward()
        g = mu.grad.numpy()[0]
        tau = 1e-5
        fd = np.zeros(3)
        for j in range(3):
            e = np.zeros(3)
            e[j] = tau
            jp = PeriodicQoI.apply(torch.tensor((MU_C0 + e)[None, :]), s)[0, 0].item()
            jm = PeriodicQoI.apply(torch.tensor((MU_C0 - e)[None, :]), s)[0, 0].item()
            fd[j] = (jp - jm) / (2 * tau)
        assert np.linalg.norm(g - fd) <= 1e-5 * np.linalg.norm(fd)
    finally:
        s.close()
