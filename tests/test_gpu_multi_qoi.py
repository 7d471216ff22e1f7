"""The multi-QoI periodic adjoint (one block GMRES for W and J_x, Sec. 4) against the
oracle's separate solves (Algorithms dual and grad per QoI) on the 32-triangle O-grid
(p = 1, 8 DIRK3 steps): multipliers, F and dF/dmu per QoI; and it needs no more adjoint
sweeps than the two separate GPU solves together."""
import numpy as np
import pytest

from gpu_common import PARITY_TOL, TIGHT, make, rel_err, to_dev, to_host
from oracle import periodic as OP
from oracle.dg import DG
from pp_inputs import CONFIGS, MU_C0, config_mesh, free_stream_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_block_adjoint_for_two_qois_matches_separate_solves():
    c = CONFIGS["tiny"]
    dg = DG(config_mesh("tiny"), c["p"], kin=c["kin"])
    u0p, tr, _ = OP.shoot_nk(dg, MU_C0, free_stream_state(dg.Ne, c["p"]).reshape(-1), c["Nt"], tol=1e-12)
    W = np.array([[1.0, 0.0], [0.0, 1.0]])
    ref = [OP.periodic_gradient(dg, tr, W[q], tol=1e-13) for q in range(2)]
    A, ctx, m = make(c["p"], c["kin"], config_mesh("tiny"), **TIGHT)
    try:
        u0 = to_dev(u0p)
        lam = torch.zeros(2 * dg.Nu, dtype=torch.float64, device="cuda")
        F, g, st = A.pp_periodic_adjoint_multi(ctx, m, MU_C0, c["Nt"], W, u0=u0, lam_Nt=lam)
        assert st["residual"] <= 1e-11
        for q in range(2):
            Fr, gr, lr = ref[q]
            assert abs(F[q] - Fr) <= PARITY_TOL * abs(Fr)
            assert rel_err(g[q], gr) <= 1e-9
            assert rel_err(to_host(lam[q * dg.Nu:(q + 1) * dg.Nu]), lr) <= 1e-9
        separate = 0
        for q in range(2):
            _, _, s1 = A.pp_periodic_adjoint(ctx, m, MU_C0, c["Nt"], W[q], u0=u0)
            separate += s1["krylov_iters"] + 2    # GMRES sweeps + the right-hand side and final sweeps
        print(f"block adjoint sweeps {st['sweeps']}, separate {separate}")
        assert st["sweeps"] <= separate
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
