"""Floquet multipliers of the periodic orbit on the GPU (Sec. 3.3, Eq. stab-def) against the
oracle's dense Phi on the 32-triangle O-grid (p = 1, 8 DIRK3 steps, N_u = 384): with m = N_u
Arnoldi steps the Ritz values are all eigenvalues of Phi; with m = 40 the largest ones have
converged.  The orbit is stable (every multiplier inside the unit circle)."""
import numpy as np
import pytest

from gpu_common import TIGHT, make, to_dev
from oracle import periodic as OP
from oracle.dg import DG
from pp_inputs import CONFIGS, MU_C0, config_mesh, free_stream_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def orbit():
    c = CONFIGS["tiny"]
    dg = DG(config_mesh("tiny"), c["p"], kin=c["kin"])
    u0p, tr, _ = OP.shoot_nk(dg, MU_C0, free_stream_state(dg.Ne, c["p"]).reshape(-1), c["Nt"], tol=1e-12)
    ev = np.linalg.eigvals(OP.dense_phi(dg, tr))
    return dict(c=c, dg=dg, u0p=u0p, ev=ev[np.argsort(-np.abs(ev))])


def _match(got, ref):
    """max over the reference values of the distance to the nearest computed value"""
    return max(np.min(np.abs(got - r)) for r in ref)


def test_floquet_multipliers_match_dense_phi(orbit):
    c, dg, ev = orbit["c"], orbit["dg"], orbit["ev"]
    A, ctx, m = make(c["p"], c["kin"], config_mesh("tiny"), **TIGHT)
    try:
        u = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        A.pp_shoot_nk(ctx, m, MU_C0, c["Nt"], 1e-12, u, u0_guess=to_dev(orbit["u0p"]))
        rho = np.abs(ev[0])
        full, _ = A.pp_floquet(ctx, dg.Nu)
        assert np.max(np.abs(full)) < 1.0
        assert abs(np.max(np.abs(full)) - rho) <= 1e-9 * rho
        assert _match(full, ev[:20]) <= 1e-8 * rho
        part, hl = A.pp_floquet(ctx, 40)
        assert _match(part[:4], ev[:4]) <= 1e-6 * rho
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
