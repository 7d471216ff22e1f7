"""pp_mesh_ogrid builds on the device the same workload mesh the input generator describes:
its residual equals the oracle's on the generator's mesh (coordinates agree to the rounding
of the libm calls, 1e-13, far below the parity bar)."""
import numpy as np
import pytest

from gpu_common import PARITY_TOL, api, perturbed_state, rel_err, to_dev, to_host
from oracle.dg import DG
from pp_inputs import CONFIGS, config_mesh, config_mu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_mesh_ogrid_residual_parity():
    A = api()
    c = CONFIGS["c0"]
    ctx = A.pp_create(A.pp_config_default(p=3, kin=c["kin"]))
    try:
        m = A.pp_mesh_ogrid(ctx, c["n_theta"], c["n_r"], 10.0, c["seed"])
        ne, npn, nu = A.pp_mesh_info(m)
        dg = DG(config_mesh("c0"), 3, kin=c["kin"])
        assert ne == dg.Ne and nu == dg.Nu
        u = perturbed_state(dg.Ne, 3, seed=17)
        mu = config_mu("c0")
        r = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        A.pp_residual(ctx, m, mu, 1.3, to_dev(u), r)
        assert rel_err(to_host(r), dg.residual(u, mu, 1.3)) <= PARITY_TOL
        A.pp_mesh_destroy(m)
    finally:
        A.pp_destroy(ctx)
