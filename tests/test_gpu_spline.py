"""Mirrored spline kinematics (Sec. 6.2, Eq. mirror) through the GPU path: NK shooting and the
periodic gradient with respect to the 8 knot values on the 32-triangle O-grid, against the
oracle's shooting and periodic adjoint with the same kinematics."""
import numpy as np
import pytest

from gpu_common import PARITY_TOL, TIGHT, make, rel_err, to_host
from oracle import periodic as OP
from oracle.dg import DG
from pp_inputs import CONFIGS, KIN_SPLINE8, MU_SPLINE8, config_mesh, free_stream_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_spline_kinematics_shooting_and_gradient_parity():
    c = CONFIGS["tiny"]
    mesh = config_mesh("tiny")
    dg = DG(mesh, c["p"], kin=KIN_SPLINE8)
    u0 = free_stream_state(dg.Ne, c["p"]).reshape(-1)
    u0p, tr, _ = OP.shoot_nk(dg, MU_SPLINE8, u0, c["Nt"], tol=1e-12)
    w = np.array([1.0, 0.5])
    F, grad, lam = OP.periodic_gradient(dg, tr, w, tol=1e-13)
    A, ctx, m = make(c["p"], KIN_SPLINE8, mesh, **TIGHT)
    try:
        ug = torch.zeros(dg.Nu, dtype=torch.float64, device="cuda")
        qoi, st = A.pp_shoot_nk(ctx, m, MU_SPLINE8, c["Nt"], 1e-12, ug)
        assert st["residual"][-1] <= 1e-12
        assert rel_err(to_host(ug), u0p) <= PARITY_TOL
        lt = torch.zeros_like(ug)
        Fg, g, ast = A.pp_periodic_adjoint(ctx, m, MU_SPLINE8, c["Nt"], w, lam_Nt=lt)
        assert len(g) == 8
        assert abs(Fg - F) <= PARITY_TOL * abs(F)
        assert rel_err(g, grad) <= 1e-9
        assert rel_err(to_host(lt), lam) <= 1e-9
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
