"""Pins of the oracle's fixed-point solvers (Algorithm fixedpt, the m-step nonlinear
preconditioning of Sec. 6.1, and the dual fixed point on Eq. fixedpt-dual).

* Algorithm fixedpt and Newton-Krylov shooting (Algorithm primal) are independent
  algorithms for the same fixed point of the period map (Eq. fixedpt): they agree.
* Near the fixed point the primal iteration is linear with the period map's Jacobian
  Phi, and the dual iteration is exactly linear with Phi^T; both contract at the rate of
  the largest Floquet multiplier |lambda_max(Phi)| = |lambda_max(Phi^T)| (Sec. 3.3), so
  their observed asymptotic rates agree with each other and with the eigenvalue computed
  from the dense Phi.
* m = 5 fixed-point steps before Newton leave the solution unchanged and cut the Newton
  iterations (the paper's observation in Sec. 6.1).
* The dual fixed point reaches the multipliers of the GMRES solve of Algorithm dual.

Workload: the 32-triangle O-grid, p = 1, one period T = 5 in 4 DIRK3 steps."""
import numpy as np
import pytest

from oracle import periodic as OP
from oracle.dg import DG
from pp_inputs import CONFIGS, MU_C0, config_mesh, free_stream_state

NT = 4


@pytest.fixture(scope="module")
def fp():
    c = CONFIGS["tiny"]
    dg = DG(config_mesh("tiny"), c["p"], kin=c["kin"])
    u0 = free_stream_state(dg.Ne, c["p"]).reshape(-1)
    uf, trf, hf = OP.shoot_fixed_point(dg, MU_C0, u0, NT, tol=1e-9)
    un, trn, hn = OP.shoot_nk(dg, MU_C0, u0, NT, tol=1e-11)
    return dict(dg=dg, u0=u0, uf=uf, hf=hf, un=un, trn=trn, hn=hn)


def _rate(h, last=5):
    h = np.asarray(h)
    return float((h[-1] / h[-1 - last]) ** (1.0 / last))


def test_fixed_point_and_newton_krylov_agree(fp):
    # both stop within their tolerances of the same fixed point: |uf - u*| <= tol / (1 - rho)
    assert fp["hf"][-1] <= 1e-9 and fp["hn"][-1] <= 1e-11
    assert np.max(np.abs(fp["uf"] - fp["un"])) <= 1e-8
    # the iteration is not trivially converged: it started far away
    assert fp["hf"][0] > 1e-2


def test_primal_and_dual_fixed_point_rates_equal_floquet_radius(fp):
    dg, trn = fp["dg"], fp["trn"]
    rho = np.max(np.abs(np.linalg.eigvals(OP.dense_phi(dg, trn))))
    assert rho < 1.0
    w = np.array([1.0, 0.5])
    lam, hd = OP.periodic_adjoint_fixed_point(dg, trn, w, tol=1e-12)
    r_primal, r_dual = _rate(fp["hf"]), _rate(hd)
    print(f"rho(Phi) = {rho:.4f}, primal fixed-point rate {r_primal:.4f}, dual {r_dual:.4f}")
    assert abs(r_dual - rho) <= 0.25 * rho
    assert abs(r_primal - rho) <= 0.25 * rho
    # the dual fixed point solves the same periodic adjoint problem as GMRES (Algorithm dual)
    lam_g = OP.periodic_adjoint(dg, trn, w, tol=1e-13)
    assert np.max(np.abs(lam - lam_g)) <= 1e-10 * np.max(np.abs(lam_g))


def test_m_step_preconditioning_cuts_newton_iterations(fp):
    dg = fp["dg"]
    u5, _, h5 = OP.shoot_nk(dg, MU_C0, fp["u0"], NT, tol=1e-11, m_pre=5)
    assert len(h5) < len(fp["hn"])
    assert np.max(np.abs(u5 - fp["un"])) <= 1e-9
