"""Kinematics (Sec. 6.1 single Fourier mode; Sec. 6.2 mirrored cubic splines, Eq. mirror).

Oracle pins: the periodic cubic spline against SciPy's periodic CubicSpline (a library
routine: values and first derivatives), knot interpolation, the mirror condition
f(t + T/2) = -f(t), and h' of the rigid motion against the time derivative of the blended
oracle's h.  C ABI (host code, no GPU): pp_motion_eval against the oracle's motion for the
three modes, its parameter derivatives against complex steps of the oracle's motion, and its
argument checks."""
import numpy as np
import pytest
from scipy.interpolate import CubicSpline

from oracle.dg import (CS_STEP, DG, KIN_FOURIER6, KIN_HEAVE_PITCH, KIN_SPLINE8, mirrored_knots,
                       periodic_cubic_spline)
from pp_inputs import MU_C0, MU_F6_BASE, MU_SPLINE8, config_mesh

T = 5.0


def _scipy_periodic(y, t):
    knots = np.arange(len(y) + 1) * T / len(y)
    cs = CubicSpline(knots, np.concatenate([y, y[:1]]), bc_type="periodic")
    return cs(t % T), cs(t % T, 1)


def test_spline_matches_scipy_periodic_cubic_spline():
    rng = np.random.default_rng(3)
    for m in (5, 8, 11):
        y = rng.standard_normal(m)
        for t in rng.uniform(-T, 2 * T, 40):
            v, d = periodic_cubic_spline(y, T, t)
            vs, ds = _scipy_periodic(y, t)
            assert abs(v - vs) <= 1e-12 * (1 + abs(vs))
            assert abs(d - ds) <= 1e-11 * (1 + abs(ds))


def test_spline_interpolates_knots_and_mirrors():
    rng = np.random.default_rng(4)
    half = rng.standard_normal(4)
    y = mirrored_knots(half)
    assert np.array_equal(y, np.concatenate([half, -half]))
    for k in range(8):
        assert abs(periodic_cubic_spline(y, T, k * T / 8)[0] - y[k]) <= 1e-13
    for t in rng.uniform(0, T, 50):
        v0, d0 = periodic_cubic_spline(y, T, t)
        v1, d1 = periodic_cubic_spline(y, T, t + T / 2)
        assert abs(v0 + v1) <= 1e-13 and abs(d0 + d1) <= 1e-12


@pytest.fixture(scope="module")
def dgs():
    mesh = config_mesh("tiny")
    return {k: DG(mesh, 1, kin=k) for k in (KIN_HEAVE_PITCH, KIN_FOURIER6, KIN_SPLINE8)}


def test_spline_heave_rate_is_the_time_derivative_of_the_blended_heave():
    from oracle.dg_blend import BlendedDG
    bd = BlendedDG(config_mesh("tiny"), 1, kin=KIN_SPLINE8)
    for t in (0.1, 0.9, 1.7, 2.6, 4.3):
        _, _, hd = bd.motion(MU_SPLINE8, t)
        eps = 1e-6
        fd = (bd.heave(MU_SPLINE8, t + eps) - bd.heave(MU_SPLINE8, t - eps)) / (2 * eps)
        assert abs(hd - fd) <= 1e-8


@pytest.mark.parametrize("kin,mu", [(KIN_HEAVE_PITCH, MU_C0), (KIN_FOURIER6, MU_F6_BASE),
                                    (KIN_SPLINE8, MU_SPLINE8)])
def test_library_motion_matches_oracle(dgs, kin, mu):
    A = pytest.importorskip("paper_1512_00616_gb300.api")
    dg = dgs[kin]
    rng = np.random.default_rng(5)
    for t in np.concatenate([[0.0, T / 8, T / 2, T], rng.uniform(0, T, 12)]):
        out = A.pp_motion_eval(kin, T, mu, t)
        ref = np.array(dg.motion(mu, t), dtype=float)
        assert np.max(np.abs(out[0] - ref)) <= 1e-13 * (1 + np.max(np.abs(ref)))
        # parameter derivatives against complex steps of the oracle's motion
        for j in range(len(mu)):
            mc = mu.astype(complex)
            mc[j] += 1j * CS_STEP
            dref = np.imag(np.array(dg.motion(mc, t))) / CS_STEP
            assert np.max(np.abs(out[1 + j] - dref)) <= 1e-12 * (1 + np.max(np.abs(dref)))


def test_library_motion_rejects_bad_arguments():
    A = pytest.importorskip("paper_1512_00616_gb300.api")
    with pytest.raises(A.PPError):
        A.pp_motion_eval(KIN_SPLINE8, T, MU_SPLINE8[:6], 0.3)
    with pytest.raises(A.PPError):
        A.pp_motion_eval(7, T, MU_SPLINE8, 0.3)
    with pytest.raises(A.PPError):
        A.pp_motion_eval(KIN_SPLINE8, 0.0, MU_SPLINE8, 0.3)
