"""Seeded workloads shaped like the paper's flapping-airfoil case (Sec. 6).

The paper's case: NACA0012, Re 1000, Mach 0.2, one period T = 5 of a heaving
and pitching motion, DIRK3 with equally spaced steps.  The configurations
below are synthetic stand-ins on seeded O-grids (the paper's mesh is not
published).  Everything here is an *input*: meshes, motion parameters, and
seeded initial states; no step of the method is computed here.

Motion parametrizations (the kinematics mode is part of the C-ABI config):

* ``KIN_HEAVE_PITCH``: mu = (h0, theta0, phi);  h = h0 sin(w t),
  theta = theta0 sin(w t + phi)  (single Fourier mode, Eq. nominal form).
* ``KIN_FOURIER6``:   mu = (a1, b1, a2, alpha1, beta1, alpha2);
  h = a1 sin wt + b1 cos wt + a2 sin 2wt, theta likewise; w = 2 pi / T.
* ``KIN_SPLINE8``:    mu = (h0, h1, h2, h3, theta0, theta1, theta2, theta3), the knot values at
  t = 0, T/8, T/4, 3T/8 of the mirrored periodic cubic splines of Sec. 6.2 (Eq. mirror).
"""
import numpy as np

from .mesh import ogrid

KIN_HEAVE_PITCH = 0
KIN_FOURIER6 = 1
KIN_SPLINE8 = 2

DEG = np.pi / 180.0

# name -> (n_theta, n_r, mesh seed, p, Nt, kinematics mode)
CONFIGS = {
    "tiny": dict(n_theta=8, n_r=2, seed=0, p=1, Nt=8, kin=KIN_HEAVE_PITCH),
    "c0": dict(n_theta=16, n_r=2, seed=0, p=1, Nt=20, kin=KIN_HEAVE_PITCH),
    "c1": dict(n_theta=64, n_r=16, seed=1, p=3, Nt=100, kin=KIN_FOURIER6),
    "c2": dict(n_theta=128, n_r=32, seed=2, p=3, Nt=100, kin=KIN_FOURIER6),
    "c3": dict(n_theta=256, n_r=64, seed=3, p=4, Nt=200, kin=KIN_FOURIER6),
}

PHYS = dict(gamma=1.4, Pr=0.72, Mach=0.2, Re=1000.0, T=5.0)

MU_C0 = np.array([0.1, 5.0 * DEG, 90.0 * DEG])
# config-0 motion written in the 6-coefficient form: h = 0.1 sin wt, theta = 5deg cos wt
MU_F6_BASE = np.array([0.1, 0.0, 0.0, 0.0, 5.0 * DEG, 0.0])
MU_F6_SCALE = np.array([0.1, 0.1, 0.1, 5.0 * DEG, 5.0 * DEG, 5.0 * DEG])
# the same motion sampled at the spline knots t = 0, T/8, T/4, 3T/8 (h = 0.1 sin wt,
# theta = 5deg cos wt)
_R2 = np.sqrt(0.5)
MU_SPLINE8 = np.array([0.0, 0.1 * _R2, 0.1, 0.1 * _R2, 5.0 * DEG, 5.0 * DEG * _R2, 0.0, -5.0 * DEG * _R2])


def config_mesh(name):
    c = CONFIGS[name]
    return ogrid(c["n_theta"], c["n_r"], seed=c["seed"])


def fourier6_samples(n, seed, spread=0.2):
    """n seeded 6-coefficient motion vectors, uniform within +-spread of the base."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return MU_F6_BASE[None, :] + spread * MU_F6_SCALE[None, :] * rng.uniform(-1.0, 1.0, (n, 6))


def config_mu(name, seed=11):
    if CONFIGS[name]["kin"] == KIN_HEAVE_PITCH:
        return MU_C0.copy()
    return fourier6_samples(1, seed)[0]


def free_stream_state(nt, p, gamma=1.4, mach=0.2):
    """Uniform free stream (rho=1, u=(1,0), p=1/(gamma M^2)) at every node; layout [nt][4][Np]."""
    npn = (p + 1) * (p + 2) // 2
    pinf = 1.0 / (gamma * mach * mach)
    U = np.array([1.0, 1.0, 0.0, pinf / (gamma - 1.0) + 0.5])
    return np.broadcast_to(U[None, :, None], (nt, 4, npn)).copy()


def state_perturbation(nt, p, seed, amp=1e-3, scale=None):
    """Seeded smooth-in-index random perturbation, layout [nt][4][Np]."""
    npn = (p + 1) * (p + 2) // 2
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.uniform(-1.0, 1.0, (nt, 4, npn))
    if scale is None:
        scale = np.array([1.0, 1.0, 1.0, 18.0])
    return amp * d * np.asarray(scale)[None, :, None]
