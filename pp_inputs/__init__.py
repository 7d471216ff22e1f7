"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only *generates inputs*: mesh vertices and triangles with boundary
tags, motion-parameter vectors, and seeded state perturbations.  It holds none
of the method's arithmetic (no basis, quadrature, flux, time stepping or
solver), so the oracle and the CUDA path can both consume it without sharing
any code of the method.

Workloads (stand-ins for the paper's 978-element NACA0012 mesh, Sec. 6.1,
which is not published):

* ``ogrid(n_theta, n_r, seed)`` -- structured O-grid around a symmetric
  12%-thickness 4-digit airfoil (closed trailing edge), each quad split into
  two triangles, far field at radius ``r_far`` chords, interior nodes jittered
  by up to 10% of the local spacing with a seeded generator.
* ``box(nx, ny, seed)`` -- jittered rectangle with far-field boundaries all
  round (free-stream preservation tests, no wall).
"""
from .mesh import ogrid, box, Mesh  # noqa: F401
from .workloads import (  # noqa: F401
    CONFIGS, KIN_HEAVE_PITCH, KIN_FOURIER6, KIN_SPLINE8, config_mesh, config_mu,
    fourier6_samples, state_perturbation, free_stream_state, MU_C0, MU_F6_BASE, MU_F6_SCALE, MU_SPLINE8,
    PHYS,
)
