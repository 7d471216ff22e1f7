"""FP64 CPU oracle for the periodic shooting / periodic adjoint method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product (the CUDA library and its Python binding) never
imports, links or executes anything here, and this package never imports the
product.  The two share no code; only the seeded input generators in
``pp_inputs`` (which hold none of the method's arithmetic) serve both.

It is a plain, slow, step-by-step restatement of the method of Zahr, Persson
and Wilkening, "A fully discrete adjoint method for optimization of flow
problems on deforming domains with time-periodicity constraints":

* ``dirk``      -- the 3-stage DIRK scheme (Eqs. dirk, dirk-stage).
* ``refelem``   -- nodal basis and quadrature on the reference triangle.
* ``dg``        -- the ALE DG semi-discretization r(u, mu, t) of the
                   compressible Navier-Stokes equations (Sec. 6, Eqs.
                   ns1-ns5, ns-cons-ref, transform1/2-nogcl, defmap), the
                   instantaneous QoIs (Eq. qoi) and their exact derivatives
                   by the complex-step method.
* ``periodic``  -- primal sweep (Eq. dirk2), tangent sweep (Eq.
                   dirk-sens-mvp), Newton-Krylov shooting (Algorithm
                   primal), adjoint sweep (Eq. uns-disc-adj-dirk2), periodic
                   adjoint GMRES (Algorithm dual) and gradient (Eq.
                   funcl-grad-nosens-dirk, Algorithm grad).

Parity status: absolute QoI values are "parity unpinned" (the paper's numbers
are for a different, unpublished setup); every other function is pinned by a
``-m "not gpu"`` test against closed forms, invariants, finite differences or
brute force.
"""
