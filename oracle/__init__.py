"""Plain FP64 CPU oracle of the cubed-sphere shell dynamo solve path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or calls this package; only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` do.  It shares no code with the CUDA path.

It follows Yin, Yang, Ma, Cai, Zhang, "Parallel finite volume simulation of
the spherical shell dynamo with pseudo-vacuum magnetic boundary conditions"
(arXiv 2009.02171):

* ``grid``      -- equiangular cubed-sphere shell, metric (Sec. 3.2, Eq. for
                   sqrt(g), cell centres), panel-edge ghost interpolation.
* ``discrete``  -- finite-volume operators by the Gauss theorem
                   (eqn:divdiscretization), VTBE / PPBE matrices (eqn:tsvelocity
                   .. eqn:tspb), cell gradient, face divergence, nonlinear
                   conservative fluxes (eqn:nonlinearint).
* ``ilu``       -- ILU(0) factorization / solves (plain C, ``ilu0.c``).
* ``schwarz``   -- one-level RAS (eqn:onelevel) and hybrid two-level RAS
                   (eqn:twolevel, eqn:coarsesolve, eqn:finesolve).
* ``krylov``    -- right-preconditioned restarted (flexible) GMRES with the
                   stopping rule of Sec. 3.3.
* ``timestep``  -- the three-step predictor-corrector (Sec. 3.1, Steps 1-3).

Every function is written for a reader checking it against the paper: no
blocking, fusion or reordering beyond what the formulas state.
"""
