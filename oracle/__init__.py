"""Oracle: a plain, slow, FP64 CPU restatement of the ADER-DG time step with a-posteriori
finite-volume subcell limiting (Sec. 3.3-3.5 of the ExaHyPE paper, arXiv 1905.07987).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may use it.  It shares no code, tables or helpers with the CUDA library
under ``paper_1905_07987_gb300/csrc``; both sides receive the same seeded inputs from
``paper_1905_07987_gb300/synth.py``, which holds none of the method's arithmetic.

Written with plain PyTorch CPU tensor operations in float64 (so that reverse-mode automatic
differentiation of the forward step gives the reference adjoint), one function per step of
the method, in the paper's order:

* ``refelem``  - Gauss-Legendre nodes, Lagrange basis, derivative and end-value tables,
                 the time-stiffness matrix of the predictor, subcell projections.
* ``pde``      - flux / non-conservative product / eigenvalue terms of the PDEs used
                 (scalar advection, compressible Euler, linear elasticity, shallow water
                 with bathymetry).
* ``aderdg``   - CFL time step, Picard and Cauchy-Kowalevski space-time predictors, time averages, face
                 extrapolation, Rusanov Riemann solver, corrector, point source, receivers.
* ``limiter``  - subcell projection, relaxed DMP + positivity detection, MUSCL-Hancock
                 recompute of troubled cells and the conservative neighbour face fix.
* ``ck``       - brute-force (dense, Kronecker-assembled) Cauchy-Kowalevski predictor for linear
                 PDEs on one cell: an independent route that pins the Picard predictor and the
                 scheme's own Cauchy-Kowalevski predictor (``aderdg.ADERDG.predictor_ck``).

Functions whose result has no independent pin say "parity unpinned" in their docstring.
"""
