"""FP64 CPU oracle for the implicit unsteady UGKS on moving / overset meshes.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
numpy restatement of the method of arXiv 2604.09984 ("Unified Gas-Kinetic
Scheme for Unsteady Multiscale Flows with Moving Boundaries").  Only the test
suite (``tests/``), ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or execute it.  The CUDA
product path never imports it, and it imports nothing from the CUDA path: the
only code the two sides share is the seeded input generator
``paper_2604_09984_gb300.workloads`` (mesh nodes, prescribed motion and initial
primitive fields; no arithmetic of the method).

Modules
  kinetic   Shakhov model in reduced form (Sec. 2.1), discrete velocity space,
            moments, micro-slopes of the interface equilibrium, time
            coefficients of the integral solution (Eq. fullSolution).
  mesh      structured-block topology and ALE geometry (mid-time faces,
            swept-area face velocity, cell volumes at both time levels).
  ugks      reconstruction, interface flux (Eqs. microscopicFlux,
            macroscopicFlux, fullSolution, maxWalldes), residuals and the
            dual-time Crank-Nicolson step with macro + micro LU-SGS
            (Sec. 2.2, Eqs. dualTimeStepping_macro/micro, Steps 1-8).
  overset   overset assembly (Sec. 3.1) and inverse-distance interpolation
            (Sec. 3.2).
  adjoint   transposes of the step's linear operators (micro LU-SGS solve,
            receptor interpolation, velocity moments) and the tangents and
            adjoints of the macro LU-SGS and of Step 7: first pieces of a
            discrete adjoint.

Parity status
  Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
  brute force, invariants or limits, except the physical fidelity of the
  paper's experiments (figures only, no data): parity unpinned for those.
"""
