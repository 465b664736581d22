"""Plain FP64 CPU oracle for the fourth-order AMR elliptic solves of Zhao & Zhang,
"Fourth-order AMR both in space and in time for incompressible Navier-Stokes equations
with Dirichlet boundary conditions" (arXiv 2506.02663).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product path (``paper_2506_02663_gb300``) never imports it and shares no code with it.

Conventions
-----------
* Arrays are indexed by dimension: axis ``d`` of a level array is the paper's dimension
  ``d`` (x = axis 0).  A level array covers the bounding box of the level's boxes grown by
  the two ghost layers of Sec. 3 (the "two-layer wrapping" paragraph after Eq. (appProj)).
* Everything is float64; exact-rational coefficients are kept as ``fractions.Fraction`` in
  ``stencil.py`` and converted once.
* No blocking, fusion or reordering beyond what the paper's definitions state.

Modules
-------
``stencil``    Eqs. (cell2face), (discreteOps), (velBCHomoDiri5th), (Neumann5): coefficients,
               physical ghost fill, level operators G, D, L and face fluxes.
``cfi``        the conservative fifth-order coarse-fine interpolation (AMRCFI, Sec. 5.2);
               the paper only cites it, so the oracle uses the reading stated there.
``hierarchy``  Sec. 5.1: boxes, proper refinement/nesting, valid/invalid regions,
               connected components, index maps.
``composite``  Sec. 5.2-5.3: average-down, CF ghost fill, COH-1..4 composite operators,
               refluxing, composite projection (Eq. comp_ProjOp).
``solve``      sparse assembly of the composite operator, direct solves, solvability fix
               (Sec. 6.4), mean-zero, transposes (adjoint).
``mg``         Sec. 6.5 geometric multigrid (V-cycle with weighted Jacobi, omega = 2/3).
``cic``        Sec. 6.3-6.4 interface conditions of the subcycled solves: the time
               interpolation I^(4) (Eq. timeInterp), the interface faces and components, the
               per-component correction of the interface face averages (Eq.
               correctingFaceAvg), and the boundary data of single-box level problems.
``regrid``     Sec. 5.4 RDM-2/3: Berger-Rigoutsos clustering of tagged cells into the boxes
               of a new hierarchy, finest level first; the data migration after it.
``convection`` Eq. (convOp): the fourth-order cell-averaged convection operator.
``imex``       the ERK-ESDIRK tableau of Eq. (GePUP-IMEX) and one additive Runge-Kutta step.
"""
