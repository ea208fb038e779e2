"""Plain, slow FP64 CPU oracle for the monolithic ph-multigrid Stokes solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may use it.  It shares no code with the CUDA path: it has
its own meshes, Lagrange bases (Silvester's barycentric product form), Stroud
conical-product quadrature, assembly, transfers, Vanka-star patches, additive
Schwarz, Chebyshev smoothing, Arnoldi eigenvalue estimate, V-cycle, bordered
coarse solve and FGMRES.  Every function cites the section or equation of
"Monolithic Multigrid Preconditioners for High-Order Discretizations of Stokes
Equations" (Voronin, Harper, MacLachlan, Olson, Tuminaro; arXiv 2407.07253)
that it follows.

Modules:
  geometry     nested uniform refinement, Alfeld split, boundary entities
  lagrange     equispaced Lagrange basis on simplices, quadrature
  stokes       TH / SV spaces, DoF maps, assembly of K = [nu A, B^T; B, 0]
  multigrid    transfers, patches, ASM, Chebyshev, Arnoldi, V-cycle, FGMRES
  rng          SplitMix64 counter-based generator (Arnoldi start vectors)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``; the solver's iteration counts are "parity
unpinned" against the paper (its iteration tables were figures that are not
in the text), only the qualitative trends are checked.
"""
