"""Plain FP64 CPU oracle for the p-multigrid-preconditioned SEM pressure-Poisson solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or run it.  It shares no code with the CUDA path.

Every function follows the paper (arXiv 2411.14977) in its own notation and order of
steps, with assembled sparse matrices, dense element matrices and library primitives
(matrix products, Cholesky, sparse LU) only -- no blocking, fusion or reordering.

Modules
  basis  -- orthonormal Legendre basis, LGL nodes/weights, Vandermonde, D, exact mass,
            p-transfer matrices                                       (Sec. 4.3, Sec. 5.2)
  sem    -- sigma-mapped quad mesh, isoparametric metric, element stiffness, assembly,
            load vectors, Dirichlet lifting, direct solves            (Sec. 2.2, Sec. 4.2-4.3)
  mg     -- geometric p-multigrid: level hierarchy, transfers, additive-Schwarz smoother,
            coarse solve, V-cycle, PCG / FCG / PDC                    (Sec. 5)

Parity status per function is stated in each module header.
"""
