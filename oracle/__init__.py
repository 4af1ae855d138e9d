"""Slow, plain FP64 CPU oracle for the DG operators of Fehn, Wall & Kronbichler,
"Efficiency of high-performance discontinuous Galerkin spectral element methods
for under-resolved turbulent incompressible flows" (arXiv:1802.01439).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

How it computes (Sec. 3.2 of the paper): every operator is assembled from
explicit element and face matrices obtained by direct 3D quadrature over the
tensor-product LGL Lagrange basis (no sum factorization, no Kronecker
factorization, no basis change), then applied cell by cell through the periodic
neighbour map.  Linear algebra uses numpy/LAPACK primitives only.

Modules
-------
rules     1D Gauss and Legendre-Gauss-Lobatto rules, Lagrange basis (Sec. 3.2).
dg        mesh, vectors, mass / inverse mass / SIPG Laplace / viscous /
          Helmholtz / divergence / gradient / convective operators (Sec. 3.2).
mg        h-multigrid transfers, Jacobi-Chebyshev smoother, V-cycle (Sec. 3.3).
solvers   preconditioned CG and residual checks (Sec. 3.3).
timestep  BDF2 dual-splitting step and dissipation rate (Secs. 3.1, 4.2).
"""
