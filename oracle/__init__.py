"""Plain, slow FP64 CPU oracle for AGCA multigrid on Kuhn tetrahedral grids.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package; only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg use it.  It shares no code with the CUDA
library and derives every quantity its own way (geometry from vertex
coordinates, barycentric inversion, centroid containment, explicit sparse
matrices, library factorizations).

Modules:
  mesh      Kuhn meshes, geometry, parent/child maps, interpolation (Sec. 2, Eq. 2.2, Eq. 2.4)
  fem       element matrices and global assembly of Eqs. 3.4-3.5
  agca      viscosity hierarchy (arithmetic / harmonic / geometric coarse means), flags (ratio
            rule; gradient rule of Eq. 2.8), element-wise Galerkin (Eqs. 2.6-2.9), V-cycle,
            per-vertex 15-offset stencils of the level operators (Remark 5)
  stokes    Stokes operator, MINRES (Remark 6), direct solve, adjoint gradient
  fgmres    the paper's outer solver: FGMRES, block-triangular Q (Eq. 4.1), diag(A)-BFBT (Eq. 4.2)
  pointwise per-vertex rows of the fine operator for sampled checks at large sizes
  partition the hierarchy, V-cycle and MINRES split over z-slabs, one rank per slab, with
            interface-plane sums and all-reduced scalars (Remark 1; run as gloo ranks)

Parity status: every function here is pinned by tests/test_oracle_*.py
(partition: by tests/test_multirank_partition.py against the single-process
oracle)
(closed forms, invariants, brute force, library routines, convergence rates),
except the iteration counts of the preconditioned solve, which the paper
prints only as figures (parity unpinned for iteration counts; the solutions
themselves are pinned against a sparse direct solve).
"""
