"""Plain FP64 CPU oracle for the multilevel elastodynamics timestep.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library in
``paper_2508_13386_gb300`` never imports it and never falls back to it.

Everything here is written to be checked by eye against the paper
(arXiv 2508.13386, "Sparse, Geometry- and Material-Aware Bases for Multilevel
Elastodynamic Simulation"): numpy/scipy in float64, vectorised over elements
only where the per-element formula is unchanged, with library routines
(``eigh``, Cholesky, sparse LU) as the only building blocks.

Modules:
  elastic    non-inverting Neo-Hookean energy, stress, stress derivative,
             per-element PSD-projected Hessian (Sec. 4 material model)
  barrier    point-plane IPC log barrier (Eq. IP, contact term B)
  friction   lagged, mollified point-plane friction D (Eq. IP, term D)
  contact    mesh-mesh point-triangle and edge-edge barrier pairs and their
             conservative CCD (Eq. IP term B, Sec. 3.9 CCD filter)
  ip         incremental potential E, gradient, Hessian (Eq. IP, implicit
             Euler or BDF2, Sec. 3.1)
  newton     projected Newton timestep with filtered backtracking line search
             (Eq. 5 linear solve; Sec. 3.9 line search), and the paper's
             inexact timestep (Alg. 1 with Alg. 2's directions)
  subspace   LBS basis matrix U (Eq. LBS, SMS basis), restriction/prolongation,
             Galerkin operator U^T H U, two-level preconditioner algebra
             (Alg. 2, Sec. 3.7.1)
  pcg        preconditioned conjugate gradient written from its definition
  mlp        FP64 MLP forward/backward and Adam (learned warm start)

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test unless it says "parity unpinned".
"""
