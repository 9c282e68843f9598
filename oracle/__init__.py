"""CPU oracle for the FGMRES-ROMSAD solver of the parametric RTE (FP64).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import, call or link anything
in this package; the product path (paper_2410_08735_gb300) never does, and it
shares no code with this package.

Modules (each cites the passages it follows):
  discretization  quadrature, orthonormal Q1 upwind DG blocks, source, g^bc (Sec. 2)
  sweep.c         one-direction upwind block Gauss-Seidel sweep and forward operator (Sec. 3.1)
  transport       T, b~, A~, angular sweep, scalar flux, dense coupled system (Sec. 3)
  krylov          FGMRES (Alg. 1) with restarts; source iteration (Sec. 3.1); SI-SA as a preconditioned
                  Richardson iteration (Sec. 3.2)
  romsad          ROMSAD preconditioner, xi recurrence, snapshots, MGS truncation,
                  greedy ROM construction (Sec. 4, appendix B)
  mlp             MLP forward/backward/Adam used for the learned warm start
  dsa             DG central-flux and jump operators, partially / lumped / fully consistent DSA
                  (appendix A, extended to 2D axis by axis), exact sparse solves and the multigrid V-cycle
  rbf             RBF interpolation of sampled scalar fluxes (the interpolated initial guess of Sec. 5)
Pins are in tests/test_oracle_*.py.  Every function listed here is pinned;
none is "parity unpinned".
"""
from . import discretization, transport, krylov, romsad, dsa, rbf  # noqa: F401
from .discretization import Problem, with_params, gauss_legendre, slab_quadrature, cl_quadrature  # noqa: F401
