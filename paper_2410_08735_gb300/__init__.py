"""GB300 (sm_103a) FGMRES-ROMSAD solver for the parametric radiative transfer equation.

The compute path is librte_gb300.so (hand-written CUDA kernels behind the C ABI
of include/rte.h); this package only builds and binds it.
"""
from .binding import (Mlp, Problem, Rom, RteError, attach_mlp, fgmres_solve, si_solve, load, RTE_F32, RTE_F64,  # noqa: F401
                      RTE_MODE_FP64, RTE_MODE_MIXED, RTE_MODE_MIXED_F64KRYLOV, RTE_POST_IDENTITY, RTE_POST_ROM,
                      RTE_POST_DSA, RTE_DSA_PARTIAL, RTE_DSA_LUMPED)
