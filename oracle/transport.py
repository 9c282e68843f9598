"""Oracle transport operators (paper Sec. 3.1-3.2), FP64, numpy over the C sweep.

Test infrastructure only.
  T s      = sum_j omega_j (D_j + Sigma_t)^{-1} s                 (eq. memory-efficient-SI)
  b~       = sum_j omega_j (D_j + Sigma_t)^{-1} (G + g_j^bc)      (eq. memory-efficient-SI)
  A~ z     = (I - T Sigma_s) z                                     (eq. memory-efficient-rte)
  psi_j    = (D_j + Sigma_t)^{-1} s, all j (the angular-output sweep)
  phi      = Q psi = sum_j omega_j psi_j                           (Sec. 2.3)
  A        = the fully coupled N_Omega*N_DOF system                (eq. one_equation)
Every direction is swept separately (no merging of directions).
"""
from __future__ import annotations

import numpy as np

from .discretization import Problem


def sweep_all(p: Problem, s: np.ndarray, with_bc: bool = False) -> np.ndarray:
    """psi[j] = (D_j + Sigma_t)^{-1} (s + with_bc * g_j^bc) for every direction; shape [N_Omega, N_DOF]."""
    out = np.empty((p.ndir, p.ndof))
    for j in range(p.ndir):
        rhs = s + p.gbc(j) if with_bc else s
        out[j] = p.sweep(j, rhs)
    return out


def scalar_flux(p: Problem, psi: np.ndarray) -> np.ndarray:
    """phi = sum_j omega_j psi_j."""
    phi = np.zeros(p.ndof)
    for j in range(p.ndir):
        phi += p.w[j] * psi[j]
    return phi


def T_apply(p: Problem, s: np.ndarray) -> np.ndarray:
    """T s = sum_j omega_j (D_j + Sigma_t)^{-1} s."""
    phi = np.zeros(p.ndof)
    for j in range(p.ndir):
        phi += p.w[j] * p.sweep(j, s)
    return phi


def rhs_btilde(p: Problem) -> np.ndarray:
    """b~ = sum_j omega_j (D_j + Sigma_t)^{-1} (G + g_j^bc)."""
    phi = np.zeros(p.ndof)
    for j in range(p.ndir):
        phi += p.w[j] * p.sweep(j, p.G + p.gbc(j))
    return phi


def Atilde_apply(p: Problem, z: np.ndarray) -> np.ndarray:
    """A~ z = z - T (Sigma_s z)."""
    return z - T_apply(p, p.sig_s_dof * z)


def dense_coupled_system(p: Problem):
    """The fully coupled system A psi = b of eq. one_equation, assembled densely.

    Block (i, i) = D_i + Sigma_t - omega_i Sigma_s, block (i, k) = -omega_k Sigma_s,
    b = (G~_1, ..., G~_N).  Only for tiny meshes.
    """
    n = p.ndof
    N = p.ndir * n
    A = np.zeros((N, N))
    Ss = np.diag(p.sig_s_dof)
    b = np.empty(N)
    for i in range(p.ndir):
        A[i * n:(i + 1) * n, i * n:(i + 1) * n] = p.dense_L(i)
        for k in range(p.ndir):
            A[i * n:(i + 1) * n, k * n:(k + 1) * n] -= p.w[k] * Ss
        b[i * n:(i + 1) * n] = p.G + p.gbc(i)
    return A, b
