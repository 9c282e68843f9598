"""Oracle transport operators (paper Sec. 3.1-3.2), FP64, numpy over the C sweep.

Test infrastructure only.
  T s      = sum_j omega_j (D_j + Sigma_t)^{-1} s                 (eq. memory-efficient-SI)
  b~       = sum_j omega_j (D_j + Sigma_t)^{-1} (G + g_j^bc)      (eq. memory-efficient-SI)
  A~ z     = (I - T Sigma_s) z                                     (eq. memory-efficient-rte)
  psi_j    = (D_j + Sigma_t)^{-1} s, all j (the angular-output sweep)
  phi      = Q psi = sum_j omega_j psi_j                           (Sec. 2.3)
  A        = the fully coupled N_Omega*N_DOF system                (eq. one_equation)
  A_refl   = the same system of a 1D slab whose ends reflect specularly (an oracle-only boundary
             condition; the paper's problems have inflow boundaries, eq. 1c)
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
    return z - T_apply(p, p.Ss_apply(z))


def _block_diag(blocks: np.ndarray) -> np.ndarray:
    n, nd, _ = blocks.shape
    out = np.zeros((n * nd, n * nd))
    for c in range(n):
        out[c * nd:(c + 1) * nd, c * nd:(c + 1) * nd] = blocks[c]
    return out


def dense_coupled_system(p: Problem):
    """The fully coupled system A psi = b of eq. one_equation, assembled densely.

    Block (i, i) = D_i + Sigma_t - omega_i Sigma_s, block (i, k) = -omega_k Sigma_s,
    b = (G~_1, ..., G~_N).  Only for tiny meshes.
    """
    n = p.ndof
    N = p.ndir * n
    A = np.zeros((N, N))
    Ss = np.diag(p.sig_s_dof) if p.Ss_blk is None else _block_diag(p.Ss_blk)
    b = np.empty(N)
    for i in range(p.ndir):
        A[i * n:(i + 1) * n, i * n:(i + 1) * n] = p.dense_L(i)
        for k in range(p.ndir):
            A[i * n:(i + 1) * n, k * n:(k + 1) * n] -= p.w[k] * Ss
        b[i * n:(i + 1) * n] = p.G + p.gbc(i)
    return A, b


def dense_reflecting_1d(p: Problem, left: bool = True, right: bool = True):
    """The coupled system A psi = b (eq. one_equation) of a 1D slab with specular reflection at the
    chosen ends, assembled densely; vacuum at an end that does not reflect.  Only for tiny meshes.

    At a reflecting end the inflow value of ordinate mu is the outgoing value of the mirrored ordinate
    -mu at the same point, psi(x_b, mu) = psi(x_b, -mu).  In the upwind flux of eq. DG (eq. upwind) the
    inflow face term (Omega . n) eta_k psi^up of direction i then couples to the trace of direction i'
    (mu_i' = -mu_i) taken from the boundary cell itself, instead of a known g moved to the right-hand
    side.  The Gauss-Legendre ordinates are symmetric, so i' exists.
    """
    assert p.dim == 1
    A, b = dense_coupled_system(p)
    n = p.ndof
    mus = np.array([d[0] for d in p.dirs])
    e_lo = p._eta(np.array([-1.0]))[:, 0]   # basis values at the cell's low end
    e_hi = p._eta(np.array([1.0]))[:, 0]
    for i in range(p.ndir):
        mirror = int(np.argmin(np.abs(mus + mus[i])))
        assert abs(mus[mirror] + mus[i]) < 1e-14
        if mus[i] > 0 and left:          # inflow through the low face of cell 0 (n = -1)
            c = 0
            on = -mus[i]
            A[i * n + 2 * c:i * n + 2 * c + 2, mirror * n + 2 * c:mirror * n + 2 * c + 2] += on * np.outer(e_lo, e_lo)
        if mus[i] < 0 and right:         # inflow through the high face of the last cell (n = +1)
            c = p.nx - 1
            on = mus[i]
            A[i * n + 2 * c:i * n + 2 * c + 2, mirror * n + 2 * c:mirror * n + 2 * c + 2] += on * np.outer(e_hi, e_hi)
    return A, b


def solve_reflecting_1d(p: Problem, left: bool = True, right: bool = True) -> np.ndarray:
    """phi = Q A_refl^{-1} b by dense LU (numpy), for the reflecting slab of dense_reflecting_1d."""
    A, b = dense_reflecting_1d(p, left, right)
    psi = np.linalg.solve(A, b).reshape(p.ndir, p.ndof)
    return scalar_flux(p, psi)
