"""Oracle DSA (diffusion synthetic acceleration) preconditioner, FP64, numpy/scipy (test infrastructure only).

Appendix A of the paper derives a DSA discretisation consistent with the upwind DG transport operator in
1D; this module extends it to the 2D X-Y geometry axis by axis and solves the resulting systems exactly
(sparse direct solves).

Operators on the DG space (rows: test function eta_k, columns: trial eta_l), per axis d:
  (D_C,d)_{kl} = - sum_T int_T d_d eta_k eta_l  - sum_{faces F normal to d} int_F {eta_l} [eta_k]
  (D_J,d)_{kl} = - sum_{faces F normal to d} int_F [eta_l] [eta_k]
with [f] = f^+ - f^- (+: the cell on the high side of the face), {f} = (f^+ + f^-) / 2, and on boundary
faces the exterior trace taken as zero.  With that convention the upwind operator with vacuum inflow is
D_j = sum_d Omega_d (D_C,d - sign(Omega_d)/2 D_J,d), D_C,d is skew-symmetric and D_J,d symmetric
negative semi-definite.

The 0th and first angular moments (weights omega_j, sum omega = 1, quadrature symmetric under each
reflection Omega_d -> -Omega_d) of the upwind correction equation with the P1 ansatz
delta psi_j = delta phi + 3 Omega_j . delta J give
  0th:  3 sum_d mu2_d D_C,d dJ_d - sum_d kappa_d D_J,d dphi + Sigma_a dphi = Sigma_s r
  1st:  mu2_d D_C,d dphi + (3 mu2_d Sigma_t - 3/2 sum_e c_de D_J,e) dJ_d = 0
with mu2_d = sum w Omega_d^2, kappa_d = sum_{Omega_d > 0} w Omega_d, c_de = sum w Omega_d^2 |Omega_e|.  For a
quadrature exact on quadratics 3 mu2_d = 1 and, in 1D (c = 2 sum_{v>0} w v^3), these are the appendix's
two moment equations.  Fully consistent DSA solves the coupled (dphi, dJ) system; partially consistent
DSA drops the D_J term of the first-moment equation, dJ_d = -Sigma_t^{-1} D_C,d dphi / 3, leaving
  K_PC = Sigma_a - sum_d kappa_d D_J,d - sum_d mu2_d D_C,d Sigma_t^{-1} D_C,d     (symmetric positive definite).
The lumped fully consistent form ("lumped") keeps the D_J term but replaces the first-moment operator
B_d = 3 mu2_d Sigma_t - 3/2 sum_e c_de D_J,e by its cell-diagonal blocks before eliminating dJ:
  K_LFC = Sigma_a - sum_d kappa_d D_J,d - sum_d 3 mu2_d^2 D_C,d blockdiag(B_d)^{-1} D_C,d            (SPD).
As a right preconditioner of A~ = I - T Sigma_s (one source iteration plus its DSA correction):
  M_DSA^{-1} v = v + dphi(Sigma_s v).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _axis_factors(h: float):
    """1D orthonormal Legendre factors on a cell of width h (p_0 = 1/sqrt(h), p_1 = sqrt(3/h) xi):
    low-end and high-end traces, and the volume matrix V[a_k, a_l] = int p_{a_k}' p_{a_l} dx."""
    s = 1.0 / math.sqrt(h)
    lo = np.array([s, -math.sqrt(3.0) * s])
    hi = np.array([s, math.sqrt(3.0) * s])
    V = np.zeros((2, 2))
    V[1, 0] = 2.0 * math.sqrt(3.0) / h
    return lo, hi, V


def dg_operators(p):
    """(D_C, D_J) per axis as sparse matrices [ndof, ndof]: a list with one pair (x) in 1D, two (x, y) in 2D."""
    nd, nx, ny = p.nd, p.nx, p.ny
    ops = []
    axes = [0] if p.dim == 1 else [0, 1]
    for d in axes:
        h = p.hx if d == 0 else p.hy
        lo, hi, V = _axis_factors(h)
        rows, cols, vc, vj = [], [], [], []

        def add(ck, cl, k, l, c_val, j_val):
            rows.append(ck * nd + k)
            cols.append(cl * nd + l)
            vc.append(c_val)
            vj.append(j_val)

        # local dof k = a + 2b: the axis-d degree and the transverse degree (identity factor)
        def split(k):
            if p.dim == 1:
                return k, 0
            a, b = k % 2, k // 2
            return (a, b) if d == 0 else (b, a)

        locs = [split(k) for k in range(nd)]
        n_along = nx if d == 0 else ny
        n_across = 1 if p.dim == 1 else (ny if d == 0 else nx)

        def cell(i_along, i_across):
            return (i_across * nx + i_along) if d == 0 else (i_along * nx + i_across)

        for t in range(n_across):
            for i in range(n_along):
                c = cell(i, t)
                # volume: - int d_d eta_k eta_l
                for k in range(nd):
                    ak, tk = locs[k]
                    for l in range(nd):
                        al, tl = locs[l]
                        if tk == tl and V[ak, al] != 0.0:
                            add(c, c, k, l, -V[ak, al], 0.0)
                # faces on the low side of cell i (interior or boundary), and the high boundary
                for face in ("low", "high_boundary") if i == n_along - 1 else ("low",):
                    if face == "low":
                        plus = c                                   # this cell is on the high side
                        minus = cell(i - 1, t) if i > 0 else None  # None: exterior
                    else:
                        plus, minus = None, c
                    for k in range(nd):
                        ak, tk = locs[k]
                        for l in range(nd):
                            al, tl = locs[l]
                            if tk != tl:
                                continue
                            # [eta_k] and {eta_l} restricted to the cells that own k / l
                            for ck, jump_k in ((plus, lo[ak]), (minus, -hi[ak])):
                                if ck is None:
                                    continue
                                for cl, tr_l, sgn in ((plus, lo[al], 1.0), (minus, hi[al], -1.0)):
                                    if cl is None:
                                        continue
                                    avg_l = 0.5 * tr_l
                                    jmp_l = sgn * tr_l
                                    add(ck, cl, k, l, -avg_l * jump_k, -jmp_l * jump_k)
        n = p.ndof
        DC = sp.csr_matrix((vc, (rows, cols)), shape=(n, n))
        DJ = sp.csr_matrix((vj, (rows, cols)), shape=(n, n))
        DC.sum_duplicates()
        DJ.sum_duplicates()
        ops.append((DC, DJ))
    return ops


def quadrature_moments(p):
    """mu2_d = sum w Omega_d^2, kappa_d = sum_{Omega_d > 0} w Omega_d, c_de = sum w Omega_d^2 |Omega_e|."""
    naxes = 1 if p.dim == 1 else 2
    om = np.asarray(p.dirs)[:, :naxes]
    w = np.asarray(p.w)
    mu2 = np.array([np.sum(w * om[:, d] ** 2) for d in range(naxes)])
    kappa = np.array([np.sum(w * np.where(om[:, d] > 0, om[:, d], 0.0)) for d in range(naxes)])
    c = np.array([[np.sum(w * om[:, d] ** 2 * np.abs(om[:, e])) for e in range(naxes)] for d in range(naxes)])
    return mu2, kappa, c


def _cell_blocks(M, nd):
    """Keep only the cell-diagonal nd x nd blocks of a sparse matrix."""
    M = sp.coo_matrix(M)
    keep = (M.row // nd) == (M.col // nd)
    return sp.csr_matrix((M.data[keep], (M.row[keep], M.col[keep])), shape=M.shape)


def eliminated_operator(p, kind, ops=None):
    """K_PC ('partial') or K_LFC ('lumped') as a sparse matrix on the DG space."""
    ops = dg_operators(p) if ops is None else ops
    mu2, kappa, c = quadrature_moments(p)
    K = sp.diags(p.sig_t_dof - p.sig_s_dof)
    for d, (DC, DJ) in enumerate(ops):
        K = K - kappa[d] * DJ
    for d, (DC, DJ) in enumerate(ops):
        if kind == "partial":
            Binv = sp.diags(1.0 / (3.0 * mu2[d] * p.sig_t_dof))
        else:
            Bd = 3.0 * mu2[d] * sp.diags(p.sig_t_dof)
            for e, (DCe, DJe) in enumerate(ops):
                Bd = Bd - 1.5 * c[d, e] * DJe
            Bd = _cell_blocks(Bd, p.nd)
            Binv = sp.block_diag([sp.csr_matrix(np.linalg.inv(Bd[i:i + p.nd, i:i + p.nd].toarray()))
                                  for i in range(0, p.ndof, p.nd)], format="csr")
        K = K - 3.0 * mu2[d] ** 2 * (DC @ Binv @ DC)
    return sp.csr_matrix(K)


class Dsa:
    """The DSA correction of one problem: solve(rhs) returns dphi for the 0th-moment right-hand side
    Sigma_s r; apply(v) = v + solve(Sigma_s v) is the right preconditioner of A~."""

    def __init__(self, p, consistent: str = "full"):
        assert consistent in ("full", "partial", "lumped")
        self.p = p
        self.kind = consistent
        ops = dg_operators(p)
        mu2, kappa, c = quadrature_moments(p)
        n = p.ndof
        sa = sp.diags(p.sig_t_dof - p.sig_s_dof)
        st = sp.diags(p.sig_t_dof)
        Kphi = sa.copy()
        for d, (DC, DJ) in enumerate(ops):
            Kphi = Kphi - kappa[d] * DJ
        if consistent in ("partial", "lumped"):
            self.K = sp.csc_matrix(eliminated_operator(p, consistent, ops))
            self.n_unknowns = n
        else:
            naxes = len(ops)
            blocks = [[None] * (naxes + 1) for _ in range(naxes + 1)]
            blocks[0][0] = Kphi
            for d, (DC, DJ) in enumerate(ops):
                blocks[0][d + 1] = 3.0 * mu2[d] * DC
                blocks[d + 1][0] = mu2[d] * DC
                JJ = 3.0 * mu2[d] * st
                for e, (DCe, DJe) in enumerate(ops):
                    JJ = JJ - 1.5 * c[d, e] * DJe
                blocks[d + 1][d + 1] = JJ
            self.K = sp.csc_matrix(sp.bmat(blocks))
            self.n_unknowns = (naxes + 1) * n
        self._lu = spla.splu(self.K)

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        """dphi from the 0th-moment right-hand side (Sigma_s r)."""
        b = np.zeros(self.n_unknowns)
        b[:self.p.ndof] = rhs
        return self._lu.solve(b)[:self.p.ndof]

    def apply(self, v: np.ndarray) -> np.ndarray:
        return v + self.solve(self.p.sig_s_dof * v)


# ----------------------------------------------------------------------------- approximate DSA solve
# The paper solves the DSA diffusion system with algebraic multigrid and does not fix the cycle.  The
# approximate solve used with the GPU path is one multigrid V-cycle on K_LFC (or K_PC):
#   DG level:  damped 4x4 (2x2 in 1D) cell-block Jacobi, x = omega Kcc^{-1} b, then the coarse correction,
#              then x += omega Kcc^{-1} (b - K x);
#   level 1:   continuous piecewise bilinear (linear in 1D) functions on the same mesh, embedded into the
#              DG space by P_c, with the Galerkin operator P_c^T K P_c;
#   level l+1: the same on the mesh coarsened by 2 in every axis (bilinear interpolation, Galerkin
#              operator), while every axis stays even and the mesh has more than 4 cells (2 in 1D);
#   vertex levels: one damped point-Jacobi step before and after the coarse correction;
#   coarsest:  exact dense solve.
# Written with explicit sparse matrices and triple products so that every step can be read off directly.


def continuous_prolongation(p):
    """P_c: vertex values of a continuous piecewise (bi)linear function -> its DG coefficients.  On a cell of
    width h the 1D factor maps the end values (u_lo, u_hi) to (sqrt(h)(u_lo+u_hi)/2, sqrt(h)(u_hi-u_lo)/(2 sqrt 3)),
    the orthonormal Legendre coefficients of the linear interpolant; 2D is the tensor product."""
    def factor(h):
        r = math.sqrt(h)
        return np.array([[r / 2.0, r / 2.0], [-r / (2.0 * math.sqrt(3.0)), r / (2.0 * math.sqrt(3.0))]])

    Fx = factor(p.hx)
    nvx = p.nx + 1
    rows, cols, vals = [], [], []
    if p.dim == 1:
        for ix in range(p.nx):
            for a in range(2):
                for vx in range(2):
                    rows.append(ix * 2 + a)
                    cols.append(ix + vx)
                    vals.append(Fx[a, vx])
        return sp.csr_matrix((vals, (rows, cols)), shape=(p.ndof, nvx))
    Fy = factor(p.hy)
    for iy in range(p.ny):
        for ix in range(p.nx):
            c = iy * p.nx + ix
            for b in range(2):
                for a in range(2):
                    for vy in range(2):
                        for vx in range(2):
                            rows.append(c * 4 + a + 2 * b)
                            cols.append((iy + vy) * nvx + ix + vx)
                            vals.append(Fx[a, vx] * Fy[b, vy])
    return sp.csr_matrix((vals, (rows, cols)), shape=(p.ndof, nvx * (p.ny + 1)))


def _interp_1d(nc):
    """Linear interpolation from nc+1 coarse vertices to 2nc+1 fine vertices."""
    P = np.zeros((2 * nc + 1, nc + 1))
    for i in range(2 * nc + 1):
        if i % 2 == 0:
            P[i, i // 2] = 1.0
        else:
            P[i, i // 2] = P[i, i // 2 + 1] = 0.5
    return sp.csr_matrix(P)


def vertex_interpolation(ncx, ncy, dim=2):
    """Bilinear interpolation from the vertices of an ncx x ncy cell grid to those of the 2ncx x 2ncy grid
    (row-major, x fastest)."""
    if dim == 1:
        return _interp_1d(ncx)
    return sp.csr_matrix(sp.kron(_interp_1d(ncy), _interp_1d(ncx)))


def coarsen(ncx, ncy, dim=2):
    """Next coarser cell grid, or None at the coarsest level."""
    if dim == 1:
        return (ncx // 2, 1) if ncx % 2 == 0 and ncx > 2 else None
    if ncx % 2 == 0 and ncy % 2 == 0 and ncx * ncy > 4:
        return ncx // 2, ncy // 2
    return None


class MultigridDsa:
    """One V-cycle of the approximate DSA solve (see the comment above); apply(v) = v + cycle(Sigma_s v)."""

    def __init__(self, p, kind="lumped", omega=0.7, omega_v=0.7):
        assert kind in ("lumped", "partial")
        self.p = p
        self.omega, self.omega_v = omega, omega_v
        self.K = eliminated_operator(p, kind)
        nd = p.nd
        self.Kcc_inv = sp.block_diag([sp.csr_matrix(np.linalg.inv(self.K[i:i + nd, i:i + nd].toarray()))
                                      for i in range(0, p.ndof, nd)], format="csr")
        self.P = [continuous_prolongation(p)]          # P[0]: level 1 -> DG; P[l]: level l+1 -> level l
        self.A = [sp.csr_matrix(self.P[0].T @ self.K @ self.P[0])]
        self.dims = [(p.nx, p.ny)]
        nxt = coarsen(p.nx, p.ny, p.dim)
        while nxt is not None:
            Pv = vertex_interpolation(nxt[0], nxt[1], p.dim)
            self.P.append(Pv)
            self.A.append(sp.csr_matrix(Pv.T @ self.A[-1] @ Pv))
            self.dims.append(nxt)
            nxt = coarsen(nxt[0], nxt[1], p.dim)
        self.Dinv = [1.0 / A.diagonal() for A in self.A]
        self.coarsest = self.A[-1].toarray()

    def _vertex_cycle(self, l, b):
        if l == len(self.A) - 1:
            return np.linalg.solve(self.coarsest, b)
        A = self.A[l]
        u = self.omega_v * self.Dinv[l] * b
        r = b - A @ u
        u = u + self.P[l + 1] @ self._vertex_cycle(l + 1, self.P[l + 1].T @ r)
        return u + self.omega_v * self.Dinv[l] * (b - A @ u)

    def cycle(self, b):
        x = self.omega * (self.Kcc_inv @ b)
        r = b - self.K @ x
        x = x + self.P[0] @ self._vertex_cycle(0, self.P[0].T @ r)
        return x + self.omega * (self.Kcc_inv @ (b - self.K @ x))

    def apply(self, v):
        return v + self.cycle(self.p.sig_s_dof * v)
