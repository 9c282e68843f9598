"""Oracle discretisation of the steady one-group RTE (paper Sec. 2), FP64, numpy.

Test infrastructure only.  Everything here is computed from the definitions:
  * Sec. 2.1: normalised S_N quadrature (weights sum to 1); Chebyshev-Legendre
    product rule CL(N_theta, N_z) with theta_j = (2j-1) pi / N_theta, weight
    1/N_theta, times an N_z-point Gauss-Legendre rule for Omega_z normalised to
    sum 1; direction index j = (j2-1) N_theta + j1.  The 1D slab uses the
    N-point Gauss-Legendre rule in mu with weights w/2 (appendix A setting).
  * Sec. 2.2, eq. DG and eq. upwind: upwind DG on a uniform Cartesian mesh
    with the Q^1 space; every volume and face integral is evaluated by
    3-point Gauss quadrature per axis (exact for these polynomial integrands).
  * Sec. 2.3: orthonormal basis, so Sigma_t and Sigma_s are diagonal with the
    cell's cross section on each of its dofs; G_k = int G eta_k;
    (g_j^bc)_k = - int_{inflow boundary} g eta_k (Omega_j . n).

Reading of the garbled boundary term in eq. DG: the inflow integrand is
g * eta_h (the test function), as in the definition of g_j^bc in Sec. 2.3.

Basis: orthonormal tensor Legendre, eta_ab(x, y) = p_a(x) q_b(y) with
p_n(x) = sqrt(2/h_x) Ptilde_n(xi), Ptilde_n = sqrt((2n+1)/2) P_n, local dof
index k = a + 2b (1D: k = a).  Cells row-major, c = iy*nx + ix.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

from . import _lib


# ---------------------------------------------------------------- quadrature
def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes (ascending) and weights on [-1, 1].

    Newton's method on P_n evaluated by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; weights 2 / ((1 - x^2) P_n'(x)^2).
    """
    x = np.cos(np.pi * (np.arange(n) + 0.75) / (n + 0.5))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for k in range(1, n):
            p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        if n == 1:
            p0, p1 = np.ones_like(x), x.copy()
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    if n == 1:
        p0, p1 = np.ones_like(x), x.copy()
    dp = n * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def slab_quadrature(n: int):
    """1D slab S_N: directions mu_j (GL nodes) and normalised weights w_j / 2."""
    mu, w = gauss_legendre(n)
    return mu.reshape(-1, 1), w / 2.0


def cl_quadrature(n_theta: int, n_z: int):
    """CL(N_theta, N_z) product rule (Sec. 2.1): returns (Omega [N,3], omega [N])."""
    z, wz = gauss_legendre(n_z)
    wz = wz / 2.0
    dirs = []
    wts = []
    for j2 in range(1, n_z + 1):
        for j1 in range(1, n_theta + 1):
            theta = (2 * j1 - 1) * math.pi / n_theta
            s = math.sqrt(1.0 - z[j2 - 1] ** 2)
            dirs.append((math.cos(theta) * s, math.sin(theta) * s, z[j2 - 1]))
            wts.append(wz[j2 - 1] / n_theta)
    return np.array(dirs), np.array(wts)


# --------------------------------------------------------------------- basis
def _leg(n: int, xi):
    """Normalised Legendre polynomial sqrt((2n+1)/2) P_n(xi) for n = 0, 1."""
    xi = np.asarray(xi, dtype=np.float64)
    if n == 0:
        return np.full_like(xi, math.sqrt(0.5))
    return math.sqrt(1.5) * xi


def _dleg(n: int, xi):
    xi = np.asarray(xi, dtype=np.float64)
    if n == 0:
        return np.zeros_like(xi)
    return np.full_like(xi, math.sqrt(1.5))


_GQ_X, _GQ_W = gauss_legendre(3)


class Problem:
    """One parameter instance of the discretised problem (Sec. 2.1-2.3).

    spec      a workloads.ProblemSpec (only its geometry/order fields are read)
    b         which instance's mesh to use
    sigma_s, sigma_a   per-region cross sections [R]
    """

    def __init__(self, spec, b: int, sigma_s: Sequence[float], sigma_a: Sequence[float]):
        self.dim = spec.dim
        self.nx = spec.nx[b]
        self.ny = spec.ny[b] if spec.dim == 2 else 1
        x0, x1, y0, y1 = spec.box
        self.x0, self.y0 = x0, y0
        self.hx = (x1 - x0) / self.nx
        self.hy = (y1 - y0) / self.ny if spec.dim == 2 else 1.0
        self.nd = 4 if spec.dim == 2 else 2
        self.ncell = self.nx * self.ny
        self.ndof = self.ncell * self.nd
        if spec.dim == 1:
            self.dirs, self.w = slab_quadrature(spec.n_polar)
        else:
            self.dirs, self.w = cl_quadrature(spec.n_azim, spec.n_polar)
        self.ndir = len(self.w)
        self.g = float(spec.inflow_g)
        # cross sections per cell (region of the cell centre), Sec. 2.3 diagonal Sigma
        rx, ry = spec.rx, (spec.ry if spec.dim == 2 else 1)
        Lx, Ly = x1 - x0, (y1 - y0)
        ss = np.asarray(sigma_s, dtype=np.float64)
        sa = np.asarray(sigma_a, dtype=np.float64)
        self.sigma_s_region = ss
        self.sigma_a_region = sa
        region = np.empty(self.ncell, dtype=np.int64)
        for iy in range(self.ny):
            for ix in range(self.nx):
                xc = x0 + (ix + 0.5) * self.hx
                ix_r = min(int((xc - x0) / (Lx / rx)), rx - 1)
                if self.dim == 2:
                    yc = y0 + (iy + 0.5) * self.hy
                    iy_r = min(int((yc - y0) / (Ly / ry)), ry - 1)
                else:
                    iy_r = 0
                region[iy * self.nx + ix] = iy_r * rx + ix_r
        self.region = region
        self.sig_s = ss[region]
        self.sig_t = ss[region] + sa[region]
        self.sig_s_dof = np.repeat(self.sig_s, self.nd)
        self.sig_t_dof = np.repeat(self.sig_t, self.nd)
        # cross-section profiles (spec.sigma_modes): Sigma is a full block per cell, (Sigma)_kl = int_T sigma eta_k eta_l
        self.sigma_modes = getattr(spec, "sigma_modes", None)
        self.mode_blocks = None
        self.Ss_blk = self.St_blk = None
        if self.sigma_modes is not None:
            if self.sigma_modes != "variable_scattering" or self.dim != 2 or len(ss) != 2:
                raise ValueError("sigma_modes: 'variable_scattering' takes two coefficients in 2D")
            eye = np.broadcast_to(np.eye(self.nd), (self.ncell, self.nd, self.nd))
            self.mode_blocks = np.stack([self._project_profile(_varscat_profile), eye])
            _set_blocks(self, ss, sa)
        # per-direction local matrices
        self.M = np.empty((self.ndir, self.nd, self.nd))
        self.C = np.empty((self.ndir, 4, self.nd, self.nd))
        self.inflow = np.zeros((self.ndir, 4), dtype=np.int32)
        for j in range(self.ndir):
            self.M[j], self.C[j], self.inflow[j] = self._assemble_dir(self.dirs[j])
        if getattr(spec, "src_gauss", None) is not None:
            self.G = self._project_gauss(*spec.src_gauss)
        else:
            self.G = self._project_source(spec.src_q, spec.src_box)
        self.inflow_faces = tuple(getattr(spec, "inflow_faces", ("x-", "x+", "y-", "y+")))
        self._gbc = {}

    # ---------------------------------------------------------- assembly
    def _eta(self, xi, zeta=None):
        """Values of the nd basis functions at reference points; shape [nd, npts]."""
        if self.dim == 1:
            s = math.sqrt(2.0 / self.hx)
            return np.stack([s * _leg(a, xi) for a in range(2)])
        s = 2.0 / math.sqrt(self.hx * self.hy)
        return np.stack([s * _leg(k % 2, xi) * _leg(k // 2, zeta) for k in range(4)])

    def _grad_eta(self, xi, zeta=None):
        """(d/dx, d/dy) of the basis at reference points; each [nd, npts]."""
        if self.dim == 1:
            s = math.sqrt(2.0 / self.hx) * (2.0 / self.hx)
            return np.stack([s * _dleg(a, xi) for a in range(2)]), None
        s = 2.0 / math.sqrt(self.hx * self.hy)
        dx = np.stack([s * (2.0 / self.hx) * _dleg(k % 2, xi) * _leg(k // 2, zeta) for k in range(4)])
        dy = np.stack([s * (2.0 / self.hy) * _leg(k % 2, xi) * _dleg(k // 2, zeta) for k in range(4)])
        return dx, dy

    def _assemble_dir(self, omega):
        """Local blocks of D_j for direction omega (eq. DG with the upwind flux, eq. upwind).

        M[k, l] = -int_T (Omega . grad eta_k) eta_l + sum over outflow faces of
                  int_f (Omega . n_f) eta_k eta_l
        C[f][k, l] = int_f (Omega . n_f) eta_k eta_l^nbr  on inflow faces f
        """
        nd = self.nd
        M = np.zeros((nd, nd))
        C = np.zeros((4, nd, nd))
        inflow = np.zeros(4, dtype=np.int32)
        q, wq = _GQ_X, _GQ_W
        if self.dim == 1:
            mu = omega[0]
            eta = self._eta(q)
            dx, _ = self._grad_eta(q)
            jac = self.hx / 2.0
            for k in range(nd):
                for l in range(nd):
                    M[k, l] = -np.sum(wq * mu * dx[k] * eta[l]) * jac
            # faces are the end points: f=0 at xi=-1 (n=-1), f=1 at xi=+1 (n=+1)
            for f, (xi_own, xi_nbr, n) in enumerate(((-1.0, 1.0, -1.0), (1.0, -1.0, 1.0))):
                on = mu * n
                e_own = self._eta(np.array([xi_own]))[:, 0]
                e_nbr = self._eta(np.array([xi_nbr]))[:, 0]
                if on > 0:
                    M += on * np.outer(e_own, e_own)
                elif on < 0:
                    inflow[f] = 1
                    C[f] = on * np.outer(e_own, e_nbr)
            return M, C, inflow
        ox, oy = omega[0], omega[1]
        XI, ZE = np.meshgrid(q, q, indexing="ij")
        W2 = np.outer(wq, wq).ravel()
        XI, ZE = XI.ravel(), ZE.ravel()
        eta = self._eta(XI, ZE)
        dx, dy = self._grad_eta(XI, ZE)
        jac = self.hx * self.hy / 4.0
        for k in range(nd):
            for l in range(nd):
                M[k, l] = -np.sum(W2 * (ox * dx[k] + oy * dy[k]) * eta[l]) * jac
        # faces: (own coords, neighbour coords, Omega.n, face Jacobian)
        ones = np.ones_like(q)
        faces = (
            ((-ones, q), (ones, q), -ox, self.hy / 2.0),   # x-low
            ((ones, q), (-ones, q), ox, self.hy / 2.0),    # x-high
            ((q, -ones), (q, ones), -oy, self.hx / 2.0),   # y-low
            ((q, ones), (q, -ones), oy, self.hx / 2.0),    # y-high
        )
        for f, (own, nbr, on, fj) in enumerate(faces):
            e_own = self._eta(*own)
            e_nbr = self._eta(*nbr)
            if on > 0:
                for k in range(nd):
                    for l in range(nd):
                        M[k, l] += np.sum(wq * on * e_own[k] * e_own[l]) * fj
            elif on < 0:
                inflow[f] = 1
                for k in range(nd):
                    for l in range(nd):
                        C[f, k, l] = np.sum(wq * on * e_own[k] * e_nbr[l]) * fj
        return M, C, inflow

    def _project_source(self, qv: float, box) -> np.ndarray:
        """G_k = int_T G eta_k with G = qv on the box, 0 outside (exact on the intersection)."""
        G = np.zeros(self.ndof)
        xa, xb, ya, yb = box
        q, wq = _GQ_X, _GQ_W
        for iy in range(self.ny):
            for ix in range(self.nx):
                xl = self.x0 + ix * self.hx
                lo_x, hi_x = max(xl, xa), min(xl + self.hx, xb)
                if hi_x <= lo_x:
                    continue
                px = 0.5 * (lo_x + hi_x) + 0.5 * (hi_x - lo_x) * q      # physical Gauss points
                xi = (px - (xl + 0.5 * self.hx)) / (0.5 * self.hx)
                c = iy * self.nx + ix
                if self.dim == 1:
                    eta = self._eta(xi)
                    G[c * 2:(c + 1) * 2] = qv * (eta @ wq) * 0.5 * (hi_x - lo_x)
                    continue
                yl = self.y0 + iy * self.hy
                lo_y, hi_y = max(yl, ya), min(yl + self.hy, yb)
                if hi_y <= lo_y:
                    continue
                py = 0.5 * (lo_y + hi_y) + 0.5 * (hi_y - lo_y) * q
                ze = (py - (yl + 0.5 * self.hy)) / (0.5 * self.hy)
                XI, ZE = np.meshgrid(xi, ze, indexing="ij")
                W2 = np.outer(wq, wq).ravel()
                eta = self._eta(XI.ravel(), ZE.ravel())
                G[c * 4:(c + 1) * 4] = qv * (eta @ W2) * 0.25 * (hi_x - lo_x) * (hi_y - lo_y)
        return G

    def _project_gauss(self, amp: float, a: float, xc: float, yc: float, npts: int = 16) -> np.ndarray:
        """G_k = int_T G eta_k for G = amp exp(-a ((x-xc)^2 + (y-yc)^2)) (2D), by npts x npts Gauss-Legendre
        points per cell (the integrand is smooth; 16 points integrate it to rounding at the workloads' cells)."""
        assert self.dim == 2
        xg, wg = gauss_legendre(npts)
        XI, ZE = np.meshgrid(xg, xg, indexing="ij")
        W2 = np.outer(wg, wg).ravel()
        eta = self._eta(XI.ravel(), ZE.ravel())
        G = np.zeros(self.ndof)
        for iy in range(self.ny):
            for ix in range(self.nx):
                c = iy * self.nx + ix
                px = self.x0 + (ix + 0.5 + 0.5 * XI.ravel()) * self.hx
                py = self.y0 + (iy + 0.5 + 0.5 * ZE.ravel()) * self.hy
                qv = amp * np.exp(-a * ((px - xc) ** 2 + (py - yc) ** 2))
                G[c * 4:(c + 1) * 4] = (eta * qv) @ W2 * 0.25 * self.hx * self.hy
        return G

    def _project_profile(self, fn, npts: int = 16) -> np.ndarray:
        """Blocks F_c[k, l] = int_T f eta_k eta_l of a cross-section profile f(x, y), by npts x npts Gauss-Legendre
        points per cell: [ncell, nd, nd]."""
        xg, wg = gauss_legendre(npts)
        XI, ZE = np.meshgrid(xg, xg, indexing="ij")
        W2 = np.outer(wg, wg).ravel()
        eta = self._eta(XI.ravel(), ZE.ravel())
        F = np.empty((self.ncell, self.nd, self.nd))
        for iy in range(self.ny):
            for ix in range(self.nx):
                px = self.x0 + (ix + 0.5 + 0.5 * XI.ravel()) * self.hx
                py = self.y0 + (iy + 0.5 + 0.5 * ZE.ravel()) * self.hy
                fw = fn(px, py) * W2 * 0.25 * self.hx * self.hy
                F[iy * self.nx + ix] = (eta * fw) @ eta.T
        return F

    def Ss_apply(self, v: np.ndarray) -> np.ndarray:
        """Sigma_s v (diagonal per region, or the cell blocks of a cross-section profile)."""
        if self.Ss_blk is None:
            return self.sig_s_dof * v
        return np.einsum("ckl,cl->ck", self.Ss_blk, v.reshape(self.ncell, self.nd)).ravel()

    def mode_apply(self, m: int, v: np.ndarray) -> np.ndarray:
        """The m-th term of the affine split applied to v (..., N_DOF): the indicator of region m, or the blocks
        of profile m."""
        if self.mode_blocks is None:
            return v * np.repeat((self.region == m).astype(np.float64), self.nd)
        sh = v.shape
        x = v.reshape(sh[:-1] + (self.ncell, self.nd))
        return np.einsum("ckl,...cl->...ck", self.mode_blocks[m], x).reshape(sh)

    def gbc(self, j: int) -> np.ndarray:
        """(g_j^bc)_k = -int over inflow boundary faces of g eta_k (Omega_j . n)."""
        if self.g == 0.0:
            return np.zeros(self.ndof)
        if j in self._gbc:
            return self._gbc[j]
        v = np.zeros(self.ndof)
        q, wq = _GQ_X, _GQ_W
        om = self.dirs[j]
        if self.dim == 1:
            mu = om[0]
            if mu > 0:   # inflow at x0 through the x-low face of cell 0
                e = self._eta(np.array([-1.0]))[:, 0]
                v[0:2] += -self.g * e * (-mu)
            elif mu < 0:
                c = self.nx - 1
                e = self._eta(np.array([1.0]))[:, 0]
                v[c * 2:(c + 1) * 2] += -self.g * e * mu
            self._gbc[j] = v
            return v
        ox, oy = om[0], om[1]
        ones = np.ones_like(q)
        fx_lo, fx_hi = "x-" in self.inflow_faces, "x+" in self.inflow_faces
        fy_lo, fy_hi = "y-" in self.inflow_faces, "y+" in self.inflow_faces
        for iy in range(self.ny):
            for ix in range(self.nx):
                c = iy * self.nx + ix
                contrib = np.zeros(4)
                if ox > 0 and ix == 0 and fx_lo:
                    contrib += -self.g * (self._eta(-ones, q) @ wq) * (-ox) * self.hy / 2.0
                if ox < 0 and ix == self.nx - 1 and fx_hi:
                    contrib += -self.g * (self._eta(ones, q) @ wq) * ox * self.hy / 2.0
                if oy > 0 and iy == 0 and fy_lo:
                    contrib += -self.g * (self._eta(q, -ones) @ wq) * (-oy) * self.hx / 2.0
                if oy < 0 and iy == self.ny - 1 and fy_hi:
                    contrib += -self.g * (self._eta(q, ones) @ wq) * oy * self.hx / 2.0
                v[c * 4:(c + 1) * 4] += contrib
        self._gbc[j] = v
        return v

    # ---------------------------------------------------------- operators
    def sweep(self, j: int, rhs: np.ndarray, sig_t: np.ndarray | None = None) -> np.ndarray:
        """psi_j = (D_j + Sigma_t)^{-1} rhs by one upwind block Gauss-Seidel pass (Sec. 3.1).  sig_t: per-cell
        values replacing the problem's Sigma_t."""
        if sig_t is None and self.St_blk is not None:
            return _lib.sweep_dir_blk(self.nx, self.ny, self.nd, self.M[j], self.C[j], self.inflow[j], self.St_blk, rhs)
        st = self.sig_t if sig_t is None else sig_t
        return _lib.sweep_dir(self.nx, self.ny, self.nd, self.M[j], self.C[j], self.inflow[j], st, rhs)

    def apply_forward(self, j: int, x: np.ndarray, sig_t: np.ndarray | None = None) -> np.ndarray:
        """(D_j + Sigma_t) x for direction j (no inflow-boundary term)."""
        if sig_t is None and self.St_blk is not None:
            return _lib.apply_dir_blk(self.nx, self.ny, self.nd, self.M[j], self.C[j], self.inflow[j], self.St_blk, x)
        st = self.sig_t if sig_t is None else sig_t
        return _lib.apply_dir(self.nx, self.ny, self.nd, self.M[j], self.C[j], self.inflow[j], st, x)

    def dense_L(self, j: int, sig_t: np.ndarray | None = None) -> np.ndarray:
        """Dense (D_j + Sigma_t) assembled block by block in numpy (independent of the C loops)."""
        st = self.sig_t if sig_t is None else sig_t
        nd, nx, ny = self.nd, self.nx, self.ny
        L = np.zeros((self.ndof, self.ndof))
        for iy in range(ny):
            for ix in range(nx):
                c = iy * nx + ix
                if sig_t is None and self.St_blk is not None:
                    L[c * nd:(c + 1) * nd, c * nd:(c + 1) * nd] = self.M[j] + self.St_blk[c]
                else:
                    L[c * nd:(c + 1) * nd, c * nd:(c + 1) * nd] = self.M[j] + st[c] * np.eye(nd)
                nbrs = (
                    (ix - 1, iy) if ix > 0 else None,
                    (ix + 1, iy) if ix < nx - 1 else None,
                    (ix, iy - 1) if iy > 0 else None,
                    (ix, iy + 1) if iy < ny - 1 else None,
                )
                for f in range(4):
                    if self.inflow[j, f] and nbrs[f] is not None:
                        nb = nbrs[f][1] * nx + nbrs[f][0]
                        L[c * nd:(c + 1) * nd, nb * nd:(nb + 1) * nd] = self.C[j, f]
        return L


def with_params(p: Problem, sigma_s, sigma_a) -> Problem:
    """Copy of p with new per-region cross sections (mesh, quadrature and local blocks shared)."""
    import copy
    q = copy.copy(p)
    ss = np.asarray(sigma_s, dtype=np.float64)
    sa = np.asarray(sigma_a, dtype=np.float64)
    q.sigma_s_region = ss
    q.sigma_a_region = sa
    q.sig_s = ss[p.region]
    q.sig_t = ss[p.region] + sa[p.region]
    q.sig_s_dof = np.repeat(q.sig_s, p.nd)
    q.sig_t_dof = np.repeat(q.sig_t, p.nd)
    if p.mode_blocks is not None:
        _set_blocks(q, ss, sa)
    return q


def _varscat_profile(x, y):
    """The variable-scattering profile (Sec. 5): r^4 (2 - r^2)^2 for r <= 1, 1 outside."""
    r2 = x * x + y * y
    return np.where(r2 <= 1.0, r2 * r2 * (2.0 - r2) ** 2, 1.0)


def _set_blocks(p: Problem, ss, sa) -> None:
    """Cell blocks Sigma_s = sum_m sigma_s,m F_m and Sigma_t = sum_m (sigma_s,m + sigma_a,m) F_m of the profiles
    F_m; the per-cell scalars become the cell means (the (0, 0) entry: eta_0 is constant), which the DSA
    diffusion operator takes."""
    B = p.mode_blocks
    p.Ss_blk = np.einsum("m,mckl->ckl", np.asarray(ss, dtype=np.float64), B)
    p.St_blk = np.einsum("m,mckl->ckl", np.asarray(ss, dtype=np.float64) + np.asarray(sa, dtype=np.float64), B)
    p.sig_s = p.Ss_blk[:, 0, 0].copy()
    p.sig_t = p.St_blk[:, 0, 0].copy()
    p.sig_s_dof = np.repeat(p.sig_s, p.nd)
    p.sig_t_dof = np.repeat(p.sig_t, p.nd)
