"""Pins of the oracle sweep and discretisation (Sec. 2.2-3.1): P2, P3, P4, convergence order."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import Problem
from oracle.discretization import gauss_legendre

from _helpers import small_1d, small_2d


def test_p2_slab_pure_absorber_outflow_is_pade_power():
    """Upwind P1 DG on a pure absorber with unit inflow: each cell multiplies the
    outflow trace by the (1,2) Pade approximant R(z) = (1 - z/3)/(1 + 2z/3 + z^2/6),
    z = sigma_t h / mu, so after n cells the trace is R(z)^n."""
    for sig, nx in ((2.0, 10), (50.0, 7), (0.3, 32)):
        spec = small_1d(nx=nx, n_polar=8, rx=1, src_q=0.0, inflow_g=1.0)
        p = Problem(spec, 0, [0.0], [sig])
        for j in range(p.ndir):
            mu = p.dirs[j, 0]
            psi = p.sweep(j, p.G + p.gbc(j))
            z = sig * p.hx / abs(mu)
            R = (1 - z / 3) / (1 + 2 * z / 3 + z * z / 6)
            if mu > 0:
                c, sgn = nx - 1, 1.0
            else:
                c, sgn = 0, -1.0
            trace = (psi[2 * c] + sgn * math.sqrt(3.0) * psi[2 * c + 1]) / math.sqrt(p.hx)
            assert abs(trace - R ** nx) <= 1e-13 * max(1.0, abs(R ** nx)) + 1e-300


@pytest.mark.parametrize("dim", [1, 2])
def test_p3_sweep_inverts_block_lower_triangular_operator(dim):
    rng = np.random.default_rng(3)
    if dim == 1:
        p = Problem(small_1d(nx=9, n_polar=4), 0, [1, 2, 30, 4], [0.1, 0.2, 0.3, 0.4])
    else:
        p = Problem(small_2d(nx=4, ny=3, n_polar=2, n_azim=4), 0, [1, 200, 3, 4], [0.1, 0.2, 0.3, 0.4])
    for j in range(p.ndir):
        L = p.dense_L(j)
        f = rng.standard_normal(p.ndof)
        psi = p.sweep(j, f)
        assert np.max(np.abs(L @ psi - f)) < 1e-12 * np.max(np.abs(f)) * max(1, np.abs(L).max())
        np.testing.assert_allclose(p.apply_forward(j, f), L @ f, rtol=1e-13, atol=1e-13)
        # block lower triangular in the sweep order: permute to upwind order, check upper blocks vanish
        nd, nx, ny = p.nd, p.nx, p.ny
        xs = range(nx) if p.dirs[j, 0] > 0 else range(nx - 1, -1, -1)
        if dim == 2:
            ys = range(ny) if p.dirs[j, 1] > 0 else range(ny - 1, -1, -1)
        else:
            ys = range(1)
        order = [iy * nx + ix for iy in ys for ix in xs]
        perm = np.concatenate([np.arange(c * nd, (c + 1) * nd) for c in order])
        Lp = L[np.ix_(perm, perm)]
        for a in range(len(order)):
            assert np.all(Lp[a * nd:(a + 1) * nd, (a + 1) * nd:] == 0.0)


def test_p4_constant_preservation_2d():
    """Uniform sigma_t, sigma_s = 0, source q everywhere, inflow q/sigma_t: psi == q/sigma_t."""
    q, sig = 3.0, 2.5
    spec = small_2d(nx=6, ny=5, n_polar=4, n_azim=8, rx=1, ry=1, src_box=(0, 1, 0, 1), src_q=q,
                    inflow_g=q / sig)
    p = Problem(spec, 0, [0.0], [sig])
    ref = np.zeros(p.ndof)
    ref[0::4] = (q / sig) * math.sqrt(p.hx * p.hy)
    for j in range(p.ndir):
        psi = p.sweep(j, p.G + p.gbc(j))
        assert np.max(np.abs(psi - ref)) < 1e-13


def _l2_error_2d(p, psi, fexact, nq=6):
    x, w = gauss_legendre(nq)
    XI, ZE = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w).ravel()
    eta = p._eta(XI.ravel(), ZE.ravel())
    err = 0.0
    for iy in range(p.ny):
        for ix in range(p.nx):
            c = iy * p.nx + ix
            X = p.x0 + (ix + 0.5 + 0.5 * XI.ravel()) * p.hx
            Y = p.y0 + (iy + 0.5 + 0.5 * ZE.ravel()) * p.hy
            uh = psi[c * 4:(c + 1) * 4] @ eta
            err += np.sum(W * (uh - fexact(X, Y)) ** 2) * p.hx * p.hy / 4
    return math.sqrt(err)


def test_dg_convergence_order_manufactured_2d():
    """Smooth manufactured solution for one direction: the Q1 upwind DG sweep converges at order 2."""
    om_idx = 5
    sig = 1.3

    def ue(X, Y):
        return np.exp(0.5 * X) * np.cos(Y) + 2.0

    errs = []
    for n in (8, 16, 32):
        p = Problem(small_2d(nx=n, ny=n, n_polar=2, n_azim=8, rx=1, ry=1), 0, [0.0], [sig])
        ox, oy = p.dirs[om_idx, 0], p.dirs[om_idx, 1]

        def f(X, Y):
            return ox * 0.5 * np.exp(0.5 * X) * np.cos(Y) - oy * np.exp(0.5 * X) * np.sin(Y) + sig * ue(X, Y)

        x, w = gauss_legendre(5)
        XI, ZE = np.meshgrid(x, x, indexing="ij")
        W = np.outer(w, w).ravel()
        eta = p._eta(XI.ravel(), ZE.ravel())
        rhs = np.zeros(p.ndof)
        for iy in range(p.ny):
            for ix in range(p.nx):
                c = iy * p.nx + ix
                X = p.x0 + (ix + 0.5 + 0.5 * XI.ravel()) * p.hx
                Y = p.y0 + (iy + 0.5 + 0.5 * ZE.ravel()) * p.hy
                rhs[c * 4:(c + 1) * 4] = eta @ (W * f(X, Y)) * p.hx * p.hy / 4
                # inflow boundary data: -int g eta_k (Omega.n)
                for cond, xi_f, ze_f, on, fj in (
                        (ox > 0 and ix == 0, -np.ones_like(x), x, -ox, p.hy / 2),
                        (ox < 0 and ix == p.nx - 1, np.ones_like(x), x, ox, p.hy / 2),
                        (oy > 0 and iy == 0, x, -np.ones_like(x), -oy, p.hx / 2),
                        (oy < 0 and iy == p.ny - 1, x, np.ones_like(x), oy, p.hx / 2)):
                    if cond:
                        Xf = p.x0 + (ix + 0.5 + 0.5 * xi_f) * p.hx
                        Yf = p.y0 + (iy + 0.5 + 0.5 * ze_f) * p.hy
                        rhs[c * 4:(c + 1) * 4] += -(p._eta(xi_f, ze_f) @ (w * ue(Xf, Yf))) * on * fj
        psi = p.sweep(om_idx, rhs)
        errs.append(_l2_error_2d(p, psi, ue))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.85 < o < 2.3 for o in orders), (errs, orders)


def test_dg_convergence_order_manufactured_1d():
    sig = 0.7

    def ue(X):
        return np.sin(3 * X) + 1.5

    errs = []
    x, w = gauss_legendre(6)
    for n in (8, 16, 32, 64):
        p = Problem(small_1d(nx=n, n_polar=4, rx=1), 0, [0.0], [sig])
        j = 1
        mu = p.dirs[j, 0]
        eta = p._eta(x)
        rhs = np.zeros(p.ndof)
        for c in range(n):
            X = p.x0 + (c + 0.5 + 0.5 * x) * p.hx
            rhs[2 * c:2 * c + 2] = eta @ (w * (mu * 3 * np.cos(3 * X) + sig * ue(X))) * p.hx / 2
        if mu > 0:
            rhs[0:2] += mu * ue(p.x0) * p._eta(np.array([-1.0]))[:, 0]
        else:
            rhs[2 * (n - 1):2 * n] += -mu * ue(p.x0 + n * p.hx) * p._eta(np.array([1.0]))[:, 0]
        psi = p.sweep(j, rhs)
        err = 0.0
        for c in range(n):
            X = p.x0 + (c + 0.5 + 0.5 * x) * p.hx
            err += np.sum(w * (psi[2 * c:2 * c + 2] @ eta - ue(X)) ** 2) * p.hx / 2
        errs.append(math.sqrt(err))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(1.85 < o < 2.3 for o in orders), (errs, orders)


def test_local_blocks_kronecker_structure():
    """With the orthonormal tensor basis the cell block of D_j is
    Omega_x K_x (x) I + Omega_y I (x) K_y with K = (1/h)[[1, sqrt3], [-sqrt3, 3]]
    for a positive component (mirrored for a negative one)."""
    p = Problem(small_2d(nx=3, ny=5, n_polar=2, n_azim=4, rx=1, ry=1), 0, [0.0], [1.0])
    s3 = math.sqrt(3.0)
    for j in range(p.ndir):
        ox, oy = p.dirs[j, 0], p.dirs[j, 1]

        def K(o, h):
            k = np.array([[1.0, s3], [-s3, 3.0]]) / h
            if o < 0:
                S = np.diag([1.0, -1.0])
                k = S @ k @ S
            return abs(o) * k

        ref = np.kron(np.eye(2), K(ox, p.hx)) + np.kron(K(oy, p.hy), np.eye(2))
        np.testing.assert_allclose(p.M[j], ref, atol=1e-12 * np.abs(ref).max())
