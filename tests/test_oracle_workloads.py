"""Pins of the oracle's support for the paper's other 2D problems (pin-cell, two-material with parametric
inflow): the Gaussian source projection, the one-sided inflow, and the region maps of the inner square."""
import dataclasses
import math

import numpy as np
import pytest

import workloads as wl
from oracle import Problem

from _helpers import rel


def _small(spec, n=8):
    return dataclasses.replace(spec, nx=[n], ny=[n], n_polar=2, n_azim=4)


def test_gaussian_source_total_matches_the_closed_form():
    """sum_T int_T G = A (pi / a) prod over axes of (erf(sqrt(a)(x1-xc)) - erf(sqrt(a)(x0-xc))) / 2, read from the
    constant coefficients (eta_00 = 1/sqrt(hx hy)); also off-centre to break symmetry."""
    for gauss in ((1.0, 100.0, 0.0, 0.0), (10.0 / math.pi, 100.0, 0.0, 0.0), (2.0, 30.0, 0.3, -0.2)):
        spec = dataclasses.replace(_small(wl.pincell(), 20), src_gauss=gauss)
        p = Problem(spec, 0, *wl.pincell_params(0.2, 0.3))
        total = float(np.sum(p.G[0::4])) * math.sqrt(p.hx * p.hy)
        A, a, xc, yc = gauss
        sa = math.sqrt(a)
        ref = A * (math.pi / a) * 0.25 * (math.erf(sa * (1 - xc)) - math.erf(sa * (-1 - xc))) \
            * (math.erf(sa * (1 - yc)) - math.erf(sa * (-1 - yc)))
        assert abs(total - ref) < 1e-12 * ref


def test_gaussian_source_moments_are_mirror_symmetric():
    """A centred Gaussian: the coefficient of p_a(x) q_b(y) changes sign as (-1)^a under x -> -x and as
    (-1)^b under y -> -y."""
    p = Problem(_small(wl.pincell(), 10), 0, *wl.pincell_params(0.2, 0.3))
    G = p.G.reshape(p.ny, p.nx, 4)
    scale = np.abs(G).max()
    for k in range(4):
        a, b = k % 2, k // 2
        assert np.abs(G[:, ::-1, k] - (-1) ** a * G[:, :, k]).max() < 1e-14 * scale
        assert np.abs(G[::-1, :, k] - (-1) ** b * G[:, :, k]).max() < 1e-14 * scale
    assert np.abs(G[..., 1]).max() > 1e-3 * scale and np.abs(G[..., 3]).max() > 1e-3 * scale


def test_gaussian_source_one_cell_by_adaptive_quadrature():
    integ = pytest.importorskip("scipy.integrate")
    p = Problem(_small(wl.pincell(), 8), 0, *wl.pincell_params(0.2, 0.3))
    ix, iy = 3, 4
    x0, y0 = p.x0 + ix * p.hx, p.y0 + iy * p.hy
    basis = [lambda x, y: 1.0, lambda x, y: math.sqrt(3.0) * (2 * (x - x0) / p.hx - 1),
             lambda x, y: math.sqrt(3.0) * (2 * (y - y0) / p.hy - 1),
             lambda x, y: 3.0 * (2 * (x - x0) / p.hx - 1) * (2 * (y - y0) / p.hy - 1)]
    c = iy * p.nx + ix
    for k in range(4):
        val, _ = integ.dblquad(lambda y, x: math.exp(-100 * (x * x + y * y)) * basis[k](x, y) / math.sqrt(p.hx * p.hy),
                               x0, x0 + p.hx, y0, y0 + p.hy, epsabs=1e-14, epsrel=1e-12)
        assert abs(p.G[c * 4 + k] - val) < 1e-10 * max(abs(val), 1e-6)


def test_inflow_faces_add_up_and_the_left_face_is_one_sided():
    base = dataclasses.replace(_small(wl.config(2), 6), inflow_g=0.7)
    full = Problem(base, 0, [2.0] * 4, [0.5] * 4)
    parts = [Problem(dataclasses.replace(base, inflow_faces=(f,)), 0, [2.0] * 4, [0.5] * 4)
             for f in ("x-", "x+", "y-", "y+")]
    for j in range(full.ndir):
        assert np.allclose(sum(q.gbc(j) for q in parts), full.gbc(j), rtol=0, atol=1e-15)
        left = parts[0].gbc(j)
        if full.dirs[j][0] < 0:
            assert not left.any()
        else:
            assert left.any()
            assert not left.reshape(full.ny, full.nx, 4)[:, 1:, :].any()     # only the first column of cells


@pytest.mark.parametrize("maker, params", [(wl.pincell, lambda: wl.pincell_params(0.1, 0.4)),
                                           (wl.param_inflow, lambda: wl.param_inflow_params(3.0))])
def test_inner_square_regions(maker, params):
    spec = _small(maker(), 8)
    ss, sa = params()
    p = Problem(spec, 0, ss, sa)
    for iy in range(p.ny):
        for ix in range(p.nx):
            xc = p.x0 + (ix + 0.5) * p.hx
            yc = p.y0 + (iy + 0.5) * p.hy
            inner = abs(xc) < 0.5 and abs(yc) < 0.5
            r = p.region[iy * p.nx + ix]
            assert (r in (5, 6, 9, 10)) == inner
            assert p.sig_s[iy * p.nx + ix] == ss[r]


def _dense(f, n):
    return np.column_stack([f(e) for e in np.eye(n)])


@pytest.mark.parametrize("which", ["pincell", "param_inflow"])
def test_small_versions_solve_to_the_dense_solution(which):
    """Both problems on a 12 x 12 mesh with CL(4, 2): GMRES-DSA reaches the dense solution; for the two-material
    problem phi is linear in the inflow value mu_bc (b~ is, A~ does not depend on it)."""
    from oracle import romsad as RS, transport as T
    if which == "pincell":
        spec = dataclasses.replace(wl.pincell(), nx=[12], ny=[12], n_polar=2, n_azim=4)
        ss, sa = wl.pincell_params(0.3, 0.2)
    else:
        spec = dataclasses.replace(wl.param_inflow(), nx=[12], ny=[12], n_polar=2, n_azim=4, inflow_g=0.8)
        ss, sa = wl.param_inflow_params(2.5)
    p = Problem(spec, 0, ss, sa)
    A = _dense(lambda z: T.Atilde_apply(p, z), p.ndof)
    bt = T.rhs_btilde(p)
    ref = np.linalg.solve(A, bt)
    sol, st = RS.solve(p, None, post="dsa_pc", restart=60, rtol=1e-12, max_iter=600)
    assert st.converged and rel(sol, ref) < 1e-9
    if which == "param_inflow":
        p2 = Problem(dataclasses.replace(spec, inflow_g=1.2), 0, ss, sa)
        assert rel(T.rhs_btilde(p2), 1.5 * bt) < 1e-13
