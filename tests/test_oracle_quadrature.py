"""Pins of the oracle quadratures (Sec. 2.1): P1."""
import math
import os

import numpy as np

from oracle.discretization import cl_quadrature, gauss_legendre, slab_quadrature

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gauss_legendre_8.txt")


def test_gauss_legendre_matches_published_table():
    ref = np.loadtxt(GOLDEN)
    x, w = gauss_legendre(8)
    np.testing.assert_allclose(x[4:], ref[:, 0], atol=2e-15)
    np.testing.assert_allclose(w[4:], ref[:, 1], atol=2e-15)
    np.testing.assert_allclose(x[:4], -ref[::-1, 0], atol=2e-15)


def test_gauss_legendre_matches_numpy_and_is_exact_to_degree_2n_minus_1():
    for n in (1, 2, 3, 6, 8, 16, 24):
        x, w = gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        np.testing.assert_allclose(x, xr, atol=1e-14)
        np.testing.assert_allclose(w, wr, atol=1e-14)
        for d in range(2 * n):
            exact = 0.0 if d % 2 else 2.0 / (d + 1)
            assert abs(np.sum(w * x ** d) - exact) < 1e-13
        # degree 2n is NOT integrated exactly (visible for small n)
        if n <= 8:
            assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


def test_cl_quadrature_normalised_and_second_moments():
    for nt, nz in ((16, 8), (24, 8), (40, 6), (4, 2)):
        d, w = cl_quadrature(nt, nz)
        assert d.shape == (nt * nz, 3)
        assert abs(w.sum() - 1.0) < 1e-14
        np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
        # diffusion tensor of eq. diffusion-limit: (1/4pi) int Omega_i^2 = 1/3
        for i in range(3):
            assert abs(np.sum(w * d[:, i] ** 2) - 1.0 / 3.0) < 1e-14
        # odd moments vanish
        for i in range(3):
            assert abs(np.sum(w * d[:, i])) < 1e-14
        # index j = (j2-1) N_theta + j1: first direction has theta = pi / N_theta
        assert abs(math.atan2(d[0, 1], d[0, 0]) - math.pi / nt) < 1e-14
        # no direction is parallel to an axis (Chebyshev azimuths never hit 0 or pi/2 for even N_theta)
        assert np.all(np.abs(d[:, :2]) > 1e-3)


def test_slab_quadrature():
    mu, w = slab_quadrature(16)
    assert abs(w.sum() - 1.0) < 1e-14
    assert abs(np.sum(w * mu[:, 0] ** 2) - 1.0 / 3.0) < 1e-14
