"""Pins of the oracle's variable-scattering problem (paper Sec. 5, the variable-scattering problem; Sec. 2.3 for
the cell blocks (Sigma)_kl = int_T sigma eta_k eta_l, which are full 4x4 blocks when sigma varies in a cell).

* The profile blocks against exact rational integration of the polynomial profile (cells inside the unit disc)
  and against the identity (cells outside it, where the profile is 1).
* The block path against the diagonal path: with the profile's coefficient zero the problem is the constant
  scattering problem, solved by the per-region code.
* The block sweep against a dense solve, the solution against the dense coupled system (eq. one_equation).
* The affine split of the reduced operator against its direct projection (Sec. 4.1).
* Mirror symmetry of the solution (the profile and the source are even in x and in y).
"""
import dataclasses
from fractions import Fraction

import numpy as np
import pytest

import workloads as wl
from oracle import Problem, romsad as ORS, transport as OT
from oracle.discretization import with_params


def _spec(n=8, n_azim=8, n_polar=2):
    return dataclasses.replace(wl.variable_scattering().with_mesh(n, n), n_azim=n_azim, n_polar=n_polar)


def test_profile_blocks_equal_exact_integrals_inside_and_identity_outside():
    sympy = pytest.importorskip("sympy")
    n = 8
    p = Problem(_spec(n), 0, *wl.variable_scattering_params(60.0))
    F = p.mode_blocks[0]
    xi, ze = sympy.symbols("xi zeta")
    h = Fraction(2, n)
    L = [sympy.sqrt(sympy.Rational(1, 2)), sympy.sqrt(sympy.Rational(3, 2))]
    checked = outside = 0
    for iy in range(n):
        for ix in range(n):
            xl, yl = -1 + ix * h, -1 + iy * h
            corners = [(xl + a * h) ** 2 + (yl + b * h) ** 2 for a in (0, 1) for b in (0, 1)]
            c = iy * n + ix
            if max(corners) <= 1:        # the whole cell inside the disc: the profile is a polynomial there
                x = sympy.Rational(xl.numerator, xl.denominator) + sympy.Rational(h.numerator, h.denominator) * (xi + 1) / 2
                y = sympy.Rational(yl.numerator, yl.denominator) + sympy.Rational(h.numerator, h.denominator) * (ze + 1) / 2
                r2 = x * x + y * y
                poly = sympy.Poly(sympy.expand(r2 * r2 * (2 - r2) ** 2), xi, ze)

                def moment(a, b):   # exact int over [-1, 1]^2 of f xi^a zeta^b, monomial by monomial
                    return sum(cf * (Fraction(2, e0 + a + 1) if (e0 + a) % 2 == 0 else 0)
                               * (Fraction(2, e1 + b + 1) if (e1 + b) % 2 == 0 else 0)
                               for (e0, e1), cf in zip(poly.monoms(), (Fraction(int(q.p), int(q.q)) for q in poly.coeffs())))
                for k in range(4):
                    for l in range(4):
                        cst = float(L[k % 2] * L[l % 2] * L[k // 2] * L[l // 2])
                        exact = cst * float(moment(k % 2 + l % 2, k // 2 + l // 2))
                        assert abs(F[c, k, l] - exact) < 1e-14 * max(1.0, abs(exact)), (ix, iy, k, l)
                checked += 1
            else:
                cx, cy = min(max(Fraction(0), xl), xl + h), min(max(Fraction(0), yl), yl + h)   # nearest point to 0
                if cx * cx + cy * cy >= 1:       # the whole cell outside the disc: the profile is 1 there
                    np.testing.assert_allclose(F[c], np.eye(4), atol=1e-14)
                    outside += 1
    assert checked >= 4 and outside >= 4


def test_zero_profile_coefficient_reduces_to_constant_scattering():
    """sigma_s = 0 * f + c: every block is c I, so operators and solutions equal those of the per-region code with
    sigma_s = c in both regions."""
    spec = _spec(8)
    c = 7.5
    pb = Problem(spec, 0, np.array([0.0, c]), np.array([0.0, 0.3]))
    pd = Problem(dataclasses.replace(spec, sigma_modes=None), 0, np.array([c, c]), np.array([0.3, 0.3]))
    z = np.random.default_rng(1).standard_normal(pb.ndof)
    np.testing.assert_allclose(OT.Atilde_apply(pb, z), OT.Atilde_apply(pd, z), rtol=0, atol=1e-13 * np.abs(z).max())
    np.testing.assert_allclose(OT.rhs_btilde(pb), OT.rhs_btilde(pd), rtol=1e-13, atol=1e-15)
    phb, _ = ORS.solve(pb, None, post="dsa", restart=30, rtol=1e-13, max_iter=500)
    phd, _ = ORS.solve(pd, None, post="dsa", restart=30, rtol=1e-13, max_iter=500)
    assert np.linalg.norm(phb - phd) < 1e-11 * np.linalg.norm(phd)


def test_block_sweep_inverts_the_transport_block_and_solution_matches_dense_system():
    p = Problem(_spec(6, n_azim=8, n_polar=2), 0, *wl.variable_scattering_params(90.0))
    rhs = np.random.default_rng(2).standard_normal(p.ndof)
    for j in (0, 3, 6):
        L = p.dense_L(j)
        assert np.linalg.norm(p.sweep(j, rhs) - np.linalg.solve(L, rhs)) < 1e-13 * np.linalg.norm(rhs)
        assert np.linalg.norm(p.apply_forward(j, rhs) - L @ rhs) < 1e-12 * np.linalg.norm(L @ rhs)
    A, b = OT.dense_coupled_system(p)
    psi = np.linalg.solve(A, b)
    phi_dense = sum(p.w[j] * psi[j * p.ndof:(j + 1) * p.ndof] for j in range(p.ndir))
    phi, st = ORS.solve(p, None, post="dsa", restart=30, rtol=1e-13, max_iter=500)
    assert st.converged
    assert np.linalg.norm(phi - phi_dense) < 1e-11 * np.linalg.norm(phi_dense)


def test_affine_split_of_reduced_operator_with_profile_blocks():
    p = Problem(_spec(8), 0, *wl.variable_scattering_params(74.9))
    r = 5
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((p.ndir * p.ndof, r)))
    U = Q.T.reshape(r, p.ndir, p.ndof).copy()
    rom = ORS.build_rom(p, U)
    for mu in (49.9, 99.9):
        q = with_params(p, *wl.variable_scattering_params(mu))
        A1 = ORS.reduced_operator(rom, q.sigma_s_region, q.sigma_a_region)
        A2 = ORS.reduced_operator_direct(q, U)
        assert np.abs(A1 - A2).max() < 1e-13 * np.abs(A2).max()


def test_solution_is_mirror_symmetric():
    """phi(-x, y) = phi(x, y): the x-odd Legendre modes flip sign under the mirror, the others stay."""
    n = 8
    p = Problem(_spec(n), 0, *wl.variable_scattering_params(55.0))
    phi, _ = ORS.solve(p, None, post="dsa", restart=30, rtol=1e-13, max_iter=500)
    ph = phi.reshape(n, n, 4)                       # [iy, ix, mode]
    mir = ph[:, ::-1, :] * np.array([1.0, -1.0, 1.0, -1.0])
    assert np.abs(ph - mir).max() < 1e-10 * np.abs(ph).max()
    mir_y = ph[::-1, :, :] * np.array([1.0, 1.0, -1.0, -1.0])
    assert np.abs(ph - mir_y).max() < 1e-10 * np.abs(ph).max()
