"""Pins of the oracle solvers (Sec. 3, Alg. 1): P5, P6, P7, GMRES equivalence, SI identity."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import Problem, transport as T
from oracle.krylov import fgmres, source_iteration
from oracle import romsad as RS

from _helpers import rel, small_1d, small_2d


@pytest.mark.parametrize("dim", [1, 2])
def test_p5_infinite_homogeneous_medium(dim):
    """Uniform medium, source q, isotropic inflow q/sigma_a: phi == q / sigma_a exactly."""
    q, ss, sa = 1.0, 7.0, 0.5
    if dim == 1:
        spec = small_1d(nx=12, n_polar=8, rx=1, src_box=(0, 1, 0, 1), src_q=q, inflow_g=q / sa)
    else:
        spec = small_2d(nx=6, ny=5, n_polar=4, n_azim=8, rx=1, ry=1, src_box=(0, 1, 0, 1), src_q=q,
                        inflow_g=q / sa)
    p = Problem(spec, 0, [ss], [sa])
    phi, st = RS.solve(p, None, rtol=1e-13)
    ref = np.zeros(p.ndof)
    ref[0::p.nd] = (q / sa) * math.sqrt(p.hx * (p.hy if dim == 2 else 1.0))
    assert np.max(np.abs(phi - ref)) < 1e-11 * np.max(ref)
    assert st.converged


def test_p5_infinite_medium_by_reflecting_slab():
    """The infinite homogeneous medium as a slab whose two ends reflect specularly (dense LU of the coupled
    system with the mirrored ordinates coupled at the ends): phi == q / sigma_a exactly, with no inflow."""
    q, ss, sa = 1.0, 7.0, 0.5
    p = Problem(small_1d(nx=10, n_polar=8, rx=1, src_box=(0, 1, 0, 1), src_q=q, inflow_g=0.0), 0, [ss], [sa])
    phi = T.solve_reflecting_1d(p)
    ref = np.zeros(p.ndof)
    ref[0::2] = (q / sa) * math.sqrt(p.hx)
    assert np.max(np.abs(phi - ref)) < 1e-12 * np.max(ref)
    # the same medium with vacuum ends loses particles: the reflection terms are what keeps phi flat
    A, b = T.dense_coupled_system(p)
    vac = T.scalar_flux(p, np.linalg.solve(A, b).reshape(p.ndir, p.ndof))
    assert np.max(np.abs(vac - ref)) > 0.1 * np.max(ref)


def test_reflecting_end_equals_mirrored_slab():
    """A reflecting end at x = 0 is a mirror: the slab [0, 1] with reflection at 0 and vacuum at 1 has the scalar
    flux of the symmetric slab [-1, 1] (mirrored cross sections and source, vacuum at both ends) on [0, 1],
    for non-uniform cross sections and source (pins the end coupling: sign, trace and mirrored ordinate)."""
    ss, sa = [5.0, 1.0, 30.0, 2.0], [0.1, 0.3, 0.2, 0.05]
    half = small_1d(nx=8, n_polar=8, rx=4, src_box=(0.25, 0.5, 0, 1), src_q=1.0, inflow_g=0.0)
    p = Problem(half, 0, ss, sa)
    phi_refl = T.solve_reflecting_1d(p, left=True, right=False)
    full = dataclasses.replace(half, nx=[16], box=(-1.0, 1.0, 0.0, 1.0), rx=8, src_box=(-0.5, 0.5, 0, 1))
    # mirrored regions and source: [-1, 0] is the reflection of [0, 1]; the source box [0.25, 0.5] and its
    # mirror [-0.5, -0.25] are covered by one box [-0.5, 0.5] minus the centre [-0.25, 0.25]
    pf = Problem(full, 0, ss[::-1] + ss, sa[::-1] + sa)
    inner = Problem(dataclasses.replace(full, src_box=(-0.25, 0.25, 0, 1)), 0, ss[::-1] + ss, sa[::-1] + sa)
    A, b = T.dense_coupled_system(pf)
    b = b - np.tile(inner.G, pf.ndir)
    phi_full = T.scalar_flux(pf, np.linalg.solve(A, b).reshape(pf.ndir, pf.ndof))
    assert rel(phi_full[p.ndof:], phi_refl) < 1e-12
    # and the mirror image on [-1, 0]: cell order reversed, odd Legendre mode flips sign
    left = phi_full[:p.ndof].reshape(-1, 2)[::-1] * np.array([1.0, -1.0])
    assert rel(left.reshape(-1), phi_refl) < 1e-12


def test_p6_pure_absorber_one_iteration():
    """sigma_s = 0 gives A~ = I: FGMRES stops after one iteration with phi = b~."""
    p = Problem(small_2d(nx=5, ny=4), 0, [0.0] * 4, [1.0, 2.0, 3.0, 4.0])
    bt = T.rhs_btilde(p)
    phi, st = RS.solve(p, None, rtol=1e-12)
    assert st.iterations == 1
    assert rel(phi, bt) < 1e-14


@pytest.mark.parametrize("dim", [1, 2])
def test_p7_dense_lu_of_coupled_system(dim):
    """phi from FGMRES on A~ phi = b~ equals Q A^{-1} b for the coupled system (eq. one_equation)."""
    if dim == 1:
        p = Problem(small_1d(nx=10, n_polar=4, inflow_g=0.4), 0, [5, 1, 30, 2], [0.1, 0.3, 0.2, 0.05])
    else:
        p = Problem(small_2d(nx=3, ny=4, n_polar=2, n_azim=4, src_box=(0.2, 0.7, 0.1, 0.5), inflow_g=0.3),
                    0, [5, 1, 30, 2], [0.1, 0.3, 0.2, 0.05])
    A, b = T.dense_coupled_system(p)
    psi = np.linalg.solve(A, b).reshape(p.ndir, p.ndof)
    phid = T.scalar_flux(p, psi)
    phi, st = RS.solve(p, None, rtol=1e-13)
    assert rel(phi, phid) < 1e-11
    # and the angular flux: one more sweep with the converged phi reproduces psi (eq. discrete-rte)
    psi_s = T.sweep_all(p, p.sig_s_dof * phi + p.G, with_bc=False)
    for j in range(p.ndir):
        psi_s[j] = p.sweep(j, p.sig_s_dof * phi + p.G + p.gbc(j))
    assert rel(psi_s, psi) < 1e-11


def _dense_Atilde(p):
    n = p.ndof
    return np.stack([T.Atilde_apply(p, e) for e in np.eye(n)], axis=1)


def test_fgmres_with_fixed_preconditioner_is_right_preconditioned_gmres():
    """Alg. 1 with M_j = M fixed minimises ||b - A M u|| over K_k(A M, r0) (Sec. 4.2)."""
    p = Problem(small_2d(nx=3, ny=3, n_polar=2, n_azim=4), 0, [20, 1, 300, 2], [0.1, 0.3, 0.2, 0.05])
    Ad = _dense_Atilde(p)
    b = T.rhs_btilde(p)
    rng = np.random.default_rng(0)
    Mmat = np.eye(p.ndof) + 0.1 * rng.standard_normal((p.ndof, p.ndof))
    pre = lambda j, v: Mmat @ v
    AM = Ad @ Mmat
    for k in range(1, 7):
        phi, st = fgmres(lambda z: Ad @ z, b, pre, restart=50, rtol=1e-30, max_iter=k,
                         true_residual_check=False)
        assert st.iterations == k
        K = np.stack([np.linalg.matrix_power(AM, i) @ b for i in range(k)], axis=1)
        Qk, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(AM @ Qk, b, rcond=None)
        ref = Mmat @ (Qk @ y)
        assert rel(phi, ref) < 1e-9


def test_source_iteration_residual_identity_and_sweep_count():
    """r^(l-1) = phi^(l,*) - phi^(l-1) (eq. SI-residual-relation); sweeps = 1 + iterations."""
    p = Problem(small_2d(nx=4, ny=4), 0, [3, 1, 30, 2], [0.1, 0.3, 0.2, 0.05])
    bt = T.rhs_btilde(p)
    its = source_iteration(p, 4)
    for l in range(1, 5):
        r = bt - T.Atilde_apply(p, its[l - 1])
        assert rel(its[l] - its[l - 1], r) < 1e-12
    phi, st = RS.solve(p, None, rtol=1e-10, true_residual_check=False)
    assert st.sweeps == 1 + st.iterations
    phi2, st2 = RS.solve(p, None, rtol=1e-10, phi0=phi * 0.9, true_residual_check=False)
    assert st2.sweeps == 2 + st2.iterations


def test_restart_reaches_same_solution():
    p = Problem(small_2d(nx=4, ny=5), 0, [3, 1, 10, 2], [0.01, 0.3, 0.2, 0.05])
    phi_a, sa_ = RS.solve(p, None, rtol=1e-12, restart=60)
    phi_b, sb_ = RS.solve(p, None, rtol=1e-12, restart=4)
    assert sb_.restarts > 0
    assert rel(phi_b, phi_a) < 1e-10
