"""Pins of the oracle ROMSAD machinery (Sec. 4, appendix B): P8, P9."""
import numpy as np
import pytest

from oracle import Problem, transport as T, romsad as RS
from oracle.krylov import fgmres
from oracle.discretization import with_params

import workloads as wl
from _helpers import rel, small_2d, small_1d


def _problem(seed_sig=(20, 1, 300, 2), seed_abs=(0.1, 0.3, 0.2, 0.05)):
    return Problem(small_2d(nx=4, ny=4, n_polar=2, n_azim=4), 0, list(seed_sig), list(seed_abs))


def _dense_Atilde(p):
    return np.stack([T.Atilde_apply(p, e) for e in np.eye(p.ndof)], axis=1)


@pytest.mark.parametrize("pre", [None, "dsa_vcycle"])
def test_xi_recurrence_equals_dense_solve(pre):
    """xi^(l) from eqs. correction-fgmres1/2 equals A~^{-1} v^(l), for FGMRES with M = I and with the DSA
    preconditioner (the recorded z = M^{-1} v enter the recurrence; the identity holds for any M)."""
    p = _problem()
    bt = T.rhs_btilde(p)
    M = RS.make_preconditioner(None, p, 2, pre) if pre else None
    phi, st, first = fgmres(lambda z: T.Atilde_apply(p, z), bt, M, restart=200, rtol=1e-14,
                            true_residual_check=False, record_first_cycle=True)
    Ad = _dense_Atilde(p)
    xis = RS.xi_recurrence(phi, first, 4)
    assert len(xis) == 4
    for l, xi in enumerate(xis):
        ref = np.linalg.solve(Ad, first["V"][l])
        assert rel(xi, ref) < 1e-9


def test_snapshot_solves_ideal_kinetic_correction_equation():
    """delta psi of eq. fgmres-psi-correction satisfies eq. ideal-kinetic-correction-fgmres:
    (D_j + Sigma_t) dpsi_j = Sigma_s dphi + Sigma_s v, with dphi = sum_j w_j dpsi_j = T Sigma_s xi."""
    p = _problem()
    rng = np.random.default_rng(1)
    v = rng.standard_normal(p.ndof)
    Ad = _dense_Atilde(p)
    xi = np.linalg.solve(Ad, v)
    dpsi = RS.correction_snapshot(p, xi)
    dphi = T.scalar_flux(p, dpsi)
    assert rel(dphi, T.T_apply(p, p.sig_s_dof * xi)) < 1e-12      # eq. density-relation
    for j in range(p.ndir):
        lhs = p.apply_forward(j, dpsi[j])
        rhs = p.sig_s_dof * dphi + p.sig_s_dof * v
        assert rel(lhs, rhs) < 1e-10
    # and v + dphi = xi (so the ideal correction turns v into A~^{-1} v)
    assert rel(v + dphi, xi) < 1e-10


def test_affine_reduced_operator_equals_direct_projection_and_basis_orthonormal():
    p = _problem()
    rng = np.random.default_rng(2)
    cols = []
    for _ in range(6):
        RS.mgs_truncate(cols, rng.standard_normal(p.ndir * p.ndof))
    U = np.stack(cols).reshape(6, p.ndir, p.ndof)
    G = U.reshape(6, -1) @ U.reshape(6, -1).T
    assert np.max(np.abs(G - np.eye(6))) < 1e-13
    rom = RS.build_rom(p, U)
    for ss, sa in (([3, 4, 5, 6], [0.1, 0.2, 0.3, 0.4]), ([1000, 1, 1, 20], [0, 0.5, 0.5, 0])):
        q = with_params(p, ss, sa)
        A_aff = RS.reduced_operator(rom, ss, sa)
        A_dir = RS.reduced_operator_direct(q, U)
        assert np.max(np.abs(A_aff - A_dir)) < 1e-10 * np.max(np.abs(A_dir))
        # against the dense coupled system of eq. one_equation
        A, _ = T.dense_coupled_system(q)
        Uf = U.reshape(6, -1).T
        assert np.max(np.abs(Uf.T @ A @ Uf - A_dir)) < 1e-10 * np.max(np.abs(A_dir))


def test_mgs_truncation_drops_dependent_vectors():
    rng = np.random.default_rng(3)
    cols = []
    a, b = rng.standard_normal(50), rng.standard_normal(50)
    assert RS.mgs_truncate(cols, a)
    assert RS.mgs_truncate(cols, b)
    assert not RS.mgs_truncate(cols, 2.0 * a - 3.0 * b)
    assert len(cols) == 2


def test_rom_reproduction_converges_in_one_iteration():
    """If the ideal correction of the first iteration lies in span U_r, the Galerkin
    correction recovers it exactly: z_1 = A~^{-1} v_1 and FGMRES stops after 1 iteration."""
    p = _problem()
    bt = T.rhs_btilde(p)
    phi, st, first = fgmres(lambda z: T.Atilde_apply(p, z), bt, None, restart=200, rtol=1e-14,
                            true_residual_check=False, record_first_cycle=True)
    xi1 = RS.xi_recurrence(phi, first, 1)[0]
    cols = []
    RS.mgs_truncate(cols, RS.correction_snapshot(p, xi1).ravel())
    rng = np.random.default_rng(4)
    for _ in range(3):   # extra unrelated columns do not spoil the exact reproduction
        RS.mgs_truncate(cols, rng.standard_normal(p.ndir * p.ndof))
    rom = RS.build_rom(p, np.stack(cols).reshape(len(cols), p.ndir, p.ndof))
    phi_r, st_r = RS.solve(p, rom, window=1, post="identity", rtol=1e-10)
    assert st_r.iterations == 1
    assert rel(phi_r, phi) < 1e-9


def _dense_indicator(rom, q, eta0):
    A, _ = T.dense_coupled_system(q)
    U = rom.U.reshape(rom.r, -1).T
    db = np.tile(eta0, q.ndir)
    c = np.linalg.solve(U.T @ A @ U, U.T @ db)
    res = (A @ (U @ c) - db).reshape(q.ndir, q.ndof)
    return np.max(np.linalg.norm(res, axis=1)) / np.linalg.norm(eta0)


def test_greedy_brute_force_on_few_training_points():
    """Sampled order = argmax of the indicator of eq. rom-residual recomputed from the dense
    coupled system; r <= k * window; basis orthonormal."""
    spec = small_2d(nx=3, ny=3, n_polar=2, n_azim=4)
    ss, sa = wl.draw_params(spec, 5, 77)
    p0 = Problem(spec, 0, ss[0], sa[0])
    window = 2
    rom, rep = RS.greedy(p0, ss, sa, window=window, max_greedy_iter=3, max_rank=100, eps_rom=0.0,
                         hf_rtol=1e-13, restart=300)
    assert len(rep.sampled) == 3
    assert rep.rank <= len(rep.sampled) * window
    Uf = rom.U.reshape(rom.r, -1)
    assert np.max(np.abs(Uf @ Uf.T - np.eye(rom.r))) < 1e-12
    # replay: rebuild the basis after each sample and check the next argmax densely
    probs = [with_params(p0, ss[i], sa[i]) for i in range(5)]
    eta0 = [q.sig_s_dof * T.rhs_btilde(q) for q in probs]
    cols_per_sample = []
    r_so_far = 0
    for k in range(1, 3):
        # the basis after k samples is a prefix of the final basis
        r_k = min(k * window, rom.r)
        Uk = rom.U[:r_k]
        rom_k = RS.build_rom(p0, Uk)
        cand = [i for i in range(5) if i not in rep.sampled[:k]]
        ind = {i: _dense_indicator(rom_k, probs[i], eta0[i]) for i in cand}
        best = max(cand, key=lambda i: (ind[i], -i))
        assert best == rep.sampled[k]
        assert abs(rep.max_indicator[k - 1] - ind[best]) < 1e-8 * ind[best]
