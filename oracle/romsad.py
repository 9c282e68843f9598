"""Oracle ROMSAD preconditioner and greedy ROM construction (paper Sec. 4), FP64.

Test infrastructure only.

Notation: U_r in R^{N_Omega N_DOF x r} with orthonormal columns, stored as
U[r, N_Omega, N_DOF] (U[:, j, :] holds the rows U_{r,j}).
  P = sum_j U_{r,j},  W = sum_j omega_j U_{r,j}           (eq. rom-correction)
  U_r^T A_mu U_r = sum_j U_{r,j}^T (D_j + Sigma_t) U_{r,j} - P^T Sigma_s W
                                                          (A of eq. one_equation)
  M_ROM^{-1} v = v + W (U_r^T A U_r)^{-1} P^T Sigma_s v   (eq. rom-sa-preconditioner)
Affine split (Sec. 4.1): with region indicators chi_R, Sigma_t = sum_R
(sigma_a,R + sigma_s,R) chi_R and Sigma_s = sum_R sigma_s,R chi_R, so
  U^T A_mu U = A_D + sum_R (sigma_a,R + sigma_s,R) T_R - sum_R sigma_s,R S_R,
  A_D = sum_j U_j^T D_j U_j, T_R = sum_j U_j^T chi_R U_j, S_R = P^T chi_R W.
ROM data (Sec. 4.4.1): xi^(1) = (phi - phi^(0)) / ||r^(0)|| (eq. correction-fgmres1),
xi^(l) = (z^(l-1) - sum_{i<l} H_{i,l-1} xi^(i)) / H_{l,l-1} (eq. correction-fgmres2),
delta psi_j^(l) = (D_j + Sigma_t)^{-1} Sigma_s xi^(l) (eq. fgmres-psi-correction).
Greedy (Sec. 4.4.2) with the modified Gram-Schmidt + truncation of appendix B.
After the window the switch (eq. ROMSAD-preconditioner) can hand over to the DSA preconditioner of
appendix A (oracle.dsa), as in the paper.

Readings where the paper is silent:
  * truncation test of appendix B is relative: ||u|| > eps_QR * ||psi|| (the
    snapshot's norm before orthogonalisation); one MGS pass;
  * the error indicator is relative: R_mu / ||eta_mu^(0)||_2 against eps_ROM;
  * the high-fidelity solve of step 2(a) is FGMRES with M = I (the xi
    recurrence holds for any preconditioner);
  * mu_1 is the training point nearest the centroid of (log sigma_s, sigma_a);
    argmax ties go to the lowest index; the rank is capped at max_rank.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import dsa
from .discretization import Problem, with_params
from .krylov import fgmres
from .transport import Atilde_apply, rhs_btilde


@dataclasses.dataclass
class Rom:
    U: np.ndarray          # [r, N_Omega, N_DOF]
    P: np.ndarray          # [N_DOF, r]
    W: np.ndarray          # [N_DOF, r]
    A_D: np.ndarray        # [r, r]
    T_R: np.ndarray        # [R, r, r]
    S_R: np.ndarray        # [R, r, r]

    @property
    def r(self) -> int:
        return self.U.shape[0]


def build_rom(p: Problem, U: np.ndarray) -> Rom:
    """P, W and the affine reduced operators for basis U[r, N_Omega, N_DOF]."""
    r = U.shape[0]
    P = U.sum(axis=1).T.copy()
    W = np.einsum("j,rjn->nr", p.w, U)
    zero_t = np.zeros(p.ncell)
    A_D = np.zeros((r, r))
    for j in range(p.ndir):
        DU = np.stack([p.apply_forward(j, U[c, j], sig_t=zero_t) for c in range(r)])  # [r, n]
        A_D += U[:, j, :] @ DU.T
    R = len(p.sigma_s_region)
    T_R = np.zeros((R, r, r))
    S_R = np.zeros((R, r, r))
    for reg in range(R):
        # term reg of the affine split: the region's indicator, or the blocks of profile reg
        for j in range(p.ndir):
            T_R[reg] += p.mode_apply(reg, U[:, j, :]) @ U[:, j, :].T
        S_R[reg] = P.T @ p.mode_apply(reg, W.T).T
    return Rom(U, P, W, A_D, T_R, S_R)


def reduced_operator(rom: Rom, sigma_s, sigma_a) -> np.ndarray:
    """Online affine assembly sum_s a_s(mu) A_{s,r} (Sec. 4.1)."""
    ss = np.asarray(sigma_s)
    sa = np.asarray(sigma_a)
    A = rom.A_D.copy()
    for reg in range(len(ss)):
        A += (ss[reg] + sa[reg]) * rom.T_R[reg] - ss[reg] * rom.S_R[reg]
    return A


def reduced_operator_direct(p: Problem, U: np.ndarray) -> np.ndarray:
    """U_r^T A_mu U_r from the coupled operator itself (no affine split)."""
    r = U.shape[0]
    P = U.sum(axis=1).T
    W = np.einsum("j,rjn->nr", p.w, U)
    A = np.zeros((r, r))
    for j in range(p.ndir):
        LU_ = np.stack([p.apply_forward(j, U[c, j]) for c in range(r)])
        A += U[:, j, :] @ LU_.T
    A -= P.T @ np.stack([p.Ss_apply(W[:, k]) for k in range(r)], axis=1)
    return A


def romsad_apply(rom: Rom, p: Problem, v: np.ndarray, A_r: Optional[np.ndarray] = None) -> np.ndarray:
    """z = M_ROM^{-1} v = v + W (U^T A U)^{-1} P^T Sigma_s v (eq. rom-sa-preconditioner)."""
    if A_r is None:
        A_r = reduced_operator(rom, p.sigma_s_region, p.sigma_a_region)
    c = np.linalg.solve(A_r, rom.P.T @ p.Ss_apply(v))
    return v + rom.W @ c


def make_preconditioner(rom: Optional[Rom], p: Problem, window: int, post: str = "rom"):
    """M_j of eq. ROMSAD-preconditioner: ROM for j <= window; afterwards 'rom', 'identity', or the DSA
    preconditioner of appendix A ('dsa': fully consistent, 'dsa_pc': partially consistent, both solved
    exactly; 'dsa_vcycle' / 'dsa_vcycle_lumped': partially / lumped fully consistent through one V-cycle of
    dsa.MultigridDsa).  Without a ROM, the DSA options give the DSA preconditioner for every j (GMRES-DSA,
    SI-DSA) and anything else none."""
    if post in ("dsa_vcycle", "dsa_vcycle_lumped"):
        D = dsa.MultigridDsa(p, "partial" if post == "dsa_vcycle" else "lumped")
    else:
        dsa_kind = {"dsa": "full", "dsa_pc": "partial"}.get(post)
        D = dsa.Dsa(p, dsa_kind) if dsa_kind is not None else None
    if rom is None:
        if D is None:
            return None
        return lambda j, v: D.apply(v)
    A_r = reduced_operator(rom, p.sigma_s_region, p.sigma_a_region)

    def precond(j: int, v: np.ndarray) -> np.ndarray:
        if j <= window or post == "rom":
            return romsad_apply(rom, p, v, A_r)
        if D is not None:
            return D.apply(v)
        return v.copy()

    return precond


def solve(p: Problem, rom: Optional[Rom] = None, window: int = 2, post: str = "rom",
          restart: int = 30, rtol: float = 1e-10, max_iter: int = 1000, phi0=None,
          true_residual_check: bool = True, record_first_cycle: bool = False):
    """FGMRES-ROMSAD on A~ phi = b~ (Alg. 1 with eq. ROMSAD-preconditioner)."""
    bt = rhs_btilde(p)
    pre = make_preconditioner(rom, p, window, post)
    return fgmres(lambda z: Atilde_apply(p, z), bt, pre, phi0=phi0, restart=restart, rtol=rtol,
                  max_iter=max_iter, true_residual_check=true_residual_check,
                  record_first_cycle=record_first_cycle)


def si_solve(p: Problem, rom: Optional[Rom] = None, window: int = 2, post: str = "rom", rtol: float = 1e-10,
             max_iter: int = 1000, phi0=None):
    """SI-ROMSAD (Sec. 3.1-3.2, 4.2): source iteration with the ROM correction for the first `window`
    iterations and `post` afterwards, as the preconditioned Richardson iteration of eq.
    preconditioned-richardson with the M_l of eq. ROMSAD-preconditioner."""
    from .krylov import preconditioned_richardson
    bt = rhs_btilde(p)
    pre = make_preconditioner(rom, p, window, post)
    return preconditioned_richardson(lambda z: Atilde_apply(p, z), bt, pre, phi0=phi0, rtol=rtol, max_iter=max_iter)


def xi_recurrence(phi: np.ndarray, first: dict, window: int) -> List[np.ndarray]:
    """xi^(l), l = 1..window, from the converged phi and the first FGMRES cycle (eqs. correction-fgmres1/2)."""
    H, Z, beta, phi0 = first["H"], first["Z"], first["beta"], first["phi0"]
    xis = [(phi - phi0) / beta]
    for l in range(2, window + 1):
        if l - 1 > Z.shape[0] or H.shape[0] < l or H[l - 1, l - 2] == 0.0:
            break
        acc = Z[l - 2].copy()
        for i in range(1, l):
            acc -= H[i - 1, l - 2] * xis[i - 1]
        xis.append(acc / H[l - 1, l - 2])
    return xis


def correction_snapshot(p: Problem, xi: np.ndarray) -> np.ndarray:
    """delta psi_j = (D_j + Sigma_t)^{-1} Sigma_s xi for every j; shape [N_Omega, N_DOF]."""
    s = p.Ss_apply(xi)
    return np.stack([p.sweep(j, s) for j in range(p.ndir)])


def mgs_truncate(U: List[np.ndarray], psi: np.ndarray, eps_qr: float = 1e-13) -> bool:
    """Appendix B: orthogonalise psi against the columns of U (one MGS pass); append if kept."""
    u = psi.copy()
    for col in U:
        R = float(col @ u)
        u = u - R * col
    nu = float(np.linalg.norm(u))
    if nu > eps_qr * float(np.linalg.norm(psi)):
        U.append(u / nu)
        return True
    return False


def default_mu1(sigma_s: np.ndarray, sigma_a: np.ndarray) -> int:
    feats = np.concatenate([np.log(sigma_s), sigma_a], axis=1)
    d = np.sum((feats - feats.mean(axis=0)) ** 2, axis=1)
    return int(np.argmin(d))


@dataclasses.dataclass
class GreedyReport:
    sampled: List[int]
    max_indicator: List[float]
    rank: int
    labels: Optional[np.ndarray] = None     # [n_train, r] Galerkin coefficients on the final basis
    hf_iterations: List[int] = dataclasses.field(default_factory=list)


def greedy(p_template: Problem, sigma_s: np.ndarray, sigma_a: np.ndarray, window: int = 2,
           max_greedy_iter: int = 10, max_rank: int = 32, eps_rom: float = 1e-8,
           eps_qr: float = 1e-13, mu1: Optional[int] = None, hf_rtol: float = 1e-12,
           restart: int = 30, want_labels: bool = False, hf_post: Optional[str] = None):
    """Greedy ROM construction of Sec. 4.4.2.  Returns (Rom, GreedyReport).

    hf_post: preconditioner of the step 2(a) high-fidelity FGMRES, None (M = I) or one of the DSA options of
    make_preconditioner (the paper solves step 2(a) with FGMRES-DSA); the first cycle keeps the
    preconditioned vectors z that the xi recurrence reads."""
    n_train = sigma_s.shape[0]
    probs = [with_params(p_template, sigma_s[i], sigma_a[i]) for i in range(n_train)]
    # Step 1: b~_mu and eta_mu^(0) = Sigma_s r_mu^(0) with r^(0) = b~ (zero initial guess)
    bt = [rhs_btilde(q) for q in probs]
    eta0 = [q.Ss_apply(b) for q, b in zip(probs, bt)]
    k_idx = default_mu1(sigma_s, sigma_a) if mu1 is None else mu1
    sampled = [k_idx]
    cols: List[np.ndarray] = []
    rep = GreedyReport(sampled=sampled, max_indicator=[], rank=0)
    nd_ang = p_template.ndir * p_template.ndof
    rom = None
    while True:
        q = probs[k_idx]
        # Step 2(a): high-fidelity FGMRES (M = I or DSA, zero guess), keep the first cycle
        pre = make_preconditioner(None, q, window, hf_post) if hf_post else None
        phi, st, first = fgmres(lambda z: Atilde_apply(q, z), bt[k_idx], pre, restart=restart,
                                rtol=hf_rtol, true_residual_check=False, record_first_cycle=True)
        rep.hf_iterations.append(st.iterations)
        xis = xi_recurrence(phi, first, window)
        # Step 2(b): angular flux corrections by transport sweeps
        # Step 2(c): MGS with truncation, then the reduced operators
        for xi in xis:
            if len(cols) >= max_rank:
                break
            snap = correction_snapshot(q, xi).reshape(nd_ang)
            mgs_truncate(cols, snap, eps_qr)
        U = np.stack(cols).reshape(len(cols), p_template.ndir, p_template.ndof)
        rom = build_rom(p_template, U)
        if len(sampled) >= max_greedy_iter or len(cols) >= max_rank or len(sampled) == n_train:
            break
        # Step 3: reduced solutions and residual indicators for unsampled mu
        best, best_i = -1.0, -1
        for i in range(n_train):
            if i in sampled:
                continue
            Ind = rom_indicator(rom, probs[i], eta0[i])
            if Ind > best:
                best, best_i = Ind, i
        rep.max_indicator.append(best)
        if best < eps_rom:
            break
        k_idx = best_i
        sampled.append(k_idx)
    rep.rank = rom.r
    if want_labels:
        rep.labels = np.stack([galerkin_coefficients(rom, probs[i], eta0[i]) for i in range(n_train)])
    return rom, rep


def galerkin_coefficients(rom: Rom, q: Problem, eta0: np.ndarray) -> np.ndarray:
    """c solving U^T A_mu U c = P^T eta^(0) (eq. greedy-rom)."""
    A_r = reduced_operator(rom, q.sigma_s_region, q.sigma_a_region)
    return np.linalg.solve(A_r, rom.P.T @ eta0)


def rom_indicator(rom: Rom, q: Problem, eta0: np.ndarray) -> float:
    """max_j ||(D_j + Sigma_t) U_j c - Sigma_s W c - eta^(0)||_2 / ||eta^(0)||_2 (eq. rom-residual)."""
    c = galerkin_coefficients(rom, q, eta0)
    dphi = rom.W @ c
    base = q.Ss_apply(dphi) + eta0
    worst = 0.0
    for j in range(q.ndir):
        dpsi_j = np.tensordot(c, rom.U[:, j, :], axes=(0, 0))
        res = q.apply_forward(j, dpsi_j) - base
        worst = max(worst, float(np.linalg.norm(res)))
    return worst / float(np.linalg.norm(eta0))
