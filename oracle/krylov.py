"""Oracle Krylov solvers (paper Sec. 4.2, Alg. 1; Sec. 3), FP64, numpy.

Test infrastructure only.

fgmres() follows Alg. 1 (flexible GMRES, Saad 1993): z_j = M_j^{-1} v_j,
w = A z_j, modified Gram-Schmidt against v_1..v_j giving H[:, j],
H[j+1, j] = ||w||, v_{j+1} = w / H[j+1, j]; the least-squares step
y = argmin ||beta e_1 - H~ y|| is solved with numpy's lstsq (the plain
definition; no Givens recurrence), and phi = phi0 + Z~ y.

Readings where the paper is silent (Alg. 1 says only "stopping criteria"):
  * stop when ||beta e_1 - H~ y||_2 / ||b||_2 <= rtol (relative residual, as
    in Sec. 5);
  * happy breakdown when H[j+1, j] <= 1e-14 * ||w|| before orthogonalisation;
  * restarted FGMRES(m): phi0 <- phi, r0 = b - A phi0 (one operator apply);
  * after the estimate converges, the true residual b - A phi is evaluated
    once (optional); if it exceeds 2 * rtol * ||b|| the solve restarts from it;
  * the preconditioner index j counts iterations globally across restarts.
Counting (Sec. 5, remark on sweeps): with a zero initial guess the number of
operator applies is 1 (for b) + iterations; a nonzero guess adds one; each
restart adds one.  The optional final check is counted separately.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class SolveStats:
    iterations: int = 0
    sweeps: int = 0
    restarts: int = 0
    check_sweeps: int = 0
    est_rel_residual: float = float("nan")
    true_rel_residual: float = float("nan")
    true_linf_residual: float = float("nan")
    converged: bool = False
    history: List[float] = dataclasses.field(default_factory=list)


def fgmres(apply_A: Callable[[np.ndarray], np.ndarray], b: np.ndarray,
           precond: Optional[Callable[[int, np.ndarray], np.ndarray]] = None,
           phi0: Optional[np.ndarray] = None, restart: int = 30, rtol: float = 1e-10,
           max_iter: int = 1000, true_residual_check: bool = True,
           breakdown_tol: float = 1e-14, record_first_cycle: bool = False,
           rhs_sweeps: int = 1):
    """Restarted FGMRES(m) on A x = b (Alg. 1).  Returns (phi, stats[, first_cycle]).

    precond(j, v) returns z = M_j^{-1} v with j the 1-based global iteration
    index (None: M_j = I).  rhs_sweeps is the number of operator applies that
    produced b (1 for b~ of the RTE), added to stats.sweeps.
    first_cycle (when recorded): dict with V [k+1, n], Z [k, n], H [k+1, k],
    beta, phi0 of the first cycle, as needed by the xi recurrence.
    """
    n = b.shape[0]
    st = SolveStats(sweeps=rhs_sweeps)
    bnorm = float(np.linalg.norm(b))
    if phi0 is None or float(np.linalg.norm(phi0)) == 0.0:
        phi = np.zeros(n)
        r = b.copy()
    else:
        phi = phi0.astype(np.float64).copy()
        r = b - apply_A(phi)
        st.sweeps += 1
    first = None
    if bnorm == 0.0:
        st.converged = True
        st.est_rel_residual = st.true_rel_residual = 0.0
        st.true_linf_residual = 0.0
        return (phi, st, first) if record_first_cycle else (phi, st)
    while True:
        beta = float(np.linalg.norm(r))
        st.history.append(beta / bnorm)
        if beta / bnorm <= rtol:
            st.converged = True
            st.est_rel_residual = beta / bnorm
            break
        if st.iterations >= max_iter:
            st.est_rel_residual = beta / bnorm
            break
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        k = 0
        est = beta
        for j in range(m):
            jg = st.iterations + 1
            Z[j] = V[j] if precond is None else precond(jg, V[j])
            w = apply_A(Z[j])
            st.iterations += 1
            st.sweeps += 1
            w0 = float(np.linalg.norm(w))
            for i in range(j + 1):
                H[i, j] = float(w @ V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            k = j + 1
            e1 = np.zeros(k + 1)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
            est = float(np.linalg.norm(e1 - H[:k + 1, :k] @ y))
            st.history.append(est / bnorm)
            happy = H[j + 1, j] <= breakdown_tol * max(w0, 1e-300)
            if not happy:
                V[j + 1] = w / H[j + 1, j]
            if happy or est / bnorm <= rtol or st.iterations >= max_iter:
                break
        e1 = np.zeros(k + 1)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
        if first is None and record_first_cycle:
            first = dict(V=V[:k + 1].copy(), Z=Z[:k].copy(), H=H[:k + 1, :k].copy(), beta=beta,
                         phi0=phi.copy())
        phi = phi + Z[:k].T @ y
        st.est_rel_residual = est / bnorm
        if est / bnorm <= rtol or happy:
            if true_residual_check:
                r = b - apply_A(phi)
                st.check_sweeps += 1
                tr = float(np.linalg.norm(r)) / bnorm
                st.true_rel_residual = tr
                st.true_linf_residual = float(np.max(np.abs(r)))
                if tr <= 2.0 * rtol or st.iterations >= max_iter:
                    st.converged = tr <= 2.0 * rtol
                    break
                st.restarts += 1
                continue
            st.converged = True
            break
        if st.iterations >= max_iter:
            break
        r = b - apply_A(phi)
        st.sweeps += 1
        st.restarts += 1
    return (phi, st, first) if record_first_cycle else (phi, st)


def preconditioned_richardson(apply_A: Callable[[np.ndarray], np.ndarray], b: np.ndarray,
                              precond: Optional[Callable[[int, np.ndarray], np.ndarray]] = None,
                              phi0: Optional[np.ndarray] = None, rtol: float = 1e-10, max_iter: int = 1000,
                              rhs_sweeps: int = 1):
    """Source iteration with synthetic acceleration as a preconditioned Richardson iteration
    (Sec. 3.2, eq. preconditioned-richardson): phi^(l) = phi^(l-1) + M_l^{-1} r^(l-1), r = b - A phi.
    precond(l, r) returns M_l^{-1} r (None: M = I, classical SI, eq. richardson).  Stops when
    ||r||_2 <= rtol ||b||_2, checked on the residual of every iterate.  sweeps counts operator applies:
    rhs_sweeps for b, one per residual (none for the first one of a zero start, r = b)."""
    st = SolveStats(sweeps=rhs_sweeps)
    bnorm = float(np.linalg.norm(b))
    phi = np.zeros_like(b) if phi0 is None else phi0.astype(np.float64).copy()
    l = 0
    while True:
        if l == 0 and phi0 is None:
            r = b.copy()
        else:
            r = b - apply_A(phi)
            st.sweeps += 1
        rel = float(np.linalg.norm(r)) / bnorm if bnorm > 0 else 0.0
        st.history.append(rel)
        st.true_rel_residual = st.est_rel_residual = rel
        st.true_linf_residual = float(np.abs(r).max()) if r.size else 0.0
        if rel <= rtol:
            st.converged = True
            break
        if st.iterations >= max_iter:
            break
        l += 1
        phi = phi + (r if precond is None else precond(l, r))
        st.iterations += 1
    return phi, st


def source_iteration(p, n_iter: int, phi0: Optional[np.ndarray] = None):
    """Memory-efficient SI (eq. memory-efficient-SI): phi <- T Sigma_s phi + b~.

    Returns the list of iterates; used to check the Richardson identity
    r^(l-1) = phi^(l,*) - phi^(l-1) (eq. SI-residual-relation).
    """
    from .transport import T_apply, rhs_btilde
    bt = rhs_btilde(p)
    phi = np.zeros(p.ndof) if phi0 is None else phi0.copy()
    out = [phi]
    for _ in range(n_iter):
        phi = T_apply(p, p.Ss_apply(phi)) + bt
        out.append(phi)
    return out
