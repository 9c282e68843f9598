"""Pins of the oracle DSA preconditioner (appendix A, extended to 2D axis by axis).

* The central-flux / jump split of the upwind operator, D_j = sum_d Omega_d (D_C,d - sign(Omega_d)/2 D_J,d),
  is checked against the transport blocks assembled independently by the discretisation module.
* The DSA moment system is checked against the angular moments of that same transport operator applied
  to a P1 angular function, which fixes every coefficient (kappa, mu2, c) and sign.
* Fourier analysis of consistent DSA for the 1D slab (infinite medium, any cell width) bounds the spectral
  radius of the accelerated source iteration by 0.2247 c; the finite slab must respect it.
"""
import numpy as np
import pytest

from oracle import Problem, dsa, romsad as RS, transport as T
from oracle.krylov import fgmres

from _helpers import rel, small_1d, small_2d


def _dense(f, n):
    return np.column_stack([f(e) for e in np.eye(n)])


def _homogeneous(spec, sig_s, sig_a):
    R = spec.n_regions
    return Problem(spec, 0, [sig_s] * R, [sig_a] * R)


def _rho(p, kind):
    """Spectral radius of I - M^{-1} A~ (source iteration for kind None, else with its DSA correction)."""
    A = _dense(lambda z: T.Atilde_apply(p, z), p.ndof)
    if kind is None:
        E = np.eye(p.ndof) - A
    else:
        E = np.eye(p.ndof) - _dense(dsa.Dsa(p, kind).apply, p.ndof) @ A
    return float(np.abs(np.linalg.eigvals(E)).max())


@pytest.mark.parametrize("spec", [small_1d(nx=7, rx=1), small_2d(nx=5, ny=4, n_polar=2, n_azim=8)])
def test_upwind_operator_splits_into_central_flux_and_jump(spec):
    p = _homogeneous(spec, 3.0, 0.5)
    ops = dsa.dg_operators(p)
    scale = 0.0
    for j in range(p.ndir):
        Dj = p.dense_L(j, sig_t=np.zeros(p.ncell))
        R = np.zeros_like(Dj)
        for d, (DC, DJ) in enumerate(ops):
            om = p.dirs[j][d]
            R += om * (DC.toarray() - np.sign(om) / 2.0 * DJ.toarray())
        scale = max(scale, np.abs(Dj).max())
        assert np.abs(Dj - R).max() < 1e-13 * scale
    for DC, DJ in ops:
        DC, DJ = DC.toarray(), DJ.toarray()
        assert np.abs(DC + DC.T).max() < 1e-13 * scale            # skew-symmetric
        assert np.abs(DJ - DJ.T).max() == 0.0                      # symmetric
        assert np.linalg.eigvalsh(DJ).max() < 1e-12 * scale        # negative semi-definite


def test_1d_jump_operator_of_a_single_interior_face():
    """Two cells of width h: the interior face couples p_0, p_1 traces (1/sqrt(h), +-sqrt(3/h));
    D_J = -(sum over faces) [eta_l][eta_k], the boundary faces seeing only their own cell."""
    p = _homogeneous(small_1d(nx=2, rx=1), 1.0, 1.0)
    h = p.hx
    DJ = dsa.dg_operators(p)[0][1].toarray()
    lo = np.array([1.0, -np.sqrt(3.0)]) / np.sqrt(h)
    hi = np.array([1.0, np.sqrt(3.0)]) / np.sqrt(h)
    jumps = []                                                      # [eta] on faces x0, x1, x2 (dofs: 2 cells x 2)
    jumps.append(np.r_[lo, 0, 0])                                   # left boundary: + side is cell 0
    jumps.append(np.r_[-hi, lo])                                    # interior: cell 1 (+) minus cell 0 (-)
    jumps.append(np.r_[0, 0, -hi])                                  # right boundary: - side is cell 1
    ref = -sum(np.outer(jv, jv) for jv in jumps)
    assert np.abs(DJ - ref).max() < 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("spec", [small_1d(nx=6, rx=2), small_2d(nx=4, ny=3, n_polar=2, n_azim=8)])
def test_moment_system_equals_moments_of_the_transport_operator(spec):
    """For dpsi_j = dphi + 3 Omega_j . dJ: sum_j w_j (L_j dpsi_j) - Sigma_s dphi is the 0th-moment row and
    sum_j w_j Omega_j,d L_j dpsi_j the first-moment row of the fully consistent system (L_j = D_j + Sigma_t)."""
    p = Problem(spec, 0, list(np.linspace(2.0, 9.0, spec.n_regions)), list(np.linspace(0.1, 0.7, spec.n_regions)))
    naxes = 1 if p.dim == 1 else 2
    rng = np.random.default_rng(3)
    dphi = rng.standard_normal(p.ndof)
    dJ = rng.standard_normal((naxes, p.ndof))
    m0 = -p.sig_s_dof * dphi
    m1 = np.zeros((naxes, p.ndof))
    for j in range(p.ndir):
        om = p.dirs[j][:naxes]
        Lpsi = p.dense_L(j) @ (dphi + 3.0 * om @ dJ)
        m0 += p.w[j] * Lpsi
        m1 += p.w[j] * np.outer(om, Lpsi)
    D = dsa.Dsa(p, "full")
    out = D.K @ np.concatenate([dphi, dJ.ravel()])
    assert rel(out[:p.ndof], m0) < 1e-12
    for d in range(naxes):
        assert rel(out[(d + 1) * p.ndof:(d + 2) * p.ndof], m1[d]) < 1e-12


def test_quadratures_integrate_quadratics():
    """3 mu2_d = 1 for the slab and CL rules used here (the P1 closure the appendix writes)."""
    for spec in (small_1d(nx=4, rx=1), small_2d(nx=2, ny=2, n_polar=2, n_azim=8),
                 small_2d(nx=2, ny=2, n_polar=6, n_azim=16)):
        mu2, kappa, c = dsa.quadrature_moments(_homogeneous(spec, 1.0, 1.0))
        assert np.allclose(3.0 * mu2, 1.0, atol=1e-14)
    mu2, kappa, c = dsa.quadrature_moments(_homogeneous(small_1d(nx=4, n_polar=2, rx=1), 1.0, 1.0))
    v = 1.0 / np.sqrt(3.0)                                          # S_2: +-1/sqrt(3), weights 1/2
    assert abs(kappa[0] - 0.5 * v) < 1e-15 and abs(c[0, 0] - v ** 3) < 1e-15


def test_partially_consistent_operator_is_spd():
    p = Problem(small_2d(nx=4, ny=4, n_polar=2, n_azim=8), 0, [20.0, 1.0, 300.0, 2.0], [0.1, 0.3, 0.2, 0.05])
    K = dsa.Dsa(p, "partial").K.toarray()
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()
    assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > 0.0


@pytest.mark.parametrize("sig_t_h", [0.025, 0.25, 2.5, 25.0])
def test_1d_fully_consistent_dsa_meets_the_fourier_bound(sig_t_h):
    """c = 0.9999: plain source iteration stalls (rho -> c in thick cells); consistent DSA stays below
    0.2247 c at every cell optical thickness."""
    spec = small_1d(nx=40, rx=1)
    p0 = _homogeneous(spec, 1.0, 1.0)
    sig_t = sig_t_h / p0.hx
    p = _homogeneous(spec, 0.9999 * sig_t, 1e-4 * sig_t)
    rho_fc = _rho(p, "full")
    assert rho_fc <= 0.2247 * 0.9999 + 1e-3
    assert rho_fc <= _rho(p, "partial") + 1e-12
    if sig_t_h >= 0.25:
        assert _rho(p, None) > 0.97


def test_2d_dsa_removes_the_diffusive_slowdown():
    spec = small_2d(nx=6, ny=6, n_polar=2, n_azim=8)
    p0 = _homogeneous(spec, 1.0, 1.0)
    sig_t = 1.6667 / p0.hx
    p = _homogeneous(spec, 0.9999 * sig_t, 1e-4 * sig_t)
    assert _rho(p, None) > 0.95
    rho_fc, rho_pc = _rho(p, "full"), _rho(p, "partial")
    assert rho_fc < 0.2 and rho_pc < 0.5 and rho_fc <= rho_pc


@pytest.mark.parametrize("post", ["dsa", "dsa_pc"])
def test_gmres_dsa_and_romsad_with_dsa_solve_the_dense_system(post):
    """Right-preconditioned GMRES-DSA and FGMRES-ROMSAD switching to DSA after the window both reach the
    solution of the dense system, with fewer iterations than unpreconditioned GMRES."""
    p = Problem(small_2d(nx=4, ny=4, n_polar=2, n_azim=8), 0, [20.0, 1.0, 300.0, 2.0], [0.1, 0.3, 0.2, 0.05])
    A = _dense(lambda z: T.Atilde_apply(p, z), p.ndof)
    bt = T.rhs_btilde(p)
    ref = np.linalg.solve(A, bt)
    _, st_plain = RS.solve(p, None, restart=100, rtol=1e-10, max_iter=2000)
    sol, st = fgmres(lambda z: T.Atilde_apply(p, z), bt, RS.make_preconditioner(None, p, 0, post),
                     restart=100, rtol=1e-10, max_iter=2000)
    assert rel(sol, ref) < 1e-8
    assert st.iterations < st_plain.iterations
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((p.ndir * p.ndof, 6)))
    rom = RS.build_rom(p, Q.T.reshape(6, p.ndir, p.ndof))
    sol2, st2 = RS.solve(p, rom, window=2, post=post, restart=100, rtol=1e-10, max_iter=2000)
    assert rel(sol2, ref) < 1e-8


# ------------------------------------------------------------------ approximate solve (one V-cycle)
def _eval_dg(p, coef, x, y):
    """Value of a DG Q1 function (orthonormal tensor Legendre) at a point, evaluated from the basis."""
    ix = min(int((x - p.x0) / p.hx), p.nx - 1)
    iy = min(int((y - p.y0) / p.hy), p.ny - 1)
    xi = 2.0 * (x - p.x0 - (ix + 0.5) * p.hx) / p.hx
    et = 2.0 * (y - p.y0 - (iy + 0.5) * p.hy) / p.hy
    px = [1.0 / np.sqrt(p.hx), np.sqrt(3.0 / p.hx) * xi]
    py = [1.0 / np.sqrt(p.hy), np.sqrt(3.0 / p.hy) * et]
    c = iy * p.nx + ix
    return sum(coef[c * 4 + a + 2 * b] * px[a] * py[b] for a in range(2) for b in range(2))


def test_continuous_prolongation_reproduces_bilinear_functions():
    p = _homogeneous(small_2d(nx=5, ny=3, n_polar=2, n_azim=4), 1.0, 1.0)
    u = lambda x, y: 1.0 + 2.0 * x - 3.0 * y + 5.0 * x * y
    vx = p.x0 + p.hx * np.arange(p.nx + 1)
    vy = p.y0 + p.hy * np.arange(p.ny + 1)
    uv = np.array([u(x, y) for y in vy for x in vx])
    coef = dsa.continuous_prolongation(p) @ uv
    rng = np.random.default_rng(0)
    for x, y in zip(rng.uniform(p.x0, p.x0 + p.nx * p.hx, 40), rng.uniform(p.y0, p.y0 + p.ny * p.hy, 40)):
        assert abs(_eval_dg(p, coef, x, y) - u(x, y)) < 1e-12


def test_vertex_interpolation_reproduces_bilinear_functions():
    u = lambda x, y: 0.5 - x + 4.0 * y + 3.0 * x * y
    ncx, ncy = 3, 2
    coarse = np.array([u(i / ncx, j / ncy) for j in range(ncy + 1) for i in range(ncx + 1)])
    fine = dsa.vertex_interpolation(ncx, ncy) @ coarse
    ref = np.array([u(i / (2 * ncx), j / (2 * ncy)) for j in range(2 * ncy + 1) for i in range(2 * ncx + 1)])
    assert np.abs(fine - ref).max() < 1e-14


def test_lumped_first_moment_blocks_have_the_closed_form():
    """Cell-diagonal block of B_d = 3 mu2_d Sigma_t - 3/2 sum_e c_de D_J,e: the jump operator's own-cell block
    along axis e is -(lo lo^T + hi hi^T) = -diag(2, 6)/h_e in that axis' degree, so the block is diagonal,
    3 mu2_d sigma_t + 3/2 sum_e c_de (2 or 6)/h_e by the dof's degree along e."""
    p = Problem(small_2d(nx=4, ny=3, n_polar=2, n_azim=8), 0, [20.0, 1.0, 300.0, 2.0], [0.1, 0.3, 0.2, 0.05])
    ops = dsa.dg_operators(p)
    mu2, kappa, c = dsa.quadrature_moments(p)
    h = (p.hx, p.hy)
    for d in range(2):
        Bd = 3.0 * mu2[d] * np.diag(p.sig_t_dof)
        for e, (DCe, DJe) in enumerate(ops):
            Bd = Bd - 1.5 * c[d, e] * DJe.toarray()
        for cell in range(p.ncell):
            blk = Bd[cell * 4:cell * 4 + 4, cell * 4:cell * 4 + 4]
            ref = np.array([3.0 * mu2[d] * p.sig_t[cell]
                            + 1.5 * sum(c[d, e] * (2.0 if (k >> e) & 1 == 0 else 6.0) / h[e] for e in range(2))
                            for k in range(4)])
            assert np.abs(blk - np.diag(ref)).max() < 1e-12 * ref.max()


@pytest.mark.parametrize("kind", ["partial", "lumped"])
def test_galerkin_hierarchy(kind):
    """A_0 = P_c^T K P_c and A_l = P_l^T A_{l-1} P_l are SPD, and the exact coarse correction leaves a
    residual orthogonal to the coarse space."""
    p = Problem(small_2d(nx=8, ny=8, n_polar=2, n_azim=8), 0, [20.0, 1.0, 300.0, 2.0], [0.1, 0.3, 0.2, 0.05])
    mg = dsa.MultigridDsa(p, kind)
    assert mg.dims == [(8, 8), (4, 4), (2, 2)]
    for A in mg.A:
        A = A.toarray()
        assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
        assert np.linalg.eigvalsh(A).min() > 0.0
    b = np.random.default_rng(2).standard_normal(p.ndof)
    P = mg.P[0].toarray()
    x = P @ np.linalg.solve(mg.A[0].toarray(), P.T @ b)
    assert np.linalg.norm(P.T @ (b - mg.K @ x)) < 1e-10 * np.linalg.norm(P.T @ b)


@pytest.mark.parametrize("spec", [small_2d(nx=8, ny=4, n_polar=2, n_azim=8), small_1d(nx=16, rx=2)])
@pytest.mark.parametrize("kind", ["partial", "lumped"])
def test_iterated_vcycle_converges_to_the_exact_dsa_solve(spec, kind):
    R = spec.n_regions
    p = Problem(spec, 0, list(np.geomspace(1.0, 400.0, R)), list(np.linspace(0.05, 0.4, R)))
    mg = dsa.MultigridDsa(p, kind)
    b = np.random.default_rng(4).standard_normal(p.ndof)
    ref = dsa.Dsa(p, kind).solve(b)
    x = np.zeros_like(b)
    for _ in range(200):                                            # a stationary iteration: contraction < 1
        x = x + mg.cycle(b - mg.K @ x)
    assert rel(x, ref) < 1e-10


@pytest.mark.parametrize("sig_t_h", [0.025, 0.25, 2.5, 25.0])
def test_1d_partially_consistent_vcycle_is_stable(sig_t_h):
    """c = 0.9999: source iteration with the V-cycle PC-DSA correction contracts at every cell optical
    thickness.  The lumped form does not in optically thin cells (its cell-diagonal first-moment operator
    misses the inter-cell jump coupling that dominates there), which is why PC is the default."""
    spec = small_1d(nx=40, rx=1)
    p0 = _homogeneous(spec, 1.0, 1.0)
    sig_t = sig_t_h / p0.hx
    p = _homogeneous(spec, 0.9999 * sig_t, 1e-4 * sig_t)
    A = _dense(lambda z: T.Atilde_apply(p, z), p.ndof)
    for kind, bound in (("partial", 0.55), ("lumped", None)):
        M = _dense(dsa.MultigridDsa(p, kind).apply, p.ndof)
        rho = float(np.abs(np.linalg.eigvals(np.eye(p.ndof) - M @ A)).max())
        if bound is not None:
            assert rho < bound
        elif sig_t_h <= 0.25:
            assert rho > 1.0


@pytest.mark.parametrize("kind", ["partial", "lumped"])
def test_gmres_with_the_vcycle_dsa_solves_the_dense_system(kind):
    p = Problem(small_2d(nx=8, ny=8, n_polar=2, n_azim=8), 0, [20.0, 1.0, 300.0, 2.0], [0.1, 0.3, 0.2, 0.05])
    A = _dense(lambda z: T.Atilde_apply(p, z), p.ndof)
    bt = T.rhs_btilde(p)
    ref = np.linalg.solve(A, bt)
    mg = dsa.MultigridDsa(p, kind)
    _, st_plain = fgmres(lambda z: T.Atilde_apply(p, z), bt, None, restart=100, rtol=1e-10, max_iter=3000)
    sol, st = fgmres(lambda z: T.Atilde_apply(p, z), bt, lambda j, v: mg.apply(v), restart=100, rtol=1e-10,
                     max_iter=3000)
    assert rel(sol, ref) < 1e-8
    assert st.iterations * 3 < st_plain.iterations


# ------------------------------------------------------------------ SI-SA (preconditioned Richardson)
def test_unaccelerated_richardson_is_source_iteration():
    """eq. richardson: phi^(l) = phi^(l-1) + r^(l-1) reproduces the source-iteration iterates phi <- T Sigma_s phi + b~."""
    from oracle.krylov import preconditioned_richardson, source_iteration
    p = Problem(small_2d(nx=4, ny=3, n_polar=2, n_azim=4), 0, [2.0, 1.0, 3.0, 0.5], [0.5, 0.3, 0.2, 0.4])
    its = source_iteration(p, 6)
    phi, st = preconditioned_richardson(lambda z: T.Atilde_apply(p, z), T.rhs_btilde(p), None, rtol=0.0, max_iter=6)
    assert st.iterations == 6 and rel(phi, its[-1]) < 1e-13


def test_richardson_with_the_exact_inverse_converges_in_one_step():
    from oracle.krylov import preconditioned_richardson
    p = Problem(small_2d(nx=4, ny=3, n_polar=2, n_azim=4), 0, [20.0, 1.0, 300.0, 2.0], [0.1, 0.3, 0.2, 0.05])
    A = _dense(lambda z: T.Atilde_apply(p, z), p.ndof)
    phi, st = preconditioned_richardson(lambda z: A @ z, T.rhs_btilde(p), lambda l, r: np.linalg.solve(A, r),
                                        rtol=1e-12, max_iter=5)
    assert st.iterations == 1 and st.converged


def test_si_dsa_contracts_at_the_spectral_radius():
    """SI with the exact PC-DSA correction: the residual ratio of late iterations approaches the spectral radius
    of I - M^{-1} A~ (the iteration matrix of the error; left and right preconditioning share the spectrum)."""
    p = _homogeneous(small_2d(nx=6, ny=6, n_polar=2, n_azim=8), 100.0 * 0.99, 100.0 * 0.01)
    phi, st = RS.si_solve(p, None, post="dsa_pc", rtol=1e-13, max_iter=200)
    assert st.converged
    h = st.history
    ratio = (h[-2] / h[-6]) ** 0.25
    assert abs(ratio - _rho(p, "partial")) < 0.05
