"""GPU parity of the transport kernels (sweep, quadrature, T, A~, b~) against the oracle."""
import numpy as np
import pytest

import workloads as wl
from oracle import transport as OT

from gpu_common import lib, oracle_problems, rel, spec1d, spec2d, split, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

# meshes spanning several 32-row bands with ragged tails, nx both below and above the warp width
MESHES_2D = [(38, 46), (12, 70), (64, 64), (8, 8), (96, 34)]


def _params(spec, seed):
    return wl.draw_params(spec, spec.n_instances, seed)


@pytest.mark.parametrize("mesh", MESHES_2D)
def test_apply_op_fp64_matches_oracle(mesh):
    torch = torch_cuda()
    B = lib()
    spec = spec2d([mesh[0]], [mesh[1]], n_polar=4, n_azim=8)
    ss, sa = _params(spec, 11)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    rng = np.random.default_rng(5)
    z = rng.standard_normal(gp.n_dof)
    w = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.apply_op(to_dev(z), w)
    ref = OT.Atilde_apply(ops[0], z)
    assert rel(w.cpu().numpy(), ref) < 1e-13
    # T itself
    gp.apply_T(to_dev(z), w)
    assert rel(w.cpu().numpy(), OT.T_apply(ops[0], z)) < 1e-13


def test_batched_uneven_instances_match_oracle_per_instance():
    torch = torch_cuda()
    B = lib()
    spec = spec2d([32, 64, 40, 16], [32, 64, 24, 48], n_polar=4, n_azim=8, inflow_g=0.3)
    ss, sa = _params(spec, 12)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    rng = np.random.default_rng(6)
    z = rng.standard_normal(gp.n_dof)
    w = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.apply_op(to_dev(z), w)
    bt = torch.empty_like(w)
    gp.rhs(bt)
    for b, (wb, zb, bb) in enumerate(zip(split(w.cpu().numpy(), gp.offsets), split(z, gp.offsets),
                                         split(bt.cpu().numpy(), gp.offsets))):
        assert rel(wb, OT.Atilde_apply(ops[b], zb)) < 1e-13
        assert rel(bb, OT.rhs_btilde(ops[b])) < 1e-13


@pytest.mark.parametrize("g", [0.0, 0.7])
def test_rhs_fp64_matches_oracle(g):
    torch = torch_cuda()
    B = lib()
    spec = spec2d([40], [36], n_polar=4, n_azim=8, inflow_g=g)
    ss, sa = _params(spec, 13)
    gp = B.Problem(spec, ss, sa)
    op = oracle_problems(spec, ss, sa)[0]
    bt = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.rhs(bt)
    assert rel(bt.cpu().numpy(), OT.rhs_btilde(op)) < 1e-13


def test_angular_sweep_and_scalar_flux_match_oracle():
    torch = torch_cuda()
    B = lib()
    spec = spec2d([34], [40], n_polar=4, n_azim=8, inflow_g=0.25)
    ss, sa = _params(spec, 14)
    gp = B.Problem(spec, ss, sa)
    op = oracle_problems(spec, ss, sa)[0]
    rng = np.random.default_rng(7)
    s = rng.standard_normal(gp.n_dof)
    psi = torch.empty(gp.n_directions * gp.n_dof, dtype=torch.float64, device="cuda")
    gp.sweep(to_dev(s), psi, with_bc=True)
    ref = np.stack([op.sweep(j, s + op.gbc(j)) for j in range(op.ndir)])
    got = psi.cpu().numpy().reshape(op.ndir, op.ndof)
    for j in range(op.ndir):
        assert rel(got[j], ref[j]) < 1e-13, j
    phi = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.scalar_flux(psi, phi)
    assert rel(phi.cpu().numpy(), OT.scalar_flux(op, ref)) < 1e-13


def test_fp32_kernels_close_to_oracle():
    torch = torch_cuda()
    B = lib()
    spec = spec2d([48], [40], n_polar=4, n_azim=8, inflow_g=0.5)
    ss, sa = _params(spec, 15)
    gp = B.Problem(spec, ss, sa)
    op = oracle_problems(spec, ss, sa)[0]
    rng = np.random.default_rng(8)
    z = rng.standard_normal(gp.n_dof)
    w = torch.empty(gp.n_dof, dtype=torch.float32, device="cuda")
    gp.apply_op(to_dev(z, torch.float32), w)
    assert rel(w.cpu().numpy(), OT.Atilde_apply(op, z.astype(np.float32).astype(np.float64))) < 2e-5
    bt = torch.empty(gp.n_dof, dtype=torch.float32, device="cuda")
    gp.rhs(bt)
    assert rel(bt.cpu().numpy(), OT.rhs_btilde(op)) < 2e-5
    psi = torch.empty(gp.n_directions * gp.n_dof, dtype=torch.float32, device="cuda")
    gp.sweep(to_dev(z, torch.float32), psi, with_bc=False)
    ref = np.stack([op.sweep(j, z.astype(np.float32).astype(np.float64)) for j in range(op.ndir)])
    assert rel(psi.cpu().numpy().reshape(op.ndir, -1), ref) < 2e-5


def test_slab_1d_matches_oracle():
    torch = torch_cuda()
    B = lib()
    spec = spec1d([128, 64, 20], n_polar=16, inflow_g=0.4)
    ss, sa = _params(spec, 16)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    rng = np.random.default_rng(9)
    z = rng.standard_normal(gp.n_dof)
    w = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.apply_op(to_dev(z), w)
    bt = torch.empty_like(w)
    gp.rhs(bt)
    psi = torch.empty(gp.n_directions * gp.n_dof, dtype=torch.float64, device="cuda")
    gp.sweep(to_dev(z), psi, with_bc=True)
    psi_h = psi.cpu().numpy()
    for b, op in enumerate(ops):
        o = gp.offsets
        assert rel(w.cpu().numpy()[o[b]:o[b + 1]], OT.Atilde_apply(op, z[o[b]:o[b + 1]])) < 1e-13
        assert rel(bt.cpu().numpy()[o[b]:o[b + 1]], OT.rhs_btilde(op)) < 1e-13
        pb = psi_h[op.ndir * o[b]:op.ndir * o[b + 1]].reshape(op.ndir, -1)
        for j in range(op.ndir):
            assert rel(pb[j], op.sweep(j, z[o[b]:o[b + 1]] + op.gbc(j))) < 1e-13


def test_results_are_deterministic():
    torch = torch_cuda()
    B = lib()
    spec = spec2d([64, 32], [64, 32], n_polar=4, n_azim=16)
    ss, sa = _params(spec, 17)
    gp = B.Problem(spec, ss, sa)
    z = to_dev(np.random.default_rng(1).standard_normal(gp.n_dof))
    w1 = torch.empty_like(z)
    w2 = torch.empty_like(z)
    gp.apply_op(z, w1)
    gp.apply_op(z, w2)
    assert torch.equal(w1, w2)


def test_full_size_square_64_matches_oracle():
    """The 64x64, 8x16-direction workload at full size: one A~ apply and b~ against the oracle."""
    torch = torch_cuda()
    B = lib()
    spec = wl.config(2)
    ss, sa = wl.draw_params(spec, 1, wl.seed_for(2, 1))
    gp = B.Problem(spec, ss, sa)
    op = oracle_problems(spec, ss, sa)[0]
    z = np.random.default_rng(2).standard_normal(gp.n_dof)
    w = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.apply_op(to_dev(z), w)
    assert rel(w.cpu().numpy(), OT.Atilde_apply(op, z)) < 1e-13
    gp.rhs(w)
    assert rel(w.cpu().numpy(), OT.rhs_btilde(op)) < 1e-13


@pytest.mark.parametrize("mesh,smax", [((38, 46), 1e3), ((64, 64), 1e4), ((12, 70), 30.0)])
def test_apply_op_double_float_matches_oracle(mesh, smax):
    """rte_apply_op in double-float arithmetic (RTE_F64_DF, the refinement residual sweep): element by element
    within 1e-12 of the FP64 oracle, also on strongly scattering draws (sigma_s up to 1e4)."""
    torch = torch_cuda()
    B = lib()
    spec = spec2d([mesh[0]], [mesh[1]], n_polar=4, n_azim=8, sigma_s_range=(1.0, smax))
    ss, sa = _params(spec, 21)
    gp = B.Problem(spec, ss, sa)
    op = oracle_problems(spec, ss, sa)[0]
    z = np.random.default_rng(9).standard_normal(gp.n_dof)
    w = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.apply_op(to_dev(z), w, double_float=True)
    ref = OT.Atilde_apply(op, z)
    got = w.cpu().numpy()
    assert rel(got, ref) < 1e-12
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_residual_double_float_at_a_converged_solution():
    """At a converged scalar flux of a thick problem A~ phi ~ b~ cancels by orders of magnitude: the double-float
    A~ phi must still be within ~1e-13 ||phi|| of the oracle's (the accuracy the 1e-8 refinement residual needs),
    batched over uneven meshes."""
    torch = torch_cuda()
    B = lib()
    from oracle import romsad as ORS
    spec = spec2d([16, 24, 32], [16, 24, 32], n_polar=4, n_azim=8, sigma_s_range=(100.0, 1e3))
    ss, sa = _params(spec, 22)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    phis = [ORS.solve(o, None, restart=120, rtol=1e-11, max_iter=4000)[0] for o in ops]
    z = np.concatenate(phis)
    w = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.apply_op(to_dev(z), w, double_float=True)
    for b, (wb, zb) in enumerate(zip(split(w.cpu().numpy(), gp.offsets), phis)):
        ref = OT.Atilde_apply(ops[b], zb)
        assert np.linalg.norm(ref) < 0.1 * np.linalg.norm(zb)       # the cancellation is real
        assert np.linalg.norm(wb - ref) < 1e-13 * np.linalg.norm(zb), b


@pytest.mark.parametrize("variant,D,run", [(0, 1, 0), (0, 4, 0), (1, 2, 0), (2, 1, 3), (2, 2, 1), (2, 4, 5),
                                           (2, 8, 2), (2, 2, 0)])
def test_every_sweep_kernel_matches_oracle(variant, D, run):
    """Each sweep kernel pinned — one CTA per task with a warp per band (0), a warp per task (1), persistent CTAs
    pipelining runs of tasks through the bands (2, runs of 1 to 5 tasks over meshes of several sizes) — at 1 to 8
    directions per warp: FP32, FP64 and double-float A~ applies over a batch of uneven meshes against the oracle."""
    torch = torch_cuda()
    B = lib()
    spec = spec2d([32, 64, 40, 16, 64, 24], [32, 64, 24, 48, 64, 40], n_polar=4, n_azim=16)
    ss, sa = _params(spec, 25)
    gp = B.Problem(spec, ss, sa)
    gp.set_sweep_variant(variant, D, run)
    ops = oracle_problems(spec, ss, sa)
    z = np.random.default_rng(10).standard_normal(gp.n_dof)
    w64 = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    wdf = torch.empty_like(w64)
    w32 = torch.empty(gp.n_dof, dtype=torch.float32, device="cuda")
    for _ in range(2):   # the second call reuses the tuned state and the runs
        gp.apply_op(to_dev(z), w64)
        gp.apply_op(to_dev(z), wdf, double_float=True)
        gp.apply_op(to_dev(z, torch.float32), w32)
    zr = z.astype(np.float32).astype(np.float64)
    for b, op in enumerate(ops):
        zb, zrb = split(z, gp.offsets)[b], split(zr, gp.offsets)[b]
        ref = OT.Atilde_apply(op, zb)
        assert rel(split(w64.cpu().numpy(), gp.offsets)[b], ref) < 1e-13, b
        assert rel(split(wdf.cpu().numpy(), gp.offsets)[b], ref) < 1e-12, b
        assert rel(split(w32.cpu().numpy().astype(np.float64), gp.offsets)[b], OT.Atilde_apply(op, zrb)) < 2e-5, b


def test_pipelined_sweep_in_a_batched_mixed_solve():
    """The pipelined kernel inside a batched mixed solve whose instances converge at different iterations (each
    CTA drops the tasks of converged instances from its run): phi within 1e-7 of the oracle."""
    torch = torch_cuda()
    B = lib()
    from oracle import romsad as ORS
    spec = spec2d([16, 32, 24, 32], [16, 32, 24, 32], n_polar=4, n_azim=8, sigma_s_range=(1.0, 100.0))
    ss, sa = _params(spec, 26)
    gp = B.Problem(spec, ss, sa)
    gp.set_sweep_variant(2, 2, 3)
    ops = oracle_problems(spec, ss, sa)
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    st = B.fgmres_solve(gp, None, phi, restart=30, rtol=1e-8, max_iter=2000, post_mode=B.RTE_POST_DSA,
                        mode=B.RTE_MODE_MIXED, inner_rtol=1e-3, max_outer=30)
    assert len({s["iterations"] for s in st}) > 1     # the instances stop at different points
    h = phi.cpu().numpy()
    for b, op in enumerate(ops):
        ref, _ = ORS.solve(op, None, post="dsa_vcycle", restart=60, rtol=1e-12, max_iter=2000)
        assert st[b]["status"] == 0
        assert rel(split(h, gp.offsets)[b], ref) < 1e-7, b
