"""GPU parity of the DSA preconditioner (appendix A; one multigrid V-cycle per apply) and of FGMRES
with DSA after the ROMSAD window (eq. ROMSAD-preconditioner) against the oracle.

The V-cycle runs in FP32 (set-up included): its output is compared with the oracle's FP64 V-cycle at 5e-5
relative (FP32 rounding of the set-up and of a few dozen dependent stencil stages; an index or sign
slip gives O(1)).  Solves are compared on phi against the oracle's tight solution."""
import numpy as np
import pytest

import workloads as wl
from oracle import dsa as ODSA, romsad as ORS, transport as OT
from oracle.krylov import fgmres as ofgmres

from gpu_common import lib, oracle_problems, rel, spec1d, spec2d, split, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _solve_gpu(B, gp, roms=None, **kw):
    torch = torch_cuda()
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    stats = B.fgmres_solve(gp, roms, phi, **kw)
    return phi.cpu().numpy(), stats


@pytest.mark.parametrize("variant", ["partial", "lumped"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_dsa_apply_matches_the_oracle_vcycle(variant, dtype):
    B = lib()
    torch = torch_cuda()
    spec = spec2d([16, 32, 8], [16, 16, 12], n_polar=4, n_azim=8)
    ss, sa = wl.draw_params(spec, 3, 51)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    v = np.random.default_rng(5).standard_normal(gp.n_dof)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    vd = to_dev(v, tdt)
    z = torch.empty_like(vd)
    code = B.RTE_DSA_PARTIAL if variant == "partial" else B.RTE_DSA_LUMPED
    gp.dsa_apply(vd, z, variant=code)
    torch.cuda.synchronize()
    zg = z.double().cpu().numpy()
    vv = vd.double().cpu().numpy()
    for b, op in enumerate(ops):
        vb = split(vv, gp.offsets)[b]
        ref = ODSA.MultigridDsa(op, variant).apply(vb)
        assert rel(split(zg, gp.offsets)[b] - vb, ref - vb) < 5e-5


def test_dsa_rejects_meshes_it_does_not_cover():
    B = lib()
    torch = torch_cuda()
    spec = spec2d([44], [44])      # 44 -> 22 -> 11: 12 x 12 coarsest vertices
    ss, sa = wl.draw_params(spec, 1, 52)
    gp = B.Problem(spec, ss, sa)
    v = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(B.RteError) as e:
        gp.dsa_apply(v, torch.empty_like(v))
    assert e.value.status == 7
    with pytest.raises(B.RteError) as e:
        _solve_gpu(B, gp, None, restart=10, rtol=1e-8, max_iter=10, post_mode=B.RTE_POST_DSA)
    assert e.value.status == 7
    # the fully consistent variant is solved exactly in the slab only
    gp2 = B.Problem(spec2d([16], [16]), ss, sa)
    v2 = torch.zeros(gp2.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(B.RteError) as e:
        gp2.dsa_apply(v2, torch.empty_like(v2), variant=B.RTE_DSA_FULL)
    assert e.value.status == 7


@pytest.mark.parametrize("variant", ["full", "partial", "lumped"])
def test_dsa_1d_exact_solve_matches_the_oracle(variant):
    """1D slab (appendix A's geometry): the exact block-tridiagonal DSA solve of each variant equals the oracle's
    sparse direct solve of the same system (1e-11: both are direct solves of a system whose condition grows with
    the cells' optical thickness), on uneven meshes in one call, FP64 and FP32 vectors."""
    torch = torch_cuda()
    B = lib()
    from oracle import dsa as ODSA
    spec = spec1d([128, 40, 64], n_polar=16)
    ss, sa = wl.draw_params(spec, 3, 53)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    code = {"full": B.RTE_DSA_FULL, "partial": B.RTE_DSA_PARTIAL, "lumped": B.RTE_DSA_LUMPED}[variant]
    v = np.random.default_rng(54).standard_normal(gp.n_dof)
    z = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.dsa_apply(to_dev(v), z, variant=code)
    z32 = torch.empty(gp.n_dof, dtype=torch.float32, device="cuda")
    gp.dsa_apply(to_dev(v, torch.float32), z32, variant=code)
    h, h32 = z.cpu().numpy(), z32.cpu().numpy().astype(np.float64)
    for b, op in enumerate(ops):
        vb = split(v, gp.offsets)[b]
        ref = ODSA.Dsa(op, variant).apply(vb)
        assert rel(split(h, gp.offsets)[b], ref) < 1e-11, b
        ref32 = ODSA.Dsa(op, variant).apply(vb.astype(np.float32).astype(np.float64))
        assert rel(split(h32, gp.offsets)[b], ref32) < 1e-6, b


def test_gmres_dsa_1d_fully_consistent_matches_the_oracle():
    """FGMRES with the fully consistent DSA (exact) on the 1D slab workload: phi within 1e-10 of the oracle's
    solution and the same iteration count within 1; fewer iterations than with the partially consistent form."""
    torch = torch_cuda()
    B = lib()
    from oracle import romsad as ORS
    spec = wl.config(1).with_instances([128, 128], [1, 1])
    ss, sa = wl.draw_params(spec, 2, 55)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    its = {}
    for variant, code, post in (("full", B.RTE_DSA_FULL, "dsa"), ("partial", B.RTE_DSA_PARTIAL, "dsa_pc")):
        phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
        st = B.fgmres_solve(gp, None, phi, restart=30, rtol=1e-12, max_iter=500, post_mode=B.RTE_POST_DSA,
                            dsa_variant=code)
        h = phi.cpu().numpy()
        its[variant] = [x["iterations"] for x in st]
        for b, op in enumerate(ops):
            ref, ost = ORS.solve(op, None, post=post, restart=30, rtol=1e-12, max_iter=500)
            assert st[b]["status"] == 0
            assert rel(split(h, gp.offsets)[b], ref) < 1e-10, (variant, b)
            assert abs(st[b]["iterations"] - ost.iterations) <= 1, (variant, b, st[b]["iterations"], ost.iterations)
    assert sum(its["full"]) <= sum(its["partial"])


@pytest.mark.parametrize("variant", ["partial", "lumped"])
def test_gmres_dsa_fp64_matches_the_oracle(variant):
    """Right-preconditioned GMRES-DSA (no ROM, DSA from the first iteration): phi at 1e-10 of the
    oracle's tight solution, iteration count within 2 of the oracle running the FP64 V-cycle."""
    B = lib()
    spec = spec2d([16, 24], [16, 16], n_polar=4, n_azim=8, inflow_g=0.2)
    ss, sa = wl.draw_params(spec, 2, 53)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    code = B.RTE_DSA_PARTIAL if variant == "partial" else B.RTE_DSA_LUMPED
    phi, stats = _solve_gpu(B, gp, None, restart=40, rtol=1e-12, max_iter=600, post_mode=B.RTE_POST_DSA,
                            dsa_variant=code)
    phi10, stats10 = _solve_gpu(B, gp, None, restart=40, rtol=1e-10, max_iter=600, post_mode=B.RTE_POST_DSA,
                                dsa_variant=code)
    for b, op in enumerate(ops):
        ref, _ = ORS.solve(op, None, restart=200, rtol=1e-13, max_iter=3000)
        assert stats[b]["status"] == 0
        assert rel(split(phi, gp.offsets)[b], ref) < 1e-10
        mg = ODSA.MultigridDsa(op, variant)
        _, st = ofgmres(lambda z: OT.Atilde_apply(op, z), OT.rhs_btilde(op), lambda j, v: mg.apply(v),
                        restart=40, rtol=1e-10, max_iter=600)
        assert abs(stats10[b]["iterations"] - st.iterations) <= 2
        _, st_plain = ORS.solve(op, None, restart=40, rtol=1e-10, max_iter=3000)
        assert st.iterations * 2 < st_plain.iterations


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_romsad_then_dsa_matches_the_oracle(mode):
    """ROMSAD for the first two iterations, DSA afterwards; instance 1 has no ROM and takes DSA from the
    first iteration.  FP64: phi at 1e-9 of the oracle; mixed: FP64 true residual <= 1e-8 and phi at 1e-7."""
    B = lib()
    spec = spec2d([16, 16], [16, 16], n_polar=4, n_azim=8)
    ss, sa = wl.draw_params(spec, 2, 54)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    op0 = ops[0]
    Q, _ = np.linalg.qr(np.random.default_rng(6).standard_normal((op0.ndir * op0.ndof, 8)))
    U = Q.T.reshape(8, op0.ndir, op0.ndof).copy()
    rom = B.Rom.from_basis(gp, U, instance=0)
    md = B.RTE_MODE_FP64 if mode == "fp64" else B.RTE_MODE_MIXED
    phi, stats = _solve_gpu(B, gp, [rom, None], restart=40, rtol=1e-10 if mode == "fp64" else 1e-8,
                            max_iter=800, window=2, post_mode=B.RTE_POST_DSA, mode=md, inner_rtol=1e-2,
                            max_outer=30)
    orom = ORS.build_rom(op0, U)
    for b, op in enumerate(ops):
        ref, _ = ORS.solve(op, None, restart=200, rtol=1e-13, max_iter=3000)
        assert stats[b]["status"] == 0
        if mode == "fp64":
            assert rel(split(phi, gp.offsets)[b], ref) < 1e-9
        else:
            assert stats[b]["true_rel_residual"] <= 1e-8
            assert rel(split(phi, gp.offsets)[b], ref) < 1e-7
    if mode == "fp64":
        # same preconditioner sequence in the oracle for the instance with a ROM
        _, st = ORS.solve(op0, orom, window=2, post="dsa_pc", restart=40, rtol=1e-10, max_iter=800)
        mg = ODSA.MultigridDsa(op0, "partial")
        A_r = ORS.reduced_operator(orom, op0.sigma_s_region, op0.sigma_a_region)
        pre = lambda j, v: ORS.romsad_apply(orom, op0, v, A_r) if j <= 2 else mg.apply(v)
        _, st_mg = ofgmres(lambda z: OT.Atilde_apply(op0, z), OT.rhs_btilde(op0), pre, restart=40, rtol=1e-10,
                           max_iter=800)
        assert abs(stats[0]["iterations"] - st_mg.iterations) <= 2


def test_dsa_on_the_multi_phase_arnoldi_path():
    """A 128 x 128 instance has too many vector chunks for the fused Arnoldi step, so the preconditioner
    is applied at the start of every iteration (k_arnoldi_wide path).  Mixed GMRES-DSA reaches the FP64
    true residual 1e-8, recomputed by the oracle."""
    B = lib()
    spec = spec2d([128], [128], n_polar=2, n_azim=8)
    ss, sa = wl.draw_params(spec, 1, 55)
    gp = B.Problem(spec, ss, sa)
    op = oracle_problems(spec, ss, sa)[0]
    phi, stats = _solve_gpu(B, gp, None, restart=30, rtol=1e-8, max_iter=600, post_mode=B.RTE_POST_DSA,
                            mode=B.RTE_MODE_MIXED, inner_rtol=1e-2, max_outer=30)
    assert stats[0]["status"] == 0
    bt = OT.rhs_btilde(op)
    assert np.linalg.norm(bt - OT.Atilde_apply(op, phi)) / np.linalg.norm(bt) <= 1.5e-8
    assert stats[0]["iterations"] < 200


def test_dsa_on_the_64x64_workload():
    """The 64 x 64 workload (128 directions, 2 x 2 regions): mixed FGMRES with DSA reaches the FP64 true
    residual 1e-8 (recomputed by the oracle) in a small fraction of the iterations without it."""
    B = lib()
    spec = wl.config(2)
    ss, sa = wl.draw_params(spec, 1, 2001)
    gp = B.Problem(spec, ss, sa)
    op = oracle_problems(spec, ss, sa)[0]
    phi, stats = _solve_gpu(B, gp, None, restart=30, rtol=1e-8, max_iter=3000, post_mode=B.RTE_POST_DSA,
                            mode=B.RTE_MODE_MIXED, inner_rtol=1e-2, max_outer=30)
    assert stats[0]["status"] == 0
    bt = OT.rhs_btilde(op)
    assert np.linalg.norm(bt - OT.Atilde_apply(op, phi)) / np.linalg.norm(bt) <= 1.5e-8
    assert stats[0]["iterations"] < 100
