"""GPU parity of FGMRES (Alg. 1) and the ROMSAD preconditioner (Sec. 4) against the oracle."""
import os
import tempfile

import numpy as np
import pytest

import workloads as wl
from oracle import romsad as ORS, transport as OT
from oracle.discretization import with_params

from gpu_common import lib, oracle_problems, rel, spec1d, spec2d, split, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _solve_gpu(B, gp, roms=None, **kw):
    torch = torch_cuda()
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    stats = B.fgmres_solve(gp, roms, phi, **kw)
    return phi.cpu().numpy(), stats


def test_fgmres_fp64_no_preconditioner_matches_oracle():
    B = lib()
    spec = spec2d([16, 24], [16, 20], n_polar=4, n_azim=8, inflow_g=0.2)
    ss, sa = wl.draw_params(spec, 2, 21)
    ss = np.minimum(ss, 30.0)   # keep plain GMRES iteration counts small
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    phi, stats = _solve_gpu(B, gp, None, restart=40, rtol=1e-12, max_iter=400)
    for b, op in enumerate(ops):
        ref, st = ORS.solve(op, None, restart=40, rtol=1e-12, max_iter=400)
        assert rel(split(phi, gp.offsets)[b], ref) < 1e-10
        assert stats[b]["status"] == 0
        assert stats[b]["true_rel_residual"] < 2e-12
    # iteration counts at rtol 1e-10 agree with the oracle running the same algorithm (+-1)
    phi, stats = _solve_gpu(B, gp, None, restart=40, rtol=1e-10, max_iter=400)
    for b, op in enumerate(ops):
        _, st = ORS.solve(op, None, restart=40, rtol=1e-10, max_iter=400)
        assert abs(stats[b]["iterations"] - st.iterations) <= 1
        assert stats[b]["sweeps"] == 1 + stats[b]["iterations"] + stats[b]["restarts"]


def test_fgmres_with_restarts_matches_dense_solution():
    B = lib()
    spec = spec2d([8], [8], n_polar=2, n_azim=4, inflow_g=0.1)
    ss, sa = wl.draw_params(spec, 1, 22)
    ss = np.minimum(ss, 100.0)   # bounded condition number: rtol 1e-13 then pins phi to ~1e-11
    gp = B.Problem(spec, ss, sa)
    op = oracle_problems(spec, ss, sa)[0]
    A, b = OT.dense_coupled_system(op)
    ref = OT.scalar_flux(op, np.linalg.solve(A, b).reshape(op.ndir, op.ndof))
    phi, stats = _solve_gpu(B, gp, None, restart=5, rtol=1e-13, max_iter=3000)
    assert stats[0]["restarts"] > 0
    assert rel(phi, ref) < 1e-10


def _oracle_rom_1d():
    spec = wl.config(1)
    ss, sa = wl.draw_params(spec, spec.n_train, wl.seed_for(1, 0))
    from oracle import Problem
    p0 = Problem(spec, 0, ss[0], sa[0])
    rom, rep = ORS.greedy(p0, ss, sa, window=2, max_greedy_iter=5, max_rank=10, eps_rom=1e-12,
                          hf_rtol=1e-12, restart=60)
    return spec, p0, rom, rep


def test_romsad_apply_and_reduced_operator_match_oracle():
    torch = torch_cuda()
    B = lib()
    spec, p0, rom, rep = _oracle_rom_1d()
    ts, ta = wl.draw_params(spec, 3, wl.seed_for(1, 1))
    spec3 = spec.with_instances([128] * 3, [1] * 3)
    gp = B.Problem(spec3, ts, ta)
    grom = B.Rom.from_basis(gp, rom.U, instance=0)
    assert grom.rank == rom.r
    for b in range(3):
        A_gpu = grom.reduced_operator(ts[b], ta[b])
        A_ref = ORS.reduced_operator(rom, ts[b], ta[b])
        assert np.max(np.abs(A_gpu - A_ref)) < 1e-10 * np.max(np.abs(A_ref))
    v = np.random.default_rng(3).standard_normal(gp.n_dof)
    z = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    grom.apply(gp, to_dev(v), z)
    zh = split(z.cpu().numpy(), gp.offsets)
    for b in range(3):
        q = with_params(p0, ts[b], ta[b])
        assert rel(zh[b], ORS.romsad_apply(rom, q, split(v, gp.offsets)[b])) < 1e-11
    # checkpoint round trip
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "rom.bin")
        grom.save(path)
        grom2 = B.Rom.load_file(path)
        z2 = torch.empty_like(z)
        grom2.apply(gp, to_dev(v), z2)
        assert torch.equal(z, z2)


def test_rank64_rom_apply_and_solves():
    """A ROM of the largest supported rank (64) from a random orthonormal basis: reduced operator and
    ROMSAD apply against the oracle, and FP64 and mixed FGMRES-ROMSAD solves that use it (the ROM
    coefficients then span two warps' lanes and the factorisation needs 64 KiB of shared memory)."""
    torch = torch_cuda()
    B = lib()
    from oracle import Problem
    spec = wl.config(1)
    ts, ta = wl.draw_params(spec, 2, wl.seed_for(1, 1))
    p0 = Problem(spec, 0, ts[0], ta[0])
    Q, _ = np.linalg.qr(np.random.default_rng(64).standard_normal((p0.ndir * p0.ndof, 64)))
    U = Q.T.reshape(64, p0.ndir, p0.ndof).copy()
    orom = ORS.build_rom(p0, U)
    spec2 = spec.with_instances([128] * 2, [1] * 2)
    gp = B.Problem(spec2, ts, ta)
    grom = B.Rom.from_basis(gp, U, instance=0)
    assert grom.rank == 64
    for b in range(2):
        A_gpu = grom.reduced_operator(ts[b], ta[b])
        A_ref = ORS.reduced_operator(orom, ts[b], ta[b])
        assert np.max(np.abs(A_gpu - A_ref)) < 1e-10 * np.max(np.abs(A_ref))
    v = np.random.default_rng(5).standard_normal(gp.n_dof)
    z = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    grom.apply(gp, to_dev(v), z)
    zh = split(z.cpu().numpy(), gp.offsets)
    for b in range(2):
        q = with_params(p0, ts[b], ta[b])
        assert rel(zh[b], ORS.romsad_apply(orom, q, split(v, gp.offsets)[b])) < 1e-11
    ops = oracle_problems(spec2, ts, ta)
    refs = [ORS.solve(op, None, restart=200, rtol=1e-13, max_iter=3000)[0] for op in ops]
    for mode, tol in ((B.RTE_MODE_FP64, 1e-9), (B.RTE_MODE_MIXED, 1e-7), (B.RTE_MODE_MIXED_F64KRYLOV, 1e-7)):
        phi, st = _solve_gpu(B, gp, [grom, grom], restart=40, rtol=1e-10, max_iter=2000, mode=mode,
                             inner_rtol=1e-2, max_outer=30)
        for b in range(2):
            assert st[b]["status"] == 0
            assert rel(split(phi, gp.offsets)[b], refs[b]) < tol


def test_fgmres_romsad_fp64_slab_matches_oracle():
    """FP64 FGMRES-ROMSAD on the 1D slab workload (128 cells, S16, rank <= 10 ROM from 20 training
    parameters): phi within 1e-10 of the oracle, iteration counts within 1."""
    B = lib()
    spec, p0, rom, rep = _oracle_rom_1d()
    ts, ta = wl.draw_params(spec, 4, wl.seed_for(1, 1))
    spec4 = spec.with_instances([128] * 4, [1] * 4)
    gp = B.Problem(spec4, ts, ta)
    grom = B.Rom.from_basis(gp, rom.U, instance=0)
    phi, stats = _solve_gpu(B, gp, [grom] * 4, restart=30, rtol=1e-12, max_iter=500, window=2)
    phi_b = split(phi, gp.offsets)
    for b in range(4):
        q = with_params(p0, ts[b], ta[b])
        ref, st = ORS.solve(q, rom, window=2, restart=30, rtol=1e-12)
        assert rel(phi_b[b], ref) < 1e-10
    phi, stats = _solve_gpu(B, gp, [grom] * 4, restart=30, rtol=1e-10, max_iter=500, window=2)
    for b in range(4):
        q = with_params(p0, ts[b], ta[b])
        _, st = ORS.solve(q, rom, window=2, restart=30, rtol=1e-10)
        assert abs(stats[b]["iterations"] - st.iterations) <= 1, (stats[b], st.iterations)
        # the ROM must help: fewer iterations than without it
    _, st0 = _solve_gpu(B, gp, None, restart=30, rtol=1e-10, max_iter=500)
    assert sum(s["iterations"] for s in stats) < sum(s["iterations"] for s in st0)


@pytest.mark.parametrize("mode,residual", [("mixed", "df"), ("mixed", "fp64"), ("mixed_f64krylov", "df")])
def test_mixed_precision_meets_fp64_accuracy(mode, residual):
    """Mixed modes (inner solves all FP32, or FP32 sweeps with FP64 Krylov vectors, MGS and Givens), refinement
    residuals in double-float (certified by a final FP64 residual) or all in FP64: FP64 true residual <= 1e-8
    and phi within 1e-7 of the FP64 oracle, element by element."""
    B = lib()
    spec = spec2d([32, 16], [32, 16], n_polar=4, n_azim=8)
    ss, sa = wl.draw_params(spec, 2, 23)
    ss = np.minimum(ss, 50.0)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    md = B.RTE_MODE_MIXED if mode == "mixed" else B.RTE_MODE_MIXED_F64KRYLOV
    rr = B.RTE_RESIDUAL_DF if residual == "df" else B.RTE_RESIDUAL_FP64
    phi, stats = _solve_gpu(B, gp, None, restart=60, rtol=1e-8, max_iter=2000, mode=md,
                            inner_rtol=1e-4, max_outer=20, refine_residual=rr)
    for b, op in enumerate(ops):
        ref, _ = ORS.solve(op, None, restart=200, rtol=1e-13, max_iter=3000)
        st = stats[b]
        assert st["status"] == 0
        assert st["true_rel_residual"] <= 1e-8
        assert st["outer"] >= 1 and st["sweeps_fp64"] >= 2
        # b~, one residual per refinement step, at most one FP64 re-check of a double-float residual
        assert 1 + st["outer"] <= st["sweeps_fp64"] + st["sweeps_df"] <= 2 + st["outer"]
        if residual == "fp64":
            assert st["sweeps_df"] == 0
        else:
            assert st["sweeps_fp64"] <= 3
        got = split(phi, gp.offsets)[b]
        assert rel(got, ref) < 1e-7
        assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_nan_in_initial_guess_is_reported_as_numeric(mode):
    """A NaN injected from the host into the initial guess reaches the first residual: fgmres_solve returns
    RTE_ERR_NUMERIC (status of that instance too) instead of iterating on it; the other instance converges."""
    torch = torch_cuda()
    B = lib()
    spec = spec2d([16, 16], [16, 16], n_polar=4, n_azim=8)
    ss, sa = wl.draw_params(spec, 2, 41)
    ss = np.minimum(ss, 20.0)
    gp = B.Problem(spec, ss, sa)
    phi0 = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    phi0[gp.offsets[1] + 7] = float("nan")
    phi = torch.zeros_like(phi0)
    md = B.RTE_MODE_FP64 if mode == "fp64" else B.RTE_MODE_MIXED
    with pytest.raises(B.RteError) as ei:
        B.fgmres_solve(gp, None, phi, phi0=phi0, restart=30, rtol=1e-8, max_iter=500, mode=md, inner_rtol=1e-3)
    assert ei.value.status == 5   # RTE_ERR_NUMERIC
    stats = B.fgmres_solve(gp, None, phi, phi0=phi0, restart=30, rtol=1e-8, max_iter=500, mode=md, inner_rtol=1e-3,
                           raise_on_fail=False)
    assert stats[1]["status"] == 5
    assert stats[0]["status"] == 0 and stats[0]["true_rel_residual"] <= 1e-8


def test_mixed_inner_restarts_keep_their_right_hand_side():
    """Mixed mode with a short restart: every inner solve restarts several times; the inner
    right-hand side (the FP64 outer residual) must survive those restarts, so the refinement
    converges without falling back to FP64 and matches the FP64 oracle."""
    B = lib()
    spec = spec2d([24, 40], [24, 40], n_polar=4, n_azim=8)
    ss, sa = wl.draw_params(spec, 2, 31)
    ss = np.minimum(ss, 30.0)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    phi, stats = _solve_gpu(B, gp, None, restart=4, rtol=1e-8, max_iter=3000, mode=B.RTE_MODE_MIXED,
                            inner_rtol=1e-2, max_outer=30)
    for b, op in enumerate(ops):
        ref, _ = ORS.solve(op, None, restart=200, rtol=1e-13, max_iter=3000)
        assert stats[b]["status"] == 0
        assert stats[b]["escalated"] == 0
        assert stats[b]["restarts"] >= stats[b]["outer"] >= 2
        assert stats[b]["true_rel_residual"] <= 1e-8
        assert rel(split(phi, gp.offsets)[b], ref) < 1e-7


def test_mixed_escalates_to_fp64_after_max_outer():
    """max_outer = 1: one FP32 refinement step, then FP64 FGMRES from the refined iterate
    finishes the solve to the FP64 target."""
    B = lib()
    spec = spec2d([16, 24], [16, 24], n_polar=4, n_azim=8)
    ss, sa = wl.draw_params(spec, 2, 37)
    ss = np.minimum(ss, 100.0)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    phi, stats = _solve_gpu(B, gp, None, restart=40, rtol=1e-11, max_iter=3000, mode=B.RTE_MODE_MIXED,
                            inner_rtol=1e-2, max_outer=1)
    for b, op in enumerate(ops):
        ref, _ = ORS.solve(op, None, restart=200, rtol=1e-13, max_iter=3000)
        assert stats[b]["status"] == 0
        assert stats[b]["escalated"] == 1 and stats[b]["outer"] == 1
        assert stats[b]["true_rel_residual"] <= 2e-11
        assert rel(split(phi, gp.offsets)[b], ref) < 1e-8


def test_large_instance_multiphase_arnoldi_matches_oracle():
    """A 132x132 instance has 272 chunks of 256 dofs, more than the 64 per instance for which the
    fused two-barrier Arnoldi step repeats the per-instance sums in every block, so the solve runs
    the multi-phase step (k_arnoldi_wide).  FP64 and mixed solves both match the oracle."""
    B = lib()
    spec = spec2d([132], [132], n_polar=2, n_azim=8)
    ss, sa = wl.draw_params(spec, 1, 41)
    ss = np.minimum(ss, 20.0)
    gp = B.Problem(spec, ss, sa)
    op = oracle_problems(spec, ss, sa)[0]
    ref, _ = ORS.solve(op, None, restart=200, rtol=1e-13, max_iter=3000)
    phi, st = _solve_gpu(B, gp, None, restart=40, rtol=1e-11, max_iter=2000)
    assert st[0]["status"] == 0
    assert rel(phi, ref) < 1e-9
    phi, st = _solve_gpu(B, gp, None, restart=40, rtol=1e-9, max_iter=2000, mode=B.RTE_MODE_MIXED,
                         inner_rtol=1e-2, max_outer=30)
    assert st[0]["status"] == 0 and st[0]["true_rel_residual"] <= 1e-9
    assert rel(phi, ref) < 1e-7


def test_host_output_pointer_and_not_converged_status():
    torch = torch_cuda()
    B = lib()
    spec = spec2d([16], [16], n_polar=2, n_azim=8)
    ss, sa = wl.draw_params(spec, 1, 24)
    gp = B.Problem(spec, ss, sa)
    host = np.zeros(gp.n_dof)
    stats = B.fgmres_solve(gp, None, host, restart=30, rtol=1e-10, max_iter=500)
    dev = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    B.fgmres_solve(gp, None, dev, restart=30, rtol=1e-10, max_iter=500)
    assert np.array_equal(host, dev.cpu().numpy())
    stats = B.fgmres_solve(gp, None, dev, restart=30, rtol=1e-10, max_iter=2, raise_on_fail=False)
    assert stats[0]["status"] == B.RTE_ERR_NOT_CONVERGED
    assert stats[0]["iterations"] == 2


def test_invalid_arguments_are_rejected():
    B = lib()
    spec = spec2d([16], [16], n_polar=2, n_azim=8)
    ss, sa = wl.draw_params(spec, 1, 25)
    gp = B.Problem(spec, ss, sa)
    with pytest.raises(B.RteError):
        gp.set_params(ss * np.nan, sa)
    with pytest.raises(B.RteError):
        B.Problem(spec2d([15], [16], n_polar=2, n_azim=8), ss, sa)   # region grid does not divide
    with pytest.raises(B.RteError):
        B.Problem(spec2d([16], [16], n_polar=2, n_azim=7), ss, sa)   # odd number of azimuths
