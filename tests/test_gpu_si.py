"""GPU parity of source iteration with synthetic acceleration (SI-ROMSAD, Sec. 3.1-3.2, eq.
preconditioned-richardson) against the oracle: the same number of iterations gives the same iterate
(to FP64 rounding without acceleration, to the FP32 V-cycle's rounding with DSA), and converged solves
match the oracle's tight solution."""
import numpy as np
import pytest

import workloads as wl
from oracle import romsad as ORS

from gpu_common import lib, oracle_problems, rel, spec2d, split, torch_cuda

pytestmark = pytest.mark.gpu


def _si_gpu(B, gp, roms=None, **kw):
    torch = torch_cuda()
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    stats = B.si_solve(gp, roms, phi, **kw)
    return phi.cpu().numpy(), stats


def test_classical_si_iterates_match_the_oracle():
    """No correction: after exactly 12 iterations the GPU iterate is the oracle's (eq. richardson)."""
    B = lib()
    spec = spec2d([16, 24], [16, 12], n_polar=4, n_azim=8, inflow_g=0.1)
    ss, sa = wl.draw_params(spec, 2, 61)
    ss = np.minimum(ss, 10.0)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    phi, stats = _si_gpu(B, gp, None, rtol=1e-30, max_iter=12, post_mode=B.RTE_POST_IDENTITY, raise_on_fail=False)
    for b, op in enumerate(ops):
        ref, st = ORS.si_solve(op, None, post="identity", rtol=1e-30, max_iter=12)
        assert stats[b]["iterations"] == 12 == st.iterations
        assert stats[b]["sweeps"] == st.sweeps
        assert rel(split(phi, gp.offsets)[b], ref) < 1e-12
        assert abs(stats[b]["true_rel_residual"] - st.true_rel_residual) <= 1e-9 * st.true_rel_residual


def test_si_dsa_iterates_and_solution_match_the_oracle():
    """SI-DSA: after 6 iterations the GPU iterate is the oracle's with its own V-cycle (FP32 V-cycle on the
    GPU: 1e-4); converged to 1e-10, phi at 1e-8 of the oracle's tight solution with the iteration count
    within 2 of the oracle's."""
    B = lib()
    spec = spec2d([16, 24], [16, 16], n_polar=4, n_azim=8)
    ss, sa = wl.draw_params(spec, 2, 62)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    phi6, _ = _si_gpu(B, gp, None, rtol=1e-30, max_iter=6, post_mode=B.RTE_POST_DSA, raise_on_fail=False)
    phi, stats = _si_gpu(B, gp, None, rtol=1e-10, max_iter=400, post_mode=B.RTE_POST_DSA)
    for b, op in enumerate(ops):
        ref6, _ = ORS.si_solve(op, None, post="dsa_vcycle", rtol=1e-30, max_iter=6)
        assert rel(split(phi6, gp.offsets)[b], ref6) < 1e-4
        _, st = ORS.si_solve(op, None, post="dsa_vcycle", rtol=1e-10, max_iter=400)
        tight, _ = ORS.solve(op, None, restart=200, rtol=1e-13, max_iter=3000)
        assert stats[b]["status"] == 0 and stats[b]["true_rel_residual"] <= 1e-10
        assert abs(stats[b]["iterations"] - st.iterations) <= 2
        assert rel(split(phi, gp.offsets)[b], tight) < 1e-8


def test_si_romsad_then_dsa_reaches_the_solution():
    """SI-ROMSAD: the ROM correction in the first iteration, DSA afterwards; instance 1 has no ROM and takes
    DSA throughout."""
    B = lib()
    spec = spec2d([16, 16], [16, 16], n_polar=4, n_azim=8)
    ss, sa = wl.draw_params(spec, 2, 63)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    op0 = ops[0]
    Q, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((op0.ndir * op0.ndof, 8)))
    U = Q.T.reshape(8, op0.ndir, op0.ndof).copy()
    rom = B.Rom.from_basis(gp, U, instance=0)
    phi, stats = _si_gpu(B, gp, [rom, None], rtol=1e-10, max_iter=400, window=1, post_mode=B.RTE_POST_DSA)
    orom = ORS.build_rom(op0, U)
    _, st0 = ORS.si_solve(op0, orom, window=1, post="dsa_vcycle", rtol=1e-10, max_iter=400)
    assert abs(stats[0]["iterations"] - st0.iterations) <= 2
    for b, op in enumerate(ops):
        tight, _ = ORS.solve(op, None, restart=200, rtol=1e-13, max_iter=3000)
        assert stats[b]["status"] == 0
        assert rel(split(phi, gp.offsets)[b], tight) < 1e-8


def test_si_rejects_reduced_precision():
    B = lib()
    torch = torch_cuda()
    spec = spec2d([8], [8])
    ss, sa = wl.draw_params(spec, 1, 64)
    gp = B.Problem(spec, ss, sa)
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    o = B.FgmresOpts(1, 1e-8, 10, 2, B.RTE_POST_DSA, B.RTE_MODE_MIXED, 0.0, 0, 0, 0, 0, 0)
    st = (B.FgmresStats * 1)()
    import ctypes
    assert B.load().si_solve(gp.h, None, ctypes.byref(o), None, B._ptr(phi), st, None) == 7
