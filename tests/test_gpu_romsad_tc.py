"""ROMSAD products on the tensor cores (BF16 operands, FP32 accumulation): romsad_apply with FP32 vectors against
the oracle's ROMSAD apply (eq. rom-sa-preconditioner), and the mixed-precision solve that uses them in its ROM
window against the oracle's solution."""
import numpy as np
import pytest

import workloads as wl
from oracle import romsad as ORS

from gpu_common import lib, oracle_problems, rel, spec2d, split, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _rom(B, gp, op, r, seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((op.ndir * op.ndof, r)))
    U = Q.T.reshape(r, op.ndir, op.ndof).copy()
    return B.Rom.from_basis(gp, U, instance=0), ORS.build_rom(op, U)


# BF16 rounding (2^-9 relative per operand) of both factors of both products, FP32 accumulation: the ROM
# correction z - v is good to about 1e-2 of its size (the reduced solve amplifies by cond(U^T A U))
TC_TOL = 3e-2


@pytest.mark.parametrize("n_inst,r", [(3, 12), (70, 40)])
def test_romsad_apply_tensor_cores_matches_oracle(n_inst, r):
    """FP32 vectors: projection and lift as BF16 mma.sync products over the instances (two instance groups at
    70 instances, padded ranks at r = 12 and 40); the correction z - v against the oracle's, per instance."""
    torch = torch_cuda()
    B = lib()
    spec = spec2d([24] * n_inst, [20] * n_inst, n_polar=2, n_azim=8)
    ss, sa = wl.draw_params(spec, n_inst, 71)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec.with_instances([24], [20]), ss[:1], sa[:1])
    rom_g, rom_o = _rom(B, B.Problem(spec.with_instances([24], [20]), ss[:1], sa[:1]), ops[0], r, 5)
    v = np.random.default_rng(6).standard_normal(gp.n_dof).astype(np.float32)
    z = torch.empty(gp.n_dof, dtype=torch.float32, device="cuda")
    z2 = torch.empty_like(z)
    rom_g.apply(gp, to_dev(v), z)
    rom_g.apply(gp, to_dev(v), z2)
    assert torch.equal(z, z2)                      # fixed-order chunk sums: deterministic
    h = split(z.cpu().numpy().astype(np.float64), gp.offsets)
    vs = split(v.astype(np.float64), gp.offsets)
    from oracle.discretization import with_params
    for b in (0, n_inst // 2, n_inst - 1):
        q = with_params(ops[0], ss[b], sa[b])
        ref = ORS.romsad_apply(rom_o, q, vs[b])
        assert rel(h[b] - vs[b], ref - vs[b]) < TC_TOL, b


def test_mixed_solve_with_tensor_core_rom_matches_oracle():
    """Mixed FGMRES-ROMSAD then DSA with the ROM window on the tensor cores: FP64 true residual 1e-8, phi within
    1e-7 of the oracle's tight solution, and no more than two iterations above the FP32 CUDA-core products."""
    torch = torch_cuda()
    B = lib()
    spec = spec2d([32, 32, 32], [32, 32, 32], n_polar=4, n_azim=8, sigma_s_range=(1.0, 300.0))
    ss, sa = wl.draw_params(spec, 3, 72)
    tr_ss, tr_sa = wl.draw_params(spec, 12, 73)
    tmpl = B.Problem(spec.with_instances([32], [32]), tr_ss[:1], tr_sa[:1])
    rom, _ = B.Rom.greedy(tmpl, tr_ss, tr_sa, window=2, max_greedy_iter=6, max_rank=12, eps_rom=0.0, hf_rtol=1e-10,
                          hf_restart=40, hf_max_iter=2000, hf_dsa=True)
    gp = B.Problem(spec, ss, sa)
    ops = oracle_problems(spec, ss, sa)
    kw = dict(restart=40, rtol=1e-8, max_iter=2000, window=2, post_mode=B.RTE_POST_DSA, mode=B.RTE_MODE_MIXED,
              inner_rtol=1e-3, max_outer=30)
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    st_tc = B.fgmres_solve(gp, [rom] * 3, phi, rom_bf16=True, **kw)
    h = split(phi.cpu().numpy(), gp.offsets)
    st_fp = B.fgmres_solve(gp, [rom] * 3, torch.zeros_like(phi), rom_bf16=False, **kw)
    for b, op in enumerate(ops):
        ref, _ = ORS.solve(op, None, post="dsa_vcycle", restart=60, rtol=1e-12, max_iter=2000)
        assert st_tc[b]["status"] == 0 and st_tc[b]["true_rel_residual"] <= 1e-8
        assert rel(h[b], ref) < 1e-7
        assert st_tc[b]["iterations"] <= st_fp[b]["iterations"] + 2, (st_tc[b], st_fp[b])
