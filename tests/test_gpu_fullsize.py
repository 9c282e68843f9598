"""GPU parity at the full batched size (256 instances: 96 x 32^2, 96 x 64^2, 64 x 128^2, 128 directions) in the
launch configurations the benchmark times: sampled instances and directions against the oracle, and the
oracle's own residual of the batched mixed-precision solve."""
import numpy as np
import pytest

import workloads as wl
from oracle import transport as OT

from gpu_common import lib, oracle_problems, rel, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

SAMPLES = (0, 100, 200)        # one instance of each mesh size
DIRS = (0, 1, 37, 127)


def _batch(B):
    spec = wl.config(3)
    ss, sa = wl.draw_params(spec, spec.n_instances, wl.seed_for(3, 1))
    return spec, ss, sa, B.Problem(spec, ss, sa)


def _oracle(spec, ss, sa, b):
    sub = spec.with_instances([spec.nx[b]], [spec.ny[b]])
    return oracle_problems(sub, ss[b:b + 1], sa[b:b + 1])[0]


def test_batch256_angular_sweep_fp32_sampled():
    """The angular-output sweep of the HBM measurement (FP32, boundary inflow on): sampled (instance,
    direction) blocks against the oracle's sweep of the FP32-rounded source."""
    torch = torch_cuda()
    B = lib()
    spec, ss, sa, gp = _batch(B)
    off = [int(x) for x in gp.offsets]
    ndir = gp.n_directions
    s = np.random.default_rng(31).standard_normal(gp.n_dof).astype(np.float32)
    psi = torch.empty(ndir * gp.n_dof, dtype=torch.float32, device="cuda")
    for _ in range(2):          # the first call also runs the autotuner
        gp.sweep(to_dev(s), psi, with_bc=True)
    torch.cuda.synchronize()
    for b in SAMPLES:
        op = _oracle(spec, ss, sa, b)
        n = off[b + 1] - off[b]
        sb = s[off[b]:off[b + 1]].astype(np.float64)
        blk = psi[ndir * off[b]:ndir * off[b + 1]].view(ndir, n)
        for j in DIRS:
            ref = op.sweep(j, sb + op.gbc(j))
            assert rel(blk[j].cpu().numpy(), ref) < 2e-5, (b, j)


def test_batch256_operator_apply_sampled():
    """A~ z over the whole batch in FP32 (the inner solves' operator) and FP64 (the residuals)."""
    torch = torch_cuda()
    B = lib()
    spec, ss, sa, gp = _batch(B)
    off = [int(x) for x in gp.offsets]
    z = np.random.default_rng(32).standard_normal(gp.n_dof)
    w32 = torch.empty(gp.n_dof, dtype=torch.float32, device="cuda")
    w64 = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    z32 = to_dev(z, torch.float32)
    z64 = to_dev(z)
    for _ in range(2):
        gp.apply_op(z32, w32)
        gp.apply_op(z64, w64)
    h32 = w32.cpu().numpy()
    h64 = w64.cpu().numpy()
    z_r = z.astype(np.float32).astype(np.float64)
    for b in SAMPLES:
        op = _oracle(spec, ss, sa, b)
        sl = slice(off[b], off[b + 1])
        assert rel(h64[sl], OT.Atilde_apply(op, z[sl])) < 1e-13, b
        assert rel(h32[sl], OT.Atilde_apply(op, z_r[sl])) < 2e-5, b


def test_batch256_mixed_solve_true_residual_by_oracle():
    """The batched mixed-precision solve with per-mesh greedy ROMs (as benchmarked): every instance
    reports convergence, and for sampled instances the oracle recomputes ||b~ - A~ phi|| / ||b~|| <= 1e-8
    from the GPU's phi."""
    torch = torch_cuda()
    B = lib()
    spec, ss, sa, gp = _batch(B)
    off = [int(x) for x in gp.offsets]
    tr_ss, tr_sa = wl.draw_params(spec, 16, wl.seed_for(3, 0))
    roms = {}
    for n in sorted(set(spec.nx)):
        tmpl = B.Problem(spec.with_instances([n], [n]), tr_ss[:1], tr_sa[:1])
        roms[n], _ = B.Rom.greedy(tmpl, tr_ss, tr_sa, window=spec.window, max_greedy_iter=8, max_rank=16,
                                  eps_rom=0.0, hf_rtol=1e-8, hf_restart=128, hf_max_iter=6000, indicator_f32=True)
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    st = B.fgmres_solve(gp, [roms[n] for n in spec.nx], phi, restart=128, rtol=1e-8, max_iter=6000,
                        window=spec.window, mode=B.RTE_MODE_MIXED, inner_rtol=1e-2, max_outer=30)
    assert all(s["status"] == 0 for s in st)
    assert max(s["true_rel_residual"] for s in st) <= 1e-8
    h = phi.cpu().numpy()
    for b in SAMPLES:
        op = _oracle(spec, ss, sa, b)
        bt = OT.rhs_btilde(op)
        r = bt - OT.Atilde_apply(op, h[off[b]:off[b + 1]])
        assert np.linalg.norm(r) / np.linalg.norm(bt) <= 1.05e-8, b


def test_large256_angular_sweep_fp32_sampled():
    """The largest workload's angular sweep (64 x 256^2, 192 directions, 8x8 regions; 12.9 GB of FP32
    output), as the HBM measurement runs it: sampled (instance, direction) blocks against the oracle."""
    torch = torch_cuda()
    B = lib()
    spec = wl.config(5)
    ss, sa = wl.draw_params(spec, spec.n_instances, wl.seed_for(5, 1))
    gp = B.Problem(spec, ss, sa)
    off = [int(x) for x in gp.offsets]
    ndir = gp.n_directions
    s = np.random.default_rng(33).standard_normal(gp.n_dof).astype(np.float32)
    psi = torch.empty(ndir * gp.n_dof, dtype=torch.float32, device="cuda")
    for _ in range(2):
        gp.sweep(to_dev(s), psi, with_bc=True)
    torch.cuda.synchronize()
    for b in (0, 63):
        op = _oracle(spec, ss, sa, b)
        n = off[b + 1] - off[b]
        sb = s[off[b]:off[b + 1]].astype(np.float64)
        blk = psi[ndir * off[b]:ndir * off[b + 1]].view(ndir, n)
        for j in (0, 95, 96, ndir - 1):
            ref = op.sweep(j, sb + op.gbc(j))
            assert rel(blk[j].cpu().numpy(), ref) < 2e-5, (b, j)
    del psi
    torch.cuda.empty_cache()
