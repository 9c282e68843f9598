"""The variable-scattering problem on the GPU (paper Sec. 5; cross-section blocks of Sec. 2.3): sigma_s = mu_s f + 0.1
with the smooth profile f, so Sigma_s and Sigma_t are full 4x4 blocks per cell.  Parity against the oracle:
operators at 1e-13 (FP64) and 2e-5 (FP32), FP64 solves at 1e-10 of the oracle's tight solution, the greedy ROM
(FGMRES-DSA high-fidelity solves) with the oracle greedy's samples and basis, FGMRES-ROMSAD against the oracle."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import Problem, romsad as ORS, transport as OT

from gpu_common import lib, rel, split, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _spec(n, n_azim=8, n_polar=2, n_inst=1):
    return dataclasses.replace(wl.variable_scattering(), n_azim=n_azim, n_polar=n_polar).with_mesh(n, n, n_inst)


def _params(mus):
    ss = np.array([wl.variable_scattering_params(m)[0] for m in mus])
    sa = np.array([wl.variable_scattering_params(m)[1] for m in mus])
    return ss, sa


def test_operators_match_oracle():
    """A~ (FP64 and FP32), b~ and the angular sweep with the cell blocks, two instances of different mu_s on one mesh
    (the azimuths of CL(10, 2) include pi/2 and 3 pi/2)."""
    torch = torch_cuda()
    B = lib()
    spec = _spec(20, n_azim=10, n_polar=2, n_inst=2)
    ss, sa = _params([52.0, 97.5])
    gp = B.Problem(spec, ss, sa)
    ops = [Problem(spec, b, ss[b], sa[b]) for b in range(2)]
    z = np.random.default_rng(4).standard_normal(gp.n_dof)
    w = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.apply_op(to_dev(z), w)
    w32 = torch.empty(gp.n_dof, dtype=torch.float32, device="cuda")
    gp.apply_op(to_dev(z, torch.float32), w32)
    bt = torch.empty_like(w)
    gp.rhs(bt)
    psi = torch.empty(gp.n_directions * gp.n_dof, dtype=torch.float64, device="cuda")
    gp.sweep(to_dev(z), psi, with_bc=False)
    hw, hw32, hb, hp = w.cpu().numpy(), w32.cpu().numpy().astype(np.float64), bt.cpu().numpy(), psi.cpu().numpy()
    off = [int(x) for x in gp.offsets]
    zr = z.astype(np.float32).astype(np.float64)
    for b, op in enumerate(ops):
        zb = z[off[b]:off[b + 1]]
        assert rel(split(hw, gp.offsets)[b], OT.Atilde_apply(op, zb)) < 1e-13, b
        assert rel(split(hw32, gp.offsets)[b], OT.Atilde_apply(op, zr[off[b]:off[b + 1]])) < 2e-5, b
        assert rel(split(hb, gp.offsets)[b], OT.rhs_btilde(op)) < 1e-12, b
        n = off[b + 1] - off[b]
        blk = hp[gp.n_directions * off[b]:gp.n_directions * off[b + 1]].reshape(gp.n_directions, n)
        for j in (0, 2, 7, 13, 19):
            assert rel(blk[j], op.sweep(j, zb)) < 1e-13, (b, j)


def test_fp64_gmres_dsa_matches_oracle():
    """FP64 GMRES-DSA (the DSA on the cell means) to 1e-12: phi within 1e-10 of the oracle's tight solution."""
    torch = torch_cuda()
    B = lib()
    spec = _spec(32, n_azim=12, n_polar=2, n_inst=2)
    ss, sa = _params([60.0, 99.9])
    gp = B.Problem(spec, ss, sa)
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    st = B.fgmres_solve(gp, None, phi, restart=30, rtol=1e-12, max_iter=2000, post_mode=B.RTE_POST_DSA,
                        mode=B.RTE_MODE_FP64)
    h = split(phi.cpu().numpy(), gp.offsets)
    for b in range(2):
        op = Problem(spec, b, ss[b], sa[b])
        ref, _ = ORS.solve(op, None, post="dsa_vcycle", restart=60, rtol=1e-13, max_iter=2000)
        assert st[b]["status"] == 0
        assert rel(h[b], ref) < 1e-10, b


def test_greedy_matches_oracle_and_romsad_solves_match():
    """Greedy ROM on 6 training points (FGMRES-DSA high-fidelity solves): the oracle greedy's samples, rank and
    basis; then FGMRES-ROMSAD (window 2, DSA after it) in FP64 and in mixed precision (FP64 refinement residuals
    with the profiles) on two new points against the oracle's tight solution, with fewer sweeps than GMRES-DSA."""
    torch = torch_cuda()
    B = lib()
    spec = _spec(16, n_azim=8, n_polar=2)
    train = np.linspace(49.9, 99.9, 6)
    ss, sa = _params(train)
    p0 = Problem(spec, 0, ss[0], sa[0])
    rom_o, rep_o = ORS.greedy(p0, ss, sa, window=2, max_greedy_iter=3, max_rank=6, eps_rom=0.0, hf_rtol=1e-12,
                              restart=60, want_labels=True, hf_post="dsa_vcycle", mu1=2)
    gp1 = B.Problem(spec, ss[:1], sa[:1])
    rom, rep = B.Rom.greedy(gp1, ss, sa, window=2, max_greedy_iter=3, max_rank=6, eps_rom=0.0, hf_rtol=1e-12,
                            hf_restart=60, hf_max_iter=5000, want_labels=True, hf_dsa=True, mu1=2)
    assert rep["sampled"] == rep_o.sampled
    assert rep["rank"] == rom_o.r
    Ug = rom.basis(p0.ndir, p0.ndof).reshape(rom.rank, -1)
    Uo = rom_o.U.reshape(rom_o.r, -1)
    assert np.max(np.abs(Ug - Uo)) < 1e-4
    # the reduced operator from the GPU's affine terms equals the oracle's at a new point
    s_new, a_new = _params([71.3])
    A_g = rom.reduced_operator(s_new[0], a_new[0])
    A_o = ORS.reduced_operator(rom_o, s_new[0], a_new[0])
    assert np.abs(A_g - A_o).max() < 1e-4 * np.abs(A_o).max()
    test = [71.3, 88.8]
    ts, ta = _params(test)
    sp2 = spec.with_mesh(16, 16, 2)
    gp = B.Problem(sp2, ts, ta)
    kw = dict(restart=30, max_iter=2000, post_mode=B.RTE_POST_DSA)
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    st = B.fgmres_solve(gp, [rom, rom], phi, rtol=1e-12, window=2, mode=B.RTE_MODE_FP64, **kw)
    phi_d = torch.zeros_like(phi)
    st_d = B.fgmres_solve(gp, None, phi_d, rtol=1e-12, mode=B.RTE_MODE_FP64, **kw)
    phi_m = torch.zeros_like(phi)
    st_m = B.fgmres_solve(gp, [rom, rom], phi_m, rtol=1e-8, window=2, mode=B.RTE_MODE_MIXED, inner_rtol=1e-3,
                          max_outer=30, **kw)
    h, hm = split(phi.cpu().numpy(), gp.offsets), split(phi_m.cpu().numpy(), gp.offsets)
    for b in range(2):
        op = Problem(sp2, b, ts[b], ta[b])
        ref, _ = ORS.solve(op, None, post="dsa_vcycle", restart=60, rtol=1e-13, max_iter=2000)
        assert st[b]["status"] == 0 and st_m[b]["status"] == 0
        assert rel(h[b], ref) < 1e-10, b
        assert st_m[b]["true_rel_residual"] <= 1e-8 and st_m[b]["sweeps_df"] == 0
        assert rel(hm[b], ref) < 1e-7, b
        assert st[b]["sweeps"] <= st_d[b]["sweeps"], (st[b], st_d[b])


def test_unavailable_forms_are_refused():
    """No double-float sweep or allocation-free apply with the cell blocks: each call returns RTE_ERR_UNSUPPORTED
    instead of running a region-based kernel."""
    torch = torch_cuda()
    B = lib()
    spec = _spec(8, n_azim=8, n_polar=2)
    ss, sa = _params([75.0])
    gp = B.Problem(spec, ss, sa)
    z = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    w = torch.empty_like(z)
    with pytest.raises(B.RteError) as e:
        gp.apply_op(z, w, double_float=True)
    assert e.value.status == 7
    with pytest.raises(B.RteError) as e:
        gp.apply_op_noalloc(z, w)
    assert e.value.status == 7
