"""The paper's other 2D problems on the GPU (Sec. 5): the pin-cell problem (Gaussian source, CL(30, 6) whose
azimuths include pi/2 and 3pi/2) and the two-material problem with a parametric inflow on the left face only.
Parity against the oracle: operators at 1e-13, FP64 solves at 1e-10 of the oracle's tight solution."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import Problem, romsad as ORS, transport as OT

from gpu_common import lib, rel, split, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _pincell(nx, n_azim=30, n_polar=6):
    return dataclasses.replace(wl.pincell().with_mesh(nx, nx), n_azim=n_azim, n_polar=n_polar)


def _pin_params(points):
    ss, sa = zip(*(wl.pincell_params(mu_a, mu_s) for mu_a, mu_s in points))
    return np.array(ss), np.array(sa)


def test_pincell_quadrature_has_unequal_quadrants_and_matches_the_oracle():
    """CL(30, 6): the quadrants hold 24, 21, 24 and 21 unique directions; the sweep (angular output), A~ and b~
    (Gaussian source) equal the oracle's, including the directions at pi/2 and 3pi/2."""
    torch = torch_cuda()
    B = lib()
    spec = _pincell(16).with_instances([16, 24], [16, 24])
    ss, sa = _pin_params([(0.1, 0.3), (0.45, 0.05)])
    gp = B.Problem(spec, ss, sa)
    ops = [Problem(spec, b, ss[b], sa[b]) for b in range(2)]
    assert gp.info.n_unique_directions == 90
    z = np.random.default_rng(3).standard_normal(gp.n_dof)
    w = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.apply_op(to_dev(z), w)
    bt = torch.empty_like(w)
    gp.rhs(bt)
    psi = torch.empty(gp.n_directions * gp.n_dof, dtype=torch.float64, device="cuda")
    gp.sweep(to_dev(z), psi, with_bc=False)
    hw, hb, hp = w.cpu().numpy(), bt.cpu().numpy(), psi.cpu().numpy()
    off = [int(x) for x in gp.offsets]
    for b, op in enumerate(ops):
        zb = z[off[b]:off[b + 1]]
        assert rel(split(hw, gp.offsets)[b], OT.Atilde_apply(op, zb)) < 1e-13
        assert rel(split(hb, gp.offsets)[b], OT.rhs_btilde(op)) < 1e-12
        n = off[b + 1] - off[b]
        blk = hp[gp.n_directions * off[b]:gp.n_directions * off[b + 1]].reshape(gp.n_directions, n)
        # j = 7 and 22: the azimuths at pi/2 and 3pi/2 (first polar level); 0 and 29 are ordinary
        for j in (0, 7, 22, 29, 7 + 30 * 5):
            assert rel(blk[j], op.sweep(j, zb)) < 1e-13, (b, j)


def test_pincell_full_size_fgmres_romsad_matches_oracle():
    """80 x 80 pin-cell problem, CL(30, 6): greedy ROM from FGMRES-DSA high-fidelity solves on a 3 x 3 training
    grid, then FGMRES-ROMSAD (window 2) with DSA after the window, FP64 to 1e-12: phi within 1e-10 of the
    oracle's tight solution; the ROM takes fewer sweeps than GMRES-DSA."""
    torch = torch_cuda()
    B = lib()
    spec = _pincell(80)
    grid = [(a, s) for a in np.linspace(0.05, 0.5, 3) for s in np.linspace(0.05, 0.5, 3)]
    tr_ss, tr_sa = _pin_params(grid)
    tmpl = B.Problem(spec, tr_ss[:1], tr_sa[:1])
    rom, rep = B.Rom.greedy(tmpl, tr_ss, tr_sa, window=2, max_greedy_iter=9, max_rank=18, eps_rom=1e-10,
                            hf_rtol=1e-12, hf_restart=30, hf_max_iter=2000, hf_dsa=True)
    test = [(0.2, 0.4), (0.33, 0.11)]
    ts, ta = _pin_params(test)
    sp2 = spec.with_instances([80, 80], [80, 80])
    gp = B.Problem(sp2, ts, ta)
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    st = B.fgmres_solve(gp, [rom, rom], phi, restart=30, rtol=1e-12, max_iter=2000, window=2,
                        post_mode=B.RTE_POST_DSA, mode=B.RTE_MODE_FP64)
    phi_d = torch.zeros_like(phi)
    st_d = B.fgmres_solve(gp, None, phi_d, restart=30, rtol=1e-12, max_iter=2000, post_mode=B.RTE_POST_DSA,
                          mode=B.RTE_MODE_FP64)
    h = split(phi.cpu().numpy(), gp.offsets)
    for b in range(2):
        op = Problem(sp2, b, ts[b], ta[b])
        ref, ost = ORS.solve(op, None, post="dsa_vcycle", restart=60, rtol=1e-13, max_iter=2000)
        assert st[b]["status"] == 0
        assert rel(h[b], ref) < 1e-10, b
        assert st[b]["sweeps"] < st_d[b]["sweeps"], (st[b], st_d[b])


def test_two_material_parametric_inflow_matches_oracle():
    """The two-material problem: inflow mu_bc on the left face only (one-sided inflow), set per instance; no
    source.  b~ and the FP64 GMRES-DSA solution equal the oracle's (1e-12 / 1e-10), and b~ is linear in mu_bc."""
    torch = torch_cuda()
    B = lib()
    spec = dataclasses.replace(wl.param_inflow().with_mesh(32, 32), n_azim=60, n_polar=6)
    spec = spec.with_instances([32, 32, 32], [32, 32, 32])
    mus = [(1.5, 0.7), (4.0, 1.3), (4.0, 0.65)]
    ss = np.array([wl.param_inflow_params(m)[0] for m, _ in mus])
    sa = np.array([wl.param_inflow_params(m)[1] for m, _ in mus])
    gp = B.Problem(spec, ss, sa)
    gp.set_inflow([g for _, g in mus])
    bt = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
    gp.rhs(bt)
    hb = split(bt.cpu().numpy(), gp.offsets)
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    st = B.fgmres_solve(gp, None, phi, restart=30, rtol=1e-12, max_iter=2000, post_mode=B.RTE_POST_DSA,
                        mode=B.RTE_MODE_FP64)
    h = split(phi.cpu().numpy(), gp.offsets)
    for b, (mu_s, g) in enumerate(mus):
        op = Problem(dataclasses.replace(spec, inflow_g=g), b, ss[b], sa[b])
        assert rel(hb[b], OT.rhs_btilde(op)) < 1e-12, b
        ref, _ = ORS.solve(op, None, post="dsa_vcycle", restart=60, rtol=1e-13, max_iter=2000)
        assert st[b]["status"] == 0
        assert rel(h[b], ref) < 1e-10, b
    # same mu_s, inflow 1.3 vs 0.65: b~ scales with the inflow (no source)
    assert rel(hb[1], 2.0 * hb[2]) < 1e-13
