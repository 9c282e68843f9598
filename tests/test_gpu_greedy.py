"""GPU greedy ROM construction (Sec. 4.4.2) against the oracle greedy."""
import numpy as np
import pytest

import workloads as wl
from oracle import Problem, romsad as ORS
from oracle.discretization import with_params

from gpu_common import lib, rel, spec2d, split, torch_cuda

pytestmark = pytest.mark.gpu


def _subspace_cos(Ua, Ub):
    """Cosines of the principal angles between span(Ua) and span(Ub) (columns orthonormal)."""
    s = np.linalg.svd(Ua.T @ Ub, compute_uv=False)
    return s


def _compare(spec, ss, sa, window, max_iter, max_rank, restart, hf_dsa=False, tol=1e-6):
    """GPU greedy vs oracle greedy: same samples and rank, same basis columns and labels.  tol: basis and label
    tolerance (the DSA high-fidelity solve runs its V-cycle in FP32 on the GPU, FP64 in the oracle, so the
    recorded z and hence xi^(2) agree to ~1e-6 relative)."""
    B = lib()
    p0 = Problem(spec, 0, ss[0], sa[0])
    rom_o, rep_o = ORS.greedy(p0, ss, sa, window=window, max_greedy_iter=max_iter, max_rank=max_rank,
                              eps_rom=0.0, hf_rtol=1e-12, restart=restart, want_labels=True,
                              hf_post="dsa_vcycle" if hf_dsa else None)
    gp = B.Problem(spec.with_instances(spec.nx[:1], spec.ny[:1]), ss[:1], sa[:1])
    rom_g, rep_g = B.Rom.greedy(gp, ss, sa, window=window, max_greedy_iter=max_iter, max_rank=max_rank,
                                eps_rom=0.0, hf_rtol=1e-12, hf_restart=restart, hf_max_iter=5000,
                                want_labels=True, hf_dsa=hf_dsa)
    assert rep_g["sampled"] == rep_o.sampled
    assert rep_g["rank"] == rom_o.r
    n_ind = len(rep_o.max_indicator)
    np.testing.assert_allclose(rep_g["max_indicator"][:n_ind], rep_o.max_indicator, rtol=tol)
    Ug = rom_g.basis(p0.ndir, p0.ndof).reshape(rom_g.rank, -1).T
    Uo = rom_o.U.reshape(rom_o.r, -1).T
    assert np.max(np.abs(Ug.T @ Ug - np.eye(rom_g.rank))) < 1e-10
    cos = _subspace_cos(Ug, Uo)
    assert np.min(cos) > 1 - 1e-8 * (tol / 1e-6) ** 2
    # same columns (same MGS order and signs)
    assert np.max(np.abs(Ug - Uo)) < tol
    # labels are reduced solves on the basis: basis perturbations of size tol reach them amplified by the
    # conditioning of U^T A U, so they are compared at tol relative to the largest label
    lab_atol = (1e-8 * (tol / 1e-6) if tol <= 1e-6 else tol) * np.abs(rep_o.labels).max()
    np.testing.assert_allclose(rep_g["labels"], rep_o.labels, rtol=tol, atol=lab_atol)
    return rom_g, rom_o, p0


def test_greedy_with_dsa_high_fidelity_solves_matches_oracle():
    """Step 2(a) as in the paper: the high-fidelity solves are FGMRES-DSA (on strongly scattering draws, where
    M = I would need hundreds of iterations); same samples, rank, basis and labels as the oracle greedy running
    its own DSA V-cycle."""
    spec = spec2d([16], [16], n_polar=2, n_azim=8, sigma_s_range=(1.0, 1e3))
    ss, sa = wl.draw_params(spec, 6, 33)
    _compare(spec, ss, sa, window=2, max_iter=3, max_rank=12, restart=60, hf_dsa=True, tol=1e-4)


def test_greedy_slab_full_size_matches_oracle():
    """1D slab workload (128 cells, S16, 20 training parameters, window 2, rank <= 10)."""
    spec = wl.config(1)
    ss, sa = wl.draw_params(spec, spec.n_train, wl.seed_for(1, 0))
    _compare(spec, ss, sa, window=2, max_iter=5, max_rank=10, restart=60)


def test_greedy_small_2d_matches_oracle_and_preconditions():
    torch = torch_cuda()
    B = lib()
    spec = spec2d([8], [8], n_polar=2, n_azim=8)
    ss, sa = wl.draw_params(spec, 6, 31)
    ss = np.minimum(ss, 200.0)
    rom_g, rom_o, p0 = _compare(spec, ss, sa, window=2, max_iter=3, max_rank=12, restart=128)
    # FGMRES-ROMSAD with the GPU-built ROM solves to the oracle's answer for new parameters
    ts, ta = wl.draw_params(spec, 2, 32)
    ts = np.minimum(ts, 200.0)
    sp2 = spec.with_instances([8, 8], [8, 8])
    gp = B.Problem(sp2, ts, ta)
    phi = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    stats = B.fgmres_solve(gp, [rom_g, rom_g], phi, restart=60, rtol=1e-12, max_iter=2000, window=2)
    for b in range(2):
        q = with_params(p0, ts[b], ta[b])
        ref, st = ORS.solve(q, rom_o, window=2, restart=60, rtol=1e-12)
        assert rel(split(phi.cpu().numpy(), gp.offsets)[b], ref) < 1e-9


def test_greedy_fp32_indicator_picks_the_oracle_samples():
    """The FP32 indicator (basis in registers, all parameters per block), as the benchmark builds its ROMs: the
    same samples as the oracle greedy and indicator values within FP32 rounding, at ranks that exercise several
    register widths (2 to 18 columns)."""
    spec = spec2d([16], [16], n_polar=2, n_azim=8)
    ss, sa = wl.draw_params(spec, 40, 34)
    ss = np.minimum(ss, 200.0)
    B = lib()
    p0 = Problem(spec, 0, ss[0], sa[0])
    rom_o, rep_o = ORS.greedy(p0, ss, sa, window=2, max_greedy_iter=9, max_rank=18, eps_rom=0.0, hf_rtol=1e-12,
                              restart=128)
    gp = B.Problem(spec.with_instances(spec.nx[:1], spec.ny[:1]), ss[:1], sa[:1])
    rom_g, rep_g = B.Rom.greedy(gp, ss, sa, window=2, max_greedy_iter=9, max_rank=18, eps_rom=0.0, hf_rtol=1e-12,
                                hf_restart=128, hf_max_iter=5000, indicator_f32=True)
    assert rep_g["sampled"] == rep_o.sampled
    n_ind = len(rep_o.max_indicator)
    np.testing.assert_allclose(rep_g["max_indicator"][:n_ind], rep_o.max_indicator, rtol=1e-4)


def test_greedy_on_the_pincell_template_keeps_its_gaussian_source():
    """The greedy's sub-problems take the template's source kind: on the pin-cell problem (Gaussian source,
    CL(30, 6), FGMRES-DSA high-fidelity solves) the GPU greedy picks the oracle greedy's samples and reproduces its
    basis and Galerkin labels, which a box source in the sub-problems would change (its b~ is zero here)."""
    import dataclasses
    spec = dataclasses.replace(wl.pincell().with_mesh(16, 16), n_azim=30, n_polar=6)
    pts = [(a, s) for a in (0.05, 0.275, 0.5) for s in (0.05, 0.5)]
    tr = [wl.pincell_params(a, s) for a, s in pts]
    ss = np.array([x[0] for x in tr])
    sa = np.array([x[1] for x in tr])
    _compare(spec, ss, sa, window=2, max_iter=3, max_rank=6, restart=30, hf_dsa=True, tol=1e-4)
