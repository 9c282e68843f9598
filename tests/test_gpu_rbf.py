"""GPU parity of the RBF-interpolated initial guess (the interpolation baseline of Sec. 5) against the
oracle interpolant on the same data, and a solve started from it."""
import numpy as np
import pytest

import workloads as wl
from oracle import rbf as ORBF, romsad as ORS

from gpu_common import lib, oracle_problems, rel, spec2d, split, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def test_rbf_initial_guess_matches_the_oracle_and_starts_a_solve():
    B = lib()
    torch = torch_cuda()
    K = 16
    one = spec2d([16], [16], n_polar=4, n_azim=8)
    tr_ss, tr_sa = wl.draw_params(one, K, 71)
    sols = np.stack([ORS.solve(op, None, post="dsa_pc", restart=200, rtol=1e-12, max_iter=3000)[0]
                     for op in (oracle_problems(one.with_instances([16] * K, [16] * K), tr_ss, tr_sa))])
    tmpl = B.Problem(one, tr_ss[:1], tr_sa[:1])
    f = B.Rbf(tmpl, tr_ss, tr_sa, sols)
    spec = spec2d([16] * 3, [16] * 3, n_polar=4, n_azim=8)
    ts, ta = wl.draw_params(spec, 3, 72)
    gp = B.Problem(spec, ts, ta)
    phi0 = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    f.initial_guess(gp, phi0)
    g0 = phi0.cpu().numpy()
    oref = ORBF.Rbf(tr_ss, tr_sa, sols)
    ops = oracle_problems(spec, ts, ta)
    phi = torch.zeros_like(phi0)
    stats = B.fgmres_solve(gp, None, phi, phi0=phi0, restart=40, rtol=1e-10, max_iter=600,
                           post_mode=B.RTE_POST_DSA)
    for b, op in enumerate(ops):
        assert rel(split(g0, gp.offsets)[b], oref(ts[b], ta[b])) < 1e-12
        tight, _ = ORS.solve(op, None, post="dsa_pc", restart=200, rtol=1e-13, max_iter=3000)
        assert np.linalg.norm(split(g0, gp.offsets)[b] - tight) < np.linalg.norm(tight)
        assert stats[b]["status"] == 0
        assert rel(split(phi.cpu().numpy(), gp.offsets)[b], tight) < 1e-8


def test_rbf_rejects_bad_arguments():
    B = lib()
    torch = torch_cuda()
    one = spec2d([8], [8])
    ss, sa = wl.draw_params(one, 12, 73)
    tmpl = B.Problem(one, ss[:1], sa[:1])
    n = tmpl.n_dof
    with pytest.raises(B.RteError) as e:                 # fewer than 2R + 2 samples
        B.Rbf(tmpl, ss[:9], sa[:9], np.zeros((9, n)))
    assert e.value.status == 1
    f = B.Rbf(tmpl, ss, sa, np.zeros((12, n)))
    other = B.Problem(spec2d([16], [16]), ss[:1], sa[:1])
    with pytest.raises(B.RteError) as e:                 # mesh of the samples differs
        f.initial_guess(other, torch.zeros(other.n_dof, dtype=torch.float64, device="cuda"))
    assert e.value.status == 1
