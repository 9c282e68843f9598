"""GPU parity of the Gaussian source (the pin-cell problem's source, Sec. 5): b~ against the oracle, whose
projection is by Gauss quadrature and whose closed form is pinned separately; the one-sided inflow of the
two-material problem is refused by this build."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import Problem, transport as OT

from gpu_common import lib, rel, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def test_gaussian_source_rhs_matches_the_oracle():
    B = lib()
    torch = torch_cuda()
    for gauss in ((1.0, 100.0, 0.0, 0.0), (2.0, 30.0, 0.3, -0.2)):
        spec = dataclasses.replace(wl.pincell(), nx=[24], ny=[20], n_polar=2, n_azim=8, src_gauss=gauss)
        ss, sa = wl.pincell_params(0.2, 0.3)
        gp = B.Problem(spec, ss[None, :], sa[None, :])
        bt = torch.empty(gp.n_dof, dtype=torch.float64, device="cuda")
        gp.rhs(bt)
        torch.cuda.synchronize()
        ref = OT.rhs_btilde(Problem(spec, 0, ss, sa))
        assert rel(bt.cpu().numpy(), ref) < 1e-12


def test_one_sided_inflow_angular_sweep_matches_oracle():
    """Inflow on the left face only: the angular sweep with boundary data equals the oracle's for directions
    entering through that face (Omega_x > 0) and for those entering through vacuum faces only."""
    torch = torch_cuda()
    B = lib()
    spec = dataclasses.replace(wl.param_inflow(), nx=[16], ny=[16], n_polar=2, n_azim=8, inflow_g=0.8)
    ss, sa = wl.param_inflow_params(2.0)
    gp = B.Problem(spec, ss[None, :], sa[None, :])
    op = Problem(spec, 0, ss, sa)
    s = np.random.default_rng(4).standard_normal(gp.n_dof)
    psi = torch.empty(gp.n_directions * gp.n_dof, dtype=torch.float64, device="cuda")
    gp.sweep(to_dev(s), psi, with_bc=True)
    h = psi.cpu().numpy().reshape(gp.n_directions, gp.n_dof)
    for j in range(gp.n_directions):
        assert rel(h[j], op.sweep(j, s + op.gbc(j))) < 1e-13, j


def test_inflow_face_mask_validated():
    B = lib()
    s1 = dataclasses.replace(wl.config(1).with_mesh(16, 1), inflow_faces=("x-", "y+"))
    ss, sa = wl.draw_params(s1, 1, 5)
    with pytest.raises(B.RteError) as e:
        B.Problem(s1, ss, sa)    # a slab has no y faces
    assert e.value.status == 1
