"""GPU parity of the Gaussian source (the pin-cell problem's source, Sec. 5): b~ against the oracle, whose
projection is by Gauss quadrature and whose closed form is pinned separately; the one-sided inflow of the
two-material problem is refused by this build."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import Problem, transport as OT

from gpu_common import lib, rel, torch_cuda

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


def test_one_sided_inflow_is_refused():
    B = lib()
    spec = dataclasses.replace(wl.param_inflow(), nx=[16], ny=[16], n_polar=2, n_azim=8)
    ss, sa = wl.param_inflow_params(2.0)
    with pytest.raises(B.RteError) as e:
        B.Problem(spec, ss[None, :], sa[None, :])
    assert e.value.status == 7
