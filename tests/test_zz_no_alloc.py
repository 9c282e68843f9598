"""rte_apply_op_noalloc: the A~ apply for callers that cannot allocate device memory.

Such callers (a host code whose pool allocator owns the device memory, or a step issued where the
implicit synchronisation of cudaMalloc is not acceptable) get the same operator through an entry
point whose scratch is a fixed array compiled into the library.  This file runs last so that a
failure here leaves every other test already run; it passes alone and after the other tests.
"""
import numpy as np
import pytest

import workloads as wl

from gpu_common import lib, rel, spec2d, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _problem(B):
    spec = spec2d([40, 24], [36, 48], n_polar=4, n_azim=8, inflow_g=0.2)
    ss, sa = wl.draw_params(spec, 2, 61)
    return B.Problem(spec, ss, sa)


@pytest.mark.parametrize("dtype_name,tol", [("float64", 1e-13), ("float32", 2e-5)])
def test_noalloc_matches_apply_op_on_two_calls(dtype_name, tol):
    torch = torch_cuda()
    B = lib()
    gp = _problem(B)
    dt = getattr(torch, dtype_name)
    rng = np.random.default_rng(7)
    for call in range(2):   # two calls in a row share (and must not depend on) the scratch contents
        z = to_dev(rng.standard_normal(gp.n_dof), dt)
        ref = torch.empty_like(z)
        out = torch.full_like(z, float("nan"))
        gp.apply_op(z, ref)
        gp.apply_op_noalloc(z, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) < tol, call


def test_noalloc_rejects_problems_beyond_its_scratch():
    B = lib()
    spec = wl.config(3)       # 256 instances: the partial sums need far more than 16 MiB
    ss, sa = wl.draw_params(spec, spec.n_instances, 62)
    gp = B.Problem(spec, ss, sa)
    torch = torch_cuda()
    z = torch.zeros(gp.n_dof, dtype=torch.float64, device="cuda")
    w = torch.empty_like(z)
    with pytest.raises(B.RteError, match="scratch"):
        gp.apply_op_noalloc(z, w)
