"""Helpers for the GPU parity tests: build/load the library, move arrays, run the oracle per instance."""
import dataclasses

import numpy as np
import pytest

import workloads as wl


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib():
    from paper_2410_08735_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def to_dev(a, dtype=None):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def oracle_problems(spec, ss, sa):
    from oracle import Problem
    return [Problem(spec, b, ss[b], sa[b]) for b in range(spec.n_instances)]


def split(vec, offsets):
    return [vec[offsets[b]:offsets[b + 1]] for b in range(len(offsets) - 1)]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def spec2d(nx, ny, n_polar=2, n_azim=8, rx=2, ry=2, **kw):
    spec = wl.config(2)
    spec = dataclasses.replace(spec, n_polar=n_polar, n_azim=n_azim, rx=rx, ry=ry, **kw)
    return spec.with_instances(list(nx), list(ny))


def spec1d(nx, n_polar=8, rx=4, **kw):
    spec = dataclasses.replace(wl.config(1), n_polar=n_polar, rx=rx, **kw)
    return spec.with_instances(list(nx), [1] * len(nx))
