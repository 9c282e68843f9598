"""Small shared helpers for the tests (problem builders on top of workloads)."""
import dataclasses

import numpy as np

import workloads as wl


def small_2d(nx=5, ny=4, n_polar=2, n_azim=4, rx=2, ry=2, **kw):
    spec = wl.config(2).with_mesh(nx, ny)
    return dataclasses.replace(spec, n_polar=n_polar, n_azim=n_azim, rx=rx, ry=ry, **kw)


def small_1d(nx=16, n_polar=8, rx=4, **kw):
    spec = wl.config(1).with_mesh(nx, 1)
    return dataclasses.replace(spec, n_polar=n_polar, rx=rx, **kw)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))
