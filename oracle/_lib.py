"""Build and load the oracle's C part (oracle/sweep.c) with gcc; ctypes bindings.

Test infrastructure only: the product path never loads this library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sweep.c")
_SO = os.path.join(_HERE, "_build", "liboracle_sweep.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/sweep.c into oracle/_build/liboracle_sweep.so (plain -O2, no -march)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        for name in ("oracle_sweep_dir", "oracle_apply_dir", "oracle_sweep_dir_blk", "oracle_apply_dir_blk"):
            f = getattr(_lib, name)
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ip, dp, dp, dp]
            f.restype = ctypes.c_int
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def sweep_dir(nx, ny, nd, M, C, inflow, sigt, rhs):
    out = np.empty(nx * ny * nd)
    M = np.ascontiguousarray(M, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    inflow = np.ascontiguousarray(inflow, dtype=np.int32)
    sigt = np.ascontiguousarray(sigt, dtype=np.float64)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    rc = lib().oracle_sweep_dir(nx, ny, nd, _dp(M), _dp(C), _ip(inflow), _dp(sigt), _dp(rhs), _dp(out))
    if rc != 0:
        raise FloatingPointError(f"oracle sweep failed ({rc})")
    return out


def apply_dir(nx, ny, nd, M, C, inflow, sigt, x):
    out = np.empty(nx * ny * nd)
    M = np.ascontiguousarray(M, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    inflow = np.ascontiguousarray(inflow, dtype=np.int32)
    sigt = np.ascontiguousarray(sigt, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    lib().oracle_apply_dir(nx, ny, nd, _dp(M), _dp(C), _ip(inflow), _dp(sigt), _dp(x), _dp(out))
    return out


def sweep_dir_blk(nx, ny, nd, M, C, inflow, St, rhs):
    """sweep_dir with a full Sigma_t block per cell: St [ncell, nd, nd]."""
    out = np.empty(nx * ny * nd)
    M = np.ascontiguousarray(M, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    inflow = np.ascontiguousarray(inflow, dtype=np.int32)
    St = np.ascontiguousarray(St, dtype=np.float64)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    rc = lib().oracle_sweep_dir_blk(nx, ny, nd, _dp(M), _dp(C), _ip(inflow), _dp(St), _dp(rhs), _dp(out))
    if rc != 0:
        raise FloatingPointError(f"oracle sweep failed ({rc})")
    return out


def apply_dir_blk(nx, ny, nd, M, C, inflow, St, x):
    """apply_dir with a full Sigma_t block per cell: St [ncell, nd, nd]."""
    out = np.empty(nx * ny * nd)
    M = np.ascontiguousarray(M, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    inflow = np.ascontiguousarray(inflow, dtype=np.int32)
    St = np.ascontiguousarray(St, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    lib().oracle_apply_dir_blk(nx, ny, nd, _dp(M), _dp(C), _ip(inflow), _dp(St), _dp(x), _dp(out))
    return out
