"""Thin ctypes binding of include/rte.h (argument marshalling only).

Every computation runs in librte_gb300.so (hand-written CUDA for sm_103a).
Tensors are torch CUDA tensors (contiguous); their data pointers are handed to
the C ABI unchanged.  A missing or unloadable library raises immediately:
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build_lib

RTE_OK = 0
RTE_ERR_NOT_CONVERGED = 4
RTE_ERR_NUMERIC = 5
RTE_F64, RTE_F32, RTE_F64_DF = 0, 1, 2
RTE_POST_ROM, RTE_POST_IDENTITY, RTE_POST_DSA = 0, 1, 2
RTE_DSA_PARTIAL, RTE_DSA_LUMPED, RTE_DSA_FULL = 0, 1, 2
RTE_DSA_KEEP_SETUP = 16
RTE_MODE_FP64, RTE_MODE_MIXED, RTE_MODE_MIXED_F64KRYLOV = 0, 1, 2
RTE_RESIDUAL_DF, RTE_RESIDUAL_FP64 = 0, 1
RTE_SIGMA_REGIONS, RTE_SIGMA_VARSCAT = 0, 1

_lib = None


class RteError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} ({status})")
        self.status = status


class ProblemDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_instances", ctypes.c_int),
                ("nx", ctypes.POINTER(ctypes.c_int)), ("ny", ctypes.POINTER(ctypes.c_int)),
                ("box", ctypes.c_double * 4), ("n_polar", ctypes.c_int), ("n_azim", ctypes.c_int),
                ("rx", ctypes.c_int), ("ry", ctypes.c_int),
                ("sigma_s", ctypes.POINTER(ctypes.c_double)), ("sigma_a", ctypes.POINTER(ctypes.c_double)),
                ("src_q", ctypes.c_double), ("src_box", ctypes.c_double * 4), ("inflow_g", ctypes.c_double),
                ("src_kind", ctypes.c_int), ("src_gauss", ctypes.c_double * 4), ("inflow_faces", ctypes.c_int),
                ("sigma_modes", ctypes.c_int)]


class ProblemInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_instances", ctypes.c_int), ("n_directions", ctypes.c_int),
                ("n_unique_directions", ctypes.c_int), ("dofs_per_cell", ctypes.c_int),
                ("n_regions", ctypes.c_int), ("n_dof_total", ctypes.c_longlong),
                ("n_angular_total", ctypes.c_longlong)]


class GreedyOpts(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("max_greedy_iter", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("eps_rom", ctypes.c_double), ("eps_qr", ctypes.c_double), ("mu1", ctypes.c_int),
                ("hf_rtol", ctypes.c_double), ("hf_restart", ctypes.c_int), ("hf_max_iter", ctypes.c_int),
                ("indicator_f32", ctypes.c_int), ("hf_dsa", ctypes.c_int)]


class GreedyReport(ctypes.Structure):
    _fields_ = [("n_sampled", ctypes.c_int), ("sampled", ctypes.POINTER(ctypes.c_int)),
                ("max_indicator", ctypes.POINTER(ctypes.c_double)), ("rank", ctypes.c_int),
                ("labels", ctypes.POINTER(ctypes.c_double))]


class MlpTrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("bf16", ctypes.c_int)]


class FgmresOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("rtol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("window", ctypes.c_int), ("post_mode", ctypes.c_int), ("mode", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("true_residual_check", ctypes.c_int), ("warm_start", ctypes.c_int), ("learned_slot", ctypes.c_int),
                ("dsa_variant", ctypes.c_int), ("rom_bf16", ctypes.c_int), ("refine_residual", ctypes.c_int)]


class FgmresStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("sweeps_fp64", ctypes.c_int), ("sweeps_df", ctypes.c_int), ("restarts", ctypes.c_int),
                ("outer", ctypes.c_int),
                ("escalated", ctypes.c_int), ("learned_start", ctypes.c_int), ("learned_slot", ctypes.c_int),
                ("est_rel_residual", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double), ("true_linf_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_SIGS = {
    "rte_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rte_last_error": (ctypes.c_char_p, []),
    "rte_version": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "rte_kernel_launches": (ctypes.c_longlong, []),
    "rte_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "rte_problem_create": (ctypes.c_int, [ctypes.POINTER(ProblemDesc), ctypes.POINTER(ctypes.c_void_p)]),
    "rte_problem_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "rte_problem_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ProblemInfo)]),
    "rte_problem_offsets": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "rte_problem_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]),
    "rte_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "rte_scalar_flux": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "rte_apply_T": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "rte_apply_op": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "rte_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "rte_apply_op_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "rte_dsa_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "romsad_create_from_basis": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p)]),
    "romsad_build_greedy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(GreedyOpts),
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(GreedyReport)]),
    "romsad_rank": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "romsad_get_basis": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "romsad_reduced_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "romsad_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "romsad_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "romsad_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]),
    "romsad_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "rte_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "rte_mlp_num_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "rte_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "rte_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "rte_mlp_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)]),
    "rte_mlp_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(MlpTrainOpts),
                                     ctypes.POINTER(ctypes.c_double)]),
    "rte_mlp_infer": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "rte_mlp_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "romsad_attach_mlp": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "fgmres_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(FgmresOpts),
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(FgmresStats),
                                    ctypes.c_void_p]),
    "si_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(FgmresOpts),
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(FgmresStats), ctypes.c_void_p]),
    "rte_rbf_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "rte_rbf_initial_guess": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "rte_rbf_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "rte_problem_set_inflow": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "rte_problem_set_sweep_variant": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "romsad_galerkin_coefficients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
}


def lib_path() -> str:
    return build_lib.LIB


def load(build_if_missing: bool = False):
    """Load librte_gb300.so (building it first only when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = build_lib.build() if build_if_missing else build_lib.LIB
    if not os.path.exists(path):
        raise ImportError(f"librte_gb300.so not built ({path}); run paper_2410_08735_gb300.build_lib.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def kernel_launches() -> int:
    """Kernels launched by librte_gb300 so far in this process."""
    return int(load().rte_kernel_launches())


def fma_peak(dtype: int = RTE_F32, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (RTE_F32 or RTE_F64)."""
    out = ctypes.c_double(0.0)
    _check(load().rte_fma_peak(dtype, ctypes.byref(out), _stream(stream)), "rte_fma_peak")
    return out.value


def _check(status: int, where: str):
    if status != RTE_OK:
        lib = load()
        raise RteError(status, where, lib.rte_last_error().decode() or lib.rte_status_string(status).decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return RTE_F64
    if t.dtype == torch.float32:
        return RTE_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Problem:
    """Owns an rte_problem_t.  spec: a workloads.ProblemSpec; sigma_s/sigma_a: [B][R] arrays."""

    def __init__(self, spec, sigma_s, sigma_a):
        lib = load()
        B = spec.n_instances
        self.spec = spec
        ss = np.ascontiguousarray(np.asarray(sigma_s, dtype=np.float64).reshape(B, -1))
        sa = np.ascontiguousarray(np.asarray(sigma_a, dtype=np.float64).reshape(B, -1))
        nx = (ctypes.c_int * B)(*spec.nx)
        ny = (ctypes.c_int * B)(*spec.ny)
        faces = tuple(getattr(spec, "inflow_faces", ("x-", "x+", "y-", "y+")))
        d = ProblemDesc()
        d.dim = spec.dim
        d.n_instances = B
        d.nx = nx
        d.ny = ny
        d.box = (ctypes.c_double * 4)(*spec.box)
        d.n_polar = spec.n_polar
        d.n_azim = spec.n_azim
        d.rx = spec.rx
        d.ry = spec.ry if spec.dim == 2 else 1
        d.sigma_s = _dptr(ss)
        d.sigma_a = _dptr(sa)
        d.src_q = spec.src_q
        d.src_box = (ctypes.c_double * 4)(*spec.src_box)
        d.inflow_g = spec.inflow_g
        gauss = getattr(spec, "src_gauss", None)
        d.src_kind = 0 if gauss is None else 1
        d.src_gauss = (ctypes.c_double * 4)(*(gauss if gauss is not None else (0.0, 0.0, 0.0, 0.0)))
        bits = {"x-": 1, "x+": 2, "y-": 4, "y+": 8}
        mask = sum(bits[f] for f in set(faces))
        d.inflow_faces = 0 if mask == 15 else mask
        modes = getattr(spec, "sigma_modes", None)
        if modes not in (None, "variable_scattering"):
            raise ValueError(f"unknown sigma_modes {modes!r}")
        d.sigma_modes = RTE_SIGMA_VARSCAT if modes == "variable_scattering" else RTE_SIGMA_REGIONS
        h = ctypes.c_void_p()
        _check(lib.rte_problem_create(ctypes.byref(d), ctypes.byref(h)), "rte_problem_create")
        self.h = h
        info = ProblemInfo()
        _check(lib.rte_problem_get_info(h, ctypes.byref(info)), "rte_problem_get_info")
        self.info = info
        offs = (ctypes.c_longlong * (B + 1))()
        _check(lib.rte_problem_offsets(h, offs), "rte_problem_offsets")
        self.offsets = np.array(list(offs), dtype=np.int64)

    @property
    def n_dof(self) -> int:
        return int(self.info.n_dof_total)

    @property
    def n_directions(self) -> int:
        return int(self.info.n_directions)

    def set_params(self, sigma_s, sigma_a):
        ss = np.ascontiguousarray(np.asarray(sigma_s, dtype=np.float64))
        sa = np.ascontiguousarray(np.asarray(sigma_a, dtype=np.float64))
        _check(load().rte_problem_set_params(self.h, _dptr(ss), _dptr(sa)), "rte_problem_set_params")

    def set_sweep_variant(self, variant: int, directions_per_warp: int = 1, tasks_per_run: int = 0):
        """Pin the sweep kernel (0 band, 1 warp per task, 2 pipelined band; -1: autotuner)."""
        _check(load().rte_problem_set_sweep_variant(self.h, variant, directions_per_warp, tasks_per_run),
               "rte_problem_set_sweep_variant")

    def set_inflow(self, g):
        """Per-instance inflow values on the problem's inflow faces: [B]."""
        gv = np.ascontiguousarray(np.asarray(g, dtype=np.float64).reshape(-1))
        _check(load().rte_problem_set_inflow(self.h, _dptr(gv)), "rte_problem_set_inflow")

    def close(self):
        if getattr(self, "h", None):
            load().rte_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # transport ------------------------------------------------------------
    def sweep(self, src, psi, with_bc: bool = False, stream=None):
        _check(load().rte_sweep(self.h, _dtype_code(src), _ptr(src), int(with_bc), _ptr(psi), _stream(stream)),
               "rte_sweep")

    def scalar_flux(self, psi, phi, stream=None):
        _check(load().rte_scalar_flux(self.h, _dtype_code(psi), _ptr(psi), _ptr(phi), _stream(stream)),
               "rte_scalar_flux")

    def apply_T(self, s, phi, stream=None):
        _check(load().rte_apply_T(self.h, _dtype_code(s), _ptr(s), _ptr(phi), _stream(stream)), "rte_apply_T")

    def apply_op(self, z, w, stream=None, double_float=False):
        """w = A~ z; double_float=True: FP64 tensors, sweep in double-float arithmetic (RTE_F64_DF)."""
        code = RTE_F64_DF if double_float else _dtype_code(z)
        _check(load().rte_apply_op(self.h, code, _ptr(z), _ptr(w), _stream(stream)), "rte_apply_op")

    def apply_op_noalloc(self, z, w, stream=None):
        """rte_apply_op without device allocation (fixed 16 MiB scratch shared by all calls)."""
        _check(load().rte_apply_op_noalloc(self.h, _dtype_code(z), _ptr(z), _ptr(w), _stream(stream)),
               "rte_apply_op_noalloc")

    def rhs(self, out, stream=None):
        _check(load().rte_rhs(self.h, _dtype_code(out), _ptr(out), _stream(stream)), "rte_rhs")

    def dsa_apply(self, v, z, variant=RTE_DSA_PARTIAL, stream=None):
        """z = M_DSA^{-1} v (one multigrid V-cycle on the DSA system of each instance)."""
        _check(load().rte_dsa_apply(self.h, variant, _dtype_code(v), _ptr(v), _ptr(z), _stream(stream)),
               "rte_dsa_apply")


class Rom:
    """Owns a romsad_t."""

    def __init__(self, handle):
        self.h = handle

    @classmethod
    def from_basis(cls, problem: Problem, U: np.ndarray, instance: int = 0):
        U = np.ascontiguousarray(U, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(load().romsad_create_from_basis(problem.h, instance, U.shape[0], _dptr(U), ctypes.byref(h)),
               "romsad_create_from_basis")
        return cls(h)

    @classmethod
    def greedy(cls, problem: Problem, train_ss, train_sa, window=2, max_greedy_iter=10, max_rank=32,
               eps_rom=1e-8, eps_qr=1e-13, mu1=-1, hf_rtol=1e-12, hf_restart=30, hf_max_iter=2000,
               want_labels=False, indicator_f32=False, hf_dsa=False):
        ss = np.ascontiguousarray(train_ss, dtype=np.float64)
        sa = np.ascontiguousarray(train_sa, dtype=np.float64)
        n_train = ss.shape[0]
        o = GreedyOpts(window, max_greedy_iter, max_rank, eps_rom, eps_qr, mu1, hf_rtol, hf_restart, hf_max_iter,
                       int(indicator_f32), int(hf_dsa))
        sampled = (ctypes.c_int * max_greedy_iter)()
        ind = (ctypes.c_double * max_greedy_iter)()
        labels = np.zeros((n_train, max_rank)) if want_labels else None
        rep = GreedyReport(0, sampled, ind, 0, _dptr(labels) if labels is not None else None)
        h = ctypes.c_void_p()
        _check(load().romsad_build_greedy(problem.h, n_train, _dptr(ss), _dptr(sa), ctypes.byref(o), ctypes.byref(h),
                                          ctypes.byref(rep)), "romsad_build_greedy")
        rom = cls(h)
        r = rep.rank
        report = {"sampled": [sampled[i] for i in range(min(rep.n_sampled, max_greedy_iter))],
                  "max_indicator": [ind[i] for i in range(min(rep.n_sampled, max_greedy_iter))],
                  "rank": r, "labels": labels[:, :r] if labels is not None else None}
        return rom, report

    @classmethod
    def load_file(cls, path: str):
        h = ctypes.c_void_p()
        _check(load().romsad_load(path.encode(), ctypes.byref(h)), "romsad_load")
        return cls(h)

    @property
    def rank(self) -> int:
        r = ctypes.c_int()
        _check(load().romsad_rank(self.h, ctypes.byref(r)), "romsad_rank")
        return r.value

    def basis(self, n_dir: int, n_dof: int) -> np.ndarray:
        U = np.zeros((self.rank, n_dir, n_dof))
        _check(load().romsad_get_basis(self.h, _dptr(U)), "romsad_get_basis")
        return U

    def reduced_operator(self, sigma_s, sigma_a) -> np.ndarray:
        r = self.rank
        A = np.zeros((r, r))
        ss = np.ascontiguousarray(sigma_s, dtype=np.float64)
        sa = np.ascontiguousarray(sigma_a, dtype=np.float64)
        _check(load().romsad_reduced_operator(self.h, _dptr(ss), _dptr(sa), _dptr(A)), "romsad_reduced_operator")
        return A

    def galerkin_coefficients(self, problem: Problem) -> np.ndarray:
        """Galerkin coefficients c_mu (eq. greedy-rom) of every instance of the problem: [B][rank]."""
        out = np.zeros((problem.spec.n_instances, self.rank))
        _check(load().romsad_galerkin_coefficients(self.h, problem.h, _dptr(out)), "romsad_galerkin_coefficients")
        return out

    def apply(self, problem: Problem, v, z, stream=None):
        _check(load().romsad_apply(self.h, problem.h, _dtype_code(v), _ptr(v), _ptr(z), _stream(stream)),
               "romsad_apply")

    def save(self, path: str):
        _check(load().romsad_save(self.h, path.encode()), "romsad_save")

    def close(self):
        if getattr(self, "h", None):
            load().romsad_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Mlp:
    """Owns an rte_mlp_t (learned warm start network)."""

    def __init__(self, n_in: int, hidden: int, n_out: int, seed: int = 0):
        h = ctypes.c_void_p()
        _check(load().rte_mlp_create(n_in, hidden, n_out, seed, ctypes.byref(h)), "rte_mlp_create")
        self.h = h
        self.n_in, self.hidden, self.n_out = n_in, hidden, n_out
        n = ctypes.c_int()
        _check(load().rte_mlp_num_params(h, ctypes.byref(n)), "rte_mlp_num_params")
        self.n_params = n.value

    def set_params(self, flat, mean=None, stdv=None):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        m = None if mean is None else _fptr(np.ascontiguousarray(mean, dtype=np.float32))
        s = None if stdv is None else _fptr(np.ascontiguousarray(stdv, dtype=np.float32))
        _check(load().rte_mlp_set_params(self.h, _fptr(flat), m, s), "rte_mlp_set_params")

    def get_params(self):
        flat = np.zeros(self.n_params, dtype=np.float32)
        mean = np.zeros(self.n_in, dtype=np.float32)
        stdv = np.zeros(self.n_in, dtype=np.float32)
        _check(load().rte_mlp_get_params(self.h, _fptr(flat), _fptr(mean), _fptr(stdv)), "rte_mlp_get_params")
        return flat, mean, stdv

    def loss_grad(self, mu, c, bf16=False):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.float64)
        loss = ctypes.c_double()
        grad = np.zeros(self.n_params, dtype=np.float32)
        _check(load().rte_mlp_loss_grad(self.h, mu.shape[0], _dptr(mu), _dptr(c), int(bf16), ctypes.byref(loss),
                                        _fptr(grad)), "rte_mlp_loss_grad")
        return loss.value, grad

    def train(self, mu, c, epochs=200, batch=256, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, bf16=True):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.float64)
        o = MlpTrainOpts(epochs, batch, lr, beta1, beta2, eps, int(bf16))
        loss = ctypes.c_double()
        _check(load().rte_mlp_train(self.h, mu.shape[0], _dptr(mu), _dptr(c), ctypes.byref(o), ctypes.byref(loss)),
               "rte_mlp_train")
        return loss.value

    def infer(self, mu):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        out = np.zeros((mu.shape[0], self.n_out))
        _check(load().rte_mlp_infer(self.h, mu.shape[0], _dptr(mu), _dptr(out)), "rte_mlp_infer")
        return out

    def close(self):
        if getattr(self, "h", None):
            load().rte_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def attach_mlp(rom: "Rom", mlp: Optional[Mlp]):
    _check(load().romsad_attach_mlp(rom.h, mlp.h if mlp is not None else None), "romsad_attach_mlp")
    rom._mlp = mlp


def fgmres_solve(problem: Problem, roms: Optional[Sequence[Optional[Rom]]], phi, phi0=None, restart=30,
                 rtol=1e-10, max_iter=1000, window=2, post_mode=RTE_POST_ROM, mode=RTE_MODE_FP64,
                 inner_rtol=1e-2, max_outer=20, true_residual_check=True, stream=None, raise_on_fail=True,
                 learned_warm_start=False, learned_slot=False, dsa_variant=RTE_DSA_PARTIAL,
                 refine_residual=RTE_RESIDUAL_DF, rom_bf16=False):
    """FGMRES-ROMSAD for all instances; phi: FP64 device tensor or host (numpy/pinned) buffer.
    post_mode=RTE_POST_DSA switches to DSA after the window (with roms=None: GMRES-DSA).

    Returns the list of per-instance stats dicts.
    """
    B = problem.spec.n_instances
    ws = 2 if learned_warm_start else int(phi0 is not None)
    o = FgmresOpts(restart, rtol, max_iter, window, post_mode, mode, inner_rtol, max_outer,
                   int(true_residual_check), ws, int(learned_slot), int(dsa_variant), int(rom_bf16),
                   int(refine_residual))
    st = (FgmresStats * B)()
    if roms is None:
        rarr = None
    else:
        rarr = (ctypes.c_void_p * B)(*[(r.h.value if r is not None else None) for r in roms])
    if isinstance(phi, np.ndarray):
        assert phi.dtype == np.float64 and phi.flags["C_CONTIGUOUS"]
        phi_ptr = ctypes.c_void_p(phi.ctypes.data)
    else:
        phi_ptr = _ptr(phi)
    s = load().fgmres_solve(problem.h, rarr, ctypes.byref(o), _ptr(phi0), phi_ptr, st, _stream(stream))
    stats = [st[b].as_dict() for b in range(B)]
    if s != RTE_OK and (raise_on_fail or s not in (RTE_ERR_NOT_CONVERGED, RTE_ERR_NUMERIC)):
        _check(s, "fgmres_solve")
    return stats


def si_solve(problem: Problem, roms: Optional[Sequence[Optional[Rom]]], phi, phi0=None, rtol=1e-10, max_iter=1000,
             window=2, post_mode=RTE_POST_DSA, dsa_variant=RTE_DSA_PARTIAL, stream=None, raise_on_fail=True):
    """SI-ROMSAD (source iteration, ROM correction in the window, then post_mode) for all instances, FP64.
    phi: FP64 device tensor or host (numpy) buffer.  Returns the list of per-instance stats dicts."""
    B = problem.spec.n_instances
    o = FgmresOpts(1, rtol, max_iter, window, post_mode, RTE_MODE_FP64, 0.0, 0, 0, 0, 0, int(dsa_variant), 0, 0)
    st = (FgmresStats * B)()
    rarr = None if roms is None else (ctypes.c_void_p * B)(*[(r.h.value if r is not None else None) for r in roms])
    if isinstance(phi, np.ndarray):
        assert phi.dtype == np.float64 and phi.flags["C_CONTIGUOUS"]
        phi_ptr = ctypes.c_void_p(phi.ctypes.data)
    else:
        phi_ptr = _ptr(phi)
    s = load().si_solve(problem.h, rarr, ctypes.byref(o), _ptr(phi0), phi_ptr, st, _stream(stream))
    stats = [st[b].as_dict() for b in range(B)]
    if s != RTE_OK and (raise_on_fail or s not in (RTE_ERR_NOT_CONVERGED, RTE_ERR_NUMERIC)):
        _check(s, "si_solve")
    return stats


class Rbf:
    """Owns an rte_rbf_t: the RBF interpolant of sampled scalar fluxes (the interpolated initial guess)."""

    def __init__(self, tmpl: Problem, sigma_s, sigma_a, solutions):
        """sigma_s, sigma_a: [K][R]; solutions: [K][N] FP64 (device tensor or numpy array), copied."""
        ss = np.ascontiguousarray(sigma_s, dtype=np.float64)
        sa = np.ascontiguousarray(sigma_a, dtype=np.float64)
        if isinstance(solutions, np.ndarray):
            sol = np.ascontiguousarray(solutions, dtype=np.float64)
            sptr = ctypes.c_void_p(sol.ctypes.data)
        else:
            sptr = _ptr(solutions)
        h = ctypes.c_void_p()
        _check(load().rte_rbf_create(tmpl.h, ss.shape[0], _dptr(ss), _dptr(sa), sptr, ctypes.byref(h)),
               "rte_rbf_create")
        self.h = h

    def initial_guess(self, problem: Problem, phi0, stream=None):
        _check(load().rte_rbf_initial_guess(self.h, problem.h, _ptr(phi0), _stream(stream)), "rte_rbf_initial_guess")

    def __del__(self):
        try:
            if getattr(self, "h", None) and self.h.value:
                load().rte_rbf_destroy(self.h)
                self.h = ctypes.c_void_p()
        except Exception:
            pass
