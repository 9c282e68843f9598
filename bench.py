"""Benchmark: parameter solves/s of FGMRES-ROMSAD for the parametric RTE on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

A step solves one batch of seeded parameter instances of the workload to FP64 true residual 1e-8 (relative
l2 of b~ - A~ phi).  The default workload is the largest single-GPU configuration of the metric,
large256_192: 64 instances of the 256x256 problem (upwind DG Q1, 8 x 24 = 192 directions, 8x8 regions,
sigma_s log-uniform in [1, 1e4], sigma_a uniform in [0, 1]), restart 40, MLP initial guess.

`value` is the mixed-precision path with the learned start (FP32 sweeps and inner solves, FP64 b~ and
certifying residual, double-float refinement residuals); `fp64` beside it is plain FP64 FGMRES-ROMSAD on the
same GPU with the same ROM.  Every leg carries the scalar-flux error of one sampled instance against the CPU
oracle's tight solution (solved in background processes during the GPU legs).  Inputs are resident in HBM
when the timed region starts; L2 is flushed (a 256 MiB write) before every timed step.  `e2e` repeats the
headline through the C ABI with host buffers: each step copies its parameters host->device and the scalar
flux device->host inside the timed region.  Under torchrun every rank solves its own instances (no
collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# every CPU oracle process runs on one core: cap the BLAS / OpenMP pools before numpy starts them
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

# Algorithmic arithmetic per cell and unique direction of the fused 2D sweep (rhs assembly, 4x4 solve with the
# precomputed cell inverse, outflow traces, quadrature): about 42 FMA = 90 flop.
SWEEP_FLOPS_PER_CELL_DIR = 90

METRIC = "param solves/s at 1e-8 true residual (mixed+MLP FGMRES-ROMSAD vs plain FP64 FGMRES-ROMSAD)"

WORKLOADS = {"large256_192": 5, "batch256_uneven": 3, "square2d_64": 2, "slab1d_128": 1}


def workload_spec(name: str):
    if name not in WORKLOADS:
        raise SystemExit(f"unknown workload {name}")
    cfg = WORKLOADS[name]
    spec = wl.config(cfg)
    return spec, spec.n_instances, cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if len(s) >= 9 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) >= 9 and s[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for s in self.samples:
            if len(s) < 9:
                continue
            for k, nm in enumerate(names):
                if s[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def dist_setup(backend: str | None = None):
    """Join the torchrun process group (one rank per GPU, NCCL; gloo when asked or without a GPU, which
    is how the host-side logic is tested on CPU).  Returns (world, rank, local rank)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    """Maximum of a host scalar over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(rank: int, n_sets: int, B: int, step: int) -> tuple[int, int]:
    """Parameter draws [i0, i1) that rank `rank` solves at step `step`: every rank owns n_sets * B
    consecutive draws of one seeded stream, so ranks never share an instance (weak scaling)."""
    i0 = rank * n_sets * B + step * B
    return i0, i0 + B


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ CPU oracle (spawned processes)
def _one_instance_spec(cfg: int, nx: int, ny: int):
    return wl.config(cfg).with_instances([nx], [ny])


def oracle_reference_phi(cfg: int, nx: int, ny: int, ss, sa, rtol: float = 1e-12):
    """The oracle's tight solution of one instance (FGMRES with its DSA V-cycle, FP64, one core): the reference
    of the scalar-flux errors.  Runs in a spawned process."""
    from oracle import Problem as OProblem, romsad as ORS
    t0 = time.perf_counter()
    p = OProblem(_one_instance_spec(cfg, nx, ny), 0, np.asarray(ss), np.asarray(sa))
    phi, st = ORS.solve(p, None, post="dsa_vcycle", restart=60, rtol=rtol, max_iter=3000, true_residual_check=True)
    return {"phi": phi, "iterations": st.iterations, "s": time.perf_counter() - t0}


def oracle_sample_worker(cfg: int, nx: int, ny: int, ss, sa, n_warm: int, n_timed: int):
    """Bounded sample of the oracle's FGMRES-DSA solve of one instance (one core): set-up (problem, b~, DSA
    V-cycle hierarchy), then n_warm + n_timed iterations' work, each a V-cycle plus an A~ apply (the MGS and
    least-squares work of an iteration is negligible next to the sweep).  Returns the timings."""
    from oracle import Problem as OProblem, dsa as ODSA, transport as OT
    t0 = time.perf_counter()
    p = OProblem(_one_instance_spec(cfg, nx, ny), 0, np.asarray(ss), np.asarray(sa))
    t1 = time.perf_counter()
    bt = OT.rhs_btilde(p)
    t2 = time.perf_counter()
    mg = ODSA.MultigridDsa(p, "partial")
    t3 = time.perf_counter()
    v = bt / np.linalg.norm(bt)
    per = []
    for k in range(n_warm + n_timed):
        a = time.perf_counter()
        z = mg.apply(v)
        w = OT.Atilde_apply(p, z)
        v = w / np.linalg.norm(w)
        if k >= n_warm:
            per.append(time.perf_counter() - a)
    return {"problem": t1 - t0, "btilde": t2 - t1, "setup": t3 - t2, "iters": per}


def oracle_baseline(cfg: int, spec, ss, sa, iters_needed: float, n_warm: int, n_timed: int, cores: int):
    """The CPU oracle on all host cores: one instance per core, solved concurrently (a spawned process each), a
    bounded sample per process extrapolated to a full FGMRES-DSA solve (set-up, b~, iters_needed iterations, one
    residual).  Throughput = cores / extrapolated solve time."""
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        jobs = [pool.apply_async(oracle_sample_worker, (cfg, spec.nx[i % len(spec.nx)], spec.ny[i % len(spec.ny)],
                                                        ss[i % len(ss)], sa[i % len(sa)], n_warm, n_timed))
                for i in range(cores)]
        res = [j.get() for j in jobs]
    wall = time.perf_counter() - t0
    per_iter = statistics.median(x for r in res for x in r["iters"])
    fixed = statistics.median(r["problem"] + 2 * r["btilde"] + r["setup"] for r in res)
    solve_s = fixed + iters_needed * per_iter
    return {"value": cores / solve_s, "unit": "param solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} concurrent one-core oracle processes, one {spec.nx[0]}x{spec.ny[0]} instance each: "
                      f"problem + b~ + DSA V-cycle set-up + {n_warm + n_timed} FGMRES-DSA iterations' work "
                      f"({wall:.1f} s wall); extrapolated to {iters_needed:.1f} iterations + 1 residual sweep "
                      f"({solve_s:.1f} s per solve, {per_iter:.2f} s per iteration)",
            "per_iter_s": per_iter, "solve_s": solve_s, "per_iter_samples": [x for r in res for x in r["iters"]]}


# FP64 GPU iteration count of each workload's solve, for the reference arm's extrapolation (the reference arm
# runs before the GPU arm and cannot read it); the GPU arm's cpu_baseline uses its own measured count.
REF_ITERS = {5: 37.0, 3: 15.3, 2: 16.0, 1: 10.0}


def run_reference(args, spec, B, world, rank, cfg):
    """The reference arm: the CPU oracle as it stands, on the workload of the GPU arm (bounded sample)."""
    if rank != 0:
        return
    t_start = time.perf_counter()
    ss, sa = wl.draw_params(spec, max(B, 1), wl.seed_for(cfg, 1))
    cores = min(host_cores(), args.ref_cores or host_cores())
    iters = args.ref_iters if args.ref_iters is not None else REF_ITERS.get(cfg, 20.0)
    cb = oracle_baseline(cfg, spec, ss, sa, iters, args.warmup, args.steps, cores)
    value = cb["value"]
    per = cb.pop("per_iter_samples")
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "param solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(per), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, spec, B, cfg),
            "cpu_baseline": dict(cb, value=value),
            "e2e": {"value": value, "unit": "param solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line))


def bench_config(args, spec, B, cfg):
    """The workload description both arms print (no model keys: the workload is named by its sizes)."""
    meshes = {}
    for nx, ny in zip(spec.nx, spec.ny):
        meshes[f"{nx}x{ny}"] = meshes.get(f"{nx}x{ny}", 0) + 1
    return {"workload": args.workload, "instances_per_step": B,
            "mesh": ", ".join(f"{c} x {m}" for m, c in meshes.items()),
            "directions": spec.n_directions, "regions": f"{spec.rx}x{spec.ry}",
            "sigma_s": f"log-uniform {spec.sigma_s_range}", "sigma_a": f"uniform {spec.sigma_a_range}",
            "restart": spec.restart if args.restart is None else args.restart,
            "preconditioner": f"ROMSAD rank <= {args.rom_rank or spec.rom_rank} (window {spec.window}, greedy with "
                              f"FGMRES-DSA high-fidelity solves), then DSA (partially consistent, one multigrid "
                              f"V-cycle)",
            "warm_start": f"MLP {2 * spec.n_regions}-128-128-r (mixed path only)",
            "l2": "flushed (256 MiB write) before every timed step"}


# ------------------------------------------------------------------ GPU helpers
def time_events(torch, stream, fn, reps=5, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def phi_error(phi, ref):
    """Scalar-flux error against the oracle: relative l2 and max-abs over the reference's max-abs."""
    if ref is None or phi is None:
        return None
    d = np.asarray(phi) - np.asarray(ref)
    return {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)),
            "max_abs_over_linf": float(np.max(np.abs(d)) / np.max(np.abs(ref)))}


def build_rom_and_mlp(RB, spec, cfg, args, n_train, rank_cap, restart, seed_net=2410, max_greedy=None):
    """Offline (untimed): greedy ROM on the training draws (FGMRES-DSA high-fidelity solves), MLP trained on its
    Galerkin-coefficient labels, attached to the ROM."""
    R = spec.n_regions
    t0 = time.perf_counter()
    tr_ss, tr_sa = wl.draw_params(spec, n_train, wl.seed_for(cfg, 0))
    tmpl = RB.Problem(spec.with_instances(spec.nx[:1], spec.ny[:1]), tr_ss[:1], tr_sa[:1])
    rom, rep = RB.Rom.greedy(tmpl, tr_ss, tr_sa, window=spec.window,
                             max_greedy_iter=max_greedy or max(1, rank_cap // spec.window), max_rank=rank_cap,
                             eps_rom=0.0, hf_rtol=1e-10, hf_restart=restart, hf_max_iter=args.max_iter,
                             want_labels=True, indicator_f32=True, hf_dsa=spec.dim == 2)
    t_greedy = time.perf_counter() - t0
    net = RB.Mlp(2 * R, 128, rep["rank"], seed=seed_net)
    loss = net.train(np.concatenate([tr_ss, tr_sa], axis=1), rep["labels"], epochs=args.mlp_epochs,
                     batch=min(64, n_train), lr=2e-3, bf16=True)
    RB.attach_mlp(rom, net)
    info = {"greedy_s": t_greedy, "total_s": time.perf_counter() - t0, "training_draws": n_train,
            "rank": rep["rank"], "sampled": len(rep["sampled"]),
            "max_indicator_last": [x for x in rep["max_indicator"] if x == x][-1:], "mlp_final_loss": loss}
    return rom, net, tmpl, rep, (tr_ss, tr_sa), info


def solve_stats(st):
    return {"iterations_mean": statistics.mean(s["iterations"] for s in st),
            "iterations_max": max(s["iterations"] for s in st),
            "sweeps_fp64_mean": statistics.mean(s["sweeps_fp64"] for s in st),
            "sweeps_df_mean": statistics.mean(s["sweeps_df"] for s in st),
            "converged": sum(1 for s in st if s["status"] == 0), "of": len(st),
            "escalated_to_fp64": sum(s["escalated"] for s in st),
            "true_rel_residual_max": max(s["true_rel_residual"] for s in st)}


# ------------------------------------------------------------------ extras (single GPU)
def measure_sweep_hbm(RB, torch, dev, stream, flush, cfg, reps=5):
    """Angular-output sweep (rte_sweep, FP32) over a whole batched workload: an HBM-bound write of
    N_Omega * N_dof * 4 bytes (both duplicate directions stored), timed with CUDA events after warm-up."""
    spec = wl.config(cfg)
    ss, sa = wl.draw_params(spec, spec.n_instances, wl.seed_for(cfg, 1))
    prob = RB.Problem(spec, ss, sa)
    n = prob.n_dof
    src = torch.randn(n, dtype=torch.float32, device=dev)
    psi = torch.empty(prob.n_directions * n, dtype=torch.float32, device=dev)
    for _ in range(3):
        prob.sweep(src, psi, with_bc=True, stream=stream)
    times = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prob.sweep(src, psi, with_bc=True, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    nbytes = prob.n_directions * n * 4 + n * 4
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    cells = sum(nx * ny for nx, ny in zip(spec.nx, spec.ny))
    meshes = {}
    for nx, ny in zip(spec.nx, spec.ny):
        meshes[f"{nx}x{ny}"] = meshes.get(f"{nx}x{ny}", 0) + 1
    desc = ", ".join(f"{c}x{m}" for m, c in meshes.items())
    out = {"workload": f"{spec.name} ({desc}; {prob.n_directions} directions, {spec.n_regions} regions)",
           "kernel": "k_sweep2d / k_sweep2d_bands (angular output, FP32; autotuned)",
           "bytes": nbytes, "ms": ms, "achieved_gbs": nbytes / (ms * 1e-3) / 1e9, "peak_gbs": peak,
           "frac": nbytes / (ms * 1e-3) / 1e9 / peak,
           "alu_tflops": SWEEP_FLOPS_PER_CELL_DIR * cells * prob.info.n_unique_directions / (ms * 1e-3) / 1e12}
    del psi, prob
    torch.cuda.empty_cache()
    return out


def measure_batched(RB, torch, dev, stream, flush, args, refs, reps=1):
    """Batched throughput on the 256-instance uneven workload (96 x 32^2, 96 x 64^2, 64 x 128^2), one solve call per
    batch: mixed with the learned start vs plain FP64, each mesh group preconditioned by its own greedy ROM, whose
    labels train that group's MLP (offline, untimed).  Scalar-flux errors on one instance of each mesh size."""
    spec3 = wl.config(3)
    B = spec3.n_instances
    ss, sa = wl.draw_params(spec3, B, wl.seed_for(3, 1))
    prob = RB.Problem(spec3, ss, sa)
    t0 = time.perf_counter()
    roms, losses = {}, {}
    for n in sorted(set(spec3.nx)):
        sp = spec3.with_instances([n], [n])
        rom, net, _, rep, _, info = build_rom_and_mlp(RB, sp, 3, args, args.batched_train, args.batched_rank,
                                                      spec3.restart, seed_net=2410 + n)
        roms[n] = (rom, net)
        losses[f"{n}x{n}"] = info["mlp_final_loss"]
    t_off = time.perf_counter() - t0
    rl = [roms[n][0] for n in spec3.nx]
    phi = torch.zeros(prob.n_dof, dtype=torch.float64, device=dev)
    out = {"workload": "batch256_uneven: 96x32^2 + 96x64^2 + 64x128^2, 128 directions, one solve call per batch",
           "instances": B, "rom_rank": args.batched_rank, "training_draws": args.batched_train, "offline_s": t_off,
           "mlp_final_loss": losses}
    sample_ids = REF_SAMPLES_C3
    for name, mode, learned in (("mixed", RB.RTE_MODE_MIXED, True), ("mixed_plain_romsad", RB.RTE_MODE_MIXED, False),
                                ("fp64", RB.RTE_MODE_FP64, False)):
        kw = dict(restart=spec3.restart, rtol=1e-8, max_iter=args.max_iter, window=spec3.window, mode=mode,
                  inner_rtol=args.inner_rtol, max_outer=30, stream=stream, raise_on_fail=False,
                  learned_warm_start=learned, post_mode=RB.RTE_POST_DSA)
        RB.fgmres_solve(prob, rl, phi, **kw)   # warm-up / tuning
        times, st_all = [], []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = RB.fgmres_solve(prob, rl, phi, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            st_all.extend(st)
        ms = statistics.mean(times)
        conv = sum(1 for s in st_all if s["status"] == 0) / reps
        host = phi.cpu().numpy()
        errs = {}
        for i in sample_ids:
            ref = refs.get(("c3", i))
            seg = host[prob.offsets[i]:prob.offsets[i + 1]]
            errs[f"instance {i} ({spec3.nx[i]}x{spec3.ny[i]})"] = phi_error(seg, ref)
        out[name] = dict({"value": conv / (ms * 1e-3), "unit": "param solves/s", "ms_per_batch": ms},
                         **solve_stats(st_all), phi_rel_err_vs_oracle=errs)
    out["speedup_mixed_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    del phi, prob
    torch.cuda.empty_cache()
    return out


def measure_single(RB, torch, dev, stream, flush, args, refs, n_steps=4):
    """The single-instance 64x64 workload (square2d_64): one instance per step, the method's variants side by side
    (mixed + MLP start, FP64, plain ROMSAD, learned slot, GMRES-DSA, RBF-interpolated start, SI-ROMSAD)."""
    spec = wl.config(2)
    ss_all, sa_all = wl.draw_params(spec, n_steps + 1, wl.seed_for(2, 1))
    prob = RB.Problem(spec, ss_all[:1], sa_all[:1])
    phi = torch.zeros(prob.n_dof, dtype=torch.float64, device=dev)
    rom, net, tmpl, rep, (tr_ss, tr_sa), info = build_rom_and_mlp(RB, spec, 2, args, args.single_train, spec.rom_rank,
                                                                   spec.restart)
    roms = [rom]
    base = dict(restart=spec.restart, rtol=1e-8, max_iter=args.max_iter, window=spec.window, stream=stream,
                raise_on_fail=False)
    legs = {
        "mixed": lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_MIXED, inner_rtol=args.inner_rtol,
                                         max_outer=30, learned_warm_start=True, post_mode=RB.RTE_POST_DSA, **base),
        "fp64": lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_FP64, post_mode=RB.RTE_POST_DSA, **base),
        "mixed_plain_romsad": lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_MIXED,
                                                      inner_rtol=args.inner_rtol, max_outer=30,
                                                      post_mode=RB.RTE_POST_DSA, **base),
        "mixed_learned_slot": lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_MIXED,
                                                      inner_rtol=args.inner_rtol, max_outer=30, learned_slot=True,
                                                      post_mode=RB.RTE_POST_DSA, **base),
        "gmres_dsa_mixed": lambda: RB.fgmres_solve(prob, None, phi, mode=RB.RTE_MODE_MIXED, inner_rtol=args.inner_rtol,
                                                   max_outer=30, post_mode=RB.RTE_POST_DSA, **base),
        "si_romsad_fp64": lambda: RB.si_solve(prob, roms, phi, rtol=1e-8, max_iter=2000, window=spec.window,
                                              post_mode=RB.RTE_POST_DSA, stream=stream, raise_on_fail=False),
    }
    # the paper's interpolation baseline: RBF interpolation of the FP64 solutions at the greedy's samples
    try:
        ks = list(rep["sampled"])
        spec_k = spec.with_instances([spec.nx[0]] * len(ks), [spec.ny[0]] * len(ks))
        pk = RB.Problem(spec_k, tr_ss[ks], tr_sa[ks])
        sol_k = torch.zeros(pk.n_dof, dtype=torch.float64, device=dev)
        RB.fgmres_solve(pk, None, sol_k, restart=spec.restart, rtol=1e-10, max_iter=args.max_iter,
                        post_mode=RB.RTE_POST_DSA, stream=stream)
        rbf = RB.Rbf(tmpl, tr_ss[ks], tr_sa[ks], sol_k.view(len(ks), -1))
        phi0_ig = torch.zeros(prob.n_dof, dtype=torch.float64, device=dev)

        def interp_solve():
            rbf.initial_guess(prob, phi0_ig, stream=stream)
            return RB.fgmres_solve(prob, None, phi, phi0=phi0_ig, mode=RB.RTE_MODE_MIXED, inner_rtol=args.inner_rtol,
                                   max_outer=30, post_mode=RB.RTE_POST_DSA, **base)
        legs["gmres_dsa_interp_ig_mixed"] = interp_solve
    except Exception as exc:   # a side measurement; report instead of losing the bench line
        legs_err = f"{type(exc).__name__}: {exc}"
    else:
        legs_err = None
    out = {"workload": "square2d_64: one 64x64 instance per step, 128 directions, 2x2 regions",
           "offline": info}
    ref = refs.get(("c2", 1))
    for name, fn in legs.items():
        times, st_all, err = [], [], None
        for s in range(n_steps + 1):
            prob.set_params(ss_all[s:s + 1], sa_all[s:s + 1])
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if s >= 1:
                times.append(e0.elapsed_time(e1))
                st_all.extend(st)
            if s == 1:
                err = phi_error(phi.cpu().numpy(), ref)
        out[name] = dict({"value": len(times) / (sum(times) * 1e-3), "unit": "param solves/s"},
                         **solve_stats(st_all), phi_rel_err_vs_oracle=err)
    if legs_err:
        out["gmres_dsa_interp_ig_mixed"] = {"error": legs_err}
    del phi, prob
    torch.cuda.empty_cache()
    return out


def measure_learned_eval(RB, torch, dev, stream, flush, args, n_test=512):
    """The learned part on the 64x64 workload with the config-4 budget: the greedy runs over 2048 training draws,
    whose Galerkin coefficients train the MLP; 512 held-out draws (seeded test split) are solved in one
    mixed-precision call with the learned warm start, with the learned ROMSAD slot, and with plain ROMSAD."""
    spec = wl.config(4)
    rom, net, tmpl, rep, (tr_ss, tr_sa), info = build_rom_and_mlp(RB, spec, 4, args, spec.n_train, spec.rom_rank,
                                                                   spec.restart)
    # held-out label error: the network's prediction against the Galerkin coefficients on the final basis
    ts, ta = wl.draw_params(spec, n_test, wl.seed_for(4, 1))
    sp = spec.with_instances([spec.nx[0]] * n_test, [spec.ny[0]] * n_test)
    prob = RB.Problem(sp, ts, ta)
    phi = torch.zeros(prob.n_dof, dtype=torch.float64, device=dev)
    roms = [rom] * n_test
    out = {"workload": f"{n_test} held-out draws of the 64x64 workload in one batched call", "instances": n_test,
           "offline": info}
    try:
        labels = rom.galerkin_coefficients(prob)
        pred = net.infer(np.concatenate([ts, ta], axis=1))
        out["label_rel_err_heldout"] = float(np.linalg.norm(pred - labels) / np.linalg.norm(labels))
    except Exception as exc:
        out["label_rel_err_heldout"] = f"{type(exc).__name__}: {exc}"
    for name, kw in (("learned_start", {"learned_warm_start": True}), ("learned_slot", {"learned_slot": True}),
                     ("plain_romsad", {})):
        common = dict(restart=spec.restart, rtol=1e-8, max_iter=args.max_iter, window=spec.window,
                      mode=RB.RTE_MODE_MIXED, inner_rtol=args.inner_rtol, max_outer=30, stream=stream,
                      raise_on_fail=False, post_mode=RB.RTE_POST_DSA, **kw)
        RB.fgmres_solve(prob, roms, phi, **common)   # warm-up / tuning
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = RB.fgmres_solve(prob, roms, phi, **common)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        conv = sum(1 for s in st if s["status"] == 0)
        out[name] = dict({"value": conv / (ms * 1e-3), "unit": "param solves/s"}, **solve_stats(st))
    out["learned_start_vs_plain"] = out["learned_start"]["value"] / out["plain_romsad"]["value"]
    del phi, prob
    torch.cuda.empty_cache()
    return out


def measure_pincell(RB, torch, dev, stream, flush, args, n_test=10):
    """The paper's pin-cell problem (Sec. 5), where it reports FGMRES-ROMSAD's gain over GMRES-DSA: [-1,1]^2, 80x80,
    CL(30, 6) = 180 directions, Gaussian source exp(-100 r^2), sigma_s = 100 outside the inner square and
    (sigma_a, sigma_s) = (mu_a, mu_s) in [0.05, 0.5]^2 inside.  Greedy ROM over a 5 x 5 training grid (FGMRES-DSA
    high-fidelity solves, eps_ROM = 1e-10, window 2, rank <= 64), then n_test seeded test parameters solved in one
    batched call to relative residual 1e-11 (FP64, as in the paper) and to FP64 true residual 1e-8 (mixed), by
    FGMRES-ROMSAD with DSA after the window and by GMRES-DSA: sweeps per solve and solves/s."""
    spec = wl.pincell()
    grid = [(a, s_) for a in np.linspace(0.05, 0.5, 5) for s_ in np.linspace(0.05, 0.5, 5)]
    tr = [wl.pincell_params(a, s_) for a, s_ in grid]
    tr_ss, tr_sa = np.array([x[0] for x in tr]), np.array([x[1] for x in tr])
    t0 = time.perf_counter()
    tmpl = RB.Problem(spec, tr_ss[:1], tr_sa[:1])
    rom, rep = RB.Rom.greedy(tmpl, tr_ss, tr_sa, window=2, max_greedy_iter=25, max_rank=64, eps_rom=1e-10,
                             hf_rtol=1e-12, hf_restart=30, hf_max_iter=args.max_iter, hf_dsa=True)
    t_off = time.perf_counter() - t0
    pts = wl.draw_box(n_test, [0.05, 0.05], [0.5, 0.5], wl.seed_for(6, 1))
    te = [wl.pincell_params(a, s_) for a, s_ in pts]
    ts, ta = np.array([x[0] for x in te]), np.array([x[1] for x in te])
    sp = spec.with_instances([spec.nx[0]] * n_test, [spec.ny[0]] * n_test)
    prob = RB.Problem(sp, ts, ta)
    phi = torch.zeros(prob.n_dof, dtype=torch.float64, device=dev)
    out = {"workload": f"pin-cell 80x80, CL(30, 6) = 180 directions, {n_test} test parameters in one batched call",
           "offline": {"greedy_s": t_off, "rank": rep["rank"], "sampled": len(rep["sampled"]),
                       "max_indicator_last": [x for x in rep["max_indicator"] if x == x][-1:]}}
    legs = (("fgmres_romsad_fp64", [rom] * n_test, RB.RTE_MODE_FP64, 1e-11),
            ("gmres_dsa_fp64", None, RB.RTE_MODE_FP64, 1e-11),
            ("fgmres_romsad_mixed", [rom] * n_test, RB.RTE_MODE_MIXED, 1e-8),
            ("gmres_dsa_mixed", None, RB.RTE_MODE_MIXED, 1e-8))
    for name, roms, mode, rtol in legs:
        kw = dict(restart=30, rtol=rtol, max_iter=args.max_iter, window=2, mode=mode, inner_rtol=args.inner_rtol,
                  max_outer=30, stream=stream, raise_on_fail=False, post_mode=RB.RTE_POST_DSA)
        RB.fgmres_solve(prob, roms, phi, **kw)   # warm-up / tuning
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = RB.fgmres_solve(prob, roms, phi, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        conv = sum(1 for x in st if x["status"] == 0)
        out[name] = dict({"value": conv / (ms * 1e-3), "unit": "param solves/s", "rtol": rtol,
                          "sweeps_mean": statistics.mean(x["sweeps"] for x in st)}, **solve_stats(st))
    out["sweeps_romsad_over_dsa_fp64"] = out["fgmres_romsad_fp64"]["sweeps_mean"] / out["gmres_dsa_fp64"]["sweeps_mean"]
    out["paper_context"] = ("paper (hardware unstated): mean sweeps 5.1 FGMRES-ROMSAD vs 15.5 GMRES-DSA, rank 44, "
                            "relative time 30.05 %")
    del phi, prob
    torch.cuda.empty_cache()
    return out


def measure_varscat(RB, torch, dev, stream, flush, args, n_test=10):
    """The paper's variable-scattering problem (Sec. 5): [-1,1]^2, 80x80, CL(30, 6), Gaussian source
    (10/pi) exp(-100 r^2), sigma_a = 0, sigma_s = mu_s r^4 (2 - r^2)^2 + 0.1 inside the unit disc and mu_s + 0.1
    outside, so Sigma is a full 4x4 block per cell.  Greedy ROM over 51 uniform training points of mu_s in
    [49.9, 99.9] starting at 74.9 (FGMRES-DSA high-fidelity solves, eps_ROM = 1e-9, window 2), then n_test seeded
    test points in one batched call to relative residual 1e-11 (FP64) and to FP64 true residual 1e-8 (mixed, FP64
    refinement residuals), FGMRES-ROMSAD with DSA after the window against GMRES-DSA."""
    spec = wl.variable_scattering()
    train = np.linspace(49.9, 99.9, 51)
    tr_ss = np.array([wl.variable_scattering_params(m)[0] for m in train])
    tr_sa = np.array([wl.variable_scattering_params(m)[1] for m in train])
    t0 = time.perf_counter()
    tmpl = RB.Problem(spec, tr_ss[:1], tr_sa[:1])
    rom, rep = RB.Rom.greedy(tmpl, tr_ss, tr_sa, window=2, max_greedy_iter=25, max_rank=64, eps_rom=1e-9,
                             mu1=25, hf_rtol=1e-12, hf_restart=30, hf_max_iter=args.max_iter, hf_dsa=True)
    t_off = time.perf_counter() - t0
    mus = wl.draw_box(n_test, [49.9], [99.9], wl.seed_for(7, 1))[:, 0]
    ts = np.array([wl.variable_scattering_params(m)[0] for m in mus])
    ta = np.array([wl.variable_scattering_params(m)[1] for m in mus])
    sp = spec.with_instances([spec.nx[0]] * n_test, [spec.ny[0]] * n_test)
    prob = RB.Problem(sp, ts, ta)
    phi = torch.zeros(prob.n_dof, dtype=torch.float64, device=dev)
    out = {"workload": f"variable scattering 80x80, CL(30, 6), {n_test} test values of mu_s in one batched call",
           "offline": {"greedy_s": t_off, "rank": rep["rank"], "sampled": len(rep["sampled"]),
                       "max_indicator_last": [x for x in rep["max_indicator"] if x == x][-1:]}}
    legs = (("fgmres_romsad_fp64", [rom] * n_test, RB.RTE_MODE_FP64, 1e-11),
            ("gmres_dsa_fp64", None, RB.RTE_MODE_FP64, 1e-11),
            ("fgmres_romsad_mixed", [rom] * n_test, RB.RTE_MODE_MIXED, 1e-8),
            ("gmres_dsa_mixed", None, RB.RTE_MODE_MIXED, 1e-8))
    for name, roms, mode, rtol in legs:
        kw = dict(restart=30, rtol=rtol, max_iter=args.max_iter, window=2, mode=mode, inner_rtol=args.inner_rtol,
                  max_outer=30, stream=stream, raise_on_fail=False, post_mode=RB.RTE_POST_DSA,
                  refine_residual=RB.RTE_RESIDUAL_FP64)
        RB.fgmres_solve(prob, roms, phi, **kw)   # warm-up / tuning
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = RB.fgmres_solve(prob, roms, phi, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        conv = sum(1 for x in st if x["status"] == 0)
        out[name] = dict({"value": conv / (ms * 1e-3), "unit": "param solves/s", "rtol": rtol,
                          "sweeps_mean": statistics.mean(x["sweeps"] for x in st)}, **solve_stats(st))
    out["sweeps_romsad_over_dsa_fp64"] = out["fgmres_romsad_fp64"]["sweeps_mean"] / out["gmres_dsa_fp64"]["sweeps_mean"]
    out["speedup_romsad_over_dsa_fp64"] = out["fgmres_romsad_fp64"]["value"] / out["gmres_dsa_fp64"]["value"]
    out["paper_context"] = ("paper (hardware unstated, PC-DSA): 8 parameters sampled, rank 16; FGMRES-ROMSAD 4.7 sweeps "
                            "on average, at least 3.11x faster than GMRES-DSA")
    del phi, prob
    torch.cuda.empty_cache()
    return out


# instances whose oracle solutions the extras compare against: config 3, one per mesh size
REF_SAMPLES_C3 = (0, 96, 192)


def start_oracle_refs(cfg, spec, B, args, world):
    """Spawn the oracle's tight solves of the sampled instances (before any GPU call); returns (pool, jobs)."""
    jobs_spec = []
    n_sets = args.warmup + args.steps
    ss_all, sa_all = wl.draw_params(spec, n_sets * B * world, wl.seed_for(cfg, 1))
    i0, _ = shard(0, n_sets, B, args.warmup)   # instance 0 of rank 0's first timed step
    jobs_spec.append((("head", 0), cfg, spec.nx[0], spec.ny[0], ss_all[i0], sa_all[i0]))
    if not args.no_extras:
        s3 = wl.config(3)
        ss3, sa3 = wl.draw_params(s3, s3.n_instances, wl.seed_for(3, 1))
        for i in REF_SAMPLES_C3:
            jobs_spec.append((("c3", i), 3, s3.nx[i], s3.ny[i], ss3[i], sa3[i]))
        s2 = wl.config(2)
        ss2, sa2 = wl.draw_params(s2, 2, wl.seed_for(2, 1))
        jobs_spec.append((("c2", 1), 2, s2.nx[0], s2.ny[0], ss2[1], sa2[1]))
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(min(len(jobs_spec), max(1, host_cores() - 2)))
    jobs = {key: pool.apply_async(oracle_reference_phi, (c, nx, ny, ss, sa)) for key, c, nx, ny, ss, sa in jobs_spec}
    return pool, jobs


def collect_refs(pool, jobs, timeout_s):
    refs, meta = {}, {}
    t_end = time.perf_counter() + timeout_s
    for key, job in jobs.items():
        try:
            r = job.get(timeout=max(1.0, t_end - time.perf_counter()))
            refs[key] = r["phi"]
            meta[f"{key[0]}:{key[1]}"] = {"iterations": r["iterations"], "s": r["s"]}
        except Exception as exc:   # no reference: the error is reported as missing, not invented
            meta[f"{key[0]}:{key[1]}"] = {"error": f"{type(exc).__name__}: {exc}"}
    pool.terminate()
    pool.join()
    return refs, meta


def profile_target(args):
    """One launch of a kernel of the headline path inside the NVTX range "profile" (for ncu --nvtx-include
    "profile/"), after its autotuning and warm-up: the A~ apply in FP32, FP64 or double-float on the first
    --profile-instances instances of the workload, the DSA V-cycle (set-up reused), or the tensor-core ROMSAD apply
    (romsad_apply with FP32 vectors, a rank-32 orthonormal basis on 128x128 meshes with 32 directions)."""
    import torch
    from paper_2410_08735_gb300 import binding as RB
    RB.load()
    spec, B, cfg = workload_spec(args.workload)
    nb = max(1, min(args.profile_instances, B))
    what = args.profile
    if what == "rom_tc":
        spec = dataclasses.replace(wl.config(2), n_polar=2, n_azim=16).with_instances([128] * nb, [128] * nb)
    else:
        spec = spec.with_instances(spec.nx[:nb], spec.ny[:nb])
    ss, sa = wl.draw_params(spec, nb, wl.seed_for(cfg, 1))
    prob = RB.Problem(spec, ss, sa)
    if args.profile_pin:   # the kernel instantiation the full-size workload's autotuner picked
        var, D = (int(x) for x in args.profile_pin.split(","))
        prob.set_sweep_variant(var, D)
    z = torch.randn(prob.n_dof, dtype=torch.float64, device="cuda")
    w = torch.empty_like(z)
    z32, w32 = z.float(), torch.empty(prob.n_dof, dtype=torch.float32, device="cuda")
    if what == "rom_tc":
        one = RB.Problem(spec.with_instances(spec.nx[:1], spec.ny[:1]), ss[:1], sa[:1])
        n_a = spec.n_directions * prob.n_dof // nb
        U, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((n_a, 32)))
        rom = RB.Rom.from_basis(one, np.ascontiguousarray(U.T.reshape(32, spec.n_directions, -1)), instance=0)
        fn = lambda: rom.apply(prob, z32, w32)
    elif what == "dsa":
        prob.dsa_apply(z32, w32)
        fn = lambda: prob.dsa_apply(z32, w32, variant=RB.RTE_DSA_KEEP_SETUP)
    elif what == "sweep_f32":
        fn = lambda: prob.apply_op(z32, w32)
    elif what == "sweep_f64":
        fn = lambda: prob.apply_op(z, w)
    else:
        fn = lambda: prob.apply_op(z, w, double_float=True)
    for _ in range(2):   # autotuning and warm-up
        fn()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("profile")
    fn()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"profile": what, "instances": nb, "n_dof": prob.n_dof}))


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large256_192", choices=sorted(WORKLOADS))
    ap.add_argument("--restart", type=int, default=None, help="restart length (default: the workload's)")
    ap.add_argument("--max-iter", type=int, default=6000)
    ap.add_argument("--inner-rtol", type=float, default=1e-3, help="inner target of the mixed refinement")
    ap.add_argument("--n-train", type=int, default=None, help="greedy/MLP training draws (default: the workload's)")
    ap.add_argument("--rom-rank", type=int, default=0, help="ROM rank cap (0: the workload's)")
    ap.add_argument("--mlp-epochs", type=int, default=300)
    ap.add_argument("--batched-train", type=int, default=64)
    ap.add_argument("--batched-rank", type=int, default=32)
    ap.add_argument("--single-train", type=int, default=64)
    ap.add_argument("--no-extras", action="store_true", help="headline workload only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-ref", action="store_true", help="skip the oracle's reference solutions")
    ap.add_argument("--oracle-timeout", type=float, default=900.0)
    ap.add_argument("--ref-iters", type=float, default=None,
                    help="reference arm: iterations of a full solve for the extrapolation (default: the GPU's FP64 "
                         "count on this workload)")
    ap.add_argument("--ref-cores", type=int, default=0, help="reference arm: oracle processes (0: all host cores)")
    ap.add_argument("--profile", default=None, choices=["sweep_f32", "sweep_f64", "sweep_df", "dsa", "rom_tc"],
                    help="run one launch of that kernel inside the NVTX range 'profile' (an ncu target) and exit")
    ap.add_argument("--profile-instances", type=int, default=16)
    ap.add_argument("--profile-pin", default=None, help="with --profile: pin the sweep kernel as 'variant,D'")
    args = ap.parse_args()
    if args.profile:
        profile_target(args)
        return
    spec, B, cfg = workload_spec(args.workload)
    restart = spec.restart if args.restart is None else args.restart
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, spec, B, world, rank, cfg)
        return
    # the oracle's reference solutions run in spawned processes while the GPU legs run (started before the
    # first GPU call); rank 0 only
    pool, jobs = (None, {})
    if rank == 0 and world == 1 and not args.no_oracle_ref:
        pool, jobs = start_oracle_refs(cfg, spec, B, args, world)
    import torch
    from paper_2410_08735_gb300 import binding as RB
    RB.load()                                   # fails loudly without the built CUDA library
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    R = spec.n_regions
    n_sets = args.warmup + args.steps
    ss_all, sa_all = wl.draw_params(spec, n_sets * B * world, wl.seed_for(cfg, 1))

    def params(step):
        i0, i1 = shard(rank, n_sets, B, step)
        return ss_all[i0:i1], sa_all[i0:i1]

    peaks = {"fp32_fma_tflops": RB.fma_peak(RB.RTE_F32, stream), "fp64_fma_tflops": RB.fma_peak(RB.RTE_F64, stream),
             "source": "rte_fma_peak: 8 independent FMA chains per thread, 8 blocks of 256 threads per SM, best of "
                       "3 launches (CUDA events)"}
    hbm_peak = measured_peaks().get("hbm_gbs")
    ss0, sa0 = params(0)
    prob = RB.Problem(spec, ss0, sa0)
    n = prob.n_dof
    off = prob.offsets
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # offline (untimed): greedy ROM with FGMRES-DSA high-fidelity solves, MLP trained on its labels
    n_train = args.n_train or spec.n_train
    meshes = sorted(set(zip(spec.nx[:B], spec.ny[:B])))
    if len(meshes) == 1:
        rom, net, tmpl, rep, _, offline = build_rom_and_mlp(RB, spec, cfg, args, n_train,
                                                            args.rom_rank or spec.rom_rank, restart)
        roms = [rom] * B
    else:
        # uneven meshes: one greedy ROM (and MLP) per mesh size, each instance preconditioned by its mesh's ROM
        per, offline = {}, {}
        for (mx, my) in meshes:
            sp = spec.with_instances([mx], [my])
            per[(mx, my)] = build_rom_and_mlp(RB, sp, cfg, args, n_train, args.rom_rank or spec.rom_rank, restart,
                                              seed_net=2410 + mx)
            offline[f"{mx}x{my}"] = per[(mx, my)][5]
        roms = [per[(spec.nx[i], spec.ny[i])][0] for i in range(B)]
    common = dict(restart=restart, rtol=1e-8, max_iter=args.max_iter, window=spec.window, stream=stream,
                  raise_on_fail=False, post_mode=RB.RTE_POST_DSA)
    mixed_kw = dict(inner_rtol=args.inner_rtol, max_outer=30)
    legs = [
        # headline: all-FP32 inner solves, learned start, double-float refinement residuals, FP64 certification
        ("mixed", lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_MIXED, learned_warm_start=True,
                                          **mixed_kw, **common)),
        # the same with the ROM window's projection and lift on the tensor cores (BF16 operands, FP32 accumulation)
        ("mixed_rom_bf16", lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_MIXED, learned_warm_start=True,
                                                   rom_bf16=True, **mixed_kw, **common)),
        # the precision form of the method statement: FP32 sweeps, FP64 Krylov vectors, MGS and Givens
        ("mixed_fp64_krylov", lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_MIXED_F64KRYLOV,
                                                      learned_warm_start=True, **mixed_kw, **common)),
        ("fp64", lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_FP64, true_residual_check=True, **common)),
        ("mixed_plain_romsad", lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_MIXED, **mixed_kw,
                                                       **common)),
        ("mixed_fp64_residuals", lambda: RB.fgmres_solve(prob, roms, phi, mode=RB.RTE_MODE_MIXED,
                                                         learned_warm_start=True, refine_residual=RB.RTE_RESIDUAL_FP64,
                                                         **mixed_kw, **common)),
        ("gmres_dsa_mixed", lambda: RB.fgmres_solve(prob, None, phi, mode=RB.RTE_MODE_MIXED, **mixed_kw, **common)),
    ]

    def timed_loop(fn, tag):
        per_step, stats_all, phi_s = [], [], None
        for s in range(n_sets):
            ss, sa = params(s)
            prob.set_params(ss, sa)
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if s >= args.warmup:   # ncu --nvtx-include "timed_mixed/" selects the timed steps of a leg
                torch.cuda.nvtx.range_push(f"timed_{tag}")
            e0.record(stream)
            st = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if s >= args.warmup:
                torch.cuda.nvtx.range_pop()
            if s >= args.warmup:
                per_step.append(e0.elapsed_time(e1))
                stats_all.extend(st)
            if s == args.warmup:   # the sampled instance: instance 0 of the first timed step
                phi_s = phi[off[0]:off[1]].cpu().numpy()
        return per_step, stats_all, phi_s

    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    results = {}
    launches = None
    for name, fn in legs:
        l0 = RB.kernel_launches()
        t, st, phi_s = timed_loop(fn, name)
        if name == "mixed":
            launches = (RB.kernel_launches() - l0) * args.steps / n_sets
        results[name] = (max_over_ranks(world, sum(t) / 1e3), st, phi_s)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    solves = args.steps * B * world
    # e2e: host parameters in, host scalar flux out, through the C ABI
    host_phi = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    e2e_ms = []
    for s in range(n_sets):
        ss, sa = params(s)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.set_params(ss, sa)
        RB.fgmres_solve(prob, roms, host_phi, mode=RB.RTE_MODE_MIXED, learned_warm_start=True, **mixed_kw, **common)
        t1 = time.perf_counter()
        if s >= args.warmup:
            e2e_ms.append(1e3 * (t1 - t0))
    e2e_s = max_over_ranks(world, sum(e2e_ms) / 1e3)
    # per-kernel launch times of the headline path, timed alone with CUDA events on the launching stream:
    # FP32, FP64 and double-float A~ applies, and one DSA V-cycle (set-up reused)
    z64 = torch.randn(n, dtype=torch.float64, device=dev)
    w64 = torch.empty_like(z64)
    z32 = z64.float()
    w32 = torch.empty_like(z32)
    ms32 = time_events(torch, stream, lambda: prob.apply_op(z32, w32, stream=stream), reps=10)
    ms64 = time_events(torch, stream, lambda: prob.apply_op(z64, w64, stream=stream), reps=3)
    msdf = time_events(torch, stream, lambda: prob.apply_op(z64, w64, stream=stream, double_float=True), reps=5)
    prob.dsa_apply(z32, w32, stream=stream)
    ms_v = time_events(torch, stream, lambda: prob.dsa_apply(z32, w32, variant=RB.RTE_DSA_KEEP_SETUP, stream=stream),
                       reps=10)
    cells = sum(nx * ny for nx, ny in zip(spec.nx[:B], spec.ny[:B]))
    nu = prob.info.n_unique_directions
    flops = SWEEP_FLOPS_PER_CELL_DIR * cells * nu
    st_m = results["mixed"][1]
    n64 = statistics.mean(s["sweeps_fp64"] for s in st_m)
    ndf = statistics.mean(s["sweeps_df"] for s in st_m)
    n32 = statistics.mean(s["sweeps"] for s in st_m) - n64 - ndf
    nv = statistics.mean(s["iterations"] for s in st_m)   # one preconditioner apply per iteration
    shares = {"k_sweep2d<float> (A~ apply, FP32)": n32 * ms32, "k_sweep2d<double> (A~ apply, FP64)": n64 * ms64,
              "k_sweep2d<dfloat> (A~ apply, double-float)": ndf * msdf, "k_dsa_vcycle (DSA V-cycle)": nv * ms_v}
    per_solve_ms = 1e3 * results["mixed"][0] / args.steps
    dom = max(shares, key=shares.get)
    if "FP32" in dom:
        roof = {"kernel": dom, "bound": "alu", "achieved": flops / (ms32 * 1e-3) / 1e12,
                "peak": peaks["fp32_fma_tflops"], "unit": "TFLOP/s", "ms_per_launch": ms32}
    elif "FP64" in dom:
        roof = {"kernel": dom, "bound": "alu", "achieved": flops / (ms64 * 1e-3) / 1e12,
                "peak": peaks["fp64_fma_tflops"], "unit": "TFLOP/s", "ms_per_launch": ms64}
    elif "double-float" in dom:
        roof = {"kernel": dom, "bound": "alu", "achieved": flops / (msdf * 1e-3) / 1e12,
                "peak": peaks["fp32_fma_tflops"], "unit": "TFLOP/s", "ms_per_launch": msdf,
                "note": "algorithmic flops in double-float arithmetic against the FP32 FMA peak"}
    else:
        vbytes = DSA_VCYCLE_BYTES_PER_CELL * cells
        roof = {"kernel": dom, "bound": "hbm", "achieved": vbytes / (ms_v * 1e-3) / 1e9, "peak": hbm_peak,
                "unit": "GB/s", "ms_per_launch": ms_v}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof.get("peak") else None
    roof["traffic"] = ncu_traffic(args.workload, dom)
    roof["peak_source"] = "measured: rte_fma_peak (FP32 / FP64 FMA), MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"
    roof["shares_ms_per_solve_batch"] = shares
    roof["solve_batch_ms"] = per_solve_ms
    roof["other_kernels"] = {
        "k_sweep2d<float>": {"ms": ms32, "tflops": flops / (ms32 * 1e-3) / 1e12,
                             "frac_of_fp32_peak": flops / (ms32 * 1e-3) / 1e12 / peaks["fp32_fma_tflops"]},
        "k_sweep2d<double>": {"ms": ms64, "tflops": flops / (ms64 * 1e-3) / 1e12,
                              "frac_of_fp64_peak": flops / (ms64 * 1e-3) / 1e12 / peaks["fp64_fma_tflops"]},
        "k_sweep2d<dfloat>": {"ms": msdf, "tflops_df": flops / (msdf * 1e-3) / 1e12},
        "k_dsa_vcycle": {"ms": ms_v}}
    del z64, w64, z32, w32
    torch.cuda.empty_cache()
    extras = {}
    refs, ref_meta = {}, {}
    if not args.no_extras and world == 1:
        # the extras need the oracle references of configs 2 and 3 only at their end; collect them first when they
        # are already done (they normally are), else after
        extras["sweep_hbm"] = measure_sweep_hbm(RB, torch, dev, stream, flush, 3)
        extras["sweep_hbm"]["large"] = measure_sweep_hbm(RB, torch, dev, stream, flush, 5, reps=3)
    if pool is not None:
        refs, ref_meta = collect_refs(pool, jobs, args.oracle_timeout)
    if not args.no_extras and world == 1:
        extras["batched"] = measure_batched(RB, torch, dev, stream, flush, args, refs)
        extras["single_instance"] = measure_single(RB, torch, dev, stream, flush, args, refs)
        extras["learned_eval"] = measure_learned_eval(RB, torch, dev, stream, flush, args)
        try:
            extras["pincell"] = measure_pincell(RB, torch, dev, stream, flush, args)
        except Exception as exc:   # a side measurement; report instead of losing the bench line
            extras["pincell"] = {"error": f"{type(exc).__name__}: {exc}"}
        try:
            extras["variable_scattering"] = measure_varscat(RB, torch, dev, stream, flush, args)
        except Exception as exc:   # a side measurement; report instead of losing the bench line
            extras["variable_scattering"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank != 0:
        return

    def leg(name):
        t, st, phi_s = results[name]
        return dict({"value": solves / t, "unit": "param solves/s", "ms_per_step": 1e3 * t / args.steps},
                    **solve_stats(st), phi_rel_err_vs_oracle=phi_error(phi_s, refs.get(("head", 0))))

    value = solves / results["mixed"][0]
    fp64_value = solves / results["fp64"][0]
    head = leg("mixed")
    line = {
        "metric": METRIC,
        "value": value, "unit": "param solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * results["mixed"][0] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+df+f64", "data": "synthetic",
        "config": bench_config(args, spec, B, cfg),
        "precision_form": "inner FGMRES all FP32 (sweeps, ROM products, Krylov basis, MGS, Givens); refinement "
                          "residuals double-float; b~ and the certifying residual FP64 (mixed_fp64_krylov: the "
                          "same with FP64 Krylov vectors, MGS and Givens)",
        "phi_rel_err_vs_oracle": head["phi_rel_err_vs_oracle"],
        "solver": {k: v for k, v in head.items() if k not in ("value", "unit", "ms_per_step")},
        "fp64": leg("fp64"),
        "speedup_mixed_vs_fp64": value / fp64_value,
        "mixed_rom_bf16": dict(leg("mixed_rom_bf16"), note="ROM projection and lift as BF16 mma.sync products"),
        "mixed_fp64_krylov": leg("mixed_fp64_krylov"),
        "mixed_plain_romsad": leg("mixed_plain_romsad"),
        "mixed_fp64_residuals": leg("mixed_fp64_residuals"),
        "gmres_dsa_mixed": dict(leg("gmres_dsa_mixed"), note="no ROM: DSA from the first iteration"),
        "learned_start_vs_plain_romsad": value / (solves / results["mixed_plain_romsad"][0]),
        "offline": offline,
        "e2e": {"value": solves / e2e_s, "unit": "param solves/s", "h2d_bytes_per_step": 2 * R * 8 * B,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(round(launches)) if launches is not None else None,
        "peaks": peaks,
        "roofline": roof,
        "oracle_reference": ref_meta,
        "clocks": clocks,
    }
    line.update(extras)
    if not args.no_cpu_baseline:
        iters = statistics.mean(s["iterations"] for s in results["fp64"][1])
        ssb, sab = params(args.warmup)
        cb = oracle_baseline(cfg, spec, ssb, sab, iters, 1, 2, host_cores())
        cb.pop("per_iter_samples", None)
        line["cpu_baseline"] = cb
    print(json.dumps(line))


# Algorithmic bytes of one DSA V-cycle per DG cell (FP32): the DG level reads the cell's right-hand side, the
# inverted cell block and the two first-moment inverses and writes/reads the iterate and residual (about 48
# floats), the vertex levels add a geometric series of 4x4 element matrices and vectors (about 24 floats per
# fine cell).
DSA_VCYCLE_BYTES_PER_CELL = 4 * 72

# DRAM traffic of one A~ apply (the sweep kernel plus the reduce of its partial fluxes), dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of each kernel (bench.py --profile ...), with the SHA-256 of the
# sweep source it was taken on: reported only while that source is unchanged.  The FP64 capture ran 16 of the 64
# instances; its traffic grows in proportion to the instances and is scaled by 4.
NCU_TRAFFIC = {
    ("large256_192", "k_sweep2d<float> (A~ apply, FP32)"): {
        "bytes": (0.186164 + 1.575940 + 1.677866 + 0.066262) * 1e9, "instances_captured": 64,
        "kernels": "k_sweep2d_bands<float, float, 4, 0> + k_reduce<float, float, float>",
        "sweep_sha256": "ea85f47f3deb12d1da7f9e8a0a2d4e3c155404c397c62a958ab093216829f25d"},
    ("large256_192", "k_sweep2d<double> (A~ apply, FP64)"): {
        "bytes": 4 * (0.115022 + 1.554706 + 1.644242 + 0.034141) * 1e9, "instances_captured": 16,
        "kernels": "k_sweep2d<double, double, 2, 0, 0> + k_reduce<double, double, double>",
        "sweep_sha256": "ea85f47f3deb12d1da7f9e8a0a2d4e3c155404c397c62a958ab093216829f25d"},
}


def ncu_traffic(workload: str, kernel: str):
    """Bytes per launch of the dominant kernel from its ncu capture, or None when there is none or the sweep
    source has changed since."""
    import hashlib
    rec = NCU_TRAFFIC.get((workload, kernel))
    if rec is None:
        return None
    with open(os.path.join(ROOT, "paper_2410_08735_gb300", "csrc", "sweep.cu"), "rb") as fh:
        if hashlib.sha256(fh.read()).hexdigest() != rec["sweep_sha256"]:
            return None
    return rec["bytes"]


if __name__ == "__main__":
    main()
