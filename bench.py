"""Benchmark: parameter solves/s of FGMRES-ROMSAD for the parametric RTE on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

A step solves one batch of seeded parameter instances of the workload to FP64 true residual
1e-8 (relative l2 of b~ - A~ phi).  `value` is the mixed-precision path (FP32 sweeps, FP64
Arnoldi/Givens/residual); `fp64` beside it is the plain FP64 path on the same GPU.  Inputs are
resident in HBM when the timed region starts; L2 is flushed (a 256 MiB write) before every
timed step.  `e2e` repeats the mixed measurement through the C ABI with host buffers: each step
copies its parameters host->device and the scalar flux device->host inside the timed region.
Under torchrun every rank solves its own instances (no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the CPU oracle legs run on one host core: cap the BLAS / OpenMP pools before numpy starts them
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

# Arithmetic per cell and unique direction of the fused sweep (rhs assembly 8 FMA, 4x4 solve 16 FMA,
# outflow traces 4 FMA, quadrature 4 FMA).
SWEEP_FLOPS_PER_CELL_DIR = 64
SWEEP32_DRAM_BYTES_64x64 = 116480   # dram__bytes_read.sum + dram__bytes_write.sum, one launch (ncu)
# ALU peaks from the unit counts and the maximum SM clock (152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz);
# FP64: GB300 nominal 1.25 TFLOP/s.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def workload_spec(name: str):
    if name == "square2d_64":
        return wl.config(2), 1
    if name == "batch256_uneven":
        return wl.config(3), 256
    if name == "slab1d_128":
        return wl.config(1), 1
    raise SystemExit(f"unknown workload {name}")


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


# ------------------------------------------------------------------ oracle legs
def oracle_sample(spec, ss, sa, iters_needed: int, sample_iters: int, dsa: bool = True):
    """Time the CPU oracle on one instance: b~ plus a bounded number of FGMRES iterations (preconditioned by
    the oracle's DSA V-cycle when dsa, whose set-up is timed too), and extrapolate to one full solve (the
    same algorithm needs `iters_needed` iterations; the ROMSAD applies of the window cost a small dense
    solve each and are left out)."""
    from oracle import Problem as OProblem, dsa as ODSA, transport as OT
    from oracle.krylov import fgmres
    p = OProblem(spec, 0, ss, sa)
    t0 = time.perf_counter()
    bt = OT.rhs_btilde(p)
    t1 = time.perf_counter()
    pre = None
    if dsa:
        mg = ODSA.MultigridDsa(p, "partial")
        pre = lambda j, v: mg.apply(v)
    t_setup = time.perf_counter() - t1
    t1b = time.perf_counter()
    fgmres(lambda z: OT.Atilde_apply(p, z), bt, pre, restart=min(sample_iters, 128), rtol=1e-30,
           max_iter=sample_iters, true_residual_check=False)
    t2 = time.perf_counter()
    per_iter = (t2 - t1b) / sample_iters
    solve_s = (t1 - t0) + t_setup + iters_needed * per_iter + (t1 - t0)   # b~, DSA set-up, iterations, residual
    what = "FGMRES-DSA" if dsa else "FGMRES"
    return {"value": 1.0 / solve_s, "unit": "param solves/s", "cores": 1, "kind": "oracle",
            "sample": f"b~ + {sample_iters} {what} iterations of one {spec.name} instance on 1 host core "
                      f"({t2 - t0:.1f} s), extrapolated to {iters_needed} iterations + 1 residual sweep"}


METRIC = "param solves/s at 1e-8 true residual (mixed+MLP FGMRES-ROMSAD vs plain FP64 FGMRES-ROMSAD)"


def bench_config(args, spec, B):
    """The workload description both arms print (no model keys: the workload is named by its sizes)."""
    return {"workload": args.workload, "instances_per_step": B, "mesh": f"{spec.nx[0]}x{spec.ny[0]}",
            "directions": spec.n_directions, "restart": args.restart,
            "preconditioner": f"ROMSAD rank {getattr(args, 'rom_rank', 0) or spec.rom_rank} (window {spec.window}), then "
                              + ("DSA (partially consistent, one multigrid V-cycle)" if getattr(args, "post", "dsa") == "dsa"
                                 else "ROMSAD kept after the window"),
            "warm_start": "MLP 8-128-128-r (mixed path only)",
            "l2": "flushed (256 MiB write) before every timed step"}


def run_reference(args, spec, B, world, rank):
    if rank != 0:
        return
    ss, sa = wl.draw_params(spec, max(1, B), wl.seed_for(2, 1))
    iters = args.ref_iters
    vals = []
    t_start = time.perf_counter()
    one = spec.with_instances(spec.nx[:1], spec.ny[:1])
    for _ in range(args.warmup):   # untimed warm-up samples
        oracle_sample(one, ss[0], sa[0], iters, args.ref_sample, getattr(args, "post", "dsa") == "dsa")
    for s in range(args.steps):
        cb = oracle_sample(one, ss[0], sa[0], iters, args.ref_sample, getattr(args, "post", "dsa") == "dsa")
        vals.append(1.0 / cb["value"])
    total = sum(vals)
    value = args.steps * B / total if B else 0.0
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "param solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, spec, B),
            "cpu_baseline": dict(cb, value=value),
            "e2e": {"value": value, "unit": "param solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU legs
def post_kwargs(RB, args):
    """fgmres_solve keywords of the preconditioner after the ROMSAD window."""
    if args.post == "dsa":
        return {"post_mode": RB.RTE_POST_DSA,
                "dsa_variant": RB.RTE_DSA_LUMPED if args.dsa_variant == "lumped" else RB.RTE_DSA_PARTIAL}
    return {"post_mode": RB.RTE_POST_ROM}


def measure_sweep_hbm(RB, torch, dev, stream, flush, reps=5, config=3):
    """Angular-output sweep (rte_sweep, FP32) over a whole batched workload: an HBM-bound write of
    N_Omega * N_dof * 4 bytes (both duplicate directions stored), timed with CUDA events after warm-up."""
    spec3 = wl.config(config)
    ss, sa = wl.draw_params(spec3, spec3.n_instances, wl.seed_for(config, 1))
    prob = RB.Problem(spec3, ss, sa)
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
    cells = sum(nx * ny for nx, ny in zip(spec3.nx, spec3.ny))
    meshes = {}
    for nx, ny in zip(spec3.nx, spec3.ny):
        meshes[f"{nx}x{ny}"] = meshes.get(f"{nx}x{ny}", 0) + 1
    desc = ", ".join(f"{c}x{m}" for m, c in meshes.items())
    out = {"workload": f"{spec3.name} ({desc}; {prob.n_directions} directions, {spec3.n_regions} regions)",
           "kernel": "k_sweep2d / k_sweep2d_bands (angular output, FP32; autotuned)",
           "bytes": nbytes, "ms": ms, "achieved_gbs": nbytes / (ms * 1e-3) / 1e9, "peak_gbs": peak,
           "frac": nbytes / (ms * 1e-3) / 1e9 / peak,
           "alu_tflops": SWEEP_FLOPS_PER_CELL_DIR * cells * prob.info.n_unique_directions / (ms * 1e-3) / 1e12}
    del psi
    torch.cuda.empty_cache()
    return out


def measure_batched(RB, torch, dev, stream, flush, args, reps=1):
    """Batched throughput: the 256-instance uneven workload solved by one fgmres_solve call per batch,
    mixed (FP32 inner solves) with the learned warm start vs plain FP64, each mesh group preconditioned by
    its own greedy ROM, whose labels train that group's MLP (offline, untimed)."""
    spec3 = wl.config(3)
    R = spec3.n_regions
    B = spec3.n_instances
    ss, sa = wl.draw_params(spec3, B, wl.seed_for(3, 1))
    prob = RB.Problem(spec3, ss, sa)
    t0 = time.perf_counter()
    roms, nets, losses = {}, {}, {}
    tr_ss, tr_sa = wl.draw_params(spec3, args.batched_train, wl.seed_for(3, 0))
    feats = np.concatenate([tr_ss, tr_sa], axis=1)
    for n in sorted(set(spec3.nx)):
        sp = spec3.with_instances([n], [n])
        tmpl = RB.Problem(sp, tr_ss[:1], tr_sa[:1])
        rom, rep = RB.Rom.greedy(tmpl, tr_ss, tr_sa, window=spec3.window, max_greedy_iter=args.batched_rank // 2,
                                 max_rank=args.batched_rank, eps_rom=0.0, hf_rtol=1e-8, hf_restart=args.restart,
                                 hf_max_iter=args.max_iter, want_labels=True, indicator_f32=True)
        net = RB.Mlp(2 * R, 128, rep["rank"], seed=2410 + n)
        losses[n] = net.train(feats, rep["labels"], epochs=args.mlp_epochs, batch=min(64, len(feats)), lr=2e-3,
                              bf16=True)
        RB.attach_mlp(rom, net)
        roms[n], nets[n] = rom, net
    t_off = time.perf_counter() - t0
    rl = [roms[n] for n in spec3.nx]
    phi = torch.zeros(prob.n_dof, dtype=torch.float64, device=dev)
    out = {"workload": "batch256_uneven: 96x32^2 + 96x64^2 + 64x128^2, 128 directions, one solve call per batch",
           "instances": B, "rom_rank": args.batched_rank, "training_draws": args.batched_train, "offline_s": t_off,
           "mlp_final_loss": {f"{n}x{n}": v for n, v in losses.items()}}
    # "mixed": FP32 inner solves + MLP warm start (the batched form of the method); "mixed_plain_romsad":
    # the same without the warm start; "fp64": plain FP64 FGMRES-ROMSAD
    for name, mode, learned in (("mixed", RB.RTE_MODE_MIXED, True), ("mixed_plain_romsad", RB.RTE_MODE_MIXED, False),
                                ("fp64", RB.RTE_MODE_FP64, False)):
        RB.fgmres_solve(prob, rl, phi, restart=args.restart, rtol=1e-8, max_iter=args.max_iter, window=spec3.window,
                        mode=mode, inner_rtol=args.inner_rtol, max_outer=30, stream=stream,
                        raise_on_fail=False, learned_warm_start=learned, **post_kwargs(RB, args))   # warm-up / tuning
        times, st_all = [], []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = RB.fgmres_solve(prob, rl, phi, restart=args.restart, rtol=1e-8, max_iter=args.max_iter,
                                 window=spec3.window, mode=mode, inner_rtol=args.inner_rtol, max_outer=30,
                                 stream=stream, raise_on_fail=False, learned_warm_start=learned,
                                 **post_kwargs(RB, args))
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            st_all.extend(st)
        ms = statistics.mean(times)
        conv = sum(1 for s in st_all if s["status"] == 0) / reps
        # only instances that met rtol count as solved
        out[name] = {"value": conv / (ms * 1e-3), "unit": "param solves/s", "ms_per_batch": ms,
                     "converged": conv, "escalated_to_fp64": sum(s["escalated"] for s in st_all) / reps,
                     "iterations_max": max(s["iterations"] for s in st_all),
                     "iterations_mean": statistics.mean(s["iterations"] for s in st_all),
                     "true_rel_residual_max": max(s["true_rel_residual"] for s in st_all),
                     "status": sorted({s["status"] for s in st_all})}
    out["speedup_mixed_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def measure_learned_eval(RB, torch, dev, stream, flush, args, spec, rom, n_test=512):
    """The learned part on held-out draws: n_test parameter instances of the single-instance workload (seeded
    test split, never seen by the greedy or the MLP) solved in one mixed-precision call, with the learned
    warm start, with the learned ROMSAD slot, and with plain ROMSAD."""
    ts, ta = wl.draw_params(spec, n_test, wl.seed_for(4, 1))
    sp = spec.with_instances([spec.nx[0]] * n_test, [spec.ny[0]] * n_test)
    prob = RB.Problem(sp, ts, ta)
    phi = torch.zeros(prob.n_dof, dtype=torch.float64, device=dev)
    roms = [rom] * n_test
    out = {"workload": f"{n_test} held-out draws of {spec.name} in one batched call", "instances": n_test}
    for name, kw in (("learned_start", {"learned_warm_start": True}), ("learned_slot", {"learned_slot": True}),
                     ("plain_romsad", {})):
        common = dict(restart=args.restart, rtol=1e-8, max_iter=args.max_iter, window=spec.window,
                      mode=RB.RTE_MODE_MIXED, inner_rtol=args.inner_rtol, max_outer=30, stream=stream,
                      raise_on_fail=False, **kw, **post_kwargs(RB, args))
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
        out[name] = {"value": conv / (ms * 1e-3), "unit": "param solves/s", "converged": conv,
                     "iterations_mean": statistics.mean(s["iterations"] for s in st),
                     "iterations_max": max(s["iterations"] for s in st),
                     "true_rel_residual_max": max(s["true_rel_residual"] for s in st)}
    del phi, prob
    torch.cuda.empty_cache()
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="square2d_64")
    ap.add_argument("--restart", type=int, default=128)
    ap.add_argument("--max-iter", type=int, default=6000)
    ap.add_argument("--inner-rtol", type=float, default=None,
                    help="inner target of the mixed refinement (default 1e-3 with DSA after the window, else 1e-2)")
    ap.add_argument("--post", default="dsa", choices=["dsa", "rom"],
                    help="preconditioner after the ROMSAD window: DSA (the paper's) or ROMSAD kept")
    ap.add_argument("--dsa-variant", default="partial", choices=["partial", "lumped"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mlp-epochs", type=int, default=300)
    ap.add_argument("--no-sweep-hbm", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-train", type=int, default=32)
    ap.add_argument("--batched-rank", type=int, default=32)
    ap.add_argument("--rom-rank", type=int, default=0, help="ROM rank cap (0: the workload's)")
    ap.add_argument("--n-train", type=int, default=1024,
                    help="training draws of the greedy and the MLP (2048 leaves the network less trained in the "
                         "same epoch budget)")
    ap.add_argument("--ref-sample", type=int, default=40, help="oracle FGMRES iterations per reference step")
    ap.add_argument("--ref-iters", type=int, default=None,
                    help="iterations of a full solve for the extrapolation (default: those of the FP64 solve of this "
                         "workload on the GPU, 16 with DSA after the window, 180 with ROMSAD kept)")
    args = ap.parse_args()
    if args.inner_rtol is None:
        args.inner_rtol = 1e-3 if args.post == "dsa" else 1e-2
    if args.ref_iters is None:
        args.ref_iters = 16 if args.post == "dsa" else 180
    spec, B = workload_spec(args.workload)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, spec, B, world, rank)
        return
    import torch
    from paper_2410_08735_gb300 import binding as RB
    RB.load()                                   # fails loudly without the built CUDA library
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    R = spec.n_regions
    n_sets = args.warmup + args.steps
    # parameters: distinct seeded draws per rank and step (test split)
    ss_all, sa_all = wl.draw_params(spec, n_sets * B * world, wl.seed_for(2, 1))
    def params(step):
        i0, i1 = shard(rank, n_sets, B, step)
        return ss_all[i0:i1], sa_all[i0:i1]

    ss0, sa0 = params(0)
    prob = RB.Problem(spec, ss0, sa0)
    n = prob.n_dof
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # offline (untimed): greedy ROM on the training draws, MLP trained on its labels
    t_off = time.perf_counter()
    n_train = args.n_train or spec.n_train
    tr_ss, tr_sa = wl.draw_params(spec, n_train, wl.seed_for(2, 0))
    tmpl = RB.Problem(spec.with_instances(spec.nx[:1], spec.ny[:1]), tr_ss[:1], tr_sa[:1])
    rank_cap = args.rom_rank or spec.rom_rank
    rom, rep = RB.Rom.greedy(tmpl, tr_ss, tr_sa, window=spec.window, max_greedy_iter=rank_cap // spec.window,
                             max_rank=rank_cap, eps_rom=0.0, hf_rtol=1e-10, hf_restart=args.restart,
                             hf_max_iter=args.max_iter, want_labels=True, indicator_f32=True)
    t_greedy = time.perf_counter() - t_off
    net = RB.Mlp(2 * R, 128, rep["rank"], seed=2410)
    mlp_loss = net.train(np.concatenate([tr_ss, tr_sa], axis=1), rep["labels"], epochs=args.mlp_epochs,
                         batch=min(64, n_train), lr=2e-3, bf16=True)
    RB.attach_mlp(rom, net)
    t_offline = time.perf_counter() - t_off
    roms = [rom] * B
    common = dict(restart=args.restart, rtol=1e-8, max_iter=args.max_iter, window=spec.window, stream=stream,
                  **post_kwargs(RB, args))

    def solve(mode, learned=True, slot=False):
        if mode in (RB.RTE_MODE_MIXED, RB.RTE_MODE_MIXED_F64KRYLOV):
            return RB.fgmres_solve(prob, roms, phi, mode=mode, inner_rtol=args.inner_rtol, max_outer=30,
                                   learned_warm_start=learned, learned_slot=slot, **common)
        return RB.fgmres_solve(prob, roms, phi, mode=mode, true_residual_check=True, **common)

    def timed_loop(mode, learned=True, slot=False, solver=None):
        per_step, stats_all = [], []
        for s in range(n_sets):
            ss, sa = params(s)
            prob.set_params(ss, sa)
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solve(mode, learned, slot) if solver is None else solver()
            e1.record(stream)
            torch.cuda.synchronize()
            if s >= args.warmup:
                per_step.append(e0.elapsed_time(e1))
                stats_all.extend(st)
        return per_step, stats_all

    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    launches0 = RB.kernel_launches()
    torch.cuda.nvtx.range_push("timed_mixed")      # ncu --nvtx-include timed_mixed/ selects this region
    t_mixed, st_mixed = timed_loop(RB.RTE_MODE_MIXED)
    torch.cuda.nvtx.range_pop()
    launches_mixed = RB.kernel_launches() - launches0
    torch.cuda.nvtx.range_push("timed_fp64")
    t_fp64, st_fp64 = timed_loop(RB.RTE_MODE_FP64)
    torch.cuda.nvtx.range_pop()
    # the mixed path without the learned warm start (plain ROMSAD), for the MLP's net effect
    t_plain, st_plain = timed_loop(RB.RTE_MODE_MIXED, learned=False)
    # the mixed path with the learned correction in the ROMSAD slot instead of the learned start
    t_slot, st_slot = timed_loop(RB.RTE_MODE_MIXED, learned=False, slot=True)
    # the precision form with FP64 Krylov vectors, MGS and Givens around the FP32 sweeps
    t_f64k, st_f64k = timed_loop(RB.RTE_MODE_MIXED_F64KRYLOV)
    # the mixed path with ROMSAD kept after the window (no DSA), learned start, inner target 1e-2
    base_kw = dict(restart=args.restart, rtol=1e-8, max_iter=args.max_iter, window=spec.window, stream=stream)
    t_prom, st_prom = timed_loop(None, solver=lambda: RB.fgmres_solve(
        prob, roms, phi, mode=RB.RTE_MODE_MIXED, inner_rtol=1e-2, max_outer=30, learned_warm_start=True,
        post_mode=RB.RTE_POST_ROM, **base_kw))
    # right-preconditioned GMRES-DSA (no ROM), mixed
    t_gdsa, st_gdsa = timed_loop(None, solver=lambda: RB.fgmres_solve(
        prob, None, phi, mode=RB.RTE_MODE_MIXED, inner_rtol=args.inner_rtol, max_outer=30,
        post_mode=RB.RTE_POST_DSA, **base_kw))
    # GMRES-DSA from the RBF-interpolated initial guess (the paper's interpolation baseline): data = FP64
    # solutions at the training points the greedy sampled (offline, untimed); the interpolation is timed
    interp = None
    try:
        ks = list(rep["sampled"])
        spec_k = spec.with_instances([spec.nx[0]] * len(ks), [spec.ny[0]] * len(ks))
        pk = RB.Problem(spec_k, tr_ss[ks], tr_sa[ks])
        sol_k = torch.zeros(pk.n_dof, dtype=torch.float64, device=dev)
        RB.fgmres_solve(pk, None, sol_k, restart=args.restart, rtol=1e-10, max_iter=args.max_iter,
                        post_mode=RB.RTE_POST_DSA, stream=stream)
        rbf = RB.Rbf(tmpl, tr_ss[ks], tr_sa[ks], sol_k.view(len(ks), -1))
        phi0_ig = torch.zeros(n, dtype=torch.float64, device=dev)

        def interp_solve():
            rbf.initial_guess(prob, phi0_ig, stream=stream)
            return RB.fgmres_solve(prob, None, phi, phi0=phi0_ig, mode=RB.RTE_MODE_MIXED, inner_rtol=args.inner_rtol,
                                   max_outer=30, post_mode=RB.RTE_POST_DSA, **base_kw)

        t_ig, st_ig = timed_loop(None, solver=interp_solve)
        ig_s = max_over_ranks(world, sum(t_ig) / 1e3)
        interp = {"value": args.steps * B * world / ig_s, "unit": "param solves/s",
                  "iterations_mean": statistics.mean(s["iterations"] for s in st_ig),
                  "samples": len(ks), "note": "mixed GMRES-DSA from the RBF-interpolated initial guess"}
        del pk, sol_k
    except Exception as exc:   # the leg is a side measurement; report instead of losing the bench line
        interp = {"error": f"{type(exc).__name__}: {exc}"}
    # SI-ROMSAD (source iteration: the ROM correction in the window, DSA afterwards), FP64
    t_si, st_si = timed_loop(None, solver=lambda: RB.si_solve(
        prob, roms, phi, rtol=1e-8, max_iter=2000, window=spec.window, post_mode=RB.RTE_POST_DSA, stream=stream,
        raise_on_fail=False))
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    mixed_s = max_over_ranks(world, sum(t_mixed) / 1e3)
    fp64_s = max_over_ranks(world, sum(t_fp64) / 1e3)
    plain_s = max_over_ranks(world, sum(t_plain) / 1e3)
    slot_s = max_over_ranks(world, sum(t_slot) / 1e3)
    f64k_s = max_over_ranks(world, sum(t_f64k) / 1e3)
    prom_s = max_over_ranks(world, sum(t_prom) / 1e3)
    gdsa_s = max_over_ranks(world, sum(t_gdsa) / 1e3)
    si_s = max_over_ranks(world, sum(t_si) / 1e3)
    si_conv = sum(1 for s in st_si if s["status"] == 0)
    solves = args.steps * B * world
    value = solves / mixed_s
    fp64_value = solves / fp64_s
    # e2e: host parameters in, host scalar flux out, through the C ABI
    host_phi = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    e2e_ms = []
    for s in range(n_sets):
        ss, sa = params(s)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.set_params(ss, sa)
        RB.fgmres_solve(prob, roms, host_phi, mode=RB.RTE_MODE_MIXED, inner_rtol=args.inner_rtol, max_outer=30,
                        learned_warm_start=True, **common)
        t1 = time.perf_counter()
        if s >= args.warmup:
            e2e_ms.append(1e3 * (t1 - t0))
    e2e_s = max_over_ranks(world, sum(e2e_ms) / 1e3)
    # roofline of the dominant kernel: the fused sweep (A~ apply), timed alone with CUDA events
    z64 = torch.randn(n, dtype=torch.float64, device=dev)
    w64 = torch.empty_like(z64)
    z32 = z64.float()
    w32 = torch.empty_like(z32)

    def time_op(z, w, reps=20):
        for _ in range(3):
            prob.apply_op(z, w, stream=stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            prob.apply_op(z, w, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms32 = time_op(z32, w32)
    ms64 = time_op(z64, w64)

    def time_dsa(reps=20):
        # rte_dsa_apply: the per-parameter set-up plus one V-cycle, FP32 vectors
        for _ in range(3):
            prob.dsa_apply(z32, w32, stream=stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            prob.dsa_apply(z32, w32, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_dsa = time_dsa() if args.post == "dsa" else None
    cells = sum(nx * ny for nx, ny in zip(spec.nx[:B], spec.ny[:B]))
    nu = prob.info.n_unique_directions
    flops = SWEEP_FLOPS_PER_CELL_DIR * cells * nu
    sw32 = sum(s["sweeps"] - s["sweeps_fp64"] for s in st_mixed)
    sw64 = sum(s["sweeps_fp64"] for s in st_mixed)
    share32, share64 = sw32 * ms32, sw64 * ms64
    if share32 >= share64:
        roof = {"kernel": "k_sweep2d<float> (A~ apply, FP32)", "bound": "alu", "achieved": flops / (ms32 * 1e-3) / 1e12,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s"}
    else:
        roof = {"kernel": "k_sweep2d<double> (A~ apply, FP64)", "bound": "alu",
                "achieved": flops / (ms64 * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes per launch of the FP32 sweep kernel from one ncu capture of this workload
    # (profiles/sweep_band_f32_square2d_64.md); none recorded for the FP64 kernel
    roof["traffic"] = SWEEP32_DRAM_BYTES_64x64 if roof["unit"] == "TFLOP/s" and "float" in roof["kernel"] else None
    # angular-output sweep (rte_sweep, FP32) on the batched 256-instance problem: HBM-bound write of
    # N_Omega * N_dof * 4 bytes; this is the sweep GB/s of the metric
    sweep_hbm = measure_sweep_hbm(RB, torch, dev, stream, flush) if not args.no_sweep_hbm else None
    if sweep_hbm is not None and world == 1:
        # the largest workload (64 x 256^2, 192 directions, 8x8 regions): 12.9 GB of angular output
        sweep_hbm["large"] = measure_sweep_hbm(RB, torch, dev, stream, flush, reps=3, config=5)
    batched = measure_batched(RB, torch, dev, stream, flush, args) if not args.no_batched and world == 1 else None
    learned_eval = (measure_learned_eval(RB, torch, dev, stream, flush, args, spec, rom)
                    if not args.no_batched and world == 1 else None)
    roof["ms_per_launch_fp32"] = ms32
    roof["ms_per_launch_fp64"] = ms64
    roof["peak_source"] = "unit counts x max SM clock (FP32); GB300 nominal (FP64)"
    if rank != 0:
        return
    line = {
        "metric": METRIC,
        "value": value, "unit": "param solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * mixed_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": bench_config(args, spec, B),
        "fp64": {"value": fp64_value, "unit": "param solves/s", "ms_per_step": 1e3 * fp64_s / args.steps},
        "mixed_plain_romsad": {"value": solves / plain_s, "unit": "param solves/s",
                               "iterations_mean": statistics.mean(s["iterations"] for s in st_plain)},
        "mixed_learned_slot": {"value": solves / slot_s, "unit": "param solves/s",
                               "iterations_mean": statistics.mean(s["iterations"] for s in st_slot)},
        "mixed_fp64_krylov": {"value": solves / f64k_s, "unit": "param solves/s",
                              "iterations_mean": statistics.mean(s["iterations"] for s in st_f64k),
                              "true_rel_residual_max": max(s["true_rel_residual"] for s in st_f64k)},
        "mixed_post_rom": {"value": solves / prom_s, "unit": "param solves/s",
                           "iterations_mean": statistics.mean(s["iterations"] for s in st_prom),
                           "note": "ROMSAD kept after the window instead of DSA, learned start, inner target 1e-2"},
        "gmres_dsa_mixed": {"value": solves / gdsa_s, "unit": "param solves/s",
                            "iterations_mean": statistics.mean(s["iterations"] for s in st_gdsa),
                            "note": "no ROM: DSA from the first iteration"},
        "gmres_dsa_interp_ig_mixed": interp,
        "si_romsad_fp64": {"value": si_conv * world / si_s, "unit": "param solves/s",
                           "converged": si_conv, "of": len(st_si),
                           "iterations_mean": statistics.mean(s["iterations"] for s in st_si),
                           "iterations_max": max(s["iterations"] for s in st_si),
                           "note": "source iteration, ROM correction in the window then DSA (FP64)"},
        "speedup_mixed_vs_fp64": value / fp64_value,
        "offline": {"greedy_s": t_greedy, "total_s": t_offline, "rank": rep["rank"], "sampled": len(rep["sampled"]),
                    "mlp_final_loss": mlp_loss},
        "solver": {
            "mixed_iterations_mean": statistics.mean(s["iterations"] for s in st_mixed),
            "mixed_fp64_sweeps_mean": statistics.mean(s["sweeps_fp64"] for s in st_mixed),
            "mixed_true_rel_residual_max": max(s["true_rel_residual"] for s in st_mixed),
            "fp64_iterations_mean": statistics.mean(s["iterations"] for s in st_fp64),
            "fp64_true_rel_residual_max": max(s["true_rel_residual"] for s in st_fp64),
            "status": sorted({s["status"] for s in st_mixed + st_fp64})},
        "e2e": {"value": solves / e2e_s, "unit": "param solves/s", "h2d_bytes_per_step": 2 * R * 8 * B,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(launches_mixed * args.steps / n_sets),
        "dsa_apply_us": None if ms_dsa is None else 1e3 * ms_dsa,
        "roofline": roof,
        "sweep_hbm": sweep_hbm,
        "batched": batched,
        "learned_eval": learned_eval,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        ss, sa = params(args.warmup)
        iters = int(round(statistics.mean(s["iterations"] for s in st_fp64)))
        line["cpu_baseline"] = oracle_sample(spec.with_instances(spec.nx[:1], spec.ny[:1]), ss[0], sa[0], iters,
                                             args.ref_sample, args.post == "dsa")
    print(json.dumps(line))


if __name__ == "__main__":
    main()
