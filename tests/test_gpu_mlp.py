"""GPU MLP kernels (learned warm start) against the oracle MLP, and the warm start's effect."""
import numpy as np
import pytest

import workloads as wl
from oracle import Problem, mlp as OM, romsad as ORS
from oracle.discretization import with_params

from gpu_common import lib, rel, spec2d, split, torch_cuda

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round float32 values to bfloat16 (round to nearest even), returned as float32."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + (((u >> 16) & 1) + 0x7FFF)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def _unpack(flat, din, H, r):
    o = 0
    out = {}
    for k, shape in (("W1", (H, din)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (r, H)), ("b3", (r,))):
        n = int(np.prod(shape))
        out[k] = flat[o:o + n].astype(np.float64).reshape(shape)
        o += n
    return out


def _features(mu, mean, stdv, R):
    raw = np.concatenate([np.log(mu[:, :R]), mu[:, R:]], axis=1)
    return ((raw - mean) / stdv).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("bf16", [False, True])
def test_loss_and_gradient_match_oracle(bf16):
    B = lib()
    R, H, r, n = 4, 32, 6, 40
    rng = np.random.default_rng(0)
    net = B.Mlp(2 * R, H, r, seed=3)
    flat = (rng.standard_normal(net.n_params) * 0.3).astype(np.float32)
    mean = rng.standard_normal(2 * R).astype(np.float32)
    stdv = (0.5 + rng.random(2 * R)).astype(np.float32)
    net.set_params(flat, mean, stdv)
    mu = np.concatenate([np.exp(rng.standard_normal((n, R))), rng.random((n, R))], axis=1)
    c = rng.standard_normal((n, r))
    loss, grad = net.loss_grad(mu, c, bf16=bf16)
    wflat = bf16_round(flat) if bf16 else flat
    params = _unpack(wflat, 2 * R, H, r)
    for k in ("b1", "b2", "b3"):      # biases are not rounded
        params[k] = _unpack(flat, 2 * R, H, r)[k]
    x = _features(mu, mean.astype(np.float64), stdv.astype(np.float64), R)
    loss_o, g_o = OM.loss_and_grads(params, x, c)
    assert abs(loss - loss_o) <= 1e-5 * loss_o
    g_gpu = _unpack(grad, 2 * R, H, r)
    for k in g_o:
        assert rel(g_gpu[k], g_o[k]) < 1e-4, k


def test_training_reduces_loss_and_inference_matches_oracle_forward():
    B = lib()
    R, H, r, n = 4, 64, 5, 512
    rng = np.random.default_rng(1)
    mu = np.concatenate([np.exp(2 * rng.random((n, R))), rng.random((n, R))], axis=1)
    c = np.stack([np.sin(np.log(mu[:, 0])), mu[:, 4] * np.log(mu[:, 1]), np.cos(mu[:, 5]), mu[:, 6] ** 2,
                  np.log(mu[:, 2] * mu[:, 3])], axis=1)
    net = B.Mlp(2 * R, H, r, seed=5)
    l0 = net.loss_grad(mu, c)[0]
    l1 = net.train(mu, c, epochs=300, batch=128, lr=3e-3, bf16=True)
    assert l1 < 0.05 * l0
    flat, mean, stdv = net.get_params()
    params = _unpack(bf16_round(flat), 2 * R, H, r)
    for k in ("b1", "b2", "b3"):
        params[k] = _unpack(flat, 2 * R, H, r)[k]
    y_o, _ = OM.forward(params, _features(mu, mean.astype(np.float64), stdv.astype(np.float64), R))
    y_g = net.infer(mu)
    assert rel(y_g, y_o) < 1e-5


def test_learned_warm_start_reduces_iterations():
    """Greedy ROM (labels) -> MLP trained on the GPU -> learned warm start phi0 = b~ + W c_hat(mu):
    the same tolerance is reached in fewer FGMRES iterations than from a zero guess, and phi
    still matches the oracle solve."""
    torch = torch_cuda()
    B = lib()
    spec = spec2d([16], [16], n_polar=2, n_azim=8)
    n_train = 48
    ss, sa = wl.draw_params(spec, n_train, 41)
    ss = np.minimum(ss, 100.0)
    gp = B.Problem(spec, ss[:1], sa[:1])
    rom, rep = B.Rom.greedy(gp, ss, sa, window=2, max_greedy_iter=8, max_rank=16, eps_rom=0.0, hf_rtol=1e-12,
                            hf_restart=128, hf_max_iter=4000, want_labels=True)
    r = rep["rank"]
    net = B.Mlp(2 * spec.n_regions, 128, r, seed=9)
    mu_train = np.concatenate([ss, sa], axis=1)
    net.train(mu_train, rep["labels"], epochs=400, batch=48, lr=2e-3, bf16=True)
    B.attach_mlp(rom, net)
    nt = 6
    ts, ta = wl.draw_params(spec, nt, 42)
    ts = np.minimum(ts, 100.0)
    sp = spec.with_instances([16] * nt, [16] * nt)
    tp = B.Problem(sp, ts, ta)
    phi0 = torch.zeros(tp.n_dof, dtype=torch.float64, device="cuda")
    phi1 = torch.zeros_like(phi0)
    common = dict(restart=100, rtol=1e-10, max_iter=3000, window=2)
    st0 = B.fgmres_solve(tp, [rom] * nt, phi0, **common)
    st1 = B.fgmres_solve(tp, [rom] * nt, phi1, learned_warm_start=True, **common)
    it0 = sum(s["iterations"] for s in st0)
    it1 = sum(s["iterations"] for s in st1)
    assert it1 < it0, (it0, it1)
    assert all(s["learned_start"] == 1 for s in st1)
    p0 = Problem(spec, 0, ss[0], sa[0])
    for b in range(nt):
        ref, _ = ORS.solve(with_params(p0, ts[b], ta[b]), None, restart=200, rtol=1e-13, max_iter=5000)
        assert rel(split(phi1.cpu().numpy(), tp.offsets)[b], ref) < 1e-8


def test_non_finite_learned_start_falls_back_to_plain_romsad():
    """A network whose outputs are not finite (NaN weights): every instance starts from zero instead
    (plain ROMSAD) and reports learned_start = 0; the solve then takes exactly the iterations of the zero
    start and gives the same phi."""
    torch = torch_cuda()
    B = lib()
    spec = spec2d([16], [16], n_polar=2, n_azim=8)
    ss, sa = wl.draw_params(spec, 24, 43)
    ss = np.minimum(ss, 100.0)
    gp = B.Problem(spec, ss[:1], sa[:1])
    rom, rep = B.Rom.greedy(gp, ss, sa, window=2, max_greedy_iter=4, max_rank=8, eps_rom=0.0, hf_rtol=1e-12,
                            hf_restart=128, hf_max_iter=4000, want_labels=True)
    net = B.Mlp(2 * spec.n_regions, 128, rep["rank"], seed=3)
    flat = net.get_params()[0]
    net.set_params(np.full(flat.shape, np.nan))
    B.attach_mlp(rom, net)
    nt = 3
    ts, ta = wl.draw_params(spec, nt, 44)
    ts = np.minimum(ts, 100.0)
    tp = B.Problem(spec.with_instances([16] * nt, [16] * nt), ts, ta)
    for mode in (B.RTE_MODE_FP64, B.RTE_MODE_MIXED):
        phi0 = torch.zeros(tp.n_dof, dtype=torch.float64, device="cuda")
        phi1 = torch.zeros_like(phi0)
        common = dict(restart=100, rtol=1e-10, max_iter=3000, window=2, mode=mode, inner_rtol=1e-2, max_outer=30)
        st0 = B.fgmres_solve(tp, [rom] * nt, phi0, **common)
        st1 = B.fgmres_solve(tp, [rom] * nt, phi1, learned_warm_start=True, **common)
        for b in range(nt):
            assert st1[b]["learned_start"] == 0
            assert st1[b]["iterations"] == st0[b]["iterations"]
        assert rel(phi1.cpu().numpy(), phi0.cpu().numpy()) < 1e-12


def _slot_setup(B, seed_net=11, nan=False):
    spec = spec2d([16], [16], n_polar=2, n_azim=8)
    ss, sa = wl.draw_params(spec, 48, 45)
    ss = np.minimum(ss, 100.0)
    gp = B.Problem(spec, ss[:1], sa[:1])
    rom, rep = B.Rom.greedy(gp, ss, sa, window=2, max_greedy_iter=8, max_rank=16, eps_rom=0.0, hf_rtol=1e-12,
                            hf_restart=128, hf_max_iter=4000, want_labels=True)
    net = B.Mlp(2 * spec.n_regions, 128, rep["rank"], seed=seed_net)
    if nan:
        net.set_params(np.full(net.get_params()[0].shape, np.nan))
    else:
        net.train(np.concatenate([ss, sa], axis=1), rep["labels"], epochs=400, batch=48, lr=2e-3, bf16=True)
    B.attach_mlp(rom, net)
    return spec, ss, sa, rom


def test_learned_romsad_slot_solves_to_the_oracle():
    """The learned correction in the ROMSAD slot (first preconditioner apply of a zero-start solve takes
    the MLP's coefficients instead of the reduced solve): FP64 and mixed solves reach the oracle's
    solution, every instance reports the slot as used, and the iteration count stays close to plain
    ROMSAD's (a perfect network would reproduce it exactly)."""
    torch = torch_cuda()
    B = lib()
    spec, ss, sa, rom = _slot_setup(B)
    nt = 4
    ts, ta = wl.draw_params(spec, nt, 46)
    ts = np.minimum(ts, 100.0)
    tp = B.Problem(spec.with_instances([16] * nt, [16] * nt), ts, ta)
    p0 = Problem(spec, 0, ss[0], sa[0])
    refs = [ORS.solve(with_params(p0, ts[b], ta[b]), None, restart=200, rtol=1e-13, max_iter=5000)[0]
            for b in range(nt)]
    for mode, tol in ((B.RTE_MODE_FP64, 1e-8), (B.RTE_MODE_MIXED, 1e-7)):
        phi0 = torch.zeros(tp.n_dof, dtype=torch.float64, device="cuda")
        phi1 = torch.zeros_like(phi0)
        common = dict(restart=100, rtol=1e-10, max_iter=3000, window=2, mode=mode, inner_rtol=1e-2, max_outer=30)
        st0 = B.fgmres_solve(tp, [rom] * nt, phi0, **common)
        st1 = B.fgmres_solve(tp, [rom] * nt, phi1, learned_slot=True, **common)
        for b in range(nt):
            assert st1[b]["learned_slot"] == 1 and st0[b]["learned_slot"] == 0
            assert st1[b]["status"] == 0
            assert abs(st1[b]["iterations"] - st0[b]["iterations"]) <= max(3, st0[b]["iterations"] // 5)
            assert rel(split(phi1.cpu().numpy(), tp.offsets)[b], refs[b]) < tol


def test_non_finite_learned_slot_keeps_plain_romsad():
    """With a network whose outputs are not finite the slot falls back to the plain ROMSAD apply: the
    solve is the plain one (same iterations, same phi) and reports learned_slot = 0."""
    torch = torch_cuda()
    B = lib()
    spec, ss, sa, rom = _slot_setup(B, nan=True)
    nt = 3
    ts, ta = wl.draw_params(spec, nt, 47)
    ts = np.minimum(ts, 100.0)
    tp = B.Problem(spec.with_instances([16] * nt, [16] * nt), ts, ta)
    for mode in (B.RTE_MODE_FP64, B.RTE_MODE_MIXED):
        phi0 = torch.zeros(tp.n_dof, dtype=torch.float64, device="cuda")
        phi1 = torch.zeros_like(phi0)
        common = dict(restart=100, rtol=1e-10, max_iter=3000, window=2, mode=mode, inner_rtol=1e-2, max_outer=30)
        st0 = B.fgmres_solve(tp, [rom] * nt, phi0, **common)
        st1 = B.fgmres_solve(tp, [rom] * nt, phi1, learned_slot=True, **common)
        for b in range(nt):
            assert st1[b]["learned_slot"] == 0
            assert st1[b]["iterations"] == st0[b]["iterations"]
        assert rel(phi1.cpu().numpy(), phi0.cpu().numpy()) < 1e-12
