"""The learned initial guess on the GPU against its oracle (oracle/guess_net.py): features,
targets, the FP32 and tensor-core forward passes, loss and gradients, one Adam step; then the
trained network against the method without it (the extrapolated guess) on held-out pulses."""
import math

import numpy as np
import pytest

from oracle import guess_net as G
from paper_2512_21697_gb300 import binding as B, learned as L, workloads as W

pytestmark = pytest.mark.gpu


def _rand_states(n, k, seed):
    import torch
    out = []
    for i in range(k):
        z = W.random_state(n, seed + i)
        out.append(torch.from_numpy(z).cuda())
    return out


def _lib_shape(t, bas):
    return t.cpu().numpy().reshape(bas.nch, bas.n // (2 * bas.nch), 2)


@pytest.fixture(scope="module")
def tiny():
    cfg = W.TINY
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg, tol=1e-12)
    return cfg, bas, op


def test_features_and_targets_match_oracle(tiny):
    import torch
    cfg, bas, op = tiny
    st = _rand_states(bas.n, 5, 40)
    # make one state a smooth continuation so that differences span several scales
    st[1] = st[0] * 0.999 + 1e-3 * st[1]
    npos = bas.nch * (cfg["N"] + 1)
    x = torch.empty((npos, 32), dtype=torch.float32, device="cuda")
    s = torch.empty(npos, dtype=torch.float32, device="cuda")
    tg = torch.empty((npos, 4), dtype=torch.float32, device="cuda")
    T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
    t_next = 0.37 * T
    B.guess_features(op, st[:4], t_next, x, s)
    B.guess_targets(op, st[:3], st[4], s, tg)
    H = np.stack([_lib_shape(z, bas) for z in st[:4]])
    xr, sr = G.features(H, bas.kappa, bas.two_mu, G.field_factors(t_next - cfg["t0"], cfg["E0"], cfg["omega"],
                                                                    cfg["n_cycles"]))
    tr = G.targets(H[:3], _lib_shape(st[4], bas), sr)
    assert np.allclose(s.cpu().numpy(), sr, rtol=1e-6, atol=0)
    assert np.max(np.abs(x.cpu().numpy() - xr)) <= 1e-6
    assert np.allclose(tg.cpu().numpy(), tr, rtol=1e-5, atol=1e-6 * np.max(np.abs(tr)))


def _net_and_batch(B_, seed):
    import torch
    p = G.init_params(seed)
    p["W4"] *= 50.0
    g = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = 0.1 * g.standard_normal(p[k].shape)
    flat = G.flatten(p)
    p = G.unflatten(flat)   # the float32 parameters the library holds
    x = g.standard_normal((B_, 32)).astype(np.float32)
    t = g.standard_normal((B_, 4)).astype(np.float32)
    net = B.GuessNet(4096, flat)
    return net, p, x, t, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()


def test_forward_fp32_and_tensor_cores_match_oracle():
    import torch
    net, p, x, _, xd, _ = _net_and_batch(3000, 11)
    out = torch.empty((3000, 4), dtype=torch.float32, device="cuda")
    ref, _ = G.forward(p, x.astype(np.float64))
    net.forward(xd, out, tensor_cores=False)
    got = out.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref)) + 1e-6
    # tensor cores keep the input and the activations in bfloat16: compare with that rounding; both
    # tensor-core kernels (1: tcgen05 with TMEM accumulators, 2: warp-level mma.sync)
    ref_b, _ = G.forward(p, x.astype(np.float64), act_bf16=True)
    for tc in (1, 2):
        out.zero_()
        net.forward(xd, out, tensor_cores=tc)
        got = out.cpu().numpy()
        print("tensor_cores=%d: max|out - ref_b| / rms(ref_b) = %.3g" %
              (tc, np.max(np.abs(got - ref_b)) / np.sqrt(np.mean(ref_b ** 2))))
        assert np.max(np.abs(got - ref_b)) <= 5e-3 * np.sqrt(np.mean(ref_b ** 2)), tc
        # and the bfloat16 activations cost little against full precision
        assert np.sqrt(np.mean((got - ref) ** 2)) <= 3e-2 * np.sqrt(np.mean(ref ** 2)), tc


@pytest.mark.parametrize("M", [1, 127, 128, 129, 5000])
def test_tcgen05_forward_sizes(M):
    # the tcgen05 kernel's 128-position tiles with a ragged last tile, a single partial tile and an
    # exact multiple; rows past M are neither read nor written
    import torch
    net, p, x, _, _, _ = _net_and_batch(M, 5)
    xd = torch.from_numpy(x).cuda()
    out = torch.full((M + 1, 4), 7.0, dtype=torch.float32, device="cuda")
    net.forward(xd, out[:M], tensor_cores=1)
    got = out.cpu().numpy()
    ref_b, _ = G.forward(p, x.astype(np.float64), act_bf16=True)
    assert np.max(np.abs(got[:M] - ref_b)) <= 5e-3 * np.sqrt(np.mean(ref_b ** 2))
    assert np.all(got[M] == 7.0)
    out2 = torch.empty((M, 4), dtype=torch.float32, device="cuda")
    net.forward(xd, out2, tensor_cores=2)
    # the two tensor-core kernels differ only in FP32 summation order and tanh rounding
    assert np.max(np.abs(got[:M] - out2.cpu().numpy())) <= 5e-3 * np.sqrt(np.mean(ref_b ** 2))


def test_loss_and_gradient_match_oracle():
    net, p, x, t, xd, td = _net_and_batch(3000, 12)   # three reduction chunks
    loss, grad = net.loss_grad(xd, td)
    lr_, gr = G.loss_and_grads(p, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lr_) <= 1e-5 * lr_
    gflat = G.flatten(gr).astype(np.float64)   # same layout
    o = 0
    for name, shp in G.SHAPES:
        n = int(np.prod(shp))
        a, b = grad[o:o + n], gflat[o:o + n]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-9, name
        o += n


def test_adam_step_matches_oracle():
    net, p, x, t, xd, td = _net_and_batch(2048, 13)
    lr = 1e-3
    net.train_step(xd, td, lr)
    got = G.unflatten(net.get_params())
    _, g = G.loss_and_grads(p, x.astype(np.float64), t.astype(np.float64))
    z = {k: np.zeros_like(v) for k, v in p.items()}
    pn, _, _ = G.adam_step(p, g, z, z, 1, lr=lr)
    # first step: every parameter moves by about lr sign(g); parameters whose gradient is at the
    # FP32 noise level may move the other way, so the bar is on the fraction that agree
    ok, tot = 0, 0
    for k in p:
        d = np.abs(got[k] - pn[k])
        ok += int(np.sum(d <= 1e-3 * lr + 1e-7))
        tot += d.size
    assert ok >= 0.999 * tot


def test_trained_network_beats_extrapolation_on_heldout_pulses():
    import torch
    base = dict(W.SMALL)
    base.update(dt=0.02, two_mu_max=1, kappa_max=3, N=50, R=40.0)
    bas = B.Basis(base)
    train_cfgs = L.pulse_variants(base, range(1000, 1024))
    test_cfgs = L.pulse_variants(base, range(2000, 2004))
    X, T, S = [], [], []
    for cfg in train_cfgs:
        tr = L.Trajectory(bas, cfg, 16)
        x, t, sc = L.samples(tr)
        X.append(x)
        T.append(t)
        S.append(sc)
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    X, T = L.importance_subsample(torch.cat(X), torch.cat(T), torch.cat(S), 400000, g)
    net = B.GuessNet(4096, G.flatten(G.init_params(7)))
    losses = L.train(net, X, T, 800, batch=4096, lr=1e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0]
    ratios, it_ext, it_net = [], 0, 0
    for cfg in test_cfgs:
        tr = L.Trajectory(bas, cfg, 16)
        e_ext, e_net = L.guess_errors(tr, net)
        ratios.append(np.mean(e_net / e_ext))
        # the same steps with the learned guess inside dirac_step (3 past states in the history)
        op = B.Operator(bas, cfg, tol=1e-12, precision=0, max_iter=1000, guess=2)
        B.set_guess(op, net)
        psi = tr.states[0].clone()
        hist = torch.zeros(3 * bas.n, dtype=torch.complex128, device="cuda")
        its, res, nh = op.step(psi, 16, cfg["t_start"], hist=hist, n_hist=0)
        assert nh == 3 and np.all(res <= 1e-12)
        assert torch.linalg.norm(psi - tr.states[-1]).item() <= 1e-9 * torch.linalg.norm(psi).item()
        it_ext += sum(tr.iters[3:])
        it_net += int(np.sum(its[3:]))
        # the captured graph driver with the learned guess gives the same steps bit for bit
        op2 = B.Operator(bas, cfg, tol=1e-12, precision=0, max_iter=1000, guess=2)
        B.set_guess(op2, net)
        psi2 = tr.states[0].clone()
        hist2 = torch.zeros(3 * bas.n, dtype=torch.complex128, device="cuda")
        its2, res2, nh2 = op2.run(psi2, 16, cfg["t_start"], hist2, n_hist=0)
        assert nh2 == 3 and np.array_equal(its, its2) and torch.equal(psi, psi2)
    print("learned / extrapolated guess error (held-out pulses):", np.round(ratios, 3),
          "iterations ext %d learned %d" % (it_ext, it_net))
    assert np.mean(ratios) < 0.7
    assert it_net <= it_ext
