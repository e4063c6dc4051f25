"""Pins of the learned-guess oracle (oracle/guess_net.py) against definitions it does not share:
bfloat16 rounding against exact halfway cases and torch's conversion, back-propagation against
finite differences, Adam's first step against its closed form, the difference features against
a cubic-in-time sequence, and the field factors against the sin^2 envelope identity."""
import math

import numpy as np
import pytest

from oracle import guess_net as G


def test_bf16_round_halfway_cases_and_library():
    # ulp(1) in bfloat16 is 2^-7: 1 + 2^-8 is halfway to an odd neighbour -> 1; 1 + 3 2^-8 is
    # halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even) -> 1 + 2^-6
    v = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 2.0 ** -130])
    r = G.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2 ** -6 and r[3] == -2.5
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).uniform(-5, 5, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(G.bf16_round(x), ref)


def _small_problem(seed=0, B=6):
    g = np.random.default_rng(seed)
    p = G.init_params(seed)
    p["W4"] *= 50.0   # a last layer of ordinary size, so every layer's gradient is exercised
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = 0.1 * g.standard_normal(p[k].shape)
    x = g.standard_normal((B, G.NIN))
    t = g.standard_normal((B, G.NOUT_NET))
    return p, x, t


def test_backprop_matches_finite_differences():
    p, x, t = _small_problem()
    _, grad = G.loss_and_grads(p, x, t, round_w=False)
    g = np.random.default_rng(5)
    h = 1e-6
    for name, shp in G.SHAPES:
        for _ in range(6):
            idx = tuple(int(g.integers(0, s)) for s in shp)
            q = {k: v.copy() for k, v in p.items()}
            q[name][idx] += h
            lp, _ = G.loss_and_grads(q, x, t, round_w=False)
            q[name][idx] -= 2 * h
            lm, _ = G.loss_and_grads(q, x, t, round_w=False)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, grad[name][idx])


def test_rounded_gradient_is_the_gradient_at_the_rounded_weights():
    p, x, t = _small_problem(1)
    l1, g1 = G.loss_and_grads(p, x, t, round_w=True)
    pr = {k: (G.bf16_round(v) if k[0] == "W" else v) for k, v in p.items()}
    l2, g2 = G.loss_and_grads(pr, x, t, round_w=False)
    assert l1 == l2
    for k in g1:
        assert np.array_equal(g1[k], g2[k])


def test_adam_first_step_closed_form():
    # t = 1: m = (1-b1) g, v = (1-b2) g^2, so the update is -lr g / (|g| + eps)
    p = {"w": np.array([0.5, -1.0, 2.0, 0.0])}
    g = {"w": np.array([3.0, -1e-3, 0.0, 1e-12])}
    z = {"w": np.zeros(4)}
    lr, eps = 1e-2, 1e-8
    pn, _, _ = G.adam_step(p, g, z, z, 1, lr=lr, eps=eps)
    exp = p["w"] - lr * g["w"] / (np.abs(g["w"]) + eps)
    assert np.allclose(pn["w"], exp, rtol=1e-12, atol=1e-15)


def test_features_and_targets_of_a_cubic_in_time():
    # psi(t) = c0 + c1 t + c2 t^2 + c3 t^3 at t = 0, -1, -2, -3 (psi_n .. psi_{n-3}) and t = 1:
    # D_3 = 6 c3 and psi(1) - x_ext = 6 c3, so the target equals the D_3 direction x[12:16]
    g = np.random.default_rng(2)
    nch, n1 = 3, 5
    c = [g.standard_normal((nch, n1, 2)) + 1j * g.standard_normal((nch, n1, 2)) for _ in range(4)]
    psi = lambda t: c[0] + c[1] * t + c[2] * t ** 2 + c[3] * t ** 3
    H = np.stack([psi(0), psi(-1), psi(-2), psi(-3)])
    H[:, 1, 2] = 0   # one position with no signal at all
    f6 = np.arange(6) * 0.1
    x, s = G.features(H, [1, -2, 3], [1, -1, 3], f6)
    nxt = psi(1)
    nxt[1, 2] = 0
    tg = G.targets(H[:3], nxt, s)
    k = 1 * n1 + 2
    assert s[k] == 0 and np.all(x[k, :19] == 0) and np.all(tg[k] == 0)
    m = np.ones(nch * n1, bool)
    m[k] = False
    assert np.allclose(tg[m], x[m, 12:16], rtol=1e-9, atol=1e-9)
    d3 = 6 * c[3]
    r3 = np.stack([d3[..., 0].real, d3[..., 0].imag, d3[..., 1].real, d3[..., 1].imag], -1).reshape(-1, 4)
    assert np.allclose(s[m], np.sqrt(np.mean(r3[m] ** 2, axis=1)), rtol=1e-9)
    assert np.allclose(x[:, 19:25], f6) and np.allclose(x[:n1, 25], 0.1) and np.allclose(x[n1:2 * n1, 26], -0.05)
    # unit-rms directions
    assert np.allclose(np.sqrt(np.mean(x[m, 0:4] ** 2, axis=1)), 1.0)


def test_field_factors_follow_the_sin2_envelope():
    E0, w, nc = 0.07, 0.057, 3.0
    T = nc * 2 * math.pi / w
    A0 = E0 / w
    for t in np.linspace(0, T, 37):
        f = G.field_factors(t, E0, w, nc)
        env = math.sin(math.pi * t / T) ** 2
        assert abs(f[0] + f[2] + f[4] - A0 * env * math.sin(w * t)) < 1e-13
        assert abs(f[1] + f[3] + f[5] - A0 * env * math.cos(w * t)) < 1e-13
    assert np.all(G.field_factors(T * 1.01, E0, w, nc) == 0) and np.all(G.field_factors(-1.0, E0, w, nc) == 0)


def test_guess_with_silent_last_layer_is_the_extrapolation():
    g = np.random.default_rng(4)
    p = G.init_params(4)
    p["W4"][:] = 0
    H = g.standard_normal((4, 2, 3, 2)) + 1j * g.standard_normal((4, 2, 3, 2))
    x = G.guess(p, H, [1, -1], [1, 1], np.zeros(6))
    assert np.allclose(x, 3 * H[0] - 3 * H[1] + H[2], rtol=0, atol=1e-15)


def test_flatten_round_trip():
    p = G.init_params(7)
    a = G.flatten(p)
    assert a.size == 32 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 4 + 4
    q = G.unflatten(a)
    for k in p:
        assert np.allclose(q[k], p[k].astype(np.float32))
