"""Plain FP64 CPU oracle of the learned initial guess (the network that predicts a step's BiCGSTAB
starting vector from the last states and the field).

TEST INFRASTRUCTURE ONLY: tests/ and ``__graft_entry__.smoke()`` are the only callers.  Plain
numpy, float64, written from the definitions below; it shares no code with the CUDA library.
Vectors are complex128 in the library's order ([channel][radial slot][DKB type], the order the
network's positions follow); nothing here depends on the basis beyond that order.

The guess is not part of the paper's method: it only changes where BiCGSTAB starts, and the
solver's own residual test still decides convergence, so the converged step is the same.

Definitions (per position p = (channel, radial slot r), both DKB types at that slot; 4 reals per
state: Re, Im of type 0, Re, Im of type 1):
  D_0 = psi_n, D_1 = psi_n - psi_{n-1}, D_2 = psi_n - 2 psi_{n-1} + psi_{n-2},
  D_3 = psi_n - 3 psi_{n-1} + 3 psi_{n-2} - psi_{n-3}        (backward differences)
  m_k = sqrt(mean of the 4 squares of D_k);  s = m_3 (the scale of the correction)
  x     = [D_k / m_k for k = 0..3 (16; zero where m_k = 0),
           clip(log10(m_j / m_3), -30, 30) / 10 for j = 0, 1, 2 (3; zero where m_j or m_3 is 0),
           the six field factors f(t_{n+1}), kappa / 10, 2 mu / 20, zeros]            (32)
  x_ext = 3 psi_n - 3 psi_{n-1} + psi_{n-2}                 (the extrapolated guess)
  net   : a1 = tanh(x W1 + b1), a2 = tanh(a1 W2 + b2), a3 = tanh(a2 W3 + b3), out = a3 W4 + b4
          with W1 32x256, W2 and W3 256x256, W4 256x4; the weights enter rounded to bfloat16
          (round to nearest, ties to even), biases in full precision
  guess = x_ext + s out                                   (zero correction where s = 0)
  target (training) = (psi_{n+1} - x_ext) / s ;  loss = mean over samples of sum_o (out - target)^2
  Adam  : m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
          w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), on the full-precision weights.
(A cubic extrapolation would add D_3 exactly, i.e. out = x[12:16]: the differences make the
correction an O(1) function of the inputs, which bfloat16 weights can represent.)
Field factors f(t): the vector potential's separable time functions, A0 = E0 / omega, three
carriers w_c = omega, omega + 2 pi / T, omega - 2 pi / T with weights 1/2, -1/4, -1/4:
  f = A0 wt_c (sin w_c t, cos w_c t) for c = 0, 1, 2, all zero outside 0 <= t <= T.
"""
import math

import numpy as np

NIN, NH, NOUT_NET, NFEAT = 32, 256, 4, 24
SHAPES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NH)), ("b3", (NH,)),
          ("W4", (NH, NOUT_NET)), ("b4", (NOUT_NET,))]


def bf16_round(w):
    """float -> nearest bfloat16 (8-bit significand), ties to even, returned as float64."""
    f = np.asarray(w, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) >> 16 << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def init_params(seed):
    """Seeded initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), last layer scaled by
    1e-2 so that the untrained network starts near the extrapolated guess; biases zero."""
    g = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name[0] == "b":
            p[name] = np.zeros(shp)
        else:
            a = 1.0 / math.sqrt(shp[0])
            w = g.uniform(-a, a, size=shp)
            if name == "W4":
                w *= 1e-2
            p[name] = w
    return p


def field_factors(t, E0, omega, n_cycles):
    T = n_cycles * 2 * math.pi / omega
    if t < 0 or t > T:
        return np.zeros(6)
    A0 = E0 / omega
    ws = [omega, omega + 2 * math.pi / T, omega - 2 * math.pi / T]
    wt = [0.5, -0.25, -0.25]
    f = []
    for w, c in zip(ws, wt):
        f += [A0 * c * math.sin(w * t), A0 * c * math.cos(w * t)]
    return np.array(f)


def differences(H):
    """H: [4][...] states psi_n .. psi_{n-3} -> the backward differences D_0 .. D_3."""
    return np.stack([H[0], H[0] - H[1], H[0] - 2 * H[1] + H[2], H[0] - 3 * H[1] + 3 * H[2] - H[3]])


def features(hist4, kappa, two_mu, f6):
    """hist4: [4][nch][n1][2] complex (psi_n, psi_{n-1}, psi_{n-2}, psi_{n-3}); returns
    x [nch * n1][32] and s [nch * n1]."""
    H = np.asarray(hist4)
    nch, n1 = H.shape[1], H.shape[2]
    D = differences(H)
    R = np.zeros((4, nch, n1, 4))
    for k in range(4):
        for t in range(2):
            R[k, :, :, 2 * t] = D[k, :, :, t].real
            R[k, :, :, 2 * t + 1] = D[k, :, :, t].imag
    m = np.sqrt(np.mean(R * R, axis=3))          # [4][nch][n1]
    x = np.zeros((nch, n1, NIN))
    for k in range(4):
        nz = m[k] > 0
        x[:, :, 4 * k:4 * k + 4][nz] = R[k][nz] / m[k][nz][:, None]
    for j in range(3):
        ok = (m[j] > 0) & (m[3] > 0)
        x[:, :, 16 + j][ok] = np.clip(np.log10(m[j][ok] / m[3][ok]), -30, 30) / 10
    x[:, :, 19:25] = f6
    x[:, :, 25] = (np.asarray(kappa, float) / 10.0)[:, None]
    x[:, :, 26] = (np.asarray(two_mu, float) / 20.0)[:, None]
    return x.reshape(nch * n1, NIN), m[3].reshape(-1)


def targets(hist3, psi_next, s):
    """(psi_{n+1} - x_ext) / s per position as [nch * n1][4] (zero where s = 0)."""
    H = np.asarray(hist3)
    d = np.asarray(psi_next) - extrapolate(H[0], H[1], H[2])
    r = np.stack([d[..., 0].real, d[..., 0].imag, d[..., 1].real, d[..., 1].imag], axis=-1).reshape(-1, 4)
    out = np.zeros_like(r)
    nz = s > 0
    out[nz] = r[nz] / s[nz][:, None]
    return out


def extrapolate(psi_n, psi_1, psi_2):
    return 3 * psi_n - 3 * psi_1 + psi_2


def forward(p, x, round_w=True, act_bf16=False):
    """Returns out and the activations (a1, a2, a3).  round_w=False uses the weights as given
    (for finite-difference checks of the gradient); act_bf16=True also rounds the input and every
    activation to bfloat16, as the tensor-core inference kernel stores them."""
    W = {k: (bf16_round(p[k]) if round_w else p[k]) for k in ("W1", "W2", "W3", "W4")}
    r = bf16_round if act_bf16 else (lambda a: a)
    a0 = r(x)
    a1 = r(np.tanh(a0 @ W["W1"] + p["b1"]))
    a2 = r(np.tanh(a1 @ W["W2"] + p["b2"]))
    a3 = r(np.tanh(a2 @ W["W3"] + p["b3"]))
    out = a3 @ W["W4"] + p["b4"]
    return out, (a1, a2, a3)


def loss_and_grads(p, x, target, round_w=True):
    """Mean squared error over the samples and its gradient with respect to every parameter (the
    gradient with respect to the bfloat16-rounded weights, applied to the full-precision ones)."""
    W = {k: (bf16_round(p[k]) if round_w else p[k]) for k in ("W1", "W2", "W3", "W4")}
    out, (a1, a2, a3) = forward(p, x, round_w)
    B = x.shape[0]
    d = out - target
    loss = float(np.sum(d * d) / B)
    g = {}
    dout = 2.0 * d / B
    g["W4"] = a3.T @ dout
    g["b4"] = dout.sum(0)
    d3 = (dout @ W["W4"].T) * (1 - a3 * a3)
    g["W3"] = a2.T @ d3
    g["b3"] = d3.sum(0)
    d2 = (d3 @ W["W3"].T) * (1 - a2 * a2)
    g["W2"] = a1.T @ d2
    g["b2"] = d2.sum(0)
    d1 = (d2 @ W["W2"].T) * (1 - a1 * a1)
    g["W1"] = x.T @ d1
    g["b1"] = d1.sum(0)
    return loss, g


def flatten(p):
    """Parameters as one float32 array in the library's order W1, b1, W2, b2, W3, b3, W4, b4."""
    return np.concatenate([np.asarray(p[k], np.float64).ravel() for k, _ in SHAPES]).astype(np.float32)


def unflatten(a):
    p, o = {}, 0
    for k, shp in SHAPES:
        n = int(np.prod(shp))
        p[k] = np.asarray(a[o:o + n], np.float64).reshape(shp)
        o += n
    return p


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (p, m, v)."""
    pn, mn, vn = {}, {}, {}
    for k in p:
        mn[k] = b1 * m[k] + (1 - b1) * g[k]
        vn[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = mn[k] / (1 - b1 ** t)
        vh = vn[k] / (1 - b2 ** t)
        pn[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return pn, mn, vn


def guess(p, hist4, kappa, two_mu, f6):
    """The network's initial guess for psi_{n+1} ([nch][n1][2] complex)."""
    H = np.asarray(hist4)
    x, s = features(H, kappa, two_mu, f6)
    out, _ = forward(p, x)
    nch, n1 = H.shape[1], H.shape[2]
    corr = (s[:, None] * out).reshape(nch, n1, 4)
    c = np.empty((nch, n1, 2), np.complex128)
    c[:, :, 0] = corr[:, :, 0] + 1j * corr[:, :, 1]
    c[:, :, 1] = corr[:, :, 2] + 1j * corr[:, :, 3]
    return extrapolate(H[0], H[1], H[2]) + c
