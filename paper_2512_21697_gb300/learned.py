"""Training and evaluation driver of the learned initial guess.

Orchestration only: the states come from the library's time step, features, targets, the
network's forward and backward passes and Adam run in the library's kernels; torch holds the
device buffers and draws the sample indices.

Workflow: generate trajectories with the method itself (dirac_step, extrapolated guess) for seeded
pulse parameters, collect (features, target) pairs at every step that has four past states, train
with Adam on random mini-batches, then attach the network to an operator (solver option guess = 2).
"""
import math

import numpy as np

from . import binding as B
from . import workloads as W


def pulse_variants(base, seeds, E0=(0.02, 0.2), wavelength=(400.0, 1600.0), cycles=(2, 6)):
    """Seeded pulse parameter sets on one basis: E0 log-uniform, wavelength uniform, integer cycles."""
    out = []
    for s in seeds:
        g = np.random.default_rng(s)
        cfg = dict(base)
        cfg["E0"] = float(np.exp(g.uniform(math.log(E0[0]), math.log(E0[1]))))
        cfg["omega"] = W.omega_from_nm(float(g.uniform(*wavelength)))
        cfg["n_cycles"] = float(g.integers(cycles[0], cycles[1] + 1))
        T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
        cfg["t_start"] = float(g.uniform(0.1, 0.9)) * T
        out.append(cfg)
    return out


class Trajectory:
    """States of one run: psi at t_start + k dt for k = 0..n_steps (device complex128 tensors), from
    the ground state.  op: an operator of this pulse to reuse (one is made otherwise); t_start:
    the start time (default cfg["t_start"]), so one operator serves several windows of a pulse."""

    def __init__(self, bas, cfg, n_steps, precision=0, tol=1e-12, op=None, t_start=None):
        import torch
        self.cfg = dict(cfg)
        if t_start is not None:
            self.cfg["t_start"] = float(t_start)
        cfg = self.cfg
        self.bas = bas
        if op is None:
            op = B.Operator(bas, cfg, tol=tol, precision=precision, max_iter=1000, tol_inner=1e-5, max_outer=30,
                            guess=1)
        psi0, _ = bas.initial_state()
        psi = torch.from_numpy(psi0).cuda()
        hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device="cuda")
        nh = 0
        t = cfg["t_start"]
        self.states = [psi.clone()]
        self.iters = []
        for _ in range(n_steps):
            it, _, nh = op.step(psi, 1, t, hist=hist, n_hist=nh)
            self.iters.append(int(it[0]))
            t += cfg["dt"]
            self.states.append(psi.clone())
        self.op = op


def samples(traj):
    """(X, T, S) float32 device tensors over every position of every step n >= 3 of a trajectory:
    features, targets and the positions' scales s (positions with s = 0 are left out)."""
    import torch
    bas, cfg, st = traj.bas, traj.cfg, traj.states
    npos = bas.nch * (cfg["N"] + 1)
    xs, ts, ss = [], [], []
    for n in range(3, len(st) - 1):
        x = torch.empty((npos, 32), dtype=torch.float32, device="cuda")
        s = torch.empty(npos, dtype=torch.float32, device="cuda")
        tg = torch.empty((npos, 4), dtype=torch.float32, device="cuda")
        t_next = cfg["t_start"] + (n + 1) * cfg["dt"]
        B.guess_features(traj.op, [st[n], st[n - 1], st[n - 2], st[n - 3]], t_next, x, s)
        B.guess_targets(traj.op, [st[n], st[n - 1], st[n - 2]], st[n + 1], s, tg)
        keep = s > 0
        xs.append(x[keep])
        ts.append(tg[keep])
        ss.append(s[keep])
    return torch.cat(xs), torch.cat(ts), torch.cat(ss)


def importance_subsample(X, T, S, k, generator):
    """k samples drawn with probability proportional to s^2: the squared guess error of a position is
    s^2 |out - target|^2, so plain mean squared error over these samples is the relative guess
    error the solver sees (positions whose amplitude is at the solver's noise level, where the
    normalised target is large and random, carry their true, negligible weight)."""
    import torch
    w = S.double() ** 2
    idx = torch.multinomial(w / w.sum(), k, replacement=True, generator=generator)
    return X[idx].contiguous(), T[idx].contiguous()


def train(net, X, T, steps, batch=4096, lr=1e-3, seed=0, log_every=0):
    """Adam on random mini-batches (indices drawn with a seeded torch generator); returns losses."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    losses = []
    for k in range(steps):
        idx = torch.randint(0, X.shape[0], (min(batch, net.max_batch),), device="cuda", generator=g)
        xb, tb = X[idx].contiguous(), T[idx].contiguous()
        loss = net.train_step(xb, tb, lr)
        losses.append(loss)
        if log_every and k % log_every == 0:
            print("step %d loss %.4e" % (k, loss))
    return losses


def guess_errors(traj, net=None):
    """Relative error ||x0 - psi_{n+1}|| / ||psi_{n+1}|| of the extrapolated guess and, with a
    network, of the learned one, for every step n >= 3 of a trajectory (computed from its states)."""
    import torch
    bas, cfg, st = traj.bas, traj.cfg, traj.states
    npos = bas.nch * (cfg["N"] + 1)
    e_ext, e_net = [], []
    for n in range(3, len(st) - 1):
        y = st[n + 1]
        xe = 3 * st[n] - 3 * st[n - 1] + st[n - 2]
        e_ext.append((torch.linalg.norm(xe - y) / torch.linalg.norm(y)).item())
        if net is not None:
            x = torch.empty((npos, 32), dtype=torch.float32, device="cuda")
            s = torch.empty(npos, dtype=torch.float32, device="cuda")
            out = torch.empty((npos, 4), dtype=torch.float32, device="cuda")
            B.guess_features(traj.op, [st[n], st[n - 1], st[n - 2], st[n - 3]],
                             cfg["t_start"] + (n + 1) * cfg["dt"], x, s)
            net.forward(x, out, tensor_cores=True)
            c = (s[:, None].double() * out.double()).reshape(-1, 2, 2)
            corr = torch.complex(c[..., 0], c[..., 1]).reshape(-1)
            e_net.append((torch.linalg.norm(xe + corr - y) / torch.linalg.norm(y)).item())
    return np.array(e_ext), (np.array(e_net) if net is not None else None)
