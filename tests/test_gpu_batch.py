"""Batched solve (dirac_solve_batch) and its schedule autotuner (dirac_batch_tune).

Instances with different pulses and radial sizes run concurrently, each through its own captured
step driver; they must give exactly what per-instance dirac_run calls give (same kernels on the
same data), whatever the window, and match the oracle."""
import math

import numpy as np
import pytest

from paper_2512_21697_gb300 import binding as B, layout, workloads as W

pytestmark = pytest.mark.gpu

STEPS = 4


def _setup(n, precision=2, seed0=100):
    import torch
    cfgs = W.batch_instances(n, seed0=seed0, kappa_max=3, l_max=2, N_lo=40, N_hi=90, R=60.0)
    dev = torch.device("cuda")
    inst = []
    for cfg in cfgs:
        bas = B.Basis(cfg)
        psi0, _ = bas.initial_state()
        T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
        op = B.Operator(bas, cfg, stream=torch.cuda.Stream(), tol=cfg["tol"], precision=precision,
                        max_iter=1000, tol_inner=1e-5, max_outer=30)
        inst.append(dict(cfg=cfg, bas=bas, op=op, psi0=psi0, t0=0.3 * T,
                         psi=torch.from_numpy(psi0).to(dev),
                         hist=torch.zeros(2 * bas.n, dtype=torch.complex128, device=dev)))
    torch.cuda.synchronize()
    return inst


def _reference(inst):
    """Per-instance dirac_run on separate ops from the same starting states."""
    import torch
    out = []
    for d in inst:
        op = B.Operator(d["bas"], d["cfg"], tol=d["cfg"]["tol"], precision=d["op"].precision, max_iter=1000,
                        tol_inner=1e-5, max_outer=30)
        psi = torch.from_numpy(d["psi0"]).cuda()
        hist = torch.zeros_like(d["hist"])
        it, res, nh = op.run(psi, STEPS, d["t0"], hist, n_hist=0)
        out.append((psi, it, res, nh))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("window", [0, 2])
def test_batch_equals_single_runs(window):
    import torch
    inst = _setup(5)
    ref = _reference(inst)
    it, res, nh = B.solve_batch([d["op"] for d in inst], [d["psi"] for d in inst], [d["hist"] for d in inst],
                                STEPS, [d["t0"] for d in inst], window=window)
    for i, d in enumerate(inst):
        assert torch.equal(d["psi"], ref[i][0]), i
        assert np.array_equal(it[i], ref[i][1]) and np.array_equal(res[i], ref[i][2])
        assert nh[i] == ref[i][3] == 2
        assert np.all(res[i] <= d["cfg"]["tol"])


def test_batch_instance_matches_oracle(oracle_mod):
    inst = _setup(2, precision=0)
    B.solve_batch([d["op"] for d in inst], [d["psi"] for d in inst], [d["hist"] for d in inst], STEPS,
                  [d["t0"] for d in inst])
    d = inst[0]
    cfg = d["cfg"]
    orc = oracle_mod.Oracle(**W.oracle_params(cfg))
    perm = layout.lib_to_paper_perm(d["bas"].kappa, d["bas"].two_mu, cfg["kappa_max"], cfg["two_mu_max"], cfg["N"])
    ref, _ = orc.run(d["psi0"][perm], STEPS, d["t0"], tol=1e-14)
    got = d["psi"].cpu().numpy()[perm]
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_batch_tune_restores_states_and_keeps_results():
    import torch
    inst = _setup(4)
    ops, psis, hists = [d["op"] for d in inst], [d["psi"] for d in inst], [d["hist"] for d in inst]
    saved = [p.clone() for p in psis]
    cand = [1, 2, 0]
    best, ms = B.batch_tune(ops, psis, hists, [d["t0"] for d in inst], cand)
    assert best in cand
    assert ms.shape == (2, 3) and np.all(ms > 0)
    for p, q in zip(psis, saved):
        assert torch.equal(p, q)
    ref = _reference(inst)
    it, res, _ = B.solve_batch(ops, psis, hists, STEPS, [d["t0"] for d in inst], window=best)
    # the tuner may switch the preconditioner schedule: both solve to tol, so the states agree to
    # cond(A_+) tol with cond(A_+) ~ 10 on these physical states
    for i, d in enumerate(inst):
        assert np.all(res[i] <= d["cfg"]["tol"])
        assert torch.linalg.norm(psis[i] - ref[i][0]).item() <= 1e-9 * torch.linalg.norm(ref[i][0]).item()


def test_batch_rejects_bad_arguments():
    import torch
    inst = _setup(2)
    ops, psis, hists = [d["op"] for d in inst], [d["psi"] for d in inst], [d["hist"] for d in inst]
    with pytest.raises(RuntimeError):
        B.solve_batch([ops[0], ops[0]], [psis[0], psis[1]], [hists[0], hists[1]], 1, [0.0, 0.0])
    # an empty batch is a no-op
    it, res, nh = B.solve_batch([], [], [], 3, [])
    assert it.shape == (0, 3)
