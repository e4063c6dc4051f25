"""Failure paths of the step, made on the host (no GPU fault): an iteration cap that cannot be met
returns DIRAC_E_NOCONV, a non-finite state returns DIRAC_E_NUMERIC, through both drivers and in
the FP64 and mixed paths; the op and the context stay usable afterwards (a valid step still
matches the oracle)."""
import math

import numpy as np
import pytest

from paper_2512_21697_gb300 import binding as B, layout, workloads as W

pytestmark = pytest.mark.gpu

E_NOCONV, E_NUMERIC = 4, 6


def _peak(cfg):
    return 0.5 * cfg["n_cycles"] * 2 * math.pi / cfg["omega"]


def _state(bas, seed):
    import torch
    return torch.from_numpy(W.random_state(bas.n, seed)).cuda()


def _valid_step_matches_oracle(op, bas, cfg, oracle_mod):
    import torch
    orc = oracle_mod.Oracle(**W.oracle_params(cfg))
    perm = layout.lib_to_paper_perm(bas.kappa, bas.two_mu, cfg["kappa_max"], cfg["two_mu_max"], cfg["N"])
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    x = W.random_state(orc.n, 9)
    x[~orc.active_mask()] = 0
    x /= np.linalg.norm(x)
    psi = torch.from_numpy(x[inv].copy()).cuda()
    t = _peak(cfg)
    _, res, _ = op.step(psi, 1, t)
    ref, _, _ = orc.step(x, t, tol=1e-14)
    assert res[0] <= 1e-12
    assert np.linalg.norm(psi.cpu().numpy()[perm] - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [0, 2])
def test_iteration_cap_returns_noconv(oracle_mod, precision):
    import torch
    cfg = W.SMALL
    bas = B.Basis(cfg)
    # FP64: one BiCGSTAB iteration cannot reach 1e-14; mixed: one refinement pass cannot either
    op = B.Operator(bas, cfg, tol=1e-14, precision=precision, max_iter=1, tol_inner=1e-5, max_outer=1)
    psi = _state(bas, 3)
    with pytest.raises(B.DiracError) as ei:
        op.step(psi, 1, _peak(cfg))
    assert ei.value.status == E_NOCONV
    hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(B.DiracError) as ei:
        op.run(_state(bas, 3), 1, _peak(cfg), hist)
    assert ei.value.status == E_NOCONV
    ok = B.Operator(bas, cfg, tol=1e-12, precision=precision, max_iter=1000, tol_inner=1e-5, max_outer=30)
    _valid_step_matches_oracle(ok, bas, cfg, oracle_mod)


@pytest.mark.parametrize("precision", [0, 2])
def test_non_finite_state_returns_numeric(oracle_mod, precision):
    import torch
    cfg = W.SMALL
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg, tol=1e-12, precision=precision, max_iter=1000, tol_inner=1e-5, max_outer=30)
    psi = _state(bas, 4)
    psi[17] = complex(float("nan"), 0.0)
    with pytest.raises(B.DiracError) as ei:
        op.step(psi, 1, _peak(cfg))
    assert ei.value.status == E_NUMERIC
    psi = _state(bas, 4)
    psi[17] = complex(float("inf"), 0.0)
    hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(B.DiracError) as ei:
        op.run(psi, 1, _peak(cfg), hist)
    assert ei.value.status == E_NUMERIC
    # the same op still steps correctly
    _valid_step_matches_oracle(op, bas, cfg, oracle_mod)
