"""The photoelectron spectrum (Sec. 4.3, Eq. dPdE) on the GPU against the oracle: propagated and
random states on the small workloads, a single eigenstate (a spike of 1 / dE at its level), window
changes and reuse, empty windows and grids; at the production size, the property that the ground
state has no continuum part."""
import numpy as np
import pytest

import oracle
from paper_2512_21697_gb300 import binding as B, layout, workloads as W

pytestmark = pytest.mark.gpu


def _setup(cfg):
    bas = B.Basis(cfg)
    orc = oracle.Oracle(**W.oracle_params(cfg))
    perm = layout.lib_to_paper_perm(bas.kappa, bas.two_mu, cfg["kappa_max"], cfg["two_mu_max"], cfg["N"])
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    return bas, orc, perm, inv


def _window_clear(orc, e_lo, e_hi):
    # no level within 1e-8 of the window's ends, so both sides select the same levels
    for kappa in set(int(k) for k in orc.kappa):
        E, _ = orc.eigen(kappa)
        assert np.all(np.abs(E - e_lo) > 1e-8) and np.all(np.abs(E - e_hi) > 1e-8)


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_spectrum_of_a_propagated_state_matches_oracle(name):
    import torch
    cfg = W.WORKLOADS[name]
    bas, orc, perm, inv = _setup(cfg)
    psi0, _ = orc.ground_state()
    x = psi0.copy()
    # a few CN steps at the pulse's peak populate the continuum
    T = cfg["n_cycles"] * 2 * np.pi / cfg["omega"]
    for s in range(4):
        x, _, _ = orc.step(x, 0.5 * T + s * cfg["dt"], tol=1e-14)
    e_lo, e_hi = 0.0, 40.0
    _window_clear(orc, e_lo, e_hi)
    grid = np.linspace(-1.0, 45.0, 777)
    ref = orc.spectrum(x, e_lo, e_hi, grid)
    op = B.Operator(bas, cfg, tol=1e-12)
    got, nl = op.spectrum(torch.from_numpy(x[inv].copy()).cuda(), e_lo, e_hi, grid)
    lv = orc.spectrum_levels(x, e_lo, e_hi)
    assert nl == sum(len(E) for E, _ in lv.values())
    assert np.max(ref) > 0
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    # the error integral through the library equals the oracle's
    e_a = B.spectrum_error(grid, got, ref * 1.01, 0.5, 30.0)
    e_b = orc.spectrum_error(grid, got, ref * 1.01, 0.5, 30.0)
    assert abs(e_a - e_b) <= 1e-12 * abs(e_b)


def test_spectrum_of_random_state_and_window_reuse():
    import torch
    cfg = W.SMALL
    bas, orc, perm, inv = _setup(cfg)
    x = W.random_state(orc.n, 21)
    x[~orc.active_mask()] = 0
    x /= np.linalg.norm(x)
    xd = torch.from_numpy(x[inv].copy()).cuda()
    op = B.Operator(bas, cfg, tol=1e-12)
    grid = np.linspace(0.0, 60.0, 501)
    res = {}
    for (lo, hi) in [(0.0, 50.0), (5.0, 25.0), (0.0, 50.0)]:
        _window_clear(orc, lo, hi)
        got, _ = op.spectrum(xd, lo, hi, grid)
        ref = orc.spectrum(x, lo, hi, grid)
        assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref)), (lo, hi)
        if (lo, hi) in res:
            assert np.array_equal(res[(lo, hi)], got)   # recomputed window: same result bit for bit
        res[(lo, hi)] = got


def test_single_eigenstate_spike():
    import torch
    cfg = W.SMALL
    bas, orc, perm, inv = _setup(cfg)
    kappa, two_mu = 2, 1
    E, V = orc.eigen(kappa)
    pos = np.nonzero((E > 0) & (E <= 30.0))[0]
    k = int(pos[len(pos) // 2])
    a = orc.channel(kappa, two_mu)
    x = np.zeros(orc.n, np.complex128)
    x[a * orc.nb:(a + 1) * orc.nb] = (0.28 + 0.96j) * V[k]
    op = B.Operator(bas, cfg, tol=1e-12)
    grid = np.array([E[k], E[k + 1], 0.5 * (E[k] + E[k + 1]), E[k - 1]])
    got, _ = op.spectrum(torch.from_numpy(x[inv].copy()).cuda(), 0.0, 30.0, grid)
    dE = 0.5 * (E[k + 1] - E[k - 1])
    # the other kappas' continua are orthogonal to this state up to rounding
    assert np.allclose(got, [1 / dE, 0.0, 0.5 / dE, 0.0], rtol=1e-9, atol=1e-9 / dE)


def test_empty_window_grid_and_bad_arguments():
    import torch
    cfg = W.TINY
    bas, orc, perm, inv = _setup(cfg)
    op = B.Operator(bas, cfg, tol=1e-12)
    xd = torch.from_numpy(W.random_state(orc.n, 2)[inv].copy()).cuda()
    E_all = np.concatenate([orc.eigen(int(k))[0] for k in set(orc.kappa)])
    top = float(np.max(E_all))
    got, nl = op.spectrum(xd, top + 1.0, top + 2.0, np.linspace(top, top + 3, 7))
    assert nl == 0 and np.all(got == 0)
    got, nl = op.spectrum(xd, 0.0, 10.0, np.zeros(0))
    assert len(got) == 0 and nl > 0
    for lo, hi in [(1.0, 1.0), (2.0, 1.0), (0.0, np.inf), (np.nan, 1.0)]:
        with pytest.raises(B.DiracError):
            op.spectrum(xd, lo, hi, np.linspace(0, 1, 3))
    with pytest.raises(B.DiracError):
        op.spectrum(xd, 0.0, 1.0, np.array([0.0, np.nan]))


def test_production_ground_state_has_no_continuum():
    import torch
    cfg = W.PRODUCTION
    bas = B.Basis(cfg)
    psi0, _ = bas.initial_state()
    op = B.Operator(bas, cfg, tol=1e-10, precision=2)
    grid = np.linspace(0.0, 2.0, 201)
    got, nl = op.spectrum(torch.from_numpy(psi0).cuda(), 0.0, 2.0, grid)
    # the ground state is an eigenvector of H0 in the basis: orthogonal to every continuum level,
    # so only rounding is left (the densities are |projection|^2 / dE with dE ~ 1e-2)
    assert nl > 1000
    assert np.all(got >= 0) and np.max(got) <= 1e-20
