"""Pins of the oracle's photoelectron spectrum (Sec. 4.3, Eq. dPdE) to facts other than itself:
completeness of the eigenvectors in the S inner product (the projections over every level add up
to the norm computed by the C oracle), the bound window against the C oracle's bound population,
a single eigenstate (a spike of height 1 / dE at its level, linear in between), closed-form level
spacings, the semiclassical density of continuum levels in a box, a library eigensolver on the
same dense matrices, and closed-form values of the error integral."""
import numpy as np
import pytest

import oracle
from paper_2512_21697_gb300 import workloads as W


@pytest.fixture(scope="module")
def orc():
    return oracle.Oracle(**W.oracle_params(W.TINY))


def _state(o, seed):
    x = W.random_state(o.n, seed)
    x[~o.active_mask()] = 0
    return x / np.linalg.norm(x)


def test_projections_over_every_level_give_the_norm(orc):
    x = _state(orc, 3)
    lv = orc.spectrum_levels(x, -np.inf, np.inf)
    tot = sum(float(np.sum(q)) for _, q in lv.values())
    nrm = orc.observables(x)["norm"]
    assert abs(tot - nrm) <= 1e-11 * nrm
    # and every level of every kappa is counted once
    for kappa, (E, q) in lv.items():
        assert len(E) == len(orc.eigen(kappa)[0])


def test_bound_window_matches_the_bound_population(orc):
    x = _state(orc, 4)
    c2 = orc.params.c ** 2
    lv = orc.spectrum_levels(x, -c2, 0.0)
    pb = sum(float(np.sum(q)) for _, q in lv.values())
    assert abs(pb - orc.observables(x)["p_bound"]) <= 1e-12
    # the windows partition the levels: negative branch + bound + continuum = norm
    neg = sum(float(np.sum(q)) for _, q in orc.spectrum_levels(x, -np.inf, -c2).values())
    pos = sum(float(np.sum(q)) for _, q in orc.spectrum_levels(x, 0.0, np.inf).values())
    assert abs(neg + pb + pos - orc.observables(x)["norm"]) <= 1e-11


def test_single_eigenstate_is_a_spike_of_inverse_spacing(orc):
    kappa, two_mu = -1, 1
    E, V = orc.eigen(kappa)
    pos = np.nonzero(E > 0)[0]
    k = int(pos[3])                      # an interior continuum level
    a = orc.channel(kappa, two_mu)
    x = np.zeros(orc.n, np.complex128)
    x[a * orc.nb:(a + 1) * orc.nb] = (0.6 - 0.8j) * V[k]   # |amplitude| = 1
    e_hi = float(E[pos[-1]])
    lv = orc.spectrum_levels(x, 0.0, e_hi)
    Ek, q = lv[kappa]
    j = int(np.nonzero(Ek == E[k])[0][0])
    expect = np.zeros(len(q))
    expect[j] = 1.0
    assert np.allclose(q, expect, atol=1e-12)
    for kap, (_, qq) in lv.items():
        if kap != kappa:
            assert np.all(qq == 0)
    dE = 0.5 * (E[k + 1] - E[k - 1])
    grid = [E[k], E[k + 1], 0.5 * (E[k] + E[k + 1]), E[k - 1], 0.25 * E[k - 1] + 0.75 * E[k]]
    P = orc.spectrum(x, 0.0, e_hi, grid)
    assert np.allclose(P, [1 / dE, 0.0, 0.5 / dE, 0.0, 0.75 / dE], rtol=1e-12, atol=1e-12 / dE)


def test_level_spacing_closed_forms():
    j = np.arange(7, dtype=np.float64)
    assert np.allclose(oracle.Oracle.level_spacing(0.3 + 0.25 * j), 0.25)
    d = oracle.Oracle.level_spacing(j ** 2)   # (j+1)^2 - (j-1)^2 = 4j inside
    assert np.allclose(d[1:-1], 2 * j[1:-1])
    assert d[0] == 1.0 and d[-1] == 36 - 25


def test_spectrum_integrates_to_the_continuum_population(orc):
    # q / dE interpolated and integrated over the levels' span is the Riemann sum of q up to the two
    # end half-cells: close to the projections' total, and far from it if dE were dropped
    x = _state(orc, 5)
    lv = orc.spectrum_levels(x, 0.0, np.inf)
    tot, inner = 0.0, 0.0
    for kappa, (E, q) in lv.items():
        tot += np.sum(q)
        inner += np.sum(q) - 0.5 * (q[0] + q[-1])
    e_max = max(E[-1] for E, _ in lv.values())
    grid = np.concatenate([np.linspace(0, 50, 20001), np.linspace(50, e_max, 20001)[1:]])
    P = orc.spectrum(x, 0.0, np.inf, grid)
    integral = float(np.sum(0.5 * (P[1:] + P[:-1]) * np.diff(grid)))
    assert abs(integral - inner) <= 0.05 * tot


def test_error_integral_closed_forms():
    g = np.linspace(0.0, 2.0, 21)
    p = np.sin(g)
    assert oracle.Oracle.spectrum_error(g, p, p, 0.0, 2.0) == 0.0
    # a constant difference 0.3 over [0.5, 1.5]: 0.09 * 1.0
    assert abs(oracle.Oracle.spectrum_error(g, p + 0.3, p, 0.5, 1.5) - 0.09) <= 1e-14
    # |difference| = E is a parabola under the square: the trapezoid rule's error h^2 (b - a) / 6
    # for f = E^2 on [0, 2] with h = 0.1 is 2 * 0.01 / 6 on top of 8 / 3
    err = oracle.Oracle.spectrum_error(g, p + g, p, 0.0, 2.0)
    assert abs(err - (8.0 / 3.0 + 0.02 / 6.0)) <= 1e-12


def test_continuum_level_spacing_follows_the_box_law():
    # continuum levels of a box of radius R: k R + ln(2 k R) / k (Coulomb phase, Z = 1) advances by
    # pi from one level to the next, so dE = k dk = pi k / (R + (1 - ln(2 k R)) / k^2) (the
    # nonrelativistic semiclassical law; k^2 = 2E(1 + E / 2c^2)).  A dropped factor in the spacing,
    # or levels from the wrong branch, miss it by far more than the 15 % allowed here.
    cfg = W.SMALL
    o = oracle.Oracle(**W.oracle_params(cfg))
    R, c = cfg["R"], cfg["c"]
    for kappa in (-1, 1, -2):
        E, _ = o.eigen(kappa)
        Ep = E[(E > 0.0) & (E < 3.0)]
        d = oracle.Oracle.level_spacing(Ep)[1:-1]
        Ei = Ep[1:-1]
        k = np.sqrt(2 * Ei * (1 + Ei / (2 * c * c)))
        pred = np.pi * k / (R + (1 - np.log(2 * k * R)) / k ** 2)
        sel = Ei > 0.2
        assert sel.sum() >= 20
        assert np.max(np.abs(d[sel] / pred[sel] - 1)) <= 0.15, kappa


def test_levels_and_projections_match_a_library_eigensolver(orc):
    # the C oracle's eigenpairs against scipy's generalised symmetric-definite solver on the same
    # dense S and H0 (only the functions the kappa uses): levels, and |v^T S psi|^2 (sign-free)
    import scipy.linalg as sl
    x = _state(orc, 6)
    lv = orc.spectrum_levels(x, -np.inf, np.inf)
    nb, N = orc.nb, orc.N
    for kappa, (E, q) in lv.items():
        S, H = orc.radial(kappa)
        act = np.ones(nb, bool)
        act[0] = kappa == -1
        act[N + 1] = kappa == 1
        Es, Vs = sl.eigh(H[np.ix_(act, act)], S[np.ix_(act, act)])
        assert np.allclose(E, Es, rtol=1e-10, atol=1e-10 * np.max(np.abs(Es)))
        qs = np.zeros(len(Es))
        for a in np.nonzero(orc.kappa == kappa)[0]:
            xa = x[a * nb:(a + 1) * nb][act]
            c = Vs.T @ (S[np.ix_(act, act)] @ xa)
            qs += np.abs(c) ** 2
        assert np.allclose(q, qs, rtol=1e-8, atol=1e-12)
