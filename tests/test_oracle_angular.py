"""Pins of the oracle's angular coupling, pulse expansion and interaction matrix elements.

Spinors (Eq. spinorbasis): orthonormality, sigma.r X_{kappa mu} = -X_{-kappa mu}.  Coupling
coefficients (Eq. Htheta): hand-derived closed forms for the 1s1/2 source, sum rules, symmetry,
brute-force 2D sphere quadrature, selection rules.  Pulse (Eq. ndpPot vs Eq. bdpA): the separable
plane-wave form equals the direct travelling sin^2 pulse.  Interaction (Eq. interactionH with
Eq. basis): Hermiticity of H(t) and a brute-force 3D quadrature of <psi_i|-c alpha.A|psi_j>.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2512_21697_gb300 import workloads as W


def lk(kappa):
    return kappa if kappa > 0 else -kappa - 1


def channels(kmax):
    for ak in range(1, kmax + 1):
        for kappa in (-ak, ak):
            for tm in range(-(2 * ak - 1), 2 * ak, 2):
                yield kappa, tm


def test_spinor_orthonormal(oracle_mod):
    x, w = np.polynomial.legendre.leggauss(24)
    nph = 16
    chans = list(channels(3))
    vals = {}
    for ch in chans:
        vals[ch] = np.array([[oracle_mod.spinor(ch[0], ch[1], math.acos(xi), 2 * math.pi * j / nph)
                              for j in range(nph)] for xi in x])
    for c1, c2 in itertools.product(chans, chans):
        ov = np.einsum("i,ijs,ijs->", w, vals[c1].conj(), vals[c2]) * 2 * math.pi / nph
        assert abs(ov - (1.0 if c1 == c2 else 0.0)) < 1e-13, (c1, c2, ov)


def test_sigma_r_maps_kappa_to_minus_kappa(oracle_mod):
    rng = np.random.default_rng(3)
    for kappa, tm in channels(4):
        for th, ph in rng.uniform([0, 0], [math.pi, 2 * math.pi], (5, 2)):
            sr = np.array([[math.cos(th), math.sin(th) * np.exp(-1j * ph)],
                           [math.sin(th) * np.exp(1j * ph), -math.cos(th)]])
            lhs = sr @ oracle_mod.spinor(kappa, tm, th, ph)
            assert np.abs(lhs + oracle_mod.spinor(-kappa, tm, th, ph)).max() < 1e-13


@pytest.mark.parametrize("l", range(0, 7))
def test_coupling_from_1s_closed_form(oracle_mod, l):
    # sigma_x (2l+1) P_l X_{-1,+1/2} = sqrt(2l+1) Y_l0 chi_down, whose projections are
    # sqrt(l+1) on X_{-l-1,-1/2} and sqrt(l) on X_{l,-1/2}; nothing else.
    tot = 0.0
    for kappa, tm in channels(l + 3):
        a = oracle_mod.angular(kappa, tm, -1, 1, l)
        if kappa == -l - 1 and tm == -1:
            assert abs(a - math.sqrt(l + 1)) < 1e-13
        elif kappa == l and tm == -1:
            assert abs(a - math.sqrt(l)) < 1e-13
        else:
            assert abs(a) < 1e-13, (kappa, tm, a)
        tot += a * a
    assert abs(tot - (2 * l + 1)) < 1e-12


def test_sigma_x_completeness(oracle_mod):
    # sigma_x^2 = 1 and sigma_x keeps the orbital l: sum over (kappa1, mu1) of a_0^2 is 1
    for kappa2, tm2 in channels(4):
        tot = sum(oracle_mod.angular(k1, t1, kappa2, tm2, 0) ** 2 for k1, t1 in channels(6))
        assert abs(tot - 1) < 1e-13, (kappa2, tm2)


def test_angular_symmetry_selection_and_bruteforce(oracle_mod):
    rng = np.random.default_rng(5)
    chans = list(channels(4))
    for _ in range(60):
        (k1, t1), (k2, t2) = chans[rng.integers(len(chans))], chans[rng.integers(len(chans))]
        l = int(rng.integers(0, 6))
        a = oracle_mod.angular(k1, t1, k2, t2, l)
        assert abs(a - oracle_mod.angular(k2, t2, k1, t1, l)) < 1e-13
        if abs(t1 - t2) != 2 or (lk(k1) + l + lk(k2)) % 2 or not (abs(lk(k1) - lk(k2)) <= l <= lk(k1) + lk(k2)):
            assert abs(a) < 1e-13
        b = oracle_mod.angular_2d(k1, t1, k2, t2, l, nth=30, nph=16)
        assert abs(a - b) < 1e-12, (k1, t1, k2, t2, l, a, b)


def test_edges_match_bruteforce_on_tiny(oracle_mod):
    p = W.oracle_params(W.TINY)
    o = oracle_mod.Oracle(**p)
    ea, eb = o.edges()
    got = set(zip(ea.tolist(), eb.tolist()))
    want = set()
    for a, b in itertools.product(range(o.nch), range(o.nch)):
        ka, ta, kb, tb = o.kappa[a], o.two_mu[a], o.kappa[b], o.two_mu[b]
        nz = any(abs(oracle_mod.angular_2d(ka, ta, -kb, tb, l, 24, 12)) > 1e-10 or
                 abs(oracle_mod.angular_2d(-ka, ta, kb, tb, l, 24, 12)) > 1e-10
                 for l in range(p["l_max"] + 1))
        if nz and a != b:
            want.add((a, b))
    assert got == want
    assert all((b, a) in got for a, b in got)


def test_edge_count_small(oracle_mod):
    o = oracle_mod.Oracle(**W.oracle_params(W.SMALL))
    ea, eb = o.edges()
    assert len(ea) == 120          # 60 coupled channel pairs at |kappa| <= 4, mu = +-1/2, l <= 2
    assert np.all(np.abs(o.two_mu[ea] - o.two_mu[eb]) == 2)


def test_spherical_bessel_closed_forms(oracle_mod):
    for x in (0.3, 1.0, 2.5, 4.0):
        s, c = math.sin(x), math.cos(x)
        assert abs(oracle_mod.sph_bessel(0, x) - s / x) < 1e-15
        assert abs(oracle_mod.sph_bessel(1, x) - (s / x ** 2 - c / x)) < 1e-15
        assert abs(oracle_mod.sph_bessel(2, x) - ((3 / x ** 2 - 1) * s / x - 3 * c / x ** 2)) < 1e-14
    x = 1e-3   # j_5(x) = x^5 / 11!! (1 - x^2 / 26 + ...)
    assert abs(oracle_mod.sph_bessel(5, x) - x ** 5 / 10395 * (1 - x * x / 26)) < 1e-14 * x ** 5 / 10395


def test_pulse_separable_form_equals_direct(oracle_mod):
    p = dict(W.oracle_params(W.SMALL), l_max=2)
    o = oracle_mod.Oracle(**p)
    T = p["n_cycles"] * 2 * math.pi / p["omega"]
    amp = p["E0"] / p["omega"]
    rng = np.random.default_rng(7)
    for t, r, ct in zip(rng.uniform(0, T, 30), rng.uniform(0.1, 50, 30), rng.uniform(-1, 1, 30)):
        d = o.field_direct(t, r, ct)
        s = o.field_series(t, r, ct, 14)
        assert abs(d - s) < 1e-14 * amp, (t, r, ct, d, s)
        # the paper's windowed pulse agrees wherever its window is open
        u = t - r * ct / p["c"]
        if 0 < u < T:
            ref = amp * math.sin(math.pi * u / T) ** 2 * math.sin(p["omega"] * u)
            assert abs(ref - d) < 1e-15 * amp
    assert o.field_F(-0.1, 1.0, 1) == 0 and o.field_F(T + 0.1, 1.0, 0) == 0


@pytest.fixture(scope="module")
def tiny(oracle_mod):
    return oracle_mod.Oracle(**dict(W.oracle_params(W.TINY), l_max=9))


def test_hamiltonian_hermitian(tiny):
    ea, eb = tiny.edges()
    t = 1.3
    for a, b in zip(ea, eb):
        if a < b:
            Xab = tiny.coupling_block(a, b, t)
            Xba = tiny.coupling_block(b, a, t)
            assert np.abs(Xab + Xba.T).max() <= 1e-14 * max(1e-300, np.abs(Xab).max())
            assert np.abs(Xab).max() > 0


def test_interaction_element_bruteforce_3d(tiny):
    # <psi_{a,i}| -c alpha.A(t) |psi_{b,j}> with the untruncated travelling pulse on a 3D grid
    ea, eb = tiny.edges()
    t = 1.3
    rng = np.random.default_rng(11)
    N1 = tiny.N + 1
    checked = 0
    for e in rng.choice(len(ea), 6, replace=False):
        a, b = int(ea[e]), int(eb[e])
        X = tiny.coupling_block(a, b, t)
        nz = np.argwhere(np.abs(X) > 1e-6 * np.abs(X).max())
        for i, j in nz[rng.choice(len(nz), 3, replace=False)]:
            ref = tiny.coupling_3d(a, int(i), b, int(j), t, nth=36, nph=16)
            assert abs(ref - 1j * X[i, j]) < 1e-11 * np.abs(X).max(), (a, b, i, j, ref, X[i, j])
            checked += 1
    assert checked == 18
    assert N1 == 13
