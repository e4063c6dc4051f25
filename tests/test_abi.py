"""Host-side checks of the C ABI (no GPU needed): every declared symbol is exported, argument
validation, and setup parity of the library's independently written basis/operator setup with
the oracle (radial matrices, initial state, angular coefficients, coupling blocks)."""
import os
import re

import numpy as np
import pytest

from paper_2512_21697_gb300 import binding as B, layout, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def libdirac():
    from paper_2512_21697_gb300 import build
    build.build()
    return B.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dirac.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dirac_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(libdirac):
    names = declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(libdirac, n), n
        assert n in B.SIGNATURES, n   # and bound in Python under the same name


def test_argument_validation(libdirac):
    import ctypes as C
    p = B.basis_params(dict(W.SMALL, N=3))       # fewer splines than the order
    h = C.c_void_p()
    assert libdirac.dirac_basis_build(C.byref(p), C.byref(h), None, None) == B.DIRAC_E_ARG
    assert b"out of range" in libdirac.dirac_last_error()
    p = B.basis_params(dict(W.SMALL, grid=1, n_lin=0))
    assert libdirac.dirac_basis_build(C.byref(p), C.byref(h), None, None) == B.DIRAC_E_ARG
    assert libdirac.dirac_basis_dim(None) == -1
    assert libdirac.dirac_step(None, None, None, None, 1, 0.0, None, None) == B.DIRAC_E_ARG
    assert libdirac.dirac_spectrum(None, None, 0.0, 1.0, 0, None, None, None) == B.DIRAC_E_ARG


def test_spectrum_error_matches_oracle(libdirac, oracle_mod):
    # host-only entry point: the trapezoid error integral against the oracle's, on closed forms too
    g = np.concatenate([np.linspace(0.0, 1.0, 11), np.linspace(1.05, 3.0, 40)])
    rng = np.random.default_rng(5)
    pn, pm = rng.random(len(g)), rng.random(len(g))
    for e1, e2 in [(0.0, 3.0), (0.33, 2.71), (1.0, 1.0), (5.0, 6.0)]:
        a = B.spectrum_error(g, pn, pm, e1, e2)
        b = oracle_mod.Oracle.spectrum_error(g, pn, pm, e1, e2)
        assert abs(a - b) <= 1e-14 * max(1.0, abs(b)), (e1, e2)
    assert abs(B.spectrum_error(g, pn + 0.3, pn, 0.0, 1.0) - 0.09) <= 1e-14
    with pytest.raises(B.DiracError):
        B.spectrum_error(g[::-1], pn, pm, 0.0, 3.0)      # a grid that does not ascend
    with pytest.raises(B.DiracError):
        B.spectrum_error(g, pn, pm, 2.0, 1.0)


def test_no_gpu_reports_state_error(libdirac):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes as C
    bas = B.Basis(W.TINY)
    pu, op = B.pulse_params(W.TINY), B.solver_opts(W.TINY)
    h = C.c_void_p()
    st = libdirac.dirac_operator_setup(bas._h, C.byref(pu), C.byref(op), None, C.byref(h))
    assert st == B.DIRAC_E_STATE


@pytest.fixture(scope="module", params=["small", "slice", "order5", "wide_l"])
def pair(request, oracle_mod, libdirac):
    cfg = W.WORKLOADS[request.param]
    return cfg, B.Basis(cfg), oracle_mod.Oracle(**W.oracle_params(cfg))


def test_radial_matrices_match_oracle(pair):
    cfg, bas, orc = pair
    p = layout.block_perm(cfg["N"])
    for kappa in (-1, 1, -2, 2, -cfg["kappa_max"], cfg["kappa_max"]):
        S, H = bas.radial(kappa)
        So, Ho = orc.radial(kappa)
        m = np.ones(orc.nb, bool)
        m[0] = kappa == -1
        m[cfg["N"] + 1] = kappa == 1
        Sp, Hp = S[np.ix_(p, p)], H[np.ix_(p, p)]
        assert np.abs(Sp - So)[np.ix_(m, m)].max() <= 1e-13 * np.abs(So).max()
        assert np.abs(Hp - Ho)[np.ix_(m, m)].max() <= 1e-13 * np.abs(Ho).max()


def test_initial_state_matches_oracle(pair):
    cfg, bas, orc = pair
    psi, e0 = bas.initial_state()
    psio, eo = orc.ground_state()
    perm = layout.lib_to_paper_perm(bas.kappa, bas.two_mu, cfg["kappa_max"], cfg["two_mu_max"], cfg["N"])
    assert abs(e0 - eo) < 1e-12
    assert np.abs(psi[perm] - psio).max() < 1e-11


def test_channel_pairs_match_oracle_edges(pair):
    cfg, bas, orc = pair
    ea, eb = orc.edges()
    assert 2 * bas.npairs == len(ea)


def test_angular_coefficients_two_routes(oracle_mod, libdirac):
    # library: Clebsch-Gordan x Gaunt (3j); oracle: quadrature of the spinors on the sphere
    rng = np.random.default_rng(4)
    chans = layout.paper_channels(12)
    for _ in range(400):
        (k1, t1), (k2, t2) = chans[rng.integers(len(chans))], chans[rng.integers(len(chans))]
        if abs(t1 - t2) != 2:
            t2 = t1 + 2 if abs(t1 + 2) <= 2 * abs(k2) - 1 else t1 - 2
            if abs(t2) > 2 * abs(k2) - 1:
                continue
        l = int(rng.integers(0, 10))
        a, b = B.angular(k1, t1, k2, t2, l), oracle_mod.angular(k1, t1, k2, t2, l)
        assert abs(a - b) < 1e-13 * max(1.0, abs(b)), (k1, t1, k2, t2, l, a, b)


def test_term_count_matches_oracle_angular(pair, oracle_mod):
    # dirac_basis_nterms: the (pair, l) terms with a nonzero angular coefficient (Eq. fullH with
    # Eq. Htheta), counted here from the oracle's quadrature of the spinors; every term couples
    # mu to mu +- 1 (x polarisation), which the factorised apply's grouping by mu relies on
    cfg, bas, _ = pair
    n = 0
    for a in range(bas.nch):
        for b in range(a + 1, bas.nch):
            ka, ta, kb, tb = int(bas.kappa[a]), int(bas.two_mu[a]), int(bas.kappa[b]), int(bas.two_mu[b])
            for l in range(cfg["l_max"] + 1):
                c1 = oracle_mod.angular(ka, ta, -kb, tb, l)
                c2 = oracle_mod.angular(-ka, ta, kb, tb, l)
                if abs(c1) > 1e-10 or abs(c2) > 1e-10:
                    assert abs(ta - tb) == 2, (ka, ta, kb, tb, l)
                    n += 1
    assert bas.nterms == n


def test_coupling_blocks_match_oracle(pair):
    cfg, bas, orc = pair
    ea, eb = orc.edges()
    p = layout.block_perm(cfg["N"])
    lib_index = {(int(k), int(m)): i for i, (k, m) in enumerate(zip(bas.kappa, bas.two_mu))}
    T = cfg["n_cycles"] * 2 * np.pi / cfg["omega"]
    rng = np.random.default_rng(2)
    for e in rng.choice(len(ea), 6, replace=False):
        a, b = int(ea[e]), int(eb[e])
        la = lib_index[(int(orc.kappa[a]), int(orc.two_mu[a]))]
        lb = lib_index[(int(orc.kappa[b]), int(orc.two_mu[b]))]
        t = float(rng.uniform(0, T))
        X = bas.coupling(cfg, la, lb, t)[np.ix_(p, p)]
        Xo = orc.coupling_block(a, b, t)
        # the two terms of Eq. fullH cancel near field zeros: compare against their scale c E0/w
        scale = cfg["c"] * cfg["E0"] / cfg["omega"]
        assert np.abs(X - Xo).max() <= 1e-13 * np.abs(Xo).max() + 1e-16 * scale, (a, b, t)
