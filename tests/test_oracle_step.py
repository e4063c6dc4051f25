"""Pins of the oracle's Crank-Nicolson step (Eq. solPsi) and BiCGSTAB (Sec. 2.4).

Dense LU vs BiCGSTAB, the exact field-free phase law of the Cayley map, conservation of psi^H S psi,
time reversal, preconditioner independence, second-order accuracy of the midpoint rule and the
observables of the initial state.
"""
import math

import numpy as np
import pytest

from paper_2512_21697_gb300 import workloads as W


@pytest.fixture(scope="module")
def tiny(oracle_mod):
    return oracle_mod.Oracle(**W.oracle_params(W.TINY))


def masked_random(o, seed):
    x = W.random_state(o.n, seed)
    x[~o.active_mask()] = 0
    return x / np.linalg.norm(x)


def test_bicgstab_matches_dense_lu(tiny):
    psi = masked_random(tiny, 1)
    t = 2.0
    x_it, it, res = tiny.step(psi, t, tol=1e-14)
    x_lu = tiny.step_dense(psi, t)
    assert np.linalg.norm(x_it - x_lu) / np.linalg.norm(x_lu) < 1e-12
    # the dense solution satisfies A_+ x = A_- psi at t* = t + dt/2
    ts = t + 0.5 * W.TINY["dt"]
    Ap, Am = tiny.dense_operator(ts, +1), tiny.dense_operator(ts, -1)
    assert np.linalg.norm(Ap @ x_lu - Am @ psi) / np.linalg.norm(Am @ psi) < 1e-13
    # and the field is doing something: the step is far from the field-free one
    assert it > 2


def test_preconditioner_does_not_change_result(oracle_mod):
    # a short step keeps the unpreconditioned system solvable by plain BiCGSTAB
    o = oracle_mod.Oracle(**dict(W.oracle_params(W.TINY), dt=0.002))
    psi = masked_random(o, 2)
    a, ia, _ = o.step(psi, 1.0, tol=1e-13, precond=True)
    b, ib, _ = o.step(psi, 1.0, tol=1e-13, precond=False, max_iter=20000)
    # both solve A_+ x = b to a relative residual of 1e-13, so they differ by at most
    # 2 cond(A_+) 1e-13 (the active part of A_+; unused slots are the identity)
    m = o.active_mask()
    Ap = o.dense_operator(1.0 + 0.001, +1)[np.ix_(m, m)]
    cond = np.linalg.cond(Ap)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 2 * cond * 1e-13
    assert ib > ia


def s_norm(o, psi):
    return o.observables(psi)["norm"]


def test_norm_conservation_and_time_reversal(oracle_mod, tiny):
    psi0 = masked_random(tiny, 3)
    dt = W.TINY["dt"]
    n0 = s_norm(tiny, psi0)
    psi = psi0.copy()
    for s in range(6):
        psi, _, _ = tiny.step(psi, 0.5 + s * dt, tol=1e-14)
    assert abs(s_norm(tiny, psi) / n0 - 1) < 1e-12
    assert np.linalg.norm(psi - psi0) > 1e-3
    # stepping back with -dt over the same midpoints undoes the steps
    back = oracle_mod.Oracle(**dict(W.oracle_params(W.TINY), dt=-dt))
    for s in reversed(range(6)):
        psi, _, _ = back.step(psi, 0.5 + (s + 1) * dt, tol=1e-14)
    assert np.linalg.norm(psi - psi0) / np.linalg.norm(psi0) < 1e-11


def test_field_free_phase_law(oracle_mod):
    p = dict(W.oracle_params(W.SMALL), E0=0.0)
    o = oracle_mod.Oracle(**p)
    psi0, E = o.ground_state()
    tau = 0.5 * p["dt"]
    psi = psi0.copy()
    for s in range(8):
        psi, _, _ = o.step(psi, s * p["dt"], tol=1e-14)
    ph = np.exp(-2j * 8 * math.atan(tau * E))
    assert np.linalg.norm(psi - ph * psi0) < 1e-12
    # per-step phase of the closed-form 1s level c^2 (sqrt(1 - (Z/c)^2) - 1) at dt = 0.01
    c = p["c"]
    e1s = -c * c * (1 / c ** 2) / (1 + math.sqrt(1 - 1 / c ** 2))
    per_step = -np.angle(np.vdot(psi0, psi) / np.vdot(psi0, psi0)) / 8
    assert abs(per_step - 2 * math.atan(tau * e1s)) < 1e-10
    assert abs(2 * math.atan(tau * e1s) + 0.00500005614892) < 1e-13


def test_midpoint_rule_is_second_order(oracle_mod):
    # H evaluated at t + dt/2 (midpoint rule, Sec. 2.4) gives a second-order propagator; the
    # printed H(t + dt) of Eq. solPsi gives a first-order one.  Below dt ~ 0.02 an error floor
    # of ~1e-5 appears: the field populates negative-energy components whose phase per step
    # (dt c^2) is never small, so only the coarse pair dt = 0.1, 0.05 is in the asymptotic range.
    base = dict(W.oracle_params(W.TINY), E0=0.1)
    T_end, t0 = 0.8, 0.4

    def run(dt, te):
        o = oracle_mod.Oracle(**dict(base, dt=dt, time_eval=te))
        psi, _ = o.ground_state()
        for s in range(int(round(T_end / dt))):
            psi, _, _ = o.step(psi, t0 + s * dt, tol=1e-14)
        return psi

    err = {}
    for te, order in ((0, 2.0), (1, 1.0)):
        ref = run(0.003125, te)
        e1 = np.linalg.norm(run(0.1, te) - ref)
        e2 = np.linalg.norm(run(0.05, te) - ref)
        assert abs(math.log2(e1 / e2) - order) < 0.2, (te, e1, e2)
        err[te] = e2
    assert err[1] > 5 * err[0]


def test_initial_state_observables(oracle_mod):
    o = oracle_mod.Oracle(**W.oracle_params(W.SMALL))
    psi0, E = o.ground_state()
    obs = o.observables(psi0)
    assert abs(obs["norm"] - 1) < 1e-13
    assert abs(obs["energy"] - E) < 1e-12
    assert abs(obs["p_ground"] - 1) < 1e-12
    assert abs(obs["p_bound"] - 1) < 1e-12


def test_bound_population_of_eigen_combination(oracle_mod):
    # psi = sum over channels of sum_e c_e v_e with S-orthonormal eigenvectors v_e of H0_kappa:
    # the norm is sum |c_e|^2 and the bound population sum over -c^2 < E_e < 0 of |c_e|^2
    # (Sec. 4.3), whatever the coefficients; a missing S, a wrong energy window or a channel left
    # out of the sum breaks one of the two
    o = oracle_mod.Oracle(**W.oracle_params(W.TINY))
    c2 = o.params.c ** 2
    rng = np.random.default_rng(3)
    psi = np.zeros(o.n, np.complex128)
    exp_b = exp_n = 0.0
    nbound = 0
    for ch, kappa in enumerate(o.kappa):
        E, V = o.eigen(int(kappa))
        coef = 0.1 * (rng.normal(size=len(E)) + 1j * rng.normal(size=len(E)))
        psi[ch * o.nb:(ch + 1) * o.nb] = coef @ V
        bound = (E > -c2) & (E < 0)
        nbound += int(bound.sum())
        exp_b += float(np.sum(np.abs(coef[bound]) ** 2))
        exp_n += float(np.sum(np.abs(coef) ** 2))
    assert 0 < nbound < o.n // 2
    obs = o.observables(psi)
    assert abs(obs["norm"] - exp_n) <= 1e-11 * exp_n
    assert abs(obs["p_bound"] - exp_b) <= 1e-11 * exp_n
