"""GPU parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (double precision everywhere):
 - operator apply: |y_gpu - y_oracle| <= 1e-12 max|y| -- sums of ~10^3 terms of size <= max|A| max|x|
   in a different order differ by ~10^3 eps relative to that scale.
 - preconditioner: relative 2-norm 1e-10 -- two LU factorisations of a matrix with condition
   number up to ~1e4 (dense vs banded, different pivot order) agree to cond * eps.
 - CN step / run: wavefunction relative L2 <= 1e-10, observables <= 1e-9 (the stated parity bar);
   the oracle solves to 1e-14.  A solve to relative residual tol leaves an error up to
   cond(A_+) tol; random states carry high-energy components where cond(A_+) reaches ~1e3, so the
   random-state step checks solve to 1e-13 (the physical-state full run uses the workload's 1e-12).
"""
STEP_TOL = 1e-13
# Mixed-precision steps (refinement passes and inner iterations).  From psi_n as the guess, a random
# state's first residual is O(||b||); each inner complex64 solve reduces it by tol_inner = 1e-5 (the
# FP32 operator's own error, ~1e-6 relative, is below that), so STEP_TOL = 1e-13 needs
# ceil(13 / 5) = 3 inner solves and 4 accurate residual passes per step, the bound asserted.  A
# wrong inner operator (relative error e) reduces the residual by about max(e, tol_inner) per pass
# instead, so an error above ~1e-5 needs a fifth pass and fails.  The inner iterations are bounded by
# twice the oracle's own preconditioned BiCGSTAB count to 1e-14 (14 decades against the inner
# solves' 15) plus 8.
MAX_PASSES_PER_STEP = 4
import math

import numpy as np
import pytest

from paper_2512_21697_gb300 import binding as B, layout, workloads as W

pytestmark = pytest.mark.gpu


def refinement_counts(op, fn):
    """Run fn() with the op's phase counters on; returns the accurate residual passes (timed launch
    groups of the 'apply' phase: in precision 1 one more per step forms b = A_- psi)."""
    op.profile(True)
    fn()
    _, cnt, _ = op.profile_read()
    op.profile(False)
    return int(cnt["apply"])


def check_refinement(op, precision, nsteps, passes, its, oracle_its):
    rhs = nsteps if precision == 1 else 0
    per_step = (passes - rhs) / nsteps
    assert per_step <= MAX_PASSES_PER_STEP, (passes, nsteps)
    for k, (a, b) in enumerate(zip(its, oracle_its)):
        assert a <= 2 * b + 8, ("inner iterations", k, a, b)
    return per_step


class Case:
    def __init__(self, cfg, oracle_mod, **opt):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.bas = B.Basis(cfg)
        self.orc = oracle_mod.Oracle(**W.oracle_params(cfg))
        self.perm = layout.lib_to_paper_perm(self.bas.kappa, self.bas.two_mu, cfg["kappa_max"],
                                             cfg["two_mu_max"], cfg["N"])
        self.inv = np.empty_like(self.perm)
        self.inv[self.perm] = np.arange(len(self.perm))
        self.op = B.Operator(self.bas, cfg, **opt)
        self.dev = torch.device("cuda")

    def to_dev(self, x_paper):
        return self.torch.from_numpy(np.ascontiguousarray(x_paper[self.inv])).to(self.dev)

    def from_dev(self, xd):
        return xd.cpu().numpy()[self.perm]

    def random(self, seed):
        x = W.random_state(self.orc.n, seed)
        x[~self.orc.active_mask()] = 0
        return x / np.linalg.norm(x)

    def T(self):
        return self.cfg["n_cycles"] * 2 * math.pi / self.cfg["omega"]


@pytest.fixture(scope="module", params=["tiny", "small", "slice", "order5"])
def case(request, oracle_mod):
    cfg = W.WORKLOADS[request.param]
    return Case(cfg, oracle_mod, tol=STEP_TOL, max_iter=1000)


def test_apply_matches_oracle(case):
    x = case.random(1)
    xd = case.to_dev(x)
    yd = case.torch.empty_like(xd)
    for sign in (+1, -1):
        for t in (0.0, 0.37 * case.T(), 0.81 * case.T()):
            case.op.apply(sign, t, xd, yd)
            y = case.from_dev(yd)
            ref = case.orc.apply(t, sign, x)
            assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max(), (sign, t)
            # unused functions stay untouched (identity)
            assert np.all(y[~case.orc.active_mask()] == 0)


@pytest.mark.parametrize("sched", [1, 2, 3])
def test_precond_matches_oracle(case, sched):
    # the complex128 schedules (warp per channel; staged through shared memory; rows fixed to lanes)
    r = case.random(2)
    rd = case.to_dev(r)
    zd = case.torch.empty_like(rd)
    keep = case.op.schedule(False)
    if sched > 1 and case.cfg["order"] != 7:
        # the staged and rotated-lane kernels are built for 13 block-diagonals: refused elsewhere
        with pytest.raises(B.DiracError):
            case.op.set_schedule(False, sched)
        return
    case.op.set_schedule(False, sched)
    case.op.precond(rd, zd)
    case.op.set_schedule(False, keep)
    z = case.from_dev(zd)
    ref = case.orc.precond(r)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)
    if sched == 3:
        # the same operations in the same order as the shifting-window warp kernel
        z1 = case.torch.empty_like(rd)
        case.op.set_schedule(False, 1)
        case.op.precond(rd, z1)
        case.op.set_schedule(False, keep)
        assert case.torch.equal(zd, z1)


@pytest.mark.parametrize("sched", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["small", "tail"])
def test_mixed_step_each_precond_schedule(oracle_mod, name, sched):
    # the complex64 inner solve with every preconditioner schedule: the refinement ends on the
    # accurate residual, so the step meets the FP64 parity bar whichever schedule the inner solve
    # used; the three warp schedules give bitwise identical states
    cfg = W.WORKLOADS[name]
    c = Case(cfg, oracle_mod, tol=STEP_TOL, max_iter=1000, precision=2, tol_inner=1e-5, max_outer=30)
    c.op.set_schedule(True, sched)
    psi0 = c.random(21)
    t0 = 0.5 * c.T()
    psid = c.to_dev(psi0)
    out = {}
    passes = refinement_counts(c.op, lambda: out.update(r=c.op.step(psid, 2, t0)))
    its, res, _ = out["r"]
    ref = psi0.copy()
    oits = []
    for s in range(2):
        ref, it, _ = c.orc.step(ref, t0 + s * cfg["dt"], tol=1e-14)
        oits.append(it)
    assert np.all(res <= STEP_TOL)
    assert np.linalg.norm(c.from_dev(psid) - ref) <= 1e-10 * np.linalg.norm(ref)
    pps = check_refinement(c.op, 2, 2, passes, its, oits)
    print("mixed %s sched %d: passes/step %.1f, inner %s, oracle %s" % (name, sched, pps, list(its), oits))
    if sched in (2, 3):
        c2 = Case(cfg, oracle_mod, tol=STEP_TOL, max_iter=1000, precision=2, tol_inner=1e-5, max_outer=30)
        c2.op.set_schedule(True, 1)
        pd2 = c2.to_dev(psi0)
        c2.op.step(pd2, 2, t0)
        assert c.torch.equal(psid, pd2)


def test_step_matches_oracle(case):
    # a few steps inside the pulse (peak-field window) from a random state
    psi0 = case.random(3)
    t0 = 0.5 * case.T()
    n = 3
    psid = case.to_dev(psi0)
    its, res, _ = case.op.step(psid, n, t0)
    ref = psi0.copy()
    for s in range(n):
        ref, _, _ = case.orc.step(ref, t0 + s * case.cfg["dt"], tol=1e-14)
    got = case.from_dev(psid)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.all(res <= STEP_TOL)
    assert np.all(got[~case.orc.active_mask()] == 0)


def test_bound_population_matches_oracle(case):
    # bound-state population (cuSOLVER eigenvectors + projection kernel) against the oracle's
    # Jacobi eigenvectors, on a random state and on the ground state.  The projector on the bound
    # subspace computed by two eigensolvers differs by ~eps ||H0|| / gap, with ||H0|| ~ 2 c^2 (the
    # negative-energy branch) and the gap between the highest bound and the lowest box state
    # ~1e-3: a few 1e-11 here; the bar is the stated observable tolerance 1e-9
    for seed in (7, 8):
        x = case.random(seed)
        got = case.op.observables(case.to_dev(x), bound=True)
        ref = case.orc.observables(x)
        for k in ("norm", "energy", "p_ground"):
            assert abs(got[k] - ref[k]) <= 1e-11 * max(1.0, abs(ref[k])), (k, got[k], ref[k])
        assert abs(got["p_bound"] - ref["p_bound"]) <= 1e-9, (got["p_bound"], ref["p_bound"])
    psi0, _ = case.orc.ground_state()
    got = case.op.observables(case.to_dev(psi0), bound=True)
    assert abs(got["p_bound"] - 1) <= 1e-11


def test_small_full_run_matches_oracle(oracle_mod):
    # the 200-step small workload from the 1s1/2 state, tol 1e-12; oracle at 1e-14
    cfg = W.SMALL
    c = Case(cfg, oracle_mod, tol=cfg["tol"], max_iter=1000)
    psi0, _ = c.orc.ground_state()
    psid = c.to_dev(psi0)
    hist = c.torch.zeros(2 * c.bas.n, dtype=c.torch.complex128, device=c.dev)
    its, res, nh = c.op.step(psid, cfg["steps"], 0.0, hist=hist, n_hist=0)
    ref, _ = c.orc.run(psi0, cfg["steps"], 0.0, tol=1e-14)
    got = c.from_dev(psid)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    o_gpu = c.op.observables(psid, bound=True)
    o_ref = c.orc.observables(ref)
    for k in ("norm", "energy", "p_ground", "p_bound"):
        assert abs(o_gpu[k] - o_ref[k]) <= 1e-9 * max(1.0, abs(o_ref[k])), k
    assert nh == 2 and np.all(res <= cfg["tol"])


def test_production_apply_sampled_rows(oracle_mod):
    # full production operator on the GPU; the oracle computes sampled rows one by one
    import torch
    cfg = W.PRODUCTION
    bas = B.Basis(cfg)
    orc = oracle_mod.Oracle(**W.oracle_params(cfg))
    op = B.Operator(bas, cfg, tol=cfg["tol"])
    perm = layout.lib_to_paper_perm(bas.kappa, bas.two_mu, cfg["kappa_max"], cfg["two_mu_max"], cfg["N"])
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    x = W.random_state(orc.n, 5)
    x[~orc.active_mask()] = 0
    xd = torch.from_numpy(x[inv]).cuda()
    yd = torch.empty_like(xd)
    T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
    t = 0.43 * T
    op.apply(+1, t, xd, yd)
    y = yd.cpu().numpy()[perm]
    rng = np.random.default_rng(9)
    nb = orc.nb
    rows = np.concatenate([rng.choice(orc.n, 40, replace=False),
                           [0, nb - 1, orc.n - 1, orc.n - nb, nb * 900 + cfg["N"], nb * 1859 + 2 * cfg["N"] + 1]])
    ch, idx = rows // nb, rows % nb
    ref = orc.apply_rows(t, +1, x, ch, idx)
    scale = np.abs(y).max()
    assert np.abs(y[rows] - ref).max() <= 1e-12 * scale


@pytest.mark.parametrize("name", ["tiny", "small", "slice", "tail", "order5"])
def test_mixed_precision_step_matches_oracle(oracle_mod, name):
    # complex64 BiCGSTAB inside double-precision refinement: the refinement stops on the FP64 true
    # residual, so the result meets the same parity bar as the FP64 path
    cfg = W.WORKLOADS[name]
    c = Case(cfg, oracle_mod, tol=STEP_TOL, max_iter=1000, precision=1, tol_inner=1e-5, max_outer=30)
    psi0 = c.random(11)
    t0 = 0.5 * c.T()
    n = 3
    psid = c.to_dev(psi0)
    out = {}
    passes = refinement_counts(c.op, lambda: out.update(r=c.op.step(psid, n, t0)))
    its, res, _ = out["r"]
    ref = psi0.copy()
    oits = []
    for s in range(n):
        ref, it, _ = c.orc.step(ref, t0 + s * cfg["dt"], tol=1e-14)
        oits.append(it)
    got = c.from_dev(psid)
    assert np.all(res <= STEP_TOL)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    pps = check_refinement(c.op, 1, n, passes, its, oits)
    print("precision 1 %s: passes/step %.1f, inner %s, oracle %s" % (name, pps, list(its), oits))


@pytest.mark.parametrize("name", ["tiny", "small", "slice", "tail", "wide_l", "order5"])
def test_double_float_apply_matches_oracle(oracle_mod, name):
    # precision 2 applies A_+- in double-float (FP32 hi/lo pairs with error-free transforms):
    # ~2^-44 relative per operation, so the bar is 1e-11 of max|y| instead of 1e-12
    cfg = W.WORKLOADS[name]
    c = Case(cfg, oracle_mod, tol=STEP_TOL, precision=2, tol_inner=1e-5, max_outer=30)
    x = c.random(13)
    xd = c.to_dev(x)
    yd = c.torch.empty_like(xd)
    for sign in (+1, -1):
        t = 0.43 * c.T()
        c.op.apply(sign, t, xd, yd)
        y = c.from_dev(yd)
        ref = c.orc.apply(t, sign, x)
        assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max(), sign


@pytest.mark.parametrize("name", ["tiny", "small", "slice", "tail", "wide_l", "order5"])
def test_double_float_step_matches_oracle(oracle_mod, name):
    cfg = W.WORKLOADS[name]
    c = Case(cfg, oracle_mod, tol=STEP_TOL, max_iter=1000, precision=2, tol_inner=1e-5, max_outer=30)
    psi0 = c.random(17)
    t0 = 0.5 * c.T()
    n = 3
    psid = c.to_dev(psi0)
    out = {}
    passes = refinement_counts(c.op, lambda: out.update(r=c.op.step(psid, n, t0)))
    its, res, _ = out["r"]
    ref = psi0.copy()
    oits = []
    for s in range(n):
        ref, it, _ = c.orc.step(ref, t0 + s * cfg["dt"], tol=1e-14)
        oits.append(it)
    got = c.from_dev(psid)
    assert np.all(res <= STEP_TOL)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    pps = check_refinement(c.op, 2, n, passes, its, oits)
    print("precision 2 %s: passes/step %.1f, inner %s, oracle %s" % (name, pps, list(its), oits))


@pytest.mark.parametrize("name", ["small", "tail"])
def test_overlapped_assembly_is_bitwise_identical(name):
    # the next step's assembly on a second stream into a second buffer set changes the schedule, not
    # the arithmetic: the states agree bit for bit with the sequential schedule, across calls
    import torch
    cfg = W.WORKLOADS[name]
    bas = B.Basis(cfg)
    kw = dict(tol=1e-12, precision=2, max_iter=1000, tol_inner=1e-5, max_outer=30)
    ops = [B.Operator(bas, cfg, **kw), B.Operator(bas, cfg, **kw)]
    ops[1].set_overlap(True)
    psi0, _ = bas.initial_state()
    T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
    out = []
    for op in ops:
        psi = torch.from_numpy(psi0).cuda()
        hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device="cuda")
        it1, r1, nh = op.step(psi, 5, 0.4 * T, hist=hist, n_hist=0)
        it2, r2, nh = op.step(psi, 4, 0.4 * T + 5 * cfg["dt"], hist=hist, n_hist=nh)
        # the graph driver on the same op afterwards (its capture follows the current buffer set)
        it3, r3, nh = op.run(psi, 3, 0.4 * T + 9 * cfg["dt"], hist, n_hist=nh)
        out.append((psi, np.concatenate([it1, it2, it3]), np.concatenate([r1, r2, r3])))
    assert torch.equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_production_mixed_step_matches_fp64():
    # full production size: the double-float refinement with the complex64 owner/gather inner solve
    # against the plain FP64 solve from the same state at peak field.  Both stop on the accurate
    # residual at 1e-10, so the states agree to cond(A_+) x 1e-10 (cond ~ 10 on physical states)
    import torch
    cfg = W.PRODUCTION
    bas = B.Basis(cfg)
    psi0, _ = bas.initial_state()
    T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
    out = []
    for prec in (0, 2):
        op = B.Operator(bas, cfg, tol=cfg["tol"], precision=prec, max_iter=1000, tol_inner=1e-5, max_outer=30)
        psi = torch.from_numpy(psi0).cuda()
        hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device="cuda")
        its, res, _ = op.step(psi, 3, 0.5 * T, hist=hist, n_hist=0)
        assert np.all(res <= cfg["tol"])
        out.append(psi)
        del op
    assert torch.linalg.norm(out[0] - out[1]).item() <= 1e-9 * torch.linalg.norm(out[0]).item()


@pytest.mark.parametrize("name,mode", [("tiny", 1), ("small", 1), ("slice", 1), ("tail", 1), ("small", 2),
                                       ("tail", 2)])
def test_factorised_inner_apply_step_matches_oracle(oracle_mod, name, mode):
    # the inner solve on the factorised complex64 apply (coupling from the radial bands and the
    # angular coefficients, never stored): the refinement still ends on the accurate residual, so
    # the step meets the same bar; the graph driver gives the same state bit for bit
    import torch
    cfg = W.WORKLOADS[name]
    c = Case(cfg, oracle_mod, tol=STEP_TOL, max_iter=1000, precision=2, tol_inner=1e-5, max_outer=30)
    c.op.set_factorised(mode)
    psi0 = c.random(23)
    t0 = 0.5 * c.T()
    psid = c.to_dev(psi0)
    hist = torch.zeros(2 * c.bas.n, dtype=torch.complex128, device="cuda")
    out = {}
    passes = refinement_counts(c.op, lambda: out.update(r=c.op.step(psid, 2, t0, hist=hist, n_hist=0)))
    its, res, _ = out["r"]
    ref = psi0.copy()
    oits = []
    for s in range(2):
        ref, it, _ = c.orc.step(ref, t0 + s * cfg["dt"], tol=1e-14)
        oits.append(it)
    assert np.all(res <= STEP_TOL)
    assert np.linalg.norm(c.from_dev(psid) - ref) <= 1e-10 * np.linalg.norm(ref)
    pps = check_refinement(c.op, 2, 2, passes, its, oits)
    print("factorised %s mode %d: passes/step %.1f, inner %s, oracle %s" % (name, mode, pps, list(its), oits))
    c2 = Case(cfg, oracle_mod, tol=STEP_TOL, max_iter=1000, precision=2, tol_inner=1e-5, max_outer=30)
    c2.op.set_factorised(mode)
    pd2 = c2.to_dev(psi0)
    hist2 = torch.zeros(2 * c2.bas.n, dtype=torch.complex128, device="cuda")
    its2, res2, _ = c2.op.run(pd2, 2, t0, hist2, n_hist=0)
    assert np.array_equal(its, its2) and torch.equal(psid, pd2)
