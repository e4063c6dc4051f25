"""Element-wise oracle parity of the complex64 parts of the mixed-precision step and of the
double-float refinement residual, through the C ABI (dirac_apply32, dirac_precond_apply32,
dirac_residual).

The refinement loop of a step ends on the accurate residual, so a moderately wrong inner operator
only costs iterations: these tests compare each part with the oracle directly.

Bars (derived from the arithmetic, u = 2^-24 the FP32 unit roundoff):
 - complex64 apply, stored coupling (owner/gather passes, per-row kernel): every operator value is
   an FP32 rounding (|rel. error| <= u; the diagonal block's tau H0 is a product of two rounded
   floats, <= 3u), and row i sums m_i real products per component (m_i = 2 x 13 x (1 + partners)
   for order-7 splines) in FP32.  Higham's bound for a sum of products gives, per component,
   |y32_i - y_i| <= (m_i + 4) u (|A| |x|)_i, with y_i the exact product of the FP64 operator and the
   complex64 input (the oracle applies its operator to the input promoted to FP64).  The test
   takes gamma_i = (2 m_i + 8) u, with |A| |x| formed from the oracle's dense operator.
 - complex64 preconditioner: an LU solve with FP32-rounded factors is backward stable,
   (M + dM) z = r with |dM| <= c kb u |L| |U|; the test checks the normwise backward error
   ||M z - r||_inf <= 8 (2 kb + 1) u || |M| |z| + |r| ||_inf (kb = 13 scalar sub-diagonals; the
   factor 8 allows a pivot growth |L||U| <= 8 |M|, far above what partial pivoting gives here).
 - factorised complex64 apply: it forms the coupling from band products (G^0 + kappa G^2) x and
   (G^1 + kappa G^3) x whose terms can exceed the assembled values by the kappa factors, so its
   bound is normwise: max_i |y32_i - y_i| <= 64 (m + 4) u max_i (|A| |x|)_i with m the largest row
   count (the factor 64 covers (1 + kappa)^2 band-term growth at |kappa| <= 7).
 - double-float residual: ~2^-44 relative per operation on sums of at most 2 x 13 x (1 + partners)
   x 2 terms: |r_i - r_ref_i| <= 1e-11 max(max|A_- psi|, max|A_+ x|), the bar of the double-float
   apply tests.
"""
import math

import numpy as np
import pytest

from paper_2512_21697_gb300 import binding as B, layout, workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


class Case32:
    def __init__(self, cfg, oracle_mod, precision=2, **opt):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.bas = B.Basis(cfg)
        self.orc = oracle_mod.Oracle(**W.oracle_params(cfg))
        self.perm = layout.lib_to_paper_perm(self.bas.kappa, self.bas.two_mu, cfg["kappa_max"],
                                             cfg["two_mu_max"], cfg["N"])
        self.inv = np.empty_like(self.perm)
        self.inv[self.perm] = np.arange(len(self.perm))
        kw = dict(tol=1e-12, max_iter=1000, precision=precision, tol_inner=1e-5, max_outer=30)
        kw.update(opt)
        self.op = B.Operator(self.bas, cfg, **kw)
        self.dev = torch.device("cuda")

    def T(self):
        return self.cfg["n_cycles"] * 2 * math.pi / self.cfg["omega"]

    def random(self, seed):
        x = W.random_state(self.orc.n, seed)
        x[~self.orc.active_mask()] = 0
        return x / np.linalg.norm(x)

    def to_dev32(self, x_paper):
        return self.torch.from_numpy(np.ascontiguousarray(x_paper[self.inv]).astype(np.complex64)).to(self.dev)

    def to_dev(self, x_paper):
        return self.torch.from_numpy(np.ascontiguousarray(x_paper[self.inv])).to(self.dev)

    def from_dev(self, xd):
        return xd.cpu().numpy().astype(np.complex128)[self.perm]

    def row_terms(self):
        """Real products per component of each row: 2 DKB types x block-diagonals x (1 + partners)."""
        ea, _ = self.orc.edges()
        deg = np.bincount(ea, minlength=self.orc.nch)
        bd = 2 * self.cfg["order"] - 1
        return np.repeat(2 * bd * (1 + deg), self.orc.nb)

    def abs_product(self, t, x):
        """(|Re A| + |Im A|) (|Re x| + |Im x|) with A = A_+(t), from the oracle's dense operator."""
        A = self.orc.dense_operator(t, +1)
        ax = np.abs(x.real) + np.abs(x.imag)
        return (np.abs(A.real) + np.abs(A.imag)) @ ax

    def abs_product_blocks(self, t, x):
        """An upper bound of abs_product built block by block (no dense operator): per channel
        (|S| + tau |H0|) |x_a| + sum over partners tau |X_ab| |x_b|, with H_ab = i X_ab."""
        o, nb = self.orc, self.orc.nb
        tau = 0.5 * self.cfg["dt"]
        ax = np.abs(x.real) + np.abs(x.imag)
        out = np.zeros(o.n)
        diag = {}
        for a in range(o.nch):
            k = int(o.kappa[a])
            if k not in diag:
                S, H = o.radial(k)
                diag[k] = np.abs(S) + tau * np.abs(H)
            out[a * nb:(a + 1) * nb] += diag[k] @ ax[a * nb:(a + 1) * nb]
        ea, eb = o.edges()
        for a, b in zip(ea, eb):
            X = o.coupling_block(int(a), int(b), t)
            out[a * nb:(a + 1) * nb] += tau * np.abs(X) @ ax[b * nb:(b + 1) * nb]
        return out


# workloads small enough for the oracle's dense operator (n <= 10^4)
DENSE = ["tiny", "small", "tail", "order5", "wide_l"]


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name", DENSE)
def test_apply32_matches_oracle_elementwise(oracle_mod, name, precision):
    # the inner solve's complex64 operator (owner/gather passes for order 7, per-row kernel for
    # order 5) against the oracle's FP64 operator on the same complex64 input, at three times
    # inside the pulse and both signs, with the per-row bound gamma_i (|A| |x|)_i
    c = Case32(W.WORKLOADS[name], oracle_mod, precision=precision)
    x = c.random(31)
    xd = c.to_dev32(x)
    x = c.from_dev(xd)                       # the input as the kernel sees it, promoted to FP64
    yd = c.torch.empty_like(xd)
    gamma = (2 * c.row_terms() + 8) * U32
    worst = 0.0
    for t in (0.21 * c.T(), 0.5 * c.T(), 0.77 * c.T()):
        bound = gamma * c.abs_product(t, x)
        for sign in (+1, -1):
            c.op.apply32(sign, t, xd, yd)
            y = c.from_dev(yd)
            ref = c.orc.apply(t, sign, x)
            err = np.maximum(np.abs(y.real - ref.real), np.abs(y.imag - ref.imag))
            assert np.all(err <= bound), (sign, t, float(np.max(err / np.maximum(bound, 1e-300))))
            assert np.all(y[~c.orc.active_mask()] == 0)
            worst = max(worst, float(np.max(err / np.maximum(bound, 1e-300))))
    print("apply32 %s precision %d: max err / bound = %.3g" % (name, precision, worst))


def test_apply32_matches_oracle_slice(oracle_mod):
    # the production grid family at |kappa| <= 5 (two 116-row tiles, the second ragged): too large
    # for the dense operator, so |A| |x| is formed block by block from the oracle's radial blocks
    # (|S| + tau |H0|) and coupling blocks (tau |X_ab|); same per-row bound as above
    c = Case32(W.SLICE, oracle_mod, precision=2)
    x = c.random(32)
    xd = c.to_dev32(x)
    x = c.from_dev(xd)
    yd = c.torch.empty_like(xd)
    gamma = (2 * c.row_terms() + 8) * U32
    worst = 0.0
    for t in (0.3 * c.T(), 0.6 * c.T()):
        bound = gamma * c.abs_product_blocks(t, x)
        for sign in (+1, -1):
            c.op.apply32(sign, t, xd, yd)
            y = c.from_dev(yd)
            ref = c.orc.apply(t, sign, x)
            err = np.maximum(np.abs(y.real - ref.real), np.abs(y.imag - ref.imag))
            assert np.all(err <= bound), (sign, t, float(np.max(err / np.maximum(bound, 1e-300))))
            worst = max(worst, float(np.max(err / np.maximum(bound, 1e-300))))
    print("apply32 slice: max err / bound = %.3g" % worst)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", ["tiny", "small", "tail", "wide_l"])
def test_factorised_apply32_matches_oracle(oracle_mod, name, mode):
    # the factorised complex64 apply (coupling from the radial bands and the angular coefficients,
    # never stored; mode 1 subgroup form, 2 per-channel form) against the oracle, normwise bar
    # 64 (m + 4) u max (|A| |x|)
    c = Case32(W.WORKLOADS[name], oracle_mod, precision=2)
    c.op.set_factorised(mode)
    x = c.random(33)
    xd = c.to_dev32(x)
    x = c.from_dev(xd)
    yd = c.torch.empty_like(xd)
    m = int(c.row_terms().max())
    worst = 0.0
    for t in (0.21 * c.T(), 0.5 * c.T(), 0.77 * c.T()):
        scale = c.abs_product(t, x).max()
        for sign in (+1, -1):
            c.op.apply32(sign, t, xd, yd)
            y = c.from_dev(yd)
            ref = c.orc.apply(t, sign, x)
            err = np.maximum(np.abs(y.real - ref.real), np.abs(y.imag - ref.imag)).max()
            assert err <= 64 * (m + 4) * U32 * scale, (sign, t, err / scale)
            worst = max(worst, err / ((m + 4) * U32 * scale))
    print("factorised apply32 %s mode %d: max err / ((m+4) u max|A||x|) = %.3g" % (name, mode, worst))


@pytest.mark.parametrize("sched", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["tiny", "small", "tail", "order5"])
def test_precond32_backward_error(oracle_mod, name, sched):
    # every complex64 preconditioner schedule solves M z = r with a small backward error (M applied
    # by the oracle: A_+ after the pulse, where the field is zero, is M = S + i tau H0), and agrees
    # with the oracle's FP64 solve to the forward error that backward error allows
    c = Case32(W.WORKLOADS[name], oracle_mod, precision=2)
    order7 = c.cfg["order"] == 7
    if sched != 1 and not order7:
        with pytest.raises(B.DiracError):
            c.op.set_schedule(True, sched)
        return
    c.op.set_schedule(True, sched)
    r = c.random(34)
    rd = c.to_dev32(r)
    r = c.from_dev(rd)
    zd = c.torch.empty_like(rd)
    c.op.precond32(rd, zd)
    z = c.from_dev(zd)
    t_free = 2.0 * c.T()
    Mz = c.orc.apply(t_free, +1, z)
    A = c.orc.dense_operator(t_free, +1)
    absMz = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(z.real) + np.abs(z.imag))
    kb = 2 * (c.cfg["order"] - 1) + 1
    be = np.abs(Mz - r).max() / (absMz + np.abs(r.real) + np.abs(r.imag)).max()
    assert be <= 8 * (2 * kb + 1) * U32, (sched, be)
    zr = c.orc.precond(r)
    fe = np.linalg.norm(z - zr) / np.linalg.norm(zr)
    assert np.all(z[~c.orc.active_mask()] == 0)
    print("precond32 %s sched %d: backward %.3g (bound %.3g), forward %.3g" %
          (name, sched, be, 8 * (2 * kb + 1) * U32, fe))


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", ["tiny", "small", "slice", "tail", "wide_l", "order5"])
def test_residual_matches_oracle(oracle_mod, name, mode):
    # the refinement residual r = A_- psi - A_+ x as the step forms it (double-float owner/gather
    # passes for order 7, per-row double-float kernel otherwise), against the oracle's two applies;
    # mode 1: Dot2 accumulators, mode 2: fixed-binade accumulators with offsets (order 7 only)
    c = Case32(W.WORKLOADS[name], oracle_mod, precision=2)
    c.op.set_residual_mode(mode)
    psi = c.random(35)
    x = psi + 0.01 * c.random(36)            # an iterate near psi, so the residual cancels partly
    pd, xd = c.to_dev(psi), c.to_dev(x)
    rd = c.torch.empty_like(pd)
    for t in (0.3 * c.T(), 0.62 * c.T()):
        bn = c.op.residual(t, pd, xd, rd)
        r = c.from_dev(rd)
        b = c.orc.apply(t, -1, psi)
        ax = c.orc.apply(t, +1, x)
        ref = b - ax
        scale = max(np.abs(b).max(), np.abs(ax).max())
        assert np.abs(r - ref).max() <= 1e-11 * scale, (t, np.abs(r - ref).max() / scale)
        print("residual %s mode %d t=%.3g: max err / scale %.3g, ||err|| / ||b|| %.3g" %
              (name, mode, t, np.abs(r - ref).max() / scale, np.linalg.norm(r - ref) / np.linalg.norm(b)))
        # ||b|| from FP32 products: relative 1e-6
        assert abs(bn - np.linalg.norm(b)) <= 1e-6 * np.linalg.norm(b)


@pytest.mark.parametrize("name", ["tiny", "small", "tail", "wide_l"])
def test_offset_residual_step_meets_tolerance(oracle_mod, name):
    # a precision-2 step with the fixed-binade accumulators (mode 2, the default at tolerances
    # >= 1e-11) ends on a state that solves the CN system to the tolerance: the oracle's FP64
    # operator gives ||A_- psi - A_+ psi'|| <= 2 tol ||A_- psi|| (the residual the refinement tests
    # carries an error of about 1e-13 ||b|| at most, far below tol), from a random state at
    # peak-field times; the Dot2 form (mode 1) on the same inputs for comparison
    tol = 1e-11
    for mode in (2, 1):
        c = Case32(W.WORKLOADS[name], oracle_mod, precision=2, tol=tol)
        c.op.set_residual_mode(mode)
        psi0 = c.random(51)
        t0 = 0.5 * c.T()
        pd = c.to_dev(psi0)
        its, res, _ = c.op.step(pd, 1, t0)
        psi1 = c.from_dev(pd)
        tm = t0 + 0.5 * c.cfg["dt"]   # the step's midpoint time, where the oracle forms A_-+
        b = c.orc.apply(tm, -1, psi0)
        rel = np.linalg.norm(b - c.orc.apply(tm, +1, psi1)) / np.linalg.norm(b)
        print("%s mode %d: reported %.3g, true residual %.3g, inner iterations %s" % (name, mode, res[0], rel,
                                                                                    list(its)))
        assert res[0] <= tol
        assert rel <= 2 * tol, (mode, rel)


def test_residual_mode_rejects_bad_values(oracle_mod):
    c = Case32(W.TINY, oracle_mod, precision=2)
    for bad in (-1, 3):
        with pytest.raises(B.DiracError):
            c.op.set_residual_mode(bad)


def test_residual_precision0_matches_oracle(oracle_mod):
    # the same entry point in FP64 (precision 0: b = A_- psi, r = b - A_+ x), bar 1e-12
    c = Case32(W.SMALL, oracle_mod, precision=0)
    psi = c.random(37)
    x = psi + 0.01 * c.random(38)
    pd, xd = c.to_dev(psi), c.to_dev(x)
    rd = c.torch.empty_like(pd)
    t = 0.4 * c.T()
    bn = c.op.residual(t, pd, xd, rd)
    b, ax = c.orc.apply(t, -1, psi), c.orc.apply(t, +1, x)
    scale = max(np.abs(b).max(), np.abs(ax).max())
    assert np.abs(c.from_dev(rd) - (b - ax)).max() <= 1e-12 * scale
    assert abs(bn - np.linalg.norm(b)) <= 1e-12 * np.linalg.norm(b)


def test_new_entry_points_reject_bad_arguments(oracle_mod):
    import torch
    c = Case32(W.TINY, oracle_mod, precision=2)
    x = c.to_dev32(c.random(1))
    with pytest.raises(B.DiracError):
        c.op.apply32(2, 0.0, x, torch.empty_like(x))        # sign not +-1
    with pytest.raises(B.DiracError):
        c.op.apply32(1, 0.0, x, x)                          # aliasing
    with pytest.raises(B.DiracError):
        c.op.precond32(x, x)
    c0 = Case32(W.TINY, oracle_mod, precision=0)
    with pytest.raises(B.DiracError):
        c0.op.apply32(1, 0.0, x, torch.empty_like(x))       # no complex64 operator in FP64 mode
    with pytest.raises(B.DiracError):
        c0.op.precond32(x, torch.empty_like(x))
    p = c0.to_dev(c0.random(2))
    with pytest.raises(B.DiracError):
        c0.op.residual(0.0, p, p, p)                        # r aliases psi


# ---- production size: sampled rows the oracle computes one by one ----

def _production(oracle_mod):
    import torch
    cfg = W.PRODUCTION
    bas = B.Basis(cfg)
    orc = oracle_mod.Oracle(**W.oracle_params(cfg))
    perm = layout.lib_to_paper_perm(bas.kappa, bas.two_mu, cfg["kappa_max"], cfg["two_mu_max"], cfg["N"])
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    rng = np.random.default_rng(19)
    nb = orc.nb
    rows = np.concatenate([rng.choice(orc.n, 40, replace=False),
                           [0, nb - 1, orc.n - 1, orc.n - nb, nb * 900 + cfg["N"], nb * 1859 + 2 * cfg["N"] + 1,
                            # radial slots at the 116-row tile edges of the owner/gather passes
                            nb * 7 + 2 * 116, nb * 7 + 2 * 115 + 1, nb * 1000 + 2 * 231, nb * 1500 + 2 * 928 + 1]])
    T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
    return cfg, bas, orc, perm, inv, rows, T, torch


def test_production_apply32_sampled_rows(oracle_mod):
    # the complex64 owner/gather apply at full size (the kernel of the 70 %-of-HBM figure), both
    # signs, against the oracle's rows on the same complex64 input.  Normwise form of the per-row
    # bound: (2 m + 8) u max|A| |x| with m the largest row count (2 x 13 x (1 + 56 partners)) and
    # max|A| |x| <= 4 max|y| (on every workload small enough to form |A| |x|, random inputs give
    # max|A| |x| / max|y| between 1.56 and 1.95)
    cfg, bas, orc, perm, inv, rows, T, torch = _production(oracle_mod)
    op = B.Operator(bas, cfg, tol=cfg["tol"], precision=2, tol_inner=1e-5, max_outer=20)
    x = W.random_state(orc.n, 41)
    x[~orc.active_mask()] = 0
    x = x.astype(np.complex64).astype(np.complex128)
    xd = torch.from_numpy(x[inv].astype(np.complex64)).cuda()
    yd = torch.empty_like(xd)
    ch, idx = rows // orc.nb, rows % orc.nb
    ea, _ = orc.edges()
    m = 2 * 13 * (1 + int(np.bincount(ea).max()))
    for sign in (+1, -1):
        t = 0.43 * T
        op.apply32(sign, t, xd, yd)
        y = yd.cpu().numpy().astype(np.complex128)[perm]
        ref = orc.apply_rows(t, sign, x, ch, idx)
        err = np.abs(y[rows] - ref).max()
        assert err <= (2 * m + 8) * U32 * 4 * np.abs(y).max(), (sign, err / np.abs(y).max())
        print("production apply32 sign %+d: max err / max|y| = %.3g" % (sign, err / np.abs(y).max()))
    # the factorised apply in its subgroup form (16 radial tiles, the largest subgroups), with the
    # factor 64 of the factorised bar above for the kappa-weighted band terms
    op.set_factorised(1)
    for sign in (+1, -1):
        t = 0.43 * T
        op.apply32(sign, t, xd, yd)
        y = yd.cpu().numpy().astype(np.complex128)[perm]
        ref = orc.apply_rows(t, sign, x, ch, idx)
        err = np.abs(y[rows] - ref).max()
        assert err <= 64 * (2 * m + 8) * U32 * 4 * np.abs(y).max(), (sign, err / np.abs(y).max())
        print("production factorised apply32 sign %+d: max err / max|y| = %.3g" % (sign, err / np.abs(y).max()))


def test_production_residual_sampled_rows(oracle_mod):
    # the double-float refinement residual (owner/gather passes: the step's dominant kernel) at full
    # size against the oracle's rows of A_- psi - A_+ x
    cfg, bas, orc, perm, inv, rows, T, torch = _production(oracle_mod)
    op = B.Operator(bas, cfg, tol=cfg["tol"], precision=2, tol_inner=1e-5, max_outer=20)
    psi = W.random_state(orc.n, 42)
    psi[~orc.active_mask()] = 0
    x = psi + 0.01 * W.random_state(orc.n, 43)
    x[~orc.active_mask()] = 0
    pd, xd = torch.from_numpy(psi[inv]).cuda(), torch.from_numpy(x[inv]).cuda()
    rd = torch.empty_like(pd)
    t = 0.57 * T
    op.residual(t, pd, xd, rd)
    r = rd.cpu().numpy()[perm]
    ch, idx = rows // orc.nb, rows % orc.nb
    b = orc.apply_rows(t, -1, psi, ch, idx)
    ax = orc.apply_rows(t, +1, x, ch, idx)
    scale = max(np.abs(b).max(), np.abs(ax).max())
    assert np.abs(r[rows] - (b - ax)).max() <= 1e-11 * scale
    # the same operator through the double-float apply entry point (precision 2 dirac_apply)
    yd = torch.empty_like(pd)
    op.apply(+1, t, xd, yd)
    y = yd.cpu().numpy()[perm]
    assert np.abs(y[rows] - ax).max() <= 1e-11 * np.abs(y).max()
