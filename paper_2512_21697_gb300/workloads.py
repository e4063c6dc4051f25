"""Seeded synthetic workloads shared by the tests, the smoke check and the benchmark.

This module holds parameter sets and random-number generation only -- none of the method's
arithmetic.  Every workload is synthetic: the paper's runs use no dataset on this path, so a
workload is a parameter set (atom, radial box, angular truncation, pulse, time step) plus seeded
random vectors for kernel-level checks.
"""
import numpy as np

C_AU = 137.036                   # speed of light in atomic units, as the workloads state it
NM_HARTREE = 45.5633525          # photon energy [a.u.] = 45.5633525 / wavelength [nm]


def omega_from_nm(wavelength_nm):
    return NM_HARTREE / float(wavelength_nm)


def _base(**kw):
    d = dict(Z=1.0, c=C_AU, order=7, grid=0, r_lin=0.0, n_lin=0, two_mu_max=0, quad=14,
             time_eval=0, t0=0.0)
    d.update(kw)
    return d


# Hydrogen, R = 50 a.u., 60 order-7 B-splines on a linear grid, |kappa| <= 4, mu = +-1/2,
# multipoles l <= 2, one-cycle 800 nm sin^2 pulse at E0 = 0.05, dt = 0.01, 200 steps, tol 1e-12.
SMALL = _base(R=50.0, N=60, kappa_max=4, two_mu_max=1, l_max=2, E0=0.05,
              omega=omega_from_nm(800), n_cycles=1.0, dt=0.01, steps=200, tol=1e-12)

# Production-shaped: R = 300 a.u., 1000 order-7 B-splines on a grid that is linear up to 60 a.u.
# (half of the knot intervals) and geometric beyond, |kappa| <= 30 with every mu, l <= 6,
# three-cycle 800 nm pulse at E0 = 0.1, dt = 0.005, 2000 steps, tol 1e-10.
PRODUCTION = _base(R=300.0, N=1000, grid=1, r_lin=60.0, n_lin=499, kappa_max=30, two_mu_max=0,
                   l_max=6, E0=0.1, omega=omega_from_nm(800), n_cycles=3.0, dt=0.005, steps=2000,
                   tol=1e-10)

# Tiny basis for dense direct solves and brute-force checks (a few hundred unknowns).  The strong
# field and long step make the coupling dominate the diagonal, so a wrong coupling term shows.
TINY = _base(R=12.0, N=12, kappa_max=2, two_mu_max=0, l_max=3, E0=2.0,
             omega=omega_from_nm(30), n_cycles=2.0, dt=0.05, steps=10, tol=1e-13)

# A small slice of the production system: same grid family, fewer channels and splines, for
# kernel parity at sizes with a ragged radial tail.
SLICE = _base(R=300.0, N=157, grid=1, r_lin=60.0, n_lin=76, kappa_max=5, two_mu_max=0, l_max=6,
              E0=0.1, omega=omega_from_nm(800), n_cycles=3.0, dt=0.005, steps=20, tol=1e-12)

# Medium system for profiler captures: the production grid family at |kappa| <= 14, 600 splines;
# its coupling values (a few GB) exceed the L2 cache.
MEDIUM = _base(R=300.0, N=600, grid=1, r_lin=60.0, n_lin=299, kappa_max=14, two_mu_max=0, l_max=6,
               E0=0.1, omega=omega_from_nm(800), n_cycles=3.0, dt=0.005, steps=20, tol=1e-10)

# Ragged-tail case for the kernels' row tiles: 121 radial slots are one 128-row tile but two
# 116-row tiles, so every partial count and halo of the tiled passes is exercised.
TAIL = _base(R=300.0, N=120, grid=1, r_lin=60.0, n_lin=58, kappa_max=4, two_mu_max=0, l_max=4,
             E0=0.1, omega=omega_from_nm(800), n_cycles=3.0, dt=0.005, steps=20, tol=1e-12)

# Multipoles up to l = 8 on the small system: some (kappa_a, kappa_b) groups couple through five
# multipoles of one parity, more than the grouped double-float assembly holds in registers, so
# the assembly takes its per-pair form.
WIDE_L = dict(SMALL, l_max=8, E0=0.5, omega=omega_from_nm(100))

# Order-5 B-splines on the small system: a band of 9 block-diagonals instead of 13, so every
# kernel takes its general-bandwidth form (plain warp-per-channel preconditioner, per-row applies
# and residual instead of the owner passes).
ORDER5 = dict(SMALL, order=5, N=40)

WORKLOADS = {"small": SMALL, "production": PRODUCTION, "tiny": TINY, "slice": SLICE, "medium": MEDIUM,
             "tail": TAIL, "wide_l": WIDE_L, "order5": ORDER5}


def oracle_params(cfg):
    """The subset of a workload that defines the discretised problem."""
    keys = ["Z", "c", "R", "N", "order", "grid", "r_lin", "n_lin", "kappa_max", "two_mu_max",
            "l_max", "quad", "E0", "omega", "n_cycles", "dt", "time_eval"]
    return {k: cfg[k] for k in keys}


def batch_instances(n_inst=64, seed0=0, kappa_max=20, l_max=2, N_lo=400, N_hi=1000, R=300.0):
    """Laser/basis parameter sets for the batched workload: E0 log-uniform in [0.02, 0.2],
    wavelength uniform in [400, 1600] nm, 2-6 cycles, N_lo..N_hi radial splines (default
    400-1000), box R (default 300 a.u.), linear-then-geometric grid with half the knot intervals
    linear up to R/5."""
    out = []
    for i in range(n_inst):
        g = np.random.default_rng(seed0 + i)
        E0 = float(np.exp(g.uniform(np.log(0.02), np.log(0.2))))
        lam = float(g.uniform(400, 1600))
        ncyc = int(g.integers(2, 7))
        N = int(g.integers(N_lo, N_hi + 1))
        m = N + 5 - 7
        out.append(_base(R=float(R), N=N, grid=1, r_lin=R / 5.0, n_lin=m // 2, kappa_max=kappa_max,
                         two_mu_max=0, l_max=l_max, E0=E0, omega=omega_from_nm(lam),
                         n_cycles=float(ncyc), dt=0.005, steps=2000, tol=1e-10))
    return out


def random_state(n, seed):
    """Seeded complex128 vector with standard-normal real and imaginary parts."""
    g = np.random.default_rng(seed)
    return g.standard_normal(n) + 1j * g.standard_normal(n)


def guess_net_init(seed):
    """Seeded initial parameters of the learned-guess network as one float32 array in the order
    W1 [32][256], b1, W2 [256][256], b2, W3 [256][256], b3, W4 [256][4], b4: weights uniform in
    +-1/sqrt(fan_in), the last layer scaled by 1e-2 (the untrained network starts near the
    extrapolated guess), biases zero."""
    g = np.random.default_rng(seed)
    parts = []
    for name, shp in (("W1", (32, 256)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)),
                      ("b3", (256,)), ("W4", (256, 4)), ("b4", (4,))):
        if name[0] == "b":
            parts.append(np.zeros(shp))
        else:
            a = 1.0 / np.sqrt(shp[0])
            w = g.uniform(-a, a, size=shp)
            if name == "W4":
                w = w * 1e-2
            parts.append(w)
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)
