"""Plain FP64 CPU oracle of the Crank-Nicolson step of the 3D time-dependent Dirac equation.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference arm are the only callers.  The arithmetic lives in ``oracle.c`` (plain C, double
precision); this module builds it with gcc and marshals numpy arrays through ctypes.  The
photoelectron spectrum (Eq. dPdE) is numpy post-processing of the C routines' eigenpairs.
It shares no code with the CUDA library in ``paper_2512_21697_gb300``.

Vectors are complex128 in "paper order": channel-major, nb = 2(N+1) coefficients per channel,
the N+1 large-type DKB functions first and the N+1 small-type ones after (Eq. dualkinetic),
built on B_1 .. B_{N+1}.  B_1 is used only by the large type of kappa = -1 and the small type of
kappa = +1 (the zero boundary condition at r = 0); other slots built on B_1 stay zero.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile liboracle.so next to the source (gcc, -O2, OpenMP over channels)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-D_GNU_SOURCE",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("Z", C.c_double), ("c", C.c_double), ("R", C.c_double), ("N", C.c_int),
                ("order", C.c_int), ("grid", C.c_int), ("r_lin", C.c_double), ("n_lin", C.c_int),
                ("kappa_max", C.c_int), ("two_mu_max", C.c_int), ("l_max", C.c_int),
                ("quad", C.c_int), ("E0", C.c_double), ("omega", C.c_double),
                ("n_cycles", C.c_double), ("dt", C.c_double), ("time_eval", C.c_int), ("b1_drop", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            dp, ip, vp = P(C.c_double), P(C.c_int), C.c_void_p
            sig = {
                "or_create": (vp, [P(Params)]), "or_free": (None, [vp]),
                "or_nchannels": (C.c_int, [vp]), "or_channels": (None, [vp, ip, ip]),
                "or_nknots": (C.c_int, [vp]), "or_knots": (None, [vp, dp]),
                "or_nedges": (C.c_int, [vp]), "or_edges": (None, [vp, ip, ip]),
                "or_bspline_all": (None, [vp, C.c_double, dp, dp, dp]),
                "or_gauss_legendre": (None, [C.c_int, dp, dp]),
                "or_radial_dense": (None, [vp, C.c_int, dp, dp]),
                "or_radial_rmoment": (None, [vp, C.c_int, dp]),
                "or_spinor": (None, [C.c_int, C.c_int, C.c_double, C.c_double, dp]),
                "or_angular": (C.c_double, [C.c_int] * 5),
                "or_angular_2d": (C.c_double, [C.c_int] * 7),
                "or_sph_bessel": (C.c_double, [C.c_int, C.c_double]),
                "or_field_direct": (C.c_double, [vp, C.c_double, C.c_double, C.c_double]),
                "or_field_series": (C.c_double, [vp, C.c_double, C.c_double, C.c_double, C.c_int]),
                "or_field_F": (C.c_double, [vp, C.c_double, C.c_double, C.c_int]),
                "or_coupling_block": (None, [vp, C.c_int, C.c_int, C.c_double, dp]),
                "or_coupling_3d": (None, [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                          C.c_int, C.c_int, dp]),
                "or_apply": (None, [vp, C.c_double, C.c_int, dp, dp]),
                "or_apply_rows": (None, [vp, C.c_double, C.c_int, dp, C.c_int, ip, ip, dp]),
                "or_dense_operator": (None, [vp, C.c_double, C.c_int, dp]),
                "or_dense_solve": (C.c_int, [C.c_int, dp, dp, dp]),
                "or_precond": (None, [vp, dp, dp]),
                "or_step": (C.c_int, [vp, dp, C.c_double, C.c_double, C.c_int, C.c_int, dp]),
                "or_step_dense": (C.c_int, [vp, dp, C.c_double]),
                "or_eigen": (C.c_int, [vp, C.c_int, dp, dp]),
                "or_observables": (None, [vp, dp, dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def gauss_legendre(q):
    lib = _load()
    x, w = np.zeros(q), np.zeros(q)
    lib.or_gauss_legendre(q, _dp(x), _dp(w))
    return x, w


def sph_bessel(l, x):
    return _load().or_sph_bessel(int(l), float(x))


def spinor(kappa, two_mu, theta, phi):
    out = np.zeros(4)
    _load().or_spinor(int(kappa), int(two_mu), float(theta), float(phi), _dp(out))
    return np.array([out[0] + 1j * out[1], out[2] + 1j * out[3]])


def angular(k1, tm1, k2, tm2, l):
    return _load().or_angular(int(k1), int(tm1), int(k2), int(tm2), int(l))


def angular_2d(k1, tm1, k2, tm2, l, nth=40, nph=64):
    return _load().or_angular_2d(int(k1), int(tm1), int(k2), int(tm2), int(l), nth, nph)


def dense_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    rc = _load().or_dense_solve(A.shape[0], _dp(A.view(np.float64)), _dp(b.view(np.float64)),
                                _dp(x.view(np.float64)))
    if rc:
        raise ArithmeticError("singular matrix")
    return x


class Oracle:
    """One discretised problem: basis, channels, pulse and time step."""

    FIELDS = [f[0] for f in Params._fields_]

    def __init__(self, **kw):
        lib = _load()
        vals = {f: 0 for f in self.FIELDS}
        vals.update(kw)
        self.params = Params(**{f: vals[f] for f in self.FIELDS})
        self._h = lib.or_create(C.byref(self.params))
        if not self._h:
            raise ValueError("invalid oracle parameters")
        self.lib = lib
        self.N = self.params.N
        self.nb = 2 * (self.N + 1)
        self.nch = lib.or_nchannels(self._h)
        k = np.zeros(self.nch, np.int32)
        m = np.zeros(self.nch, np.int32)
        lib.or_channels(self._h, _ip(k), _ip(m))
        self.kappa, self.two_mu = k, m
        self.n = self.nb * self.nch

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.or_free(h)
            self._h = None

    def channel(self, kappa, two_mu):
        idx = np.nonzero((self.kappa == kappa) & (self.two_mu == two_mu))[0]
        return int(idx[0]) if len(idx) else -1

    def knots(self):
        out = np.zeros(self.lib.or_nknots(self._h))
        self.lib.or_knots(self._h, _dp(out))
        return out

    def edges(self):
        ne = self.lib.or_nedges(self._h)
        a, b = np.zeros(ne, np.int32), np.zeros(ne, np.int32)
        self.lib.or_edges(self._h, _ip(a), _ip(b))
        return a, b

    def bsplines(self, x):
        ns = self.N + 4
        v, d1, d2 = np.zeros(ns), np.zeros(ns), np.zeros(ns)
        self.lib.or_bspline_all(self._h, float(x), _dp(v), _dp(d1), _dp(d2))
        return v, d1, d2

    def radial(self, kappa):
        n = self.nb
        S, H = np.zeros((n, n)), np.zeros((n, n))
        self.lib.or_radial_dense(self._h, int(kappa), _dp(S), _dp(H))
        return S, H

    def rmoment(self, kappa):
        n = self.nb
        R = np.zeros((n, n))
        self.lib.or_radial_rmoment(self._h, int(kappa), _dp(R))
        return R

    def field_direct(self, t, r, ct):
        return self.lib.or_field_direct(self._h, t, r, ct)

    def field_series(self, t, r, ct, lmax):
        return self.lib.or_field_series(self._h, t, r, ct, int(lmax))

    def field_F(self, t, r, l):
        return self.lib.or_field_F(self._h, t, r, int(l))

    def coupling_block(self, a, b, t):
        n = self.nb
        X = np.zeros((n, n))
        self.lib.or_coupling_block(self._h, int(a), int(b), float(t), _dp(X))
        return X

    def coupling_3d(self, a, i, b, j, t, nth=40, nph=32):
        out = np.zeros(2)
        self.lib.or_coupling_3d(self._h, a, i, b, j, float(t), nth, nph, _dp(out))
        return out[0] + 1j * out[1]

    def apply(self, t, sign, x):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.zeros_like(x)
        self.lib.or_apply(self._h, float(t), int(sign), _dp(x.view(np.float64)), _dp(y.view(np.float64)))
        return y

    def apply_rows(self, t, sign, x, ch, idx):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        ch = np.ascontiguousarray(ch, dtype=np.int32)
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        out = np.zeros(len(ch), np.complex128)
        self.lib.or_apply_rows(self._h, float(t), int(sign), _dp(x.view(np.float64)), len(ch),
                               _ip(ch), _ip(idx), _dp(out.view(np.float64)))
        return out

    def dense_operator(self, t, sign):
        A = np.zeros((self.n, self.n), np.complex128)
        self.lib.or_dense_operator(self._h, float(t), int(sign), _dp(A.view(np.float64)))
        return A

    def precond(self, r):
        r = np.ascontiguousarray(r, dtype=np.complex128)
        z = np.zeros_like(r)
        self.lib.or_precond(self._h, _dp(r.view(np.float64)), _dp(z.view(np.float64)))
        return z

    def step(self, psi, t_n, tol=1e-14, max_iter=500, precond=True):
        """One CN step in place on a copy; returns (psi_next, iterations, residual)."""
        x = np.array(psi, dtype=np.complex128, copy=True)
        res = C.c_double(0)
        it = self.lib.or_step(self._h, _dp(x.view(np.float64)), float(t_n), float(tol), int(max_iter),
                              1 if precond else 0, C.byref(res))
        if it < 0:
            raise ArithmeticError("oracle BiCGSTAB did not converge (res %g)" % res.value)
        return x, it, res.value

    def step_dense(self, psi, t_n):
        x = np.array(psi, dtype=np.complex128, copy=True)
        if self.lib.or_step_dense(self._h, _dp(x.view(np.float64)), float(t_n)):
            raise ArithmeticError("singular")
        return x

    def run(self, psi, n_steps, t0=0.0, tol=1e-14, max_iter=500):
        x = np.array(psi, dtype=np.complex128, copy=True)
        iters = []
        for s in range(n_steps):
            x, it, _ = self.step(x, t0 + s * self.params.dt, tol=tol, max_iter=max_iter)
            iters.append(it)
        return x, iters

    def eigen(self, kappa):
        """Eigenpairs of H0 v = E S v for one kappa (only the functions this kappa uses)."""
        n = self.nb
        E, V = np.zeros(n), np.zeros((n, n))
        na = self.lib.or_eigen(self._h, int(kappa), _dp(E), _dp(V))
        return E[:na], V[:na]

    def ground_state(self):
        """1s1/2 (kappa=-1, mu=+1/2) state: lowest eigenvalue above -c^2 (Sec. 2.3)."""
        E, V = self.eigen(-1)
        c2 = self.params.c ** 2
        e = int(np.nonzero(E > -c2)[0][0])
        psi = np.zeros(self.n, np.complex128)
        a = self.channel(-1, 1)
        psi[a * self.nb:(a + 1) * self.nb] = V[e]
        return psi, E[e]

    def observables(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.zeros(4)
        self.lib.or_observables(self._h, _dp(psi.view(np.float64)), _dp(out))
        return dict(norm=out[0], energy=out[1], p_ground=out[2], p_bound=out[3])

    # -- photoelectron spectrum (Sec. 4.3, Eq. dPdE): numpy post-processing of the eigenpairs above --

    def spectrum_levels(self, psi, e_lo, e_hi):
        """Discrete spectrum of psi per kappa in use: the eigenvalues E_j of H0 v = E S v with
        e_lo < E_j <= e_hi (ascending) and q_j = sum over the channels (kappa, mu) of
        |v_j^T S psi_{kappa mu}|^2 (v_j normalised v^T S v = 1).  Returns {kappa: (E, q)}."""
        psi = np.asarray(psi, dtype=np.complex128)
        out = {}
        for kappa in sorted(set(int(k) for k in self.kappa)):
            E, V = self.eigen(kappa)
            S, _ = self.radial(kappa)
            sel = (E > e_lo) & (E <= e_hi)
            Vs = V[sel]
            q = np.zeros(int(sel.sum()))
            for a in np.nonzero(self.kappa == kappa)[0]:
                c = Vs @ (S @ psi[a * self.nb:(a + 1) * self.nb])
                q += c.real ** 2 + c.imag ** 2
            out[kappa] = (E[sel].copy(), q)
        return out

    @staticmethod
    def level_spacing(E):
        """Local level spacing of ascending levels: (E_{j+1} - E_{j-1}) / 2 inside, the one-sided
        difference at the two ends.  The box-normalised eigenvectors become energy-normalised
        continuum states when divided by its square root (density of states 1 / dE)."""
        E = np.asarray(E, dtype=np.float64)
        d = np.empty_like(E)
        d[1:-1] = 0.5 * (E[2:] - E[:-2])
        d[0] = E[1] - E[0]
        d[-1] = E[-1] - E[-2]
        return d

    def spectrum(self, psi, e_lo, e_hi, grid):
        """dP/dE (Eq. dPdE) on an energy grid: per kappa the densities q_j / dE_j at its levels,
        linearly interpolated in E (zero outside the kappa's first and last level in the window;
        a kappa with fewer than two levels there contributes nothing), summed over kappa."""
        grid = np.asarray(grid, dtype=np.float64)
        P = np.zeros(len(grid))
        for kappa, (E, q) in self.spectrum_levels(psi, e_lo, e_hi).items():
            if len(E) < 2:
                continue
            P += np.interp(grid, E, q / self.level_spacing(E), left=0.0, right=0.0)
        return P

    @staticmethod
    def spectrum_error(grid, p_n, p_m, e1, e2):
        """Err_{n,m} = integral over [e1, e2] of |P_n(E) - P_m(E)|^2 dE (Sec. 4.3), by the trapezoid
        rule over the grid points inside [e1, e2] (ascending grid)."""
        grid = np.asarray(grid, dtype=np.float64)
        sel = (grid >= e1) & (grid <= e2)
        e = grid[sel]
        f = np.abs(np.asarray(p_n)[sel] - np.asarray(p_m)[sel]) ** 2
        return float(np.sum(0.5 * (f[1:] + f[:-1]) * (e[1:] - e[:-1]))) if len(e) > 1 else 0.0

    def active_mask(self):
        """Boolean mask over the full vector: True where a basis function is used."""
        m = np.ones((self.nch, self.nb), bool)
        m[:, 0] = self.kappa == -1
        m[:, self.N + 1] = self.kappa == 1
        return m.reshape(-1)
