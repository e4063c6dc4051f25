"""ctypes binding of libdirac_gb300.so: the C ABI of include/dirac.h under the same names.

Argument marshalling only; every step of the method runs in the library (host setup in C++,
the time step in CUDA kernels).  Device buffers are torch CUDA tensors (complex128, contiguous).
Importing works without a GPU; a missing library raises immediately -- there is no fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# DIRAC_BOUNDS_CHECK=1 selects the debug build (index checks compiled in, build(debug=True))
LIB_PATH = os.path.join(HERE, "libdirac_gb300_dbg.so" if os.environ.get("DIRAC_BOUNDS_CHECK") == "1"
                        else "libdirac_gb300.so")

DIRAC_OK, DIRAC_E_ARG, DIRAC_E_NOMEM, DIRAC_E_CUDA, DIRAC_E_NOCONV, DIRAC_E_BREAKDOWN, DIRAC_E_NUMERIC, \
    DIRAC_E_STATE = range(8)
STATUS_NAMES = ["OK", "E_ARG", "E_NOMEM", "E_CUDA", "E_NOCONV", "E_BREAKDOWN", "E_NUMERIC", "E_STATE"]


class DiracError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


class dirac_basis_params(C.Structure):
    _fields_ = [("Z", C.c_double), ("c", C.c_double), ("R", C.c_double), ("n_splines", C.c_int),
                ("order", C.c_int), ("grid", C.c_int), ("r_lin", C.c_double), ("n_lin", C.c_int),
                ("kappa_max", C.c_int), ("two_mu_max", C.c_int), ("l_max", C.c_int), ("quad_pts", C.c_int)]


class dirac_pulse(C.Structure):
    _fields_ = [("E0", C.c_double), ("omega", C.c_double), ("n_cycles", C.c_double), ("t0", C.c_double)]


class dirac_solver_opts(C.Structure):
    _fields_ = [("dt", C.c_double), ("tol", C.c_double), ("tol_inner", C.c_double), ("max_iter", C.c_int),
                ("precision", C.c_int), ("max_outer", C.c_int), ("guess", C.c_int), ("time_eval", C.c_int),
                ("precond", C.c_int)]


_lib = None
_VP, _DP, _IP = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
SIGNATURES = {
    "dirac_basis_build": (C.c_int, [C.POINTER(dirac_basis_params), C.POINTER(_VP), _DP, _DP]),
    "dirac_basis_free": (None, [_VP]),
    "dirac_basis_dim": (C.c_int64, [_VP]),
    "dirac_basis_nchannels": (C.c_int, [_VP]),
    "dirac_basis_channels": (C.c_int, [_VP, _IP, _IP]),
    "dirac_basis_npairs": (C.c_int64, [_VP]),
    "dirac_basis_nterms": (C.c_int64, [_VP]),
    "dirac_basis_radial": (C.c_int, [_VP, C.c_int, _DP, _DP]),
    "dirac_basis_coupling": (C.c_int, [_VP, C.POINTER(dirac_pulse), C.c_int, C.c_int, C.c_double, _DP]),
    "dirac_angular": (C.c_double, [C.c_int] * 5),
    "dirac_operator_setup": (C.c_int, [_VP, C.POINTER(dirac_pulse), C.POINTER(dirac_solver_opts), _VP,
                                       C.POINTER(_VP)]),
    "dirac_op_free": (None, [_VP]),
    "dirac_op_device_bytes": (C.c_int64, [_VP]),
    "dirac_apply": (C.c_int, [_VP, C.c_int, C.c_double, _VP, _VP]),
    "dirac_precond_apply": (C.c_int, [_VP, _VP, _VP]),
    "dirac_step": (C.c_int, [_VP, _VP, _VP, _IP, C.c_int, C.c_double, _IP, _DP]),
    "dirac_observables": (C.c_int, [_VP, _VP, _DP, C.c_int]),
    "dirac_run": (C.c_int, [_VP, _VP, _VP, _IP, C.c_int, C.c_double, _IP, _DP]),
    "dirac_apply_assembled": (C.c_int, [_VP, C.c_int, _VP, _VP]),
    "dirac_apply32": (C.c_int, [_VP, C.c_int, C.c_double, _VP, _VP]),
    "dirac_precond_apply32": (C.c_int, [_VP, _VP, _VP]),
    "dirac_residual": (C.c_int, [_VP, C.c_double, _VP, _VP, _VP, _DP]),
    "dirac_profile": (C.c_int, [_VP, C.c_int]),
    "dirac_profile_read": (C.c_int, [_VP, _DP, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "dirac_observables_static": (C.c_int, [_VP, _VP, _DP, C.c_int]),
    "dirac_solve_batch": (C.c_int, [C.POINTER(_VP), C.c_int, C.POINTER(_VP), C.POINTER(_VP), _IP, C.c_int, _DP,
                                    C.c_int, _IP, _DP]),
    "dirac_batch_tune": (C.c_int, [C.POINTER(_VP), C.c_int, C.POINTER(_VP), C.POINTER(_VP), _IP, _DP, _IP,
                                   C.c_int, _IP, _DP]),
    "dirac_guess_param_count": (C.c_int64, []),
    "dirac_guess_create": (C.c_int, [C.c_int, C.POINTER(_VP)]),
    "dirac_guess_free": (None, [_VP]),
    "dirac_guess_set_params": (C.c_int, [_VP, C.POINTER(C.c_float), C.c_int64]),
    "dirac_guess_get_params": (C.c_int, [_VP, C.POINTER(C.c_float), C.c_int64]),
    "dirac_guess_features": (C.c_int, [_VP, C.POINTER(_VP), C.c_double, _VP, _VP]),
    "dirac_guess_targets": (C.c_int, [_VP, C.POINTER(_VP), _VP, _VP, _VP]),
    "dirac_guess_forward": (C.c_int, [_VP, _VP, C.c_int64, _VP, C.c_int, _VP]),
    "dirac_guess_loss_grad": (C.c_int, [_VP, _VP, _VP, C.c_int, _DP, C.POINTER(C.c_float), _VP]),
    "dirac_guess_train_step": (C.c_int, [_VP, _VP, _VP, C.c_int, C.c_double, _DP, _VP]),
    "dirac_op_set_guess": (C.c_int, [_VP, _VP]),
    "dirac_op_set_overlap": (C.c_int, [_VP, C.c_int]),
    "dirac_op_set_residual_mode": (C.c_int, [_VP, C.c_int]),
    "dirac_op_set_schedule": (C.c_int, [_VP, C.c_int, C.c_int]),
    "dirac_selftest_wait": (C.c_int, [_VP, C.c_double, C.POINTER(C.c_int)]),
    "dirac_bounds_word": (C.c_int, [_VP, C.POINTER(C.c_uint), C.POINTER(C.c_int)]),
    "dirac_spectrum": (C.c_int, [_VP, _VP, C.c_double, C.c_double, C.c_int, _DP, _DP, C.POINTER(C.c_int64)]),
    "dirac_spectrum_error": (C.c_int, [C.c_int, _DP, _DP, _DP, C.c_double, C.c_double, _DP]),
    "dirac_op_set_factorised": (C.c_int, [_VP, C.c_int]),
    "dirac_op_get_schedule": (C.c_int, [_VP, C.c_int]),
    "dirac_last_error": (C.c_char_p, []),
}


def lib():
    """Load libdirac_gb300.so (built by ``paper_2512_21697_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s is not built (run __graft_entry__.build()); " % os.path.basename(LIB_PATH) +
                              "there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, what):
    if status != DIRAC_OK:
        raise DiracError(status, "%s: %s" % (what, lib().dirac_last_error().decode()))


def _dp(a):
    return a.ctypes.data_as(_DP)


def _ip(a):
    return a.ctypes.data_as(_IP)


def _fptr(t):
    """Device pointer of a contiguous float32 CUDA tensor."""
    import torch
    if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.float32):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _ptr(t):
    """Device pointer of a contiguous complex128 CUDA tensor."""
    import torch
    if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.complex128):
        raise ValueError("expected a contiguous complex128 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _ptr32(t):
    """Device pointer of a contiguous complex64 CUDA tensor."""
    import torch
    if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.complex64):
        raise ValueError("expected a contiguous complex64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def basis_params(cfg):
    return dirac_basis_params(Z=cfg["Z"], c=cfg["c"], R=cfg["R"], n_splines=cfg["N"], order=cfg["order"],
                              grid=cfg["grid"], r_lin=cfg["r_lin"], n_lin=cfg["n_lin"],
                              kappa_max=cfg["kappa_max"], two_mu_max=cfg["two_mu_max"], l_max=cfg["l_max"],
                              quad_pts=cfg["quad"])


def pulse_params(cfg):
    return dirac_pulse(E0=cfg["E0"], omega=cfg["omega"], n_cycles=cfg["n_cycles"], t0=cfg.get("t0", 0.0))


def solver_opts(cfg, **over):
    d = dict(dt=cfg["dt"], tol=cfg.get("tol", 1e-12), tol_inner=cfg.get("tol_inner", 1e-5),
             max_iter=cfg.get("max_iter", 500), precision=cfg.get("precision", 0),
             max_outer=cfg.get("max_outer", 20), guess=cfg.get("guess", 1),
             time_eval=cfg.get("time_eval", 0), precond=cfg.get("precond", 1))
    d.update(over)
    return dirac_solver_opts(**d)


class Basis:
    """dirac_basis: host-side basis, radial/pulse/angular setup data and the initial state."""

    def __init__(self, cfg):
        L = lib()
        self.cfg = dict(cfg)
        self.params = basis_params(cfg)
        h = _VP()
        n_guess = None
        # first call sizes the state; psi0 written in library order
        st = L.dirac_basis_build(C.byref(self.params), C.byref(h), None, None)
        _check(st, "dirac_basis_build")
        self._h = h
        self.n = L.dirac_basis_dim(h)
        self.nch = L.dirac_basis_nchannels(h)
        self.N = cfg["N"]
        self.nb = 2 * (self.N + 1)
        k = np.zeros(self.nch, np.int32)
        m = np.zeros(self.nch, np.int32)
        _check(L.dirac_basis_channels(h, _ip(k), _ip(m)), "dirac_basis_channels")
        self.kappa, self.two_mu = k, m
        self.npairs = L.dirac_basis_npairs(h)
        self.nterms = L.dirac_basis_nterms(h)
        del n_guess

    def initial_state(self):
        """(psi0, e0): the 1s1/2 mu=+1/2 state in library order and its energy."""
        L = lib()
        psi = np.zeros(self.n, np.complex128)
        e0 = C.c_double(0)
        h = _VP()
        _check(L.dirac_basis_build(C.byref(self.params), C.byref(h), _dp(psi.view(np.float64)), C.byref(e0)),
               "dirac_basis_build")
        L.dirac_basis_free(h)
        return psi, e0.value

    def radial(self, kappa):
        S = np.zeros((self.nb, self.nb))
        H = np.zeros((self.nb, self.nb))
        _check(lib().dirac_basis_radial(self._h, int(kappa), _dp(S), _dp(H)), "dirac_basis_radial")
        return S, H

    def coupling(self, cfg, a, b, t):
        X = np.zeros((self.nb, self.nb))
        p = pulse_params(cfg)
        _check(lib().dirac_basis_coupling(self._h, C.byref(p), int(a), int(b), float(t), _dp(X)),
               "dirac_basis_coupling")
        return X

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.dirac_basis_free(h)
            self._h = None


def angular(k1, tm1, k2, tm2, l):
    return lib().dirac_angular(int(k1), int(tm1), int(k2), int(tm2), int(l))


class Operator:
    """dirac_op: the device operator of one basis, pulse and solver setting."""

    def __init__(self, basis, cfg, stream=None, **opt_over):
        import torch
        self.basis = basis
        self.pulse = pulse_params(cfg)
        self.opts = solver_opts(cfg, **opt_over)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = _VP()
        _check(lib().dirac_operator_setup(basis._h, C.byref(self.pulse), C.byref(self.opts),
                                          C.c_void_p(stream.cuda_stream), C.byref(h)), "dirac_operator_setup")
        self._h = h
        self.n = basis.n

    @property
    def precision(self):
        return self.opts.precision

    def set_factorised(self, enable=True):
        """dirac_op_set_factorised: factorised complex64 apply in the inner solve (True or 1: subgroup
        form, 2: per-channel form, False or 0: stored coupling)."""
        mode = int(enable) if not isinstance(enable, bool) else int(enable)
        _check(lib().dirac_op_set_factorised(self._h, mode), "dirac_op_set_factorised")

    def spectrum(self, psi, e_lo, e_hi, grid, counts=False):
        """dirac_spectrum: (dP/dE on the host grid, levels in the window) or, with counts=True,
        (dP/dE, levels, channel-level projections formed)."""
        g = np.ascontiguousarray(grid, dtype=np.float64)
        out = np.zeros(len(g))
        cn = (C.c_int64 * 2)()
        _check(lib().dirac_spectrum(self._h, _ptr(psi), float(e_lo), float(e_hi), len(g), _dp(g), _dp(out), cn),
               "dirac_spectrum")
        return (out, int(cn[0]), int(cn[1])) if counts else (out, int(cn[0]))

    def bounds_word(self):
        """dirac_bounds_word: (bits of failed index checks since the last call, 1 if the library
        checks indexes -- a debug build -- else 0)."""
        w, c = C.c_uint(0), C.c_int(0)
        _check(lib().dirac_bounds_word(self._h, C.byref(w), C.byref(c)), "dirac_bounds_word")
        return int(w.value), int(c.value)

    def selftest_wait(self, limit_cycles):
        """dirac_selftest_wait: 1 if a wait on a never-completed mbarrier ran out of time."""
        t = C.c_int(0)
        _check(lib().dirac_selftest_wait(self._h, float(limit_cycles), C.byref(t)), "dirac_selftest_wait")
        return t.value

    def set_schedule(self, complex64, sched):
        """dirac_op_set_schedule: 0 lane / 1 warp / 2 staged-warp / 3 rotated-lane-warp preconditioner
        schedule."""
        _check(lib().dirac_op_set_schedule(self._h, int(bool(complex64)), int(sched)), "dirac_op_set_schedule")

    def schedule(self, complex64):
        return int(lib().dirac_op_get_schedule(self._h, int(bool(complex64))))

    def set_overlap(self, enable=True):
        """dirac_op_set_overlap: assemble the next step's coupling values during the current solve."""
        _check(lib().dirac_op_set_overlap(self._h, int(bool(enable))), "dirac_op_set_overlap")

    def set_residual_mode(self, mode):
        """dirac_op_set_residual_mode: 0 automatic (by tolerance), 1 Dot2, 2 fixed-binade offsets."""
        _check(lib().dirac_op_set_residual_mode(self._h, int(mode)), "dirac_op_set_residual_mode")

    def device_bytes(self):
        return lib().dirac_op_device_bytes(self._h)

    def apply(self, sign, t, x, y):
        _check(lib().dirac_apply(self._h, int(sign), float(t), _ptr(x), _ptr(y)), "dirac_apply")

    def apply32(self, sign, t, x, y):
        """dirac_apply32: the inner solve's complex64 operator (x, y complex64 CUDA tensors)."""
        _check(lib().dirac_apply32(self._h, int(sign), float(t), _ptr32(x), _ptr32(y)), "dirac_apply32")

    def precond32(self, r, z):
        """dirac_precond_apply32: the inner solve's complex64 preconditioner (current schedule)."""
        _check(lib().dirac_precond_apply32(self._h, _ptr32(r), _ptr32(z)), "dirac_precond_apply32")

    def residual(self, t, psi, x, r):
        """dirac_residual: r = A_-(t) psi - A_+(t) x as the step computes it; returns ||A_- psi||."""
        bn = C.c_double(0)
        _check(lib().dirac_residual(self._h, float(t), _ptr(psi), _ptr(x), _ptr(r), C.byref(bn)), "dirac_residual")
        return bn.value

    def apply_assembled(self, sign, x, y):
        _check(lib().dirac_apply_assembled(self._h, int(sign), _ptr(x), _ptr(y)), "dirac_apply_assembled")

    def profile(self, enable=True):
        _check(lib().dirac_profile(self._h, 1 if enable else 0), "dirac_profile")

    PHASES = ("assemble", "apply", "precond", "vector", "apply32", "guess", "owner")

    def profile_read(self):
        """({phase: ms}, {phase: timed launch groups}, kernel launches) since the last reset."""
        ms = np.zeros(len(self.PHASES))
        cnt = np.zeros(len(self.PHASES), np.int64)
        nl = C.c_int64(0)
        _check(lib().dirac_profile_read(self._h, _dp(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(nl)),
               "dirac_profile_read")
        return dict(zip(self.PHASES, ms)), dict(zip(self.PHASES, cnt)), nl.value

    def precond(self, r, z):
        _check(lib().dirac_precond_apply(self._h, _ptr(r), _ptr(z)), "dirac_precond_apply")

    def step(self, psi, n_steps, t_start, hist=None, n_hist=0):
        """Advance psi (CUDA complex128 tensor) in place; returns (iters, resid, n_hist)."""
        it = np.zeros(max(n_steps, 1), np.int32)
        res = np.zeros(max(n_steps, 1))
        nh = C.c_int(n_hist)
        st = lib().dirac_step(self._h, _ptr(psi), _ptr(hist) if hist is not None else None,
                              C.byref(nh), int(n_steps), float(t_start), _ip(it), _dp(res))
        _check(st, "dirac_step")
        return it[:n_steps], res[:n_steps], nh.value

    def run(self, psi, n_steps, t_start, hist, n_hist=0):
        """dirac_run: n_steps in one captured CUDA graph; returns (iters, resid, n_hist)."""
        it = np.zeros(max(n_steps, 1), np.int32)
        res = np.zeros(max(n_steps, 1))
        nh = C.c_int(n_hist)
        st = lib().dirac_run(self._h, _ptr(psi), _ptr(hist), C.byref(nh), int(n_steps), float(t_start), _ip(it),
                             _dp(res))
        _check(st, "dirac_run")
        return it[:n_steps], res[:n_steps], nh.value

    def observables(self, psi, bound=False):
        """norm, energy, ground-state population; with bound=True also the bound-state population
        (its eigenvectors are computed on the first such call)."""
        k = 4 if bound else 3
        out = np.zeros(k)
        _check(lib().dirac_observables(self._h, _ptr(psi), _dp(out), k), "dirac_observables")
        d = dict(norm=out[0], energy=out[1], p_ground=out[2])
        if bound:
            d["p_bound"] = out[3]
        return d

    def observables_static(self, psi):
        """dirac_observables_static: the same observables with library-static scratch."""
        out = np.zeros(3)
        _check(lib().dirac_observables_static(self._h, _ptr(psi), _dp(out), 3), "dirac_observables_static")
        return dict(norm=out[0], energy=out[1], p_ground=out[2])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.dirac_op_free(h)
            self._h = None


def _batch_args(ops, psis, hists, n_hist, t_start):
    n = len(ops)
    if not (len(psis) == len(hists) == n):
        raise ValueError("ops, states and histories differ in number")
    oa = (_VP * n)(*[o._h for o in ops])
    pa = (_VP * n)(*[_ptr(p) for p in psis])
    ha = (_VP * n)(*[_ptr(h) for h in hists])
    nh = (C.c_int * n)(*([0] * n if n_hist is None else [int(v) for v in n_hist]))
    ts = (C.c_double * n)(*[float(t) for t in (t_start if np.ndim(t_start) else [t_start] * n)])
    return n, oa, pa, ha, nh, ts


def solve_batch(ops, psis, hists, n_steps, t_start, n_hist=None, window=0):
    """dirac_solve_batch: advance every instance n_steps; returns (iters [n, n_steps],
    resid [n, n_steps], n_hist list)."""
    n, oa, pa, ha, nh, ts = _batch_args(ops, psis, hists, n_hist, t_start)
    it = np.zeros((n, max(n_steps, 1)), np.int32)
    res = np.zeros((n, max(n_steps, 1)))
    st = lib().dirac_solve_batch(oa, n, pa, ha, nh, int(n_steps), ts, int(window), _ip(it), _dp(res))
    _check(st, "dirac_solve_batch")
    return it[:, :n_steps], res[:, :n_steps], list(nh)


def batch_tune(ops, psis, hists, t_start, candidates, n_hist=None):
    """dirac_batch_tune: best window over the candidates (the ops keep the best preconditioner
    schedule); returns (best_window, ms [2, len(candidates)])."""
    n, oa, pa, ha, nh, ts = _batch_args(ops, psis, hists, n_hist, t_start)
    cand = (C.c_int * len(candidates))(*[int(c) for c in candidates])
    best = C.c_int(0)
    ms = np.zeros(2 * len(candidates))
    st = lib().dirac_batch_tune(oa, n, pa, ha, nh, ts, cand, len(candidates), C.byref(best), _dp(ms))
    _check(st, "dirac_batch_tune")
    return best.value, ms.reshape(2, len(candidates))


class GuessNet:
    """dirac_guess: the learned initial-guess network (parameters as one float32 array in the order
    W1, b1, W2, b2, W3, b3, W4, b4)."""

    def __init__(self, max_batch, params=None):
        h = _VP()
        _check(lib().dirac_guess_create(int(max_batch), C.byref(h)), "dirac_guess_create")
        self._h = h
        self.max_batch = int(max_batch)
        self.nparams = int(lib().dirac_guess_param_count())
        if params is not None:
            self.set_params(params)

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(lib().dirac_guess_set_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size),
               "dirac_guess_set_params")

    def get_params(self):
        a = np.zeros(self.nparams, np.float32)
        _check(lib().dirac_guess_get_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size),
               "dirac_guess_get_params")
        return a

    def forward(self, x, out, tensor_cores=True, stream=None):
        """dirac_guess_forward: tensor_cores True or 1 = tcgen05 kernel, 2 = mma.sync kernel, False or
        0 = the FP32 kernels."""
        tc = int(tensor_cores) if not isinstance(tensor_cores, bool) else int(tensor_cores)
        _check(lib().dirac_guess_forward(self._h, _fptr(x), x.shape[0], _fptr(out), tc,
                                         _VP(_stream_ptr(stream))), "dirac_guess_forward")

    def loss_grad(self, x, t, stream=None):
        B = x.shape[0]
        loss = C.c_double(0)
        g = np.zeros(self.nparams, np.float32)
        _check(lib().dirac_guess_loss_grad(self._h, _fptr(x), _fptr(t), B, C.byref(loss),
                                           g.ctypes.data_as(C.POINTER(C.c_float)), _VP(_stream_ptr(stream))),
               "dirac_guess_loss_grad")
        return loss.value, g

    def train_step(self, x, t, lr, stream=None):
        loss = C.c_double(0)
        _check(lib().dirac_guess_train_step(self._h, _fptr(x), _fptr(t), x.shape[0], float(lr), C.byref(loss),
                                            _VP(_stream_ptr(stream))), "dirac_guess_train_step")
        return loss.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.dirac_guess_free(h)
            self._h = None


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def spectrum_error(grid, p_n, p_m, e1, e2):
    """dirac_spectrum_error: trapezoid integral of |p_n - p_m|^2 over the grid points in [e1, e2]."""
    g = np.ascontiguousarray(grid, dtype=np.float64)
    a = np.ascontiguousarray(p_n, dtype=np.float64)
    b = np.ascontiguousarray(p_m, dtype=np.float64)
    if not (len(a) == len(b) == len(g)):
        raise ValueError("grid and spectra differ in length")
    err = C.c_double(0)
    _check(lib().dirac_spectrum_error(len(g), _dp(g), _dp(a), _dp(b), float(e1), float(e2), C.byref(err)),
           "dirac_spectrum_error")
    return float(err.value)


def guess_features(op, states, t_next, x, s):
    arr = (_VP * 4)(*[_ptr(z) for z in states])
    _check(lib().dirac_guess_features(op._h, arr, float(t_next), _fptr(x), _fptr(s)), "dirac_guess_features")


def guess_targets(op, states, psi_next, s, t):
    arr = (_VP * 3)(*[_ptr(z) for z in states[:3]])
    _check(lib().dirac_guess_targets(op._h, arr, _ptr(psi_next), _fptr(s), _fptr(t)), "dirac_guess_targets")


def set_guess(op, net):
    op._net = net   # keep the network alive while attached
    _check(lib().dirac_op_set_guess(op._h, net._h if net is not None else None), "dirac_op_set_guess")
