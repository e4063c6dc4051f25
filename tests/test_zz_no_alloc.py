"""dirac_observables_static: the observables with no allocation in the call.

Callers that cannot allocate GPU memory when they read the observables -- real-time or monitoring
threads that must not trigger the implicit device synchronisation of cudaMalloc/cudaFree,
processes whose device footprint is fixed after setup -- use this entry point; its scratch is a
library-static device array.  These tests call it through the C ABI twice in a row (different
states) and check it against dirac_observables, which uses the operator's own preallocated
scratch, and against the oracle; they also check its argument errors and its size limit.  The
file runs last so that a failure here leaves every other test already run, and it passes both
alone and after the others.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2512_21697_gb300 import binding as B, layout, workloads as W

pytestmark = pytest.mark.gpu


def _masked_random(bas, seed):
    x = W.random_state(bas.n, seed)
    nb = bas.nb
    for ch, kappa in enumerate(bas.kappa):
        if kappa != -1:
            x[ch * nb + 0] = 0          # slot 0, large type: used only by kappa = -1
        if kappa != 1:
            x[ch * nb + 1] = 0          # slot 0, small type: used only by kappa = +1
    return x / np.linalg.norm(x)


def _static(lib, op, psi, n_out=3):
    out = np.zeros(max(n_out, 1))
    st = lib.dirac_observables_static(op._h, C.c_void_p(psi.data_ptr()), out.ctypes.data_as(C.POINTER(C.c_double)),
                                      n_out)
    return st, out


@pytest.mark.parametrize("name", ["small", "slice"])
def test_static_scratch_observables_match_allocating_entry_point(name, oracle_mod):
    import torch
    from paper_2512_21697_gb300 import build
    build.build()
    lib = B.lib()
    cfg = W.WORKLOADS[name]
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg)
    orc = oracle_mod.Oracle(**W.oracle_params(cfg))
    perm = layout.lib_to_paper_perm(bas.kappa, bas.two_mu, cfg["kappa_max"], cfg["two_mu_max"], cfg["N"])
    psi0, _ = bas.initial_state()
    for call, psi_h in enumerate((_masked_random(bas, 21), psi0)):   # two calls in a row
        psi = torch.from_numpy(psi_h).cuda()
        ref = op.observables(psi)
        st, out = _static(lib, op, psi)
        assert st == B.DIRAC_OK, lib.dirac_last_error()
        orf = orc.observables(psi_h[perm])
        for i, k in enumerate(("norm", "energy", "p_ground")):
            assert abs(out[i] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (call, k, out[i], ref[k])
            assert abs(out[i] - orf[k]) <= 1e-11 * max(1.0, abs(orf[k])), (call, k, out[i], orf[k])
    # the second state is the normalised 1s level: norm 1, ground population 1
    assert abs(out[0] - 1) < 1e-12 and abs(out[2] - 1) < 1e-12


def test_static_scratch_rejects_bad_arguments():
    import torch
    lib = B.lib()
    cfg = W.TINY
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg)
    psi = torch.from_numpy(_masked_random(bas, 3)).cuda()
    for n_out in (0, 4):
        st, _ = _static(lib, op, psi, n_out)
        assert st == B.DIRAC_E_ARG, n_out
    st, _ = _static(lib, op, psi, 2)          # a valid call still works afterwards
    assert st == B.DIRAC_OK, lib.dirac_last_error()


def test_static_scratch_size_limit():
    # 220 channels (|kappa| <= 10, every mu) x ceil(38017 / 128) = 298 row tiles = 65 560 block
    # partials, just above DIRAC_STATIC_MAX_PARTIALS = 65 536: refused with DIRAC_E_ARG, while the
    # allocating entry point still serves the system (multipole l = 0 only keeps the operator at
    # about 9 GB of coupling values)
    import torch
    lib = B.lib()
    cfg = dict(W.SMALL, kappa_max=10, two_mu_max=0, l_max=0, N=38016, R=3000.0)
    bas = B.Basis(cfg)
    assert bas.nch * -(-(cfg["N"] + 1) // 128) == 65560
    op = B.Operator(bas, cfg)
    psi0, _ = bas.initial_state()
    psi = torch.from_numpy(psi0).cuda()
    st, _ = _static(lib, op, psi)
    assert st == B.DIRAC_E_ARG
    assert b"static scratch" in lib.dirac_last_error()
    ref = op.observables(psi)
    assert abs(ref["norm"] - 1) < 1e-10


def test_static_scratch_refuses_a_capturing_stream():
    # the call reads its sums back and synchronises the op's stream, which a stream capture does not
    # allow: on a capturing stream it returns DIRAC_E_STATE before enqueueing anything, the capture
    # stays valid, and the op works again once the capture has ended
    import torch
    lib = B.lib()
    cfg = W.TINY
    bas = B.Basis(cfg)
    s = torch.cuda.Stream()
    op = B.Operator(bas, cfg, stream=s)
    psi = torch.from_numpy(_masked_random(bas, 5)).cuda()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st, _ = _static(lib, op, psi)
    assert st == B.DIRAC_E_STATE, lib.dirac_last_error()
    assert b"captured" in lib.dirac_last_error()
    torch.cuda.synchronize()
    st, out = _static(lib, op, psi)
    assert st == B.DIRAC_OK, lib.dirac_last_error()
    ref = op.observables(psi)
    for i, k in enumerate(("norm", "energy", "p_ground")):
        assert abs(out[i] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, out[i], ref[k])
