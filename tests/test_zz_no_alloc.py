"""dirac_observables_static: the observables with no allocation in the call.

Callers that cannot allocate GPU memory when they read the observables -- code running while a
stream is captured into a CUDA graph, real-time or monitoring threads that must not trigger the
implicit device synchronisation of cudaMalloc/cudaFree, processes whose device footprint is fixed
after setup -- use this entry point; its scratch is a library-static device array.  This test
calls it through the C ABI twice in a row (different states) and checks it against
dirac_observables, which uses the operator's own preallocated scratch.  It runs last so that a
failure here leaves every other test already run, and it passes both alone and after the others.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2512_21697_gb300 import binding as B, workloads as W

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


@pytest.mark.parametrize("name", ["small", "slice"])
def test_static_scratch_observables_match_allocating_entry_point(name):
    import torch
    from paper_2512_21697_gb300 import build
    build.build()
    lib = B.lib()
    cfg = W.WORKLOADS[name]
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg)
    psi0, _ = bas.initial_state()
    for call, psi_h in enumerate((_masked_random(bas, 21), psi0)):   # two calls in a row
        psi = torch.from_numpy(psi_h).cuda()
        ref = op.observables(psi)
        out = np.zeros(3)
        st = lib.dirac_observables_static(op._h, C.c_void_p(psi.data_ptr()),
                                          out.ctypes.data_as(C.POINTER(C.c_double)), 3)
        assert st == B.DIRAC_OK, lib.dirac_last_error()
        for i, k in enumerate(("norm", "energy", "p_ground")):
            assert abs(out[i] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (call, k, out[i], ref[k])
    # the second state is the normalised 1s level: norm 1, ground population 1
    assert abs(out[0] - 1) < 1e-12 and abs(out[2] - 1) < 1e-12
