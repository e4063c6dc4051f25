"""Bounded waits on the GPU: a wait that nothing completes runs out of time, the kernel records it
in the op's error word and returns, and the context stays usable (the next step still matches
the oracle).  No fault, trap or hang: the wait has a cycle limit and no copy is in flight."""
import numpy as np
import pytest

from paper_2512_21697_gb300 import binding as B, workloads as W

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_context_survives(oracle_mod):
    import torch
    cfg = W.TINY
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg, tol=1e-12, precision=2, max_iter=1000, tol_inner=1e-5, max_outer=30)
    assert op.selftest_wait(2e6) == 1          # about a millisecond at 2 GHz, then the error word
    assert op.selftest_wait(0) == 1            # the limit is checked before any completion
    with pytest.raises(B.DiracError):
        op.selftest_wait(-1.0)
    # the context and the op still work: one step against the oracle
    orc = oracle_mod.Oracle(**W.oracle_params(cfg))
    from paper_2512_21697_gb300 import layout
    perm = layout.lib_to_paper_perm(bas.kappa, bas.two_mu, cfg["kappa_max"], cfg["two_mu_max"], cfg["N"])
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    x = W.random_state(orc.n, 5)
    x[~orc.active_mask()] = 0
    x /= np.linalg.norm(x)
    psi = torch.from_numpy(x[inv].copy()).cuda()
    its, res, _ = op.step(psi, 1, 1.0)
    ref, _, _ = orc.step(x, 1.0, tol=1e-14)
    got = psi.cpu().numpy()[perm]
    assert res[0] <= 1e-12
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
