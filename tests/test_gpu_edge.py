"""Degenerate inputs of the step: a zero state (b = 0, so the relative criterion is met by the zero
solution at once), zero steps (nothing changes), for the FP64 and the mixed paths and for both
drivers.  The results are exact: no arithmetic can make a zero state nonzero."""
import numpy as np
import pytest

from paper_2512_21697_gb300 import binding as B, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 2])
def test_zero_state_stays_zero(precision):
    import torch
    cfg = W.SMALL
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg, tol=1e-12, precision=precision, max_iter=1000, tol_inner=1e-5, max_outer=30)
    psi = torch.zeros(bas.n, dtype=torch.complex128, device="cuda")
    its, res, _ = op.step(psi, 3, 0.3)
    assert torch.count_nonzero(psi).item() == 0
    assert np.all(res == 0)
    hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device="cuda")
    its, res, _ = op.run(psi, 3, 0.3, hist)
    assert torch.count_nonzero(psi).item() == 0
    assert np.all(res == 0)


@pytest.mark.parametrize("precision", [0, 2])
def test_zero_steps_leave_the_state(precision):
    import torch
    cfg = W.SMALL
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg, tol=1e-12, precision=precision, max_iter=1000, tol_inner=1e-5, max_outer=30)
    x = torch.from_numpy(W.random_state(bas.n, 4)).cuda()
    psi = x.clone()
    hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device="cuda")
    its, res, nh = op.step(psi, 0, 0.3, hist=hist, n_hist=0)
    assert len(its) == 0 and nh == 0 and torch.equal(psi, x)
    its, res, nh = op.run(psi, 0, 0.3, hist, n_hist=0)
    assert len(its) == 0 and nh == 0 and torch.equal(psi, x)
    with pytest.raises(B.DiracError):
        op.step(psi, -1, 0.3)
