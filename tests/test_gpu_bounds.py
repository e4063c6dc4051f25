"""The debug build (index checks compiled in, -DDG_BOUNDS): every computed global index of the
owner and gather passes and of the grouped assembly stays inside its buffer on the parity
workloads -- several radial tiles with a ragged last tile, one tile, kappa groups of every size --
and the checks change no result.  The debug library runs in a child process (the binding picks
the library at import); the parent compares its states with the release library's."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (workload, precision, driver, factorised): the mixed paths use the owner/gather passes and the
# grouped assembly; "run" is the captured graph driver
CASES = [("tiny", 2, "step", 0), ("small", 2, "step", 0), ("tail", 2, "step", 0), ("slice", 2, "run", 0),
         ("small", 1, "step", 0), ("tail", 1, "run", 0), ("small", 2, "step", 1), ("tail", 2, "run", 2),
         ("order5", 2, "step", 0)]

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2512_21697_gb300 import binding as B, workloads as W
out = {}
for name, prec, drv, fact in json.loads(sys.argv[2]):
    cfg = W.WORKLOADS[name]
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg, tol=1e-12, precision=prec, max_iter=1000, tol_inner=1e-5, max_outer=30)
    if fact:
        op.set_factorised(fact)
    psi = torch.from_numpy(W.random_state(bas.n, 11)).cuda()
    hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device="cuda")
    t = 0.25 * cfg["n_cycles"] * 2 * np.pi / cfg["omega"]
    if drv == "step":
        op.step(psi, 2, t, hist=hist, n_hist=0)
    else:
        op.run(psi, 2, t, hist, n_hist=0)
    word, checked = op.bounds_word()
    np.save(sys.argv[3] + "/%s_%d_%s_%d.npy" % (name, prec, drv, fact), psi.cpu().numpy())
    out["%s_%d_%s_%d" % (name, prec, drv, fact)] = [word, checked]
print("BOUNDS " + json.dumps(out))
"""


def _run_release(name, prec, drv, fact):
    import torch
    from paper_2512_21697_gb300 import binding as B, workloads as W
    cfg = W.WORKLOADS[name]
    bas = B.Basis(cfg)
    op = B.Operator(bas, cfg, tol=1e-12, precision=prec, max_iter=1000, tol_inner=1e-5, max_outer=30)
    if fact:
        op.set_factorised(fact)
    psi = torch.from_numpy(W.random_state(bas.n, 11)).cuda()
    hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device="cuda")
    t = 0.25 * cfg["n_cycles"] * 2 * np.pi / cfg["omega"]
    if drv == "step":
        op.step(psi, 2, t, hist=hist, n_hist=0)
    else:
        op.run(psi, 2, t, hist, n_hist=0)
    word, checked = op.bounds_word()
    assert (word, checked) == (0, 0)   # a release build carries no checks
    return psi.cpu().numpy()


def test_debug_build_indexes_stay_in_bounds(tmp_path):
    sys.path.insert(0, ROOT)
    from paper_2512_21697_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, DIRAC_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(CASES), str(tmp_path)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("BOUNDS ")][-1]
    words = json.loads(line[len("BOUNDS "):])
    for key, (word, checked) in words.items():
        assert checked == 1, key            # the child really loaded the debug build
        assert word == 0, "%s: failed index checks, site bits %#x" % (key, word)
    for name, prec, drv, fact in CASES:
        key = "%s_%d_%s_%d" % (name, prec, drv, fact)
        dbg = np.load(str(tmp_path / (key + ".npy")))
        rel = _run_release(name, prec, drv, fact)
        # the checks only guard accesses: the same arithmetic, so the same states to rounding
        assert np.linalg.norm(dbg - rel) <= 1e-13 * np.linalg.norm(rel), key
