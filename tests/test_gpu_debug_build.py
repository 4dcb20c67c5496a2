"""The index-checked debug library (libdks_debug.so: every sphere <-> grid and plane index of the
FFT kernels is checked before use, a failed check records its code and skips the access) on the
GPU, on valid inputs: the same H' results as the oracle, a full solve, and no recorded failure.
It runs in a child process, since a process holds one of the two libraries."""
import json
import os
import subprocess
import sys

import pytest

from ._helpers import gpu

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import paper_1211_1446_gb300 as P
from paper_1211_1446_gb300 import build
P.load_library(build.build(debug=True))
import workloads as W
from oracle import basis, lobpcgf, operator
out = {}
for name, kw in (("small", {}), ("dimer", {"ecut": 4.0}), ("small", {"grid": (20, 21, 14)})):
    wl = W.make(name, **kw)
    ctx = P.Context.from_workload(wl)
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    x = W.random_block(len(q), 3, 5)
    ref = operator.MatrixFreeH(wl, m, q)(x)
    xd = torch.from_numpy(x).cuda()
    hx = torch.empty_like(xd)
    ctx.apply_H(0, xd, hx)
    ctx.apply_H(0, xd, hx, emulated=True)
    torch.cuda.synchronize()
    out[name + str(kw)] = float(np.abs(hx.cpu().numpy() - ref).max() / np.abs(ref).max())
wl = W.make("cubic")
ctx = P.Context.from_workload(wl)
m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
lam_ref, _, _ = lobpcgf.dense_eigs(operator.dense_hamiltonian(wl, m, q), wl.c, 8)
x0 = torch.from_numpy(W.start_block(len(q), 8, wl.seed)).cuda()
lam, rep, rc = ctx.solve([x0], 8, mode=P.MODE_MIXED, check=False)
out["solve_rc"] = rc
out["solve_err"] = float(np.abs(lam[0] - lam_ref).max())
compiled, code = P.debug_check()
out["compiled"] = compiled
out["code"] = code
print("RESULT " + json.dumps(out))
"""


def test_debug_build_runs_clean_on_valid_inputs():
    gpu()
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert res["compiled"] is True and res["code"] == 0, res
    assert res["solve_rc"] == 0 and res["solve_err"] < 1e-8, res
    for k, v in res.items():
        if k.startswith(("small", "dimer")):
            assert v < 1e-11, (k, v)
