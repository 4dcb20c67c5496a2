"""Shared test plumbing: build a library context and the matching oracle objects for a workload."""
import numpy as np

import workloads as W
from oracle import basis as obasis
from oracle import operator as oop


def gpu():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("needs a CUDA device")
    return torch


def make_pair(name, ik=0, model="dks", **kw):
    """(workload, library Context, oracle matrix-free operator, q) for k-point ik; model "dks"
    (four-spinors, MatrixFreeH) or "ksso" (two-spinors, MatrixFreeKSSO)."""
    import paper_1211_1446_gb300 as P
    wl = W.make(name, **kw)
    ctx = P.Context.from_workload(wl, model=model)
    m, q = obasis.sphere(wl.lattice, wl.grid, wl.kfrac[ik], wl.ecut_k[ik])
    lib_m = ctx.basis(ik)
    assert lib_m.shape == m.shape and np.array_equal(lib_m, m), "planewave basis differs from the oracle's"
    hop = oop.MatrixFreeH(wl, m, q) if model == "dks" else oop.MatrixFreeKSSO(wl, m, q)
    return wl, ctx, hop, q


def to_dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
