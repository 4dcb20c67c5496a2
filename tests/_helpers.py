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


def cluster_sines(lam_ref, u_ref, x, gap=1e-6):
    """Largest principal-angle sine between span(u_ref[:, cluster]) and span(x[:, cluster]) over the
    clusters of lam_ref (eigenvalues closer than `gap` form one cluster, Kramers pairs included);
    a cluster that reaches the last column may continue beyond it and is left out.  u_ref and x
    are column matrices with orthonormal columns."""
    lam_ref = np.asarray(lam_ref)
    n = len(lam_ref)
    worst = 0.0
    i = 0
    while i < n:
        j = i + 1
        while j < n and lam_ref[j] - lam_ref[j - 1] < gap:
            j += 1
        if j < n:
            s = np.linalg.svd(u_ref[:, i:j].conj().T @ x[:, i:j], compute_uv=False)
            worst = max(worst, float(np.sqrt(max(0.0, 1.0 - min(s) ** 2))))
        i = j
    return worst
