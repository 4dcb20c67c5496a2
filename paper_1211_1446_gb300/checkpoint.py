"""Checkpoint and resume of solves (the paper's warm start, Sec. 3.1: a converged X becomes the
next start block with N_init = 1).

save() writes, per k-point, the eigenvector block X [nev_k + nbuf, ncomp, npw] (complex128), its
eigenvalues and the planewave basis (Miller triples) to one .npz file; load() reads them back as
device tensors, and checks that the basis of every k-point matches the context it resumes in
(the same cell, cutoff and k-points give the same canonical planewave order).
"""
from __future__ import annotations

import numpy as np


def save(path, ctx, xs, lams, **meta):
    """Write the blocks xs (device or host complex tensors, one per k-point), the eigenvalues lams
    (arrays, one per k-point) and the context's basis to path (.npz); meta: extra scalars."""
    if len(xs) != ctx.nk or len(lams) != ctx.nk:
        raise ValueError(f"need one block and one eigenvalue array per k-point ({ctx.nk})")
    arrays = {"nk": np.int64(ctx.nk), "ncomp": np.int64(ctx.ncomp), "grid": np.asarray(ctx.grid, dtype=np.int64)}
    for ik in range(ctx.nk):
        x = xs[ik].detach().cpu().numpy() if hasattr(xs[ik], "detach") else np.asarray(xs[ik])
        arrays[f"x{ik}"] = np.ascontiguousarray(x, dtype=np.complex128)
        arrays[f"lam{ik}"] = np.asarray(lams[ik], dtype=np.float64)
        arrays[f"miller{ik}"] = np.asarray(ctx.basis(ik), dtype=np.int32)
    for k, v in meta.items():
        arrays[f"meta_{k}"] = np.asarray(v)
    np.savez(path, **arrays)


def load(path, ctx, device="cuda"):
    """Read a checkpoint for ctx: returns (xs as complex128 tensors on device, lams, meta dict).
    Raises ValueError when the k-points, components, grid or any planewave basis differ."""
    import torch
    with np.load(path) as f:
        if int(f["nk"]) != ctx.nk or int(f["ncomp"]) != ctx.ncomp or tuple(f["grid"]) != tuple(ctx.grid):
            raise ValueError("checkpoint was written for another context (k-points, components or grid)")
        xs, lams = [], []
        for ik in range(ctx.nk):
            if not np.array_equal(f[f"miller{ik}"], ctx.basis(ik)):
                raise ValueError(f"planewave basis of k-point {ik} differs from the checkpoint's")
            xs.append(torch.from_numpy(np.array(f[f"x{ik}"])).to(device))
            lams.append(np.array(f[f"lam{ik}"]))
        meta = {k[5:]: f[k][()] for k in f.files if k.startswith("meta_")}
    return xs, lams, meta
