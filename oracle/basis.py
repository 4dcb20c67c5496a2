"""Planewave sphere for one k-point (Sec. 2.3; grid convention of Sec. 4).

The basis for k is every reciprocal vector G = m1 b1 + m2 b2 + m3 b3 with
|k+G|^2 / 2 <= Ecut.  The same grid resolves wavefunctions and the potential,
so the sphere must fit inside the FFT grid without touching the Nyquist plane:
|m_i| <= (N_i - 1) // 2, else the workload is rejected.
"""
from __future__ import annotations

import numpy as np

from workloads import reciprocal_rows


def sphere(lattice, grid, kfrac, ecut):
    """Return (miller[npw,3] int64, q[npw,3] cartesian k+G) in canonical order."""
    lattice = np.asarray(lattice, dtype=np.float64)
    brow = reciprocal_rows(lattice)
    k = np.asarray(kfrac, dtype=np.float64) @ brow
    gmax = np.sqrt(2.0 * ecut)
    # |m_i| is bounded by (|k| + gmax) |a_i| / (2 pi)
    lim = [int(np.floor((np.linalg.norm(k) + gmax) * np.linalg.norm(lattice[i]) / (2 * np.pi))) + 1
           for i in range(3)]
    r = [np.arange(-l, l + 1) for l in lim]
    m = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    q = k + m @ brow
    keep = 0.5 * np.einsum("ij,ij->i", q, q) <= ecut
    m, q = m[keep], q[keep]
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0]))
    m, q = m[order], q[order]
    for i in range(3):
        if np.abs(m[:, i]).max(initial=0) > (grid[i] - 1) // 2:
            raise ValueError(f"planewave sphere does not fit the FFT grid along axis {i}")
    return m.astype(np.int64), q


def grid_index(miller, grid):
    """Flat index (i1*N2 + i2)*N3 + i3 of each planewave with i = m mod N."""
    n1, n2, n3 = grid
    i = np.mod(miller, np.asarray(grid))
    return (i[:, 0] * n2 + i[:, 1]) * n3 + i[:, 2]
