"""Write the stored expected values under tests/golden/ by calling the CPU oracle only.

    python tests/golden/make_golden.py [cubic] [dimer]

cubic_dense_eigs.txt   lowest 8 eigenvalues above the gap of the dense shifted H'
                       for the cubic workload (zheevd, FP64).
dimer_lobpcgf_eigs.txt lowest 32 eigenvalues of the dimer workload from the oracle's
                       Algorithm 1 (FP64, Teter, N_init = 3, block of 32 + 8 buffer columns,
                       every checked residual below 5e-7).
dimer_ksso_eigs.txt    lowest 32 eigenvalues of the dimer's KSSO two-component operator from
                       the oracle's Algorithm 1 without the filter (standard LOBPCG, Teter,
                       32 + 8 buffer columns, every checked residual below 5e-7).
dimer_ecut2_dense_eigs.txt
                       lowest 40 eigenvalues above the gap of the dense shifted H' of the dimer
                       cell, grid and 36 projector channels at Ecut 2 Ha (1295 planewaves,
                       dimension 5180), zheevd (FP64).
layered_k<i>_eigs.txt  lowest 48 eigenvalues of the layered crystal at k-point i from the oracle's
                       Algorithm 1 (FP64, Teter, N_init = 3, 48 + 8 buffer columns, every checked
                       residual below 5e-7): one k-point of the batched configuration, about an
                       hour of CPU time each (python tests/golden/make_golden.py layered0 layered4).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import basis, lobpcgf as lb, operator as op  # noqa: E402


def cubic():
    wl = W.make("cubic")
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    lam, _, _ = lb.dense_eigs(op.dense_hamiltonian(wl, m, q), wl.c, 8)
    np.savetxt(os.path.join(HERE, "cubic_dense_eigs.txt"), lam, fmt="%.15e",
               header="cubic workload: lowest 8 eigenvalues (Ha, shifted by -c^2) of dense H', zheevd")


def dimer():
    wl = W.make("dimer")
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    hop = op.MatrixFreeH(wl, m, q)
    cs, om = op.filter_constants(wl, q)
    x0 = W.start_block(len(q), 40, wl.seed)
    r = lb.lobpcgf(hop, q, x0, 40, cs, om, tol=5e-7, nconv=32,
                   callback=lambda it, lam, n: print(it, n[:32].max(), flush=True))
    assert r.converged and np.all(r.lam > -wl.c ** 2)
    np.savetxt(os.path.join(HERE, "dimer_lobpcgf_eigs.txt"), r.lam[:32], fmt="%.15e",
               header=f"dimer workload: lowest 32 eigenvalues (Ha, shifted) from the oracle's "
                      f"Algorithm 1, 32 + 8 buffer columns, tol 5e-7, {r.iterations} iterations")


def dimer_ksso():
    wl = W.make("dimer")
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    hop = op.MatrixFreeKSSO(wl, m, q)
    x0 = W.start_block(len(q), 40, wl.seed, ncomp=2)
    r = lb.lobpcgf(hop, q, x0, 40, 0.0, 1.0, tol=5e-7, nconv=32, use_filter=False,
                   callback=lambda it, lam, n: print(it, n[:32].max(), flush=True))
    assert r.converged
    np.savetxt(os.path.join(HERE, "dimer_ksso_eigs.txt"), r.lam[:32], fmt="%.15e",
               header=f"dimer workload, KSSO operator: lowest 32 eigenvalues (Ha) from the oracle's "
                      f"Algorithm 1 without the filter, 32 + 8 buffer columns, tol 5e-7, "
                      f"{r.iterations} iterations")


def dimer_ecut2():
    wl = W.make("dimer", ecut=2.0)
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    h = op.dense_hamiltonian(wl, m, q)
    lam, _, _ = lb.dense_eigs(h, wl.c, 40)
    np.savetxt(os.path.join(HERE, "dimer_ecut2_dense_eigs.txt"), lam, fmt="%.15e",
               header=f"dimer cell at Ecut 2 Ha (npw {len(q)}, dimension {h.shape[0]}, 36 projector "
                      f"channels): lowest 40 eigenvalues (Ha, shifted by -c^2) of dense H', zheevd")


def layered(ik, nev=48, nbuf=8):
    wl = W.make("layered")
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[ik], wl.ecut_k[ik])
    hop = op.MatrixFreeH(wl, m, q)
    cs, om = op.filter_constants(wl, q)
    x0 = W.start_block(len(q), nev + nbuf, wl.seed, ik)
    r = lb.lobpcgf(hop, q, x0, nev + nbuf, cs, om, tol=5e-7, nconv=nev,
                   callback=lambda it, lam, n: print(it, n[:nev].max(), flush=True))
    assert r.converged and np.all(r.lam > -wl.c ** 2)
    np.savetxt(os.path.join(HERE, f"layered_k{ik}_eigs.txt"), r.lam[:nev], fmt="%.15e",
               header=f"layered crystal, k-point {ik} (fractional {[float(v) for v in wl.kfrac[ik]]}, npw {len(q)}): "
                      f"lowest {nev} eigenvalues (Ha, shifted) from the oracle's Algorithm 1, "
                      f"{nev} + {nbuf} buffer columns, tol 5e-7, {r.iterations} iterations")


def layered0():
    layered(0)


def layered4():
    layered(4)


if __name__ == "__main__":
    which = sys.argv[1:] or ["cubic"]
    for w in which:
        globals()[w]()
