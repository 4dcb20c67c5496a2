"""The layered-crystal configuration at its full size: hexagonal cell a = 7.8, c = 28 bohr with
15 sites in three quintuple layers (270 spin-orbit projector channels), 60 x 60 x 216 grid,
16 k-points on a 4 x 4 x 1 mesh with per-k cutoffs jittered by +-3 % (about 39,000-41,000
planewaves each) and nev_k between 48 and 96.

Dense diagonalisation is out of reach at ~160,000 rows, so parity is checked on outputs the
oracle computes one by one and on properties that hold at any size:
  * H' x for sampled columns at two k-points against the oracle's matrix-free operator;
  * a mixed-precision solve of all 16 k-points by concurrent workers (8 buffer columns per k):
    every checked residual below 1e-6, and for sampled columns recomputed here with the
    oracle's operator; orthonormal vectors; no eigenvalue below the gap midpoint; Kramers pairs
    at the four time-reversal-invariant k-points of the mesh; the 48 lowest eigenvalues at
    k = 0 within 1e-8 Ha of the oracle's Algorithm 1 run on that k-point alone (stored by
    tests/golden/make_golden.py).
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import basis as obasis, operator as oop
from tests._helpers import gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

TRIM = (0, 2, 8, 10)      # k = (0,0), (0,1/2), (1/2,0), (1/2,1/2)


@pytest.fixture(scope="module")
def layered():
    gpu()
    import paper_1211_1446_gb300 as P
    wl = W.make("layered")
    ctx = P.Context.from_workload(wl)
    return wl, ctx


@pytest.mark.parametrize("ik", [0, 5])
def test_layered_apply_h_sampled(layered, ik):
    import torch
    wl, ctx = layered
    m, q = obasis.sphere(wl.lattice, wl.grid, wl.kfrac[ik], wl.ecut_k[ik])
    assert np.array_equal(ctx.basis(ik), m)
    hop = oop.MatrixFreeH(wl, m, q)
    rng = np.random.default_rng(ik)
    x = rng.standard_normal((2, 4, len(m))) + 1j * rng.standard_normal((2, 4, len(m)))
    want = hop(x)
    hx = torch.empty((2, 4, len(m)), dtype=torch.complex128, device="cuda")
    ctx.apply_H(ik, to_dev(x, torch.complex128), hx)
    assert rel_err(hx.cpu().numpy(), want) < 1e-12
    ctx.apply_H(ik, to_dev(x, torch.complex128), hx, emulated=True)
    assert rel_err(hx.cpu().numpy(), want) < 1e-12


def test_layered_solve_all_kpoints(layered):
    import torch
    import paper_1211_1446_gb300 as P
    wl, ctx = layered
    nbuf = 8
    nev_k = [int(v) for v in wl.nev_k]
    xs = [torch.from_numpy(W.start_block(ctx.npw(ik), nev_k[ik] + nbuf, wl.seed, ik)).cuda() for ik in range(wl.nk)]
    lam, rep, rc = ctx.solve(xs, 0, nev_k=nev_k, nbuf=nbuf, tol=1e-6, mode=P.MODE_MIXED, check=False)
    print(f"layered: 16 k-points, {sum(nev_k)} eigenpairs in {rep['seconds']:.2f} s, iterations "
          f"{rep['iterations'][:wl.nk]}, FP64-phase {rep['fp64_iterations'][:wl.nk]}")
    assert rc == 0, (rep["message"], rep["iterations"][:wl.nk], rep["max_residual"][:wl.nk])
    assert max(rep["max_residual"][:wl.nk]) < 1e-6
    for ik in range(wl.nk):
        assert lam[ik].shape == (nev_k[ik],) and np.all(np.diff(lam[ik]) >= -1e-12)
        assert lam[ik][0] > -wl.c ** 2                           # above the gap midpoint
    for ik in TRIM:                                              # Kramers pairs
        assert np.abs(lam[ik][0::2] - lam[ik][1::2]).max() < 1e-7, ik
    # eigenvalues at k = 0 against the oracle's Algorithm 1 on that k-point alone (48 lowest,
    # tests/golden/layered_k0_eigs.txt): a state skipped inside the wanted window fails here
    gold = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "layered_k0_eigs.txt"))
    assert np.abs(lam[0][:len(gold)] - gold).max() < 1e-8, np.abs(lam[0][:len(gold)] - gold).max()
    # orthonormal columns (all nev + nbuf of them) at two k-points.  X = Z V with V orthonormal
    # in the metric S = Z^H Z of the last Rayleigh-Ritz step, so X^H X - I is the rounding of that
    # FP64 step times the conditioning of S, which grows as the directions of P converge; on a
    # GB300 the largest entry was 6.5e-10 (k = 13, among the buffer columns), the bound leaves a
    # factor 15
    for ik in (0, 13):
        x = xs[ik].reshape(xs[ik].shape[0], -1)
        g = (x.conj() @ x.T).cpu().numpy()
        assert np.abs(g - np.eye(g.shape[0])).max() < 1e-8
    # residuals of sampled columns with the oracle's operator
    for ik in (0, 13):
        m, q = obasis.sphere(wl.lattice, wl.grid, wl.kfrac[ik], wl.ecut_k[ik])
        hop = oop.MatrixFreeH(wl, m, q)
        cols = [0, nev_k[ik] // 2, nev_k[ik] - 1]
        x = xs[ik][cols].cpu().numpy()
        r = hop(x) - lam[ik][cols][:, None, None] * x
        assert np.linalg.norm(r.reshape(len(cols), -1), axis=1).max() < 1.5e-6
