"""GPU eigenvectors against the dense oracle, compared per cluster of degenerate eigenvalues as
subspaces (largest principal-angle sine, the parity measure for vectors: inside a Kramers pair
or a degenerate cluster any orthonormal basis is correct).  At residual tol the sines are of
order tol / gap; the small cell's lowest clusters are at least 0.11 Ha apart, so 1e-4 leaves a wide
margin."""
import numpy as np
import pytest

import workloads as W
from oracle import lobpcgf as olb, operator as oop

from ._helpers import cluster_sines, gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1])
def test_eigenvectors_match_dense_subspaces(mode):
    torch = gpu()
    import paper_1211_1446_gb300 as P
    import oracle.basis as ob
    wl = W.make("small")
    ctx = P.Context.from_workload(wl)
    nev, nbuf = 8, 2
    m, q = ob.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    x = torch.from_numpy(W.start_block(ctx.npw(0), nev + nbuf, wl.seed)).cuda()
    lam, rep, rc = ctx.solve([x], nev, nbuf=nbuf, tol=1e-6, mode=mode, check=False)
    assert rc == 0, rep["message"]
    h = oop.dense_hamiltonian(wl, m, q)
    ref, u, _ = olb.dense_eigs(h, wl.c, nev)
    assert np.abs(lam[0] - ref).max() < 1e-8
    xv = x[:nev].reshape(nev, -1).cpu().numpy().T
    assert np.abs(xv.conj().T @ xv - np.eye(nev)).max() < 1e-8
    assert cluster_sines(ref, u, xv) < 1e-4
