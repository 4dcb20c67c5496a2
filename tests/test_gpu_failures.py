"""Failure detection without a GPU fault: every failure here is made on the host (a poisoned input
column, a tolerance that forces the fallback branch, a wait limit of zero polls), and each test
checks that the library answers with its status codes or its fallback path and that the same
context keeps working afterwards.  Nothing traps, faults or hangs the GPU.
"""
import numpy as np
import pytest

import workloads as W
from oracle import basis as ob
from oracle import lobpcgf as olb
from oracle import operator as oop

from ._helpers import gpu, make_pair, to_dev

pytestmark = pytest.mark.gpu


def _dense_ref(wl, q, nev):
    m, _ = ob.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    ref, _, _ = olb.dense_eigs(oop.dense_hamiltonian(wl, m, q), wl.c, nev)
    return ref


@pytest.mark.parametrize("mode", [0, 1])
def test_nan_start_column_is_refused_and_context_recovers(mode):
    """A start block with a NaN in one column: the solve returns INVALID_ARG naming that column
    before any other work (the block is left as it was), and the next solve on the same context
    with a clean block reaches the dense eigenvalues."""
    torch = gpu()
    import paper_1211_1446_gb300 as P
    wl, ctx, hop, q = make_pair("small")
    x = W.start_block(len(q), 8, wl.seed)
    x[3, 1, 17] = np.nan
    xd = torch.from_numpy(x.copy()).cuda()
    lam, rep, rc = ctx.solve([xd], 6, nbuf=2, mode=mode, check=False)
    assert rc == P.ERR_INVALID_ARG and "column 3" in rep["message"], (rc, rep["message"])
    back = xd.cpu().numpy()
    assert np.isnan(back[3, 1, 17]) and np.array_equal(np.delete(back, 3, axis=0), np.delete(x, 3, axis=0))
    xd = torch.from_numpy(W.start_block(len(q), 8, wl.seed)).cuda()
    lam, rep, rc = ctx.solve([xd], 6, nbuf=2, mode=mode, check=False)
    assert rc == 0, rep["message"]
    assert np.abs(lam[0] - _dense_ref(wl, q, 6)).max() < 1e-8


@pytest.mark.parametrize("mode", [0, 1])
def test_forced_svqb_gives_the_same_eigenpairs(mode):
    """A Cholesky tolerance no pivot can meet sends every Rayleigh-Ritz step to the SVQB branch
    of the single-CTA kernel (the route a failed factorisation takes); the solve still reaches
    the dense eigenvalues and matches the default route."""
    torch = gpu()
    wl, ctx, hop, q = make_pair("small")
    ref = _dense_ref(wl, q, 6)
    out = {}
    for chol in (None, 1e300):
        xd = torch.from_numpy(W.start_block(len(q), 8, wl.seed)).cuda()
        lam, rep, rc = ctx.solve([xd], 6, nbuf=2, mode=mode, chol_tol=chol, check=False)
        assert rc == 0, (chol, rep["message"])
        out[chol] = lam[0]
    assert np.abs(out[1e300] - ref).max() < 1e-8
    assert np.abs(out[1e300] - out[None]).max() < 1e-8


def test_rr_staging_wait_gives_up_and_single_cta_kernel_redoes_the_step():
    """With the first staging wait of the per-column Rayleigh-Ritz kernels limited to zero polls,
    every such wait gives up (the copy still lands: the draining wait keeps its limit), the
    kernels raise their flag and the single-CTA kernel redoes the step: the Ritz pairs equal the
    oracle's, the redo counter shows it ran, and restoring the limit brings back the cluster
    route (no further redos)."""
    torch = gpu()
    import paper_1211_1446_gb300 as P
    rng = np.random.default_rng(41)
    nz, n = 120, 40
    zz = rng.standard_normal((3 * nz, nz)) + 1j * rng.standard_normal((3 * nz, nz))
    hh = rng.standard_normal((3 * nz, 3 * nz)) + 1j * rng.standard_normal((3 * nz, 3 * nz))
    hh = hh + hh.conj().T
    a, s = zz.conj().T @ hh @ zz, zz.conj().T @ zz
    lam_ref, v_ref, _ = olb.rayleigh_ritz(a, s, n)

    def run():
        v = torch.empty((n, nz), dtype=torch.complex128, device="cuda")
        lam = torch.empty(n, dtype=torch.float64, device="cuda")
        info = torch.zeros(3, dtype=torch.int32, device="cuda")
        P.rayleigh_ritz(to_dev(a.T.copy(), torch.complex128), to_dev(s.T.copy(), torch.complex128), n, v, lam, info)
        torch.cuda.synchronize()
        return lam.cpu().numpy(), info.cpu().numpy()

    P.debug_rr_wait(1 << 24)                      # clear the counter
    try:
        P.debug_rr_wait(0)
        lam, info = run()
        redone = P.debug_rr_wait(0)
        assert redone >= 1
        scale = max(1.0, np.abs(lam_ref).max())
        assert np.abs(lam - lam_ref).max() < 1e-9 * scale and info[1] == nz and info[2] == 0
        # a whole solve on that route
        wl, ctx, hop, q = make_pair("cubic")
        xd = torch.from_numpy(W.start_block(len(q), 8, wl.seed)).cuda()
        lam_s, rep, rc = ctx.solve([xd], 8, mode=1, check=False)
        assert rc == 0, rep["message"]
        assert np.abs(lam_s[0] - _dense_ref(wl, q, 8)).max() < 1e-8
    finally:
        P.debug_rr_wait(1 << 24)
    lam, info = run()
    assert P.debug_rr_wait(1 << 24) == 0
    assert np.abs(lam - lam_ref).max() < 1e-9 * max(1.0, np.abs(lam_ref).max())
