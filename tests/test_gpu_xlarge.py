"""GPU paths for problems beyond one CTA or one block, and the tuner that chooses between forms:
the split plane FFT (row and column kernels through an L2-resident plane buffer) for planes above
one CTA's shared memory, band blocks with deflation for more pairs than one Rayleigh-Ritz pencil
holds, and the launch-parameter tuner.  Each is checked against the oracle, and the alternative
forms against each other (they run the same line transforms).
"""
import numpy as np
import pytest

import workloads as W
from oracle import lobpcgf as olb, operator as oop, scf as oscf

from ._helpers import gpu, make_pair, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _unit_block(nb, nc, npw, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nb, nc, npw)) + 1j * rng.standard_normal((nb, nc, npw))
    return x / np.linalg.norm(x.reshape(nb, -1), axis=1)[:, None, None]


@pytest.mark.parametrize("name,kw,nb", [("small", dict(ecut=4.0), 5), ("dimer", dict(), 32)])
def test_density_split_plane_matches_oracle(name, kw, nb):
    """The density with the plane transforms forced into the split form."""
    torch = gpu()
    wl, ctx, hop, q = make_pair(name, **kw)
    ctx.set_tuning(64 << 20, 0, 1)
    m = ctx.basis(0)
    x = _unit_block(nb, 4, len(m), 11)
    occ = np.linspace(1.0, 0.25, nb)
    rho = torch.zeros(wl.grid, dtype=torch.float64, device="cuda")
    ctx.density(0, to_dev(x, torch.complex128), occ, rho)
    assert rel_err(rho.cpu().numpy(), oscf.density(x, m, wl.grid, wl.volume, occ)) < 1e-11


def test_plane_too_large_for_one_cta():
    """A 120 x 120 plane of complex128 (232 KB) exceeds one CTA's shared memory: H' runs the split
    plane FFT in FP64 and double-float and the one-kernel form in FP32 (116 KB), the density the
    split form; all against the oracle."""
    torch = gpu()
    from oracle import scf as oscf
    wl, ctx, hop, q = make_pair("cubic", ecut=4.0, grid=(120, 120, 10))
    npw = ctx.npw(0)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((3, 4, npw)) + 1j * rng.standard_normal((3, 4, npw))
    want = hop(x)
    for dt, emu, tol in ((torch.complex128, False, 1e-11), (torch.complex128, True, 1e-11), (torch.complex64, False, 2e-6)):
        xd = to_dev(x, dt)
        hx = torch.empty_like(xd)
        ctx.apply_H(0, xd, hx, emulated=emu)
        assert rel_err(hx.cpu().numpy(), want) < tol, (dt, emu)
    xn = x / np.linalg.norm(x.reshape(3, -1), axis=1)[:, None, None]
    rho = torch.zeros(wl.grid, dtype=torch.float64, device="cuda")
    ctx.density(0, to_dev(xn, torch.complex128), [1.0, 0.5, 0.25], rho)
    dens = oscf.density(xn, ctx.basis(0), wl.grid, wl.volume, [1.0, 0.5, 0.25])
    assert rel_err(rho.cpu().numpy(), dens) < 1e-11


def test_autotune_changes_time_not_results(tmp_path):
    """dks_autotune times its candidates (4 chunk budgets x {one-kernel plane FFT with 4 CTA sizes,
    split plane FFT}) and then the projector contraction schedule (tensor cores or CUDA cores)
    at the chosen FFT parameters, keeps the fastest, and H' x is the same under every choice
    (every line transform is the same butterfly arithmetic, whichever kernel and thread runs it;
    the two contraction schedules agree to the FP32 bar); the JSON cache returns the stored
    choice."""
    torch = gpu()
    import paper_1211_1446_gb300 as P
    wl, ctx, hop, q = make_pair("dimer", ecut=4.0)
    npw = ctx.npw(0)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((6, 4, npw)) + 1j * rng.standard_normal((6, 4, npw))
    want = hop(x)
    cache = str(tmp_path / "tune.json")
    r = ctx.autotune(0, nb=8, prec=P.PREC_FP32, cache=cache)
    assert not r["cached"] and len(r["candidates"]) == 20
    assert all(c["ms"] > 0 for c in r["candidates"])
    # the projector contraction schedule (tensor cores or CUDA cores) is tuned as well
    assert r["proj_tc"] in (0, 1) and all(v > 0 for v in r["proj_ms"])
    assert ctx.tuning() == dict(chunk_bytes=r["chunk_bytes"], plane_threads=r["plane_threads"],
                                plane_split=r["plane_split"], proj_tc=r["proj_tc"])
    x32 = to_dev(x, torch.complex64)
    h32 = []
    for ptc in (0, 1):
        ctx.set_tuning(r["chunk_bytes"], r["plane_threads"], r["plane_split"], proj_tc=ptc)
        hx = torch.empty_like(x32)
        ctx.apply_H(0, x32, hx)
        h32.append(hx.cpu().numpy().astype(np.complex128))
    assert rel_err(h32[1], h32[0]) < 2e-6 and rel_err(h32[0], want) < 2e-6
    xd = to_dev(x, torch.complex128)
    for emulated in (False, True):
        outs = []
        for chunk, thr, split in [(r["chunk_bytes"], r["plane_threads"], r["plane_split"]), (16 << 20, 128, 0),
                                  (128 << 20, 512, 0), (64 << 20, 0, 1), (16 << 20, 0, 1)]:
            ctx.set_tuning(chunk, thr, split)
            hx = torch.empty_like(xd)
            ctx.apply_H(0, xd, hx, emulated=emulated)
            outs.append(hx.cpu().numpy())
        assert rel_err(outs[0], want) < 1e-11
        for o in outs[1:]:
            assert rel_err(o, outs[0]) < 1e-14                 # the same line transforms
    r2 = ctx.autotune(0, nb=8, prec=P.PREC_FP32, cache=cache)
    assert r2["cached"] and all(r2[k] == r[k] for k in ("chunk_bytes", "plane_threads", "plane_split", "proj_tc"))
    assert ctx.tuning()["proj_tc"] == r["proj_tc"]


@pytest.mark.parametrize("mode", [0, 1])
def test_band_blocks_with_deflation(mode):
    """20 pairs in band blocks of 8 wanted + 4 buffer columns (FP64 and mixed precision): the
    eigenvalues are the dense ones, the locked vectors orthonormal and eigenvectors of H'."""
    torch = gpu()
    import paper_1211_1446_gb300 as P
    import oracle.basis as ob
    wl = W.make("small", ecut=4.0)
    ctx = P.Context.from_workload(wl)
    n, blk, nbuf = 20, 8, 4
    m, q = ob.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    x = torch.from_numpy(W.start_block(ctx.npw(0), n + nbuf, wl.seed)).cuda()
    lam, rep, rc = ctx.solve([x], n, nbuf=nbuf, tol=1e-7, mode=mode, block=blk, check=False)
    assert rc == 0, rep["message"]
    h = oop.dense_hamiltonian(wl, m, q)
    ref, _, _ = olb.dense_eigs(h, wl.c, n)
    assert np.abs(lam[0] - ref).max() < 1e-8
    xv = x[:n].reshape(n, -1).cpu().numpy().T
    assert np.abs(xv.conj().T @ xv - np.eye(n)).max() < 1e-8
    assert np.abs(h @ xv - xv * lam[0][None, :]).max() < 1e-6
