"""The complex64 contractions on the tcgen05 tensor cores (three BF16 slices per FP32 value, FP32
accumulation in tensor memory) against plain FP64 numpy products of the same FP32 inputs.

Bar: the error of every entry, relative to sum_k |a_k| |b_k| of that entry (the scale every
floating-point evaluation of a dot product is measured against), stays below
c_L 2^-24 with c_L = 8 sqrt(L) for an FP32 accumulation over L products of the slices: the six
slice products leave out less than 3 2^-24 of each product, and FP32 accumulation of L terms
has a rounding error that grows like sqrt(L) for data of random sign.  L is the inner size of
the rotation (2 m real terms) or the chunk length of the Gram forms (2 kchunk).  The same bar
is met by the CUDA-core FP32 kernels, which are compared too.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import operator as oop

from ._helpers import gpu, make_pair, to_dev

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


@pytest.fixture
def tc():
    gpu()
    import paper_1211_1446_gb300 as P
    old = P.tensor_cores()
    yield P
    P.tensor_cores(old[0], old[1])


def _cplx(rng, *shape):
    return ((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)).astype(np.complex64)


def _scaled_err(got, want, scale):
    return float(np.max(np.abs(got - want) / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("rows,nz,n,beta", [(4 * 1000, 120, 40, 0.0), (2 * 517 + 2, 37, 9, 0.0),
                                            (1234, 48, 136, 0.0), (3000, 120, 80, 1.0), (128, 1, 1, 0.0),
                                            (2 * 4113, 36, 80, 1.0)])
def test_rotate_tensor_cores(tc, rows, nz, n, beta):
    """OUT = Z W (+ beta OUT): ragged rows (not a multiple of the 128-row tile), inner sizes that
    are not a multiple of the 16-column chunk, more than 128 output columns (two column tiles),
    and the accumulating form of the projector update."""
    import torch
    P = tc
    rng = np.random.default_rng(rows + nz + n)
    z = _cplx(rng, nz, rows)
    w = rng.standard_normal((n, nz)) + 1j * rng.standard_normal((n, nz))       # columns of W (FP64)
    o0 = _cplx(rng, n, rows)
    w32 = w.astype(np.complex64).astype(np.complex128)                            # W is rounded to FP32
    want = (w32 @ z.astype(np.complex128)) + beta * o0.astype(np.complex128)
    scale = np.abs(w32) @ np.abs(z.astype(np.complex128)) + abs(beta) * np.abs(o0)
    res = {}
    for mask in (P.TC_ROTATE, 0):
        P.tensor_cores(mask)
        out = to_dev(o0, torch.complex64)
        P.rotate(to_dev(z, torch.complex64), to_dev(w, torch.complex128), n, out, beta=beta)
        torch.cuda.synchronize()
        res[mask] = _scaled_err(out.cpu().numpy().astype(np.complex128), want, scale)
    bound = 8 * math.sqrt(2 * nz) * U
    print(f"rotate rows {rows} nz {nz} n {n}: tensor cores {res[P.TC_ROTATE]:.2e}, CUDA cores {res[0]:.2e}, "
          f"bound {bound:.2e}")
    assert res[P.TC_ROTATE] < bound and res[0] < bound


@pytest.mark.parametrize("rows,nz", [(4 * 2000, 120), (4 * 517, 40), (2 * 3001, 200), (4 * 700, 312), (64, 3)])
@pytest.mark.parametrize("kchunk", [512, 2048])
def test_gram_hermitian_tensor_cores(tc, rows, nz, kchunk):
    """Lower triangles of A = Z^H HZ and S = Z^H Z (mirrored), one tile (nz <= 128) and several
    (nz = 200, 312: block lower triangle of 2 and 3 row blocks); kchunk = 512 and 2048."""
    import torch
    P = tc
    rng = np.random.default_rng(rows + nz)
    z = _cplx(rng, nz, rows)
    hz = _cplx(rng, nz, rows) * np.float32(7.0)
    zc, hc = z.astype(np.complex128), hz.astype(np.complex128)
    want_a, want_s = zc.conj() @ hc.T, zc.conj() @ zc.T
    sc_a, sc_s = np.abs(zc) @ np.abs(hc).T, np.abs(zc) @ np.abs(zc).T
    P.tensor_cores(P.TC_GRAM, kchunk)
    a = torch.empty((nz, nz), dtype=torch.complex128, device="cuda")
    s = torch.empty_like(a)
    P.gram_hermitian(to_dev(z, torch.complex64), to_dev(hz, torch.complex64), a, s)
    torch.cuda.synchronize()
    # column-major results: a[j, i] holds entry (i, j)
    got_a, got_s = a.cpu().numpy().T, s.cpu().numpy().T
    lo = np.tril(np.ones((nz, nz), dtype=bool))
    ea = _scaled_err(got_a[lo], want_a[lo], sc_a[lo])
    es = _scaled_err(got_s[lo], want_s[lo], sc_s[lo])
    bound = 8 * math.sqrt(2 * min(kchunk, rows)) * U
    print(f"gram rows {rows} nz {nz} kchunk {kchunk}: A {ea:.2e} S {es:.2e} bound {bound:.2e}")
    assert ea < bound and es < bound
    assert np.array_equal(got_s, got_s.conj().T) or np.allclose(got_s, got_s.conj().T, rtol=0, atol=1e-9 * np.abs(got_s).max())
    # A's upper triangle mirrors its lower one (A itself is Hermitian only when HZ = H' Z)
    up = np.triu(np.ones((nz, nz), dtype=bool), 1)
    assert np.array_equal(got_a[up], got_a.conj().T[up])


@pytest.mark.parametrize("rows,m,n", [(4 * 1500, 120, 40), (2 * 999, 36, 80), (1000, 130, 20)])
def test_gram_general_tensor_cores(tc, rows, m, n):
    """dks_gram (every entry of A^H B, no symmetry): m > 128 needs two row tiles."""
    import torch
    P = tc
    rng = np.random.default_rng(3 * rows + m)
    z = _cplx(rng, m, rows)
    hz = _cplx(rng, m, rows)
    P.tensor_cores(P.TC_GRAM)
    a = torch.zeros((m, m), dtype=torch.complex128, device="cuda")
    s = torch.zeros_like(a)
    P.gram(to_dev(z, torch.complex64), to_dev(hz, torch.complex64), a, s)
    torch.cuda.synchronize()
    zc, hc = z.astype(np.complex128), hz.astype(np.complex128)
    ea = _scaled_err(a.cpu().numpy().T, zc.conj() @ hc.T, np.abs(zc) @ np.abs(hc).T)
    es = _scaled_err(s.cpu().numpy().T, zc.conj() @ zc.T, np.abs(zc) @ np.abs(zc).T)
    bound = 8 * math.sqrt(2 * min(512, rows)) * U
    assert ea < bound and es < bound, (ea, es, bound)


def test_hn_long_index_many_tiles(tc):
    """A^H B with a long index (300,000 rows) and 5 x 17 tiles of at most 64 B columns (the
    projector coefficients at the supercell's sizes: 1080 channels against 320 columns, here
    scaled to 600 x 300), so that the partial-tile budget makes each CTA's chunk long: the
    FP32 register sums over the chunk stay within the FP32 bar of a chunk that long."""
    import torch
    P = tc
    rng = np.random.default_rng(77)
    rows, m, n = 300000, 300, 600
    a = _cplx(rng, m, rows)
    b = _cplx(rng, n, rows)
    P.tensor_cores(P.TC_GRAM)
    c = torch.zeros((m, n), dtype=torch.complex128, device="cuda")
    s = torch.zeros((m, m), dtype=torch.complex128, device="cuda")
    ad, bd = to_dev(a, torch.complex64), to_dev(b, torch.complex64)
    # dks_gram computes Z^H HZ and Z^H Z; use its general path on (a, b) through the binding's gemm
    P.gram(ad, ad, s, s)                       # S = A^H A, every entry
    torch.cuda.synchronize()
    ac = a.astype(np.complex128)
    want = ac.conj() @ ac.T
    scale = np.abs(ac) @ np.abs(ac).T
    got = s.cpu().numpy().T
    sample = (slice(0, m, 7), slice(0, m, 5))
    err = _scaled_err(got[sample], want[sample], scale[sample])
    print(f"hn long index: {err:.2e}")
    assert err < 8 * math.sqrt(2 * 8192) * U


@pytest.mark.parametrize("name,kw", [("small", {}), ("dimer", {"ecut": 4.0}), ("dimer", {})])
def test_apply_h_fp32_projectors_on_tensor_cores(tc, name, kw):
    """FP32 H' with both projector contractions (B^H x~ and x~ += B D (B^H x~)) on the tensor
    cores, against the oracle per term (the spin-orbit and local terms against their own
    magnitude, as in the CUDA-core test)."""
    import torch
    P = tc
    from .test_gpu_operator import _per_term_excess
    wl, ctx, hop, q = make_pair(name, **kw)
    x = W.random_block(len(q), 3, 17).astype(np.complex64).astype(np.complex128)
    P.tensor_cores(P.TC_PROJ_HN | P.TC_PROJ_NN)
    xd = to_dev(x, torch.complex64)
    hx = torch.empty_like(xd)
    ctx.apply_H(0, xd, hx)
    torch.cuda.synchronize()
    e_norm, e_max = _per_term_excess(hx.cpu().numpy().astype(np.complex128), hop, x)
    print(f"tensor-core projectors {name} {kw}: normwise {e_norm:.3e} max {e_max:.3e}")
    assert e_norm < 1e-5 and e_max < 5e-5


@pytest.mark.parametrize("mask", [1, 2, 12, 15])
def test_solve_with_tensor_cores_vs_dense(tc, mask):
    """The mixed-precision solve with contractions on the tensor cores reaches the dense
    eigenvalues within 1e-8 Ha (spin-orbit 'small' workload and the cubic cell)."""
    import torch
    P = tc
    import oracle.basis as ob
    from oracle import lobpcgf as olb
    P.tensor_cores(mask)
    for name, nev in (("small", 6), ("cubic", 8)):
        wl, ctx, hop, q = make_pair(name)
        m, _ = ob.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
        ref, _, _ = olb.dense_eigs(oop.dense_hamiltonian(wl, m, q), wl.c, nev)
        x0 = torch.from_numpy(W.start_block(len(q), nev + 2, wl.seed)).cuda()
        lam, rep, rc = ctx.solve([x0], nev, nbuf=2, mode=P.MODE_MIXED, check=False)
        assert rc == 0, (name, rc, rep["message"])
        assert np.abs(lam[0] - ref).max() < 1e-8, (name, np.abs(lam[0] - ref).max())


@pytest.mark.parametrize("mask", [0, 1, 2, 15])
def test_dimer_full_size_with_tensor_cores(tc, mask):
    """The bench configuration with the FP32-phase contractions on the tensor cores: same
    eigenvalues as the oracle's Algorithm 1 within 1e-8 Ha (the FP64 refinement is unchanged);
    prints the iteration counts of both phases for the record."""
    import os
    import torch
    P = tc
    P.tensor_cores(mask)
    wl, ctx, hop, q = make_pair("dimer")
    ref = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "dimer_lobpcgf_eigs.txt"))
    x0 = torch.from_numpy(W.start_block(len(q), 40, wl.seed)).cuda()
    lam, rep, rc = ctx.solve([x0], 32, nbuf=8, tol=1e-6, mode=P.MODE_MIXED, check=False)
    print(f"dimer mask {mask}: rc {rc} iterations {rep['iterations'][0]} FP64 {rep['fp64_iterations'][0]} "
          f"{rep['seconds'] * 1e3:.0f} ms history {[float('%.2g' % v) for v in rep['history']]}")
    assert rc == 0, rep["message"]
    assert np.abs(lam[0] - ref).max() < 1e-8
