"""The complex128 contractions of the double-float refinement phase on the tcgen05 tensor cores,
through exact integer slices (DKS_TC_FP64): per 128-row window and column every value is
rounded to 56 fractional bits of the window's power of two and cut into seven 8-bit digits; the
28 digit products of levels 0..6 accumulate exactly (levels 0..3) or in one FP32 accumulator
(levels 4..6).

Bars: (1) integer-valued inputs give the exact products (every digit product and partial sum
is an exact integer), bit for bit; (2) random inputs with a wide dynamic range (columns scaled
over 10 decades, rows decaying like planewave coefficients) stay within 1e-13 of numpy's FP64
Gram matrices relative to sum_k |a_k| |b_k| of each entry, and rotations within 1e-13 relative
to sum_c m_c |w_c| with m_c the maximum of column c of Z over the 128-row window of the output
row -- the representation keeps 2^-57 of the window maximum per value (an entry far below its
window's maximum has fewer digits of its own), and the FP32 accumulator shared by levels 4..6
takes up to 2^-45 of the leading level over a rotation's 288 accumulation steps if every step
truncates (measured 1e-15 to 3.3e-14 in this measure; the double-float kernel is printed
beside it); (3) the same
call twice gives bitwise equal results (fixed reduction order); (4) solves with the refinement
phase on this path reach the dense eigenvalues within 1e-8 Ha.
"""
import numpy as np
import pytest

import workloads as W
from oracle import basis as ob
from oracle import lobpcgf as olb
from oracle import operator as oop

from ._helpers import gpu, make_pair, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture
def slices():
    gpu()
    import paper_1211_1446_gb300 as P
    old = P.tensor_cores()
    P.tensor_cores(old[0] | P.TC_FP64)
    yield P
    P.tensor_cores(old[0], old[1])


def _ranged(rng, nz, rows, decades=10.0):
    """nz columns of rows entries: column scales 10^[-decades+2, 2], entries decaying along the
    rows (as planewave coefficients do with |G|), a few exact zeros."""
    z = rng.standard_normal((nz, rows)) + 1j * rng.standard_normal((nz, rows))
    z *= 10.0 ** rng.uniform(2.0 - decades, 2.0, size=(nz, 1))
    z *= np.exp(-np.arange(rows) / (0.3 * rows))[None, :]
    z[:, ::97] = 0.0
    return z


def _scaled(got, want, scale):
    return float(np.max(np.abs(got - want) / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("rows,nz", [(2000, 40), (4 * 517 + 3, 120), (300, 1), (5000, 200), (1500, 300)])
def test_gram_integer_inputs_are_exact(slices, rows, nz):
    """Gaussian-integer inputs: A = Z^H HZ and S = Z^H Z equal the exact integer products."""
    import torch
    P = slices
    rng = np.random.default_rng(rows + nz)
    z = rng.integers(-100, 101, (nz, rows)) + 1j * rng.integers(-100, 101, (nz, rows))
    hz = rng.integers(-1000, 1001, (nz, rows)) + 1j * rng.integers(-1000, 1001, (nz, rows))
    a = torch.empty((nz, nz), dtype=torch.complex128, device="cuda")
    s = torch.empty_like(a)
    P.gram_hermitian(to_dev(z, torch.complex128), to_dev(hz, torch.complex128), a, s, emulated=True)
    torch.cuda.synchronize()
    got_a, got_s = a.cpu().numpy().T, s.cpu().numpy().T
    want_a, want_s = z.conj() @ hz.T, z.conj() @ z.T
    lo = np.tril(np.ones((nz, nz), dtype=bool))
    assert np.array_equal(got_a[lo], want_a[lo])
    assert np.array_equal(got_s[lo], want_s[lo])
    up = np.triu(np.ones((nz, nz), dtype=bool), 1)
    assert np.array_equal(got_a[up], got_a.conj().T[up])


@pytest.mark.parametrize("rows,nz", [(4 * 2000, 120), (4 * 517 + 2, 40), (2 * 3001, 200), (4 * 700, 312), (64, 3)])
def test_gram_ranged_inputs(slices, rows, nz):
    """Wide dynamic range, ragged rows, one and several 128-column tiles: within 1e-13 of FP64
    relative to sum |a||b|, deterministic, and at least as accurate as the double-float kernel."""
    import torch
    P = slices
    rng = np.random.default_rng(7 * rows + nz)
    z = _ranged(rng, nz, rows)
    hz = _ranged(rng, nz, rows) * 50.0
    want_a, want_s = z.conj() @ hz.T, z.conj() @ z.T
    sc_a, sc_s = np.abs(z) @ np.abs(hz).T, np.abs(z) @ np.abs(z).T
    lo = np.tril(np.ones((nz, nz), dtype=bool))
    zd, hd = to_dev(z, torch.complex128), to_dev(hz, torch.complex128)
    res = {}
    for tag in ("slices", "again", "double-float"):
        if tag == "double-float":
            P.tensor_cores(P.tensor_cores()[0] & ~P.TC_FP64)
        a = torch.empty((nz, nz), dtype=torch.complex128, device="cuda")
        s = torch.empty_like(a)
        P.gram_hermitian(zd, hd, a, s, emulated=True)
        torch.cuda.synchronize()
        res[tag] = (a.cpu().numpy().T, s.cpu().numpy().T)
    ea = _scaled(res["slices"][0][lo], want_a[lo], sc_a[lo])
    es = _scaled(res["slices"][1][lo], want_s[lo], sc_s[lo])
    da = _scaled(res["double-float"][0][lo], want_a[lo], sc_a[lo])
    ds = _scaled(res["double-float"][1][lo], want_s[lo], sc_s[lo])
    print(f"gram rows {rows} nz {nz}: slices A {ea:.2e} S {es:.2e}; double-float A {da:.2e} S {ds:.2e}")
    assert ea < 1e-13 and es < 1e-13
    assert np.array_equal(res["slices"][0], res["again"][0]) and np.array_equal(res["slices"][1], res["again"][1])


@pytest.mark.parametrize("rows,nz,n,beta", [(4 * 1000, 120, 40, 0.0), (2 * 517 + 2, 37, 9, 0.0),
                                            (1234, 48, 100, 0.0), (3000, 120, 80, 1.0), (128, 1, 1, 0.0),
                                            (2 * 4113, 300, 40, 1.0), (777, 130, 48, 0.0)])
def test_rotate_ranged_inputs(slices, rows, nz, n, beta):
    """OUT = Z W (+ beta OUT): ragged rows, inner sizes off the 16-column chunk, more than 48
    output columns (several column tiles), more than 120 inner columns (several column windows,
    later ones added in FP64), and the accumulating form; error relative to the window maxima."""
    import torch
    P = slices
    rng = np.random.default_rng(rows + 3 * nz + n)
    z = _ranged(rng, nz, rows)
    w = rng.standard_normal((n, nz)) + 1j * rng.standard_normal((n, nz))    # columns of W
    w *= 10.0 ** rng.uniform(-6, 0, size=(n, 1))
    o0 = rng.standard_normal((n, rows)) + 1j * rng.standard_normal((n, rows))
    want = w @ z + beta * o0
    # window maxima of each column of Z, spread back over the rows of the window
    zmax = np.maximum(np.abs(z.real), np.abs(z.imag))
    pad = -rows % 128
    zwin = np.pad(zmax, ((0, 0), (0, pad))).reshape(nz, -1, 128).max(axis=2)
    zwin = np.repeat(zwin, 128, axis=1)[:, :rows]
    scale = np.abs(w) @ zwin + abs(beta) * np.abs(o0)
    zd, wd = to_dev(z, torch.complex128), to_dev(w, torch.complex128)
    outs = []
    for tag in ("slices", "again", "double-float"):
        if tag == "double-float":
            P.tensor_cores(P.tensor_cores()[0] & ~P.TC_FP64)
        out = to_dev(o0, torch.complex128)
        P.rotate(zd, wd, n, out, beta=beta, emulated=True)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    err = _scaled(outs[0], want, scale)
    dfe = _scaled(outs[2], want, scale)
    print(f"rotate rows {rows} nz {nz} n {n} beta {beta}: slices {err:.2e}, double-float {dfe:.2e}")
    assert err < 1e-13
    assert np.array_equal(outs[0], outs[1])


def test_rotate_integer_inputs_are_exact(slices):
    import torch
    P = slices
    rng = np.random.default_rng(5)
    rows, nz, n = 3001, 70, 33
    z = rng.integers(-100, 101, (nz, rows)) + 1j * rng.integers(-100, 101, (nz, rows))
    w = rng.integers(-50, 51, (n, nz)) + 1j * rng.integers(-50, 51, (n, nz))
    out = torch.zeros((n, rows), dtype=torch.complex128, device="cuda")
    P.rotate(to_dev(z, torch.complex128), to_dev(w, torch.complex128), n, out, emulated=True)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), w @ z)


def test_solves_with_refinement_on_slices(slices):
    """Mixed-mode solves whose FP64 phase forms its Gram matrices and rotations from the slices:
    dense eigenvalues within 1e-8 Ha (spin-orbit 'small' workload, cubic cell), also at a
    tolerance of 1e-9 that the refinement phase must reach on its own."""
    import torch
    P = slices
    for name, nev, tol in (("small", 6, 1e-6), ("cubic", 8, 1e-6), ("small", 6, 1e-9)):
        wl, ctx, hop, q = make_pair(name)
        m, _ = ob.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
        ref, _, _ = olb.dense_eigs(oop.dense_hamiltonian(wl, m, q), wl.c, nev)
        x0 = torch.from_numpy(W.start_block(len(q), nev + 2, wl.seed)).cuda()
        lam, rep, rc = ctx.solve([x0], nev, nbuf=2, mode=P.MODE_MIXED, tol=tol, check=False)
        assert rc == 0, (name, tol, rep["message"])
        assert rep["fp64_iterations"][0] > 0
        assert np.abs(lam[0] - ref).max() < 1e-8, (name, tol, np.abs(lam[0] - ref).max())


def test_dimer_full_size_refinement_on_slices(slices):
    """The bench configuration with the refinement phase's Gram matrices and rotations on the
    slices: eigenvalues within 1e-8 Ha of the oracle's Algorithm 1; prints both phases'
    iteration counts and the time."""
    import os
    import torch
    P = slices
    wl, ctx, hop, q = make_pair("dimer")
    ref = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "dimer_lobpcgf_eigs.txt"))
    x0 = torch.from_numpy(W.start_block(len(q), 40, wl.seed)).cuda()
    lam, rep, rc = ctx.solve([x0], 32, nbuf=8, tol=1e-6, mode=P.MODE_MIXED, check=False)
    print(f"dimer on slices: rc {rc} iterations {rep['iterations'][0]} FP64 {rep['fp64_iterations'][0]} "
          f"{rep['seconds'] * 1e3:.0f} ms max err {np.abs(lam[0] - ref).max():.2e}")
    assert rc == 0, rep["message"]
    assert np.abs(lam[0] - ref).max() < 1e-8


def test_non_finite_inputs_come_out_nan(slices):
    """A NaN or an infinity in a block gives NaN wherever it enters a product (its slices are
    BF16 NaNs, which the tensor cores propagate), so that the solver's finiteness checks still
    see it: Gram entries of the poisoned columns are NaN and the others exact-slice accurate; in
    a rotation the output row of a non-finite Z entry is NaN and every other output is finite."""
    import torch
    P = slices
    rng = np.random.default_rng(9)
    rows, nz, n = 1000, 12, 5
    z = rng.standard_normal((nz, rows)) + 1j * rng.standard_normal((nz, rows))
    hz = rng.standard_normal((nz, rows)) + 1j * rng.standard_normal((nz, rows))
    zb = z.copy()
    zb[3, 700] = np.nan
    zb[5, 10] = np.inf
    a = torch.empty((nz, nz), dtype=torch.complex128, device="cuda")
    s = torch.empty_like(a)
    P.gram_hermitian(to_dev(zb, torch.complex128), to_dev(hz, torch.complex128), a, s, emulated=True)
    torch.cuda.synchronize()
    ga, gs = a.cpu().numpy().T, s.cpu().numpy().T
    lo = np.tril(np.ones((nz, nz), dtype=bool))
    poisoned = np.isin(np.arange(nz), [3, 5])
    bad = poisoned[:, None] | poisoned[None, :]
    assert np.all(np.isnan(gs[lo & bad])) and np.all(np.isfinite(gs[lo & ~bad]))
    assert np.all(np.isnan(ga[lo & poisoned[:, None]])) and np.all(np.isfinite(ga[lo & ~poisoned[:, None]]))
    want_s = z.conj() @ z.T
    scale = np.abs(z) @ np.abs(z).T
    assert _scaled(gs[lo & ~bad], want_s[lo & ~bad], scale[lo & ~bad]) < 1e-13
    # rotation: NaN in Z row 700 of column 3
    w = rng.standard_normal((n, nz)) + 1j * rng.standard_normal((n, nz))   # columns of W
    zr = z.copy()
    zr[3, 700] = np.nan
    out = torch.zeros((n, rows), dtype=torch.complex128, device="cuda")
    P.rotate(to_dev(zr, torch.complex128), to_dev(w, torch.complex128), n, out, emulated=True)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(np.isnan(o[:, 700])) and np.all(np.isfinite(np.delete(o, 700, axis=1)))
