"""GPU parity of the operator steps (H' application, filter, preconditioner) against the CPU oracle.

Tolerances: FP64 blocks agree with the FP64 oracle to a relative max-norm error of
1e-11 (FFT rounding grows like log Ng * eps times the largest operator entry
2c^2); FP32 blocks to 2e-6 relative, with the Dirac 4x4 term evaluated in FP64.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operator as oop

from ._helpers import gpu, make_pair, rel_err, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    ("cubic", {}),                                        # local potential only, 12^3 grid
    ("small", {}),                                        # projectors + local, odd grid axes 15
    ("small", {"kfrac": [[0.25, -0.125, 0.5]]}),          # general k
    ("dimer", {"ecut": 4.0}),                             # full 48x48x56 grid, reduced sphere
    ("cubic", {"potential": False}),                      # free Dirac term alone
    ("small", {"grid": (20, 21, 14)}),                    # radices 5x4, 7x3, 7x2; odd plane row length
    ("cubic", {"grid": (16, 12, 27)}),                    # radices 8x2, 6x2, 3x3x3
]


@pytest.mark.parametrize("name,kw", CASES)
@pytest.mark.parametrize("nb", [1, 5])
def test_apply_h_fp64(name, kw, nb):
    torch = gpu()
    wl, ctx, hop, q = make_pair(name, **kw)
    x = W.random_block(len(q), nb, 100 + nb)
    ref = hop(x)
    xd = to_dev(x, torch.complex128)
    hx = torch.empty_like(xd)
    ctx.apply_H(0, xd, hx)
    torch.cuda.synchronize()
    assert rel_err(hx.cpu().numpy(), ref) < 1e-11


@pytest.mark.parametrize("name,kw", CASES[:4])
def test_apply_h_fp32(name, kw):
    torch = gpu()
    wl, ctx, hop, q = make_pair(name, **kw)
    x = W.random_block(len(q), 3, 7)
    ref = hop(x)
    xd = to_dev(x, torch.complex64)
    hx = torch.empty_like(xd)
    ctx.apply_H(0, xd, hx)
    torch.cuda.synchronize()
    assert rel_err(hx.cpu().numpy(), ref) < 2e-6


def _dirac_abs(hop, x):
    """Sum of the magnitudes of the products that make up each element of the free Dirac term
    (an upper bound on what an FP32 evaluation of that term can lose to rounding, cancellation
    between the products included)."""
    c, q = hop.wl.c, hop.q
    qz, qp = np.abs(q[:, 2]), np.hypot(q[:, 0], q[:, 1])
    a = np.abs(x)
    d = np.empty(x.shape, dtype=np.float64)
    d[:, 0] = c * (qz * a[:, 2] + qp * a[:, 3])
    d[:, 1] = c * (qp * a[:, 2] + qz * a[:, 3])
    d[:, 2] = c * (qz * a[:, 0] + qp * a[:, 1]) + 2.0 * c * c * a[:, 2]
    d[:, 3] = c * (qp * a[:, 0] + qz * a[:, 1]) + 2.0 * c * c * a[:, 3]
    return d


def _per_term_excess(hx, hop, x):
    """Error of an FP32 H'x in the potential terms alone.  The oracle's FP64 Dirac part is taken
    off the GPU output and the rest is compared with the oracle's local + nonlocal terms T, after
    each element is allowed the FP32 rounding of the Dirac products that form it and of its own
    stored value (2^-22 times the sum of their magnitudes).  Returned as (normwise error over
    ||T||_2, largest element error over max |T|)."""
    d = hop.dirac(x)
    t = hop(x) - d
    full = d + t
    allow = 2.0 ** -22 * (_dirac_abs(hop, x) + np.abs(full))
    excess = np.maximum(np.abs(hx - full) - allow, 0.0)
    return float(np.linalg.norm(excess) / np.linalg.norm(t)), float(excess.max() / np.abs(t).max())


@pytest.mark.parametrize("name,kw", [("small", {}), ("dimer", {"ecut": 4.0}), ("dimer", {}),
                                     ("dimer", {"projectors": False}), ("dimer", {"potential": False}),
                                     ("small", {"c": 1.0})])
def test_apply_h_fp32_per_term(name, kw):
    """FP32 H' per term: the local-potential and spin-orbit contributions are held to their own
    magnitude, not to the 2c^2 Dirac entries that dominate the output: normwise error below
    1e-5 of ||T||_2 and no element off by more than 5e-5 of max |T| (the FP32 FFT round trip of
    the local term loses a few units of 2^-24 per radix pass; its largest-element error is the
    larger of the two).  c = 1 makes the Dirac term small, so there the whole output is held to
    1e-5 as well."""
    torch = gpu()
    wl, ctx, hop, q = make_pair(name, **kw)
    x = W.random_block(len(q), 3, 17).astype(np.complex64).astype(np.complex128)
    xd = to_dev(x, torch.complex64)
    hx = torch.empty_like(xd)
    ctx.apply_H(0, xd, hx)
    torch.cuda.synchronize()
    out = hx.cpu().numpy().astype(np.complex128)
    e_norm, e_max = _per_term_excess(out, hop, x)
    print(f"per-term excess {name} {kw}: normwise {e_norm:.3e} max {e_max:.3e}")
    assert e_norm < 1e-5 and e_max < 5e-5, (e_norm, e_max)
    if kw.get("c") == 1.0:
        assert rel_err(out, hop(x)) < 1e-5


def test_apply_h_full_dimer():
    """Full-size dimer (npw 57419, 48x48x56 grid, 36 projector channels), every output element."""
    torch = gpu()
    wl, ctx, hop, q = make_pair("dimer")
    assert ctx.nproj() == 36
    x = W.random_block(len(q), 3, 5)
    ref = hop(x)
    for dt, tol in ((torch.complex128, 1e-11), (torch.complex64, 2e-6)):
        xd = to_dev(x, dt)
        hx = torch.empty_like(xd)
        ctx.apply_H(0, xd, hx)
        torch.cuda.synchronize()
        assert rel_err(hx.cpu().numpy(), ref) < tol


@pytest.mark.parametrize("name,kw", [("dimer", {"ecut": 4.0}), CASES[5], CASES[6]])
def test_apply_h_double_float(name, kw):
    """complex128 H' with the FFTs and projector contractions in double-float arithmetic."""
    torch = gpu()
    wl, ctx, hop, q = make_pair(name, **kw)
    x = W.random_block(len(q), 5, 31)
    ref = hop(x)
    xd = to_dev(x, torch.complex128)
    hx = torch.empty_like(xd)
    ctx.apply_H(0, xd, hx, emulated=True)
    torch.cuda.synchronize()
    assert rel_err(hx.cpu().numpy(), ref) < 1e-11


def test_filter_parity():
    torch = gpu()
    wl, ctx, hop, q = make_pair("small")
    cs, om = ctx.filter_constants(0)
    cs_o, om_o = oop.filter_constants(wl, q)
    assert abs(cs - cs_o) < 1e-9 * abs(cs_o) and abs(om - om_o) < 1e-9 * abs(om_o)
    y = W.random_block(len(q), 4, 3)
    ref = oop.apply_filter(hop, y, cs, om)
    yd = to_dev(y, torch.complex128)
    fy = torch.empty_like(yd)
    ctx.filter(0, yd, fy, cs, om)
    torch.cuda.synchronize()
    assert rel_err(fy.cpu().numpy(), ref) < 1e-11


@pytest.mark.parametrize("precond", [0, 1])
def test_precond_parity(precond):
    torch = gpu()
    wl, ctx, hop, q = make_pair("small")
    npw = len(q)
    x = W.random_block(npw, 5, 21)
    hx = W.random_block(npw, 5, 22)
    lam = np.array([-1.0, 0.5, 2.0, 3.0, 7.5])
    act = np.array([4, 1, 2], dtype=np.int32)
    r = hx[act] - lam[act][:, None, None] * x[act]
    ref = oop.teter_precondition(q, x[act], r) if precond == 0 else r
    y = torch.empty((3, 4, npw), dtype=torch.complex128, device="cuda")
    ctx.precond(0, to_dev(x, torch.complex128), to_dev(hx, torch.complex128), to_dev(lam, torch.float64),
                to_dev(act, torch.int32), y, precond=precond)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy(), ref) < 1e-13


def test_zero_columns_is_noop():
    torch = gpu()
    wl, ctx, hop, q = make_pair("small")
    x = torch.zeros((0, 4, len(q)), dtype=torch.complex128, device="cuda")
    ctx.apply_H(0, x, torch.empty_like(x))


def test_invalid_arguments_are_reported():
    torch = gpu()
    import paper_1211_1446_gb300 as P
    wl, ctx, hop, q = make_pair("small")
    x = torch.zeros((1, 4, len(q)), dtype=torch.complex128, device="cuda")
    with pytest.raises(P.DKSError) as e:
        ctx.apply_H(3, x, torch.empty_like(x))
    assert e.value.code == -1
    with pytest.raises(P.DKSError) as e:
        P.Context.from_workload(W.make("dimer", grid=(40, 48, 56)))
    assert e.value.code == -8
    with pytest.raises(P.DKSError) as e:
        P.Context.from_workload(W.make("cubic", grid=(11, 12, 12)))   # prime 11 is not a supported radix
    assert e.value.code == -9


@pytest.mark.parametrize("name,kw", [CASES[0], CASES[2], CASES[3], ("dimer", {})])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_kinetic_balance(name, kw, dt):
    """Eq. (RKB): small two-spinors from the large ones, every element against the oracle; the
    large two-spinors are left bit-identical."""
    torch = gpu()
    wl, ctx, hop, q = make_pair(name, **kw)
    x = W.random_block(len(q), 3, 31)
    if dt == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    ref = oop.kinetic_balance(q, x, wl.c)
    xd = to_dev(x, torch.complex128 if dt == "c128" else torch.complex64)
    ctx.kinetic_balance(0, xd)
    torch.cuda.synchronize()
    got = xd.cpu().numpy().astype(np.complex128)
    assert np.array_equal(got[:, 0:2], x[:, 0:2])
    assert rel_err(got[:, 2:4], ref[:, 2:4]) < (1e-14 if dt == "c128" else 1e-6)


@pytest.mark.parametrize("name,kw", CASES)
@pytest.mark.parametrize("dt", ["c128", "c64", "df"])
def test_apply_h_ksso(name, kw, dt):
    """The KSSO two-component operator (kinetic + V + spin-orbit projectors) against the oracle's
    matrix-free KSSO operator, every element; complex128 in FP64 and in double-float arithmetic,
    complex64 in FP32."""
    torch = gpu()
    wl, ctx, hop, q = make_pair(name, model="ksso", **kw)
    assert ctx.ncomp == 2
    x = W.random_block(len(q), 3, 41, ncomp=2)
    if dt == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    ref = hop(x)
    xd = to_dev(x, torch.complex64 if dt == "c64" else torch.complex128)
    hx = torch.empty_like(xd)
    ctx.apply_H(0, xd, hx, emulated=(dt == "df"))
    torch.cuda.synchronize()
    assert rel_err(hx.cpu().numpy(), ref) < (2e-6 if dt == "c64" else 1e-12)


def test_kinetic_balance_rejects_ksso():
    torch = gpu()
    import paper_1211_1446_gb300 as P
    wl, ctx, hop, q = make_pair("cubic", model="ksso")
    xd = to_dev(W.random_block(len(q), 2, 3, ncomp=2), torch.complex128)
    with pytest.raises(P.DKSError):
        ctx.kinetic_balance(0, xd)


@pytest.mark.parametrize("dt", ["c64", "df"])
def test_apply_h_ksso_full_dimer(dt):
    """KSSO operator at the bench size (npw 57419, 48x48x56 grid, 36 projector channels), every
    output element against the oracle."""
    torch = gpu()
    wl, ctx, hop, q = make_pair("dimer", model="ksso")
    x = W.random_block(len(q), 3, 43, ncomp=2)
    if dt == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    ref = hop(x)
    xd = to_dev(x, torch.complex64 if dt == "c64" else torch.complex128)
    hx = torch.empty_like(xd)
    ctx.apply_H(0, xd, hx, emulated=(dt == "df"))
    torch.cuda.synchronize()
    assert rel_err(hx.cpu().numpy(), ref) < (2e-6 if dt == "c64" else 1e-12)
