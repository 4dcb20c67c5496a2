"""GPU parity of the block linear algebra of Algorithm 1: Gram matrices, the FP64 Rayleigh-Ritz
solve (Cholesky and SVQB branches), rotations and residual norms, against numpy / the oracle."""
import numpy as np
import pytest

from oracle import lobpcgf as olb

from ._helpers import gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("rows,nz", [(4 * 287, 18), (4 * 57419, 96), (1000, 33), (4 * 5, 1)])
def test_gram_fp64(rows, nz):
    torch = gpu()
    import paper_1211_1446_gb300 as P
    z = _rand((nz, rows), 1)
    hz = _rand((nz, rows), 2)
    a = torch.empty((nz, nz), dtype=torch.complex128, device="cuda")
    s = torch.empty_like(a)
    P.gram(to_dev(z, torch.complex128), to_dev(hz, torch.complex128), a, s)
    torch.cuda.synchronize()
    a_ref = z.conj() @ hz.T          # (Z^H HZ)[i,j] with columns as rows of z
    s_ref = z.conj() @ z.T
    # library matrices are column-major: tensor[j, i] = M[i, j]
    assert rel_err(a.cpu().numpy().T, a_ref) < 1e-13
    assert rel_err(s.cpu().numpy().T, s_ref) < 1e-13


def test_gram_fp32():
    torch = gpu()
    import paper_1211_1446_gb300 as P
    z = _rand((40, 4 * 3000), 3)
    a = torch.empty((40, 40), dtype=torch.complex128, device="cuda")
    s = torch.empty_like(a)
    zd = to_dev(z, torch.complex64)
    P.gram(zd, zd, a, s)
    torch.cuda.synchronize()
    z32 = z.astype(np.complex64).astype(np.complex128)
    assert rel_err(s.cpu().numpy().T, z32.conj() @ z32.T) < 1e-5


def _pencil(nz, seed, rank_def=False, degenerate=False):
    rng = np.random.default_rng(seed)
    nn = 4 * nz + 40
    zz = rng.standard_normal((nn, nz)) + 1j * rng.standard_normal((nn, nz))
    zz *= rng.uniform(0.1, 10.0, nz)[None, :]          # badly scaled columns
    if rank_def:
        zz[:, nz - 1] = 2.0 * zz[:, 1] - 0.5j * zz[:, 3]
    if degenerate:
        # pencil with exactly repeated generalized eigenvalues: A = Z^H W Z, S = Z^H Z (Z square)
        zq = zz[:nz]
        w = np.repeat(np.arange((nz + 1) // 2, dtype=float), 2)[:nz] - 3.0
        return zq.conj().T @ (w[:, None] * zq), zq.conj().T @ zq
    hm = rng.standard_normal((nn, nn)) + 1j * rng.standard_normal((nn, nn))
    hm = hm + hm.conj().T
    return zz.conj().T @ hm @ zz, zz.conj().T @ zz


@pytest.mark.parametrize("nz,n,kind", [(96, 32, "plain"), (40, 12, "rankdef"), (24, 24, "plain"),
                                       (60, 20, "degenerate"), (1, 1, "plain"), (200, 64, "plain"),
                                       (37, 9, "plain"), (2, 1, "plain"), (3, 2, "degenerate"),
                                       (301, 100, "plain")])
def test_rayleigh_ritz(nz, n, kind):
    torch = gpu()
    import paper_1211_1446_gb300 as P
    a, s = _pencil(nz, 10 + nz, rank_def=(kind == "rankdef"), degenerate=(kind == "degenerate"))
    lam_ref, v_ref, info_ref = olb.rayleigh_ritz(a, s, n)
    ad = to_dev(a.T.copy(), torch.complex128)            # column-major upload
    sd = to_dev(s.T.copy(), torch.complex128)
    v = torch.empty((n, nz), dtype=torch.complex128, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    P.rayleigh_ritz(ad, sd, n, v, lam, info)
    torch.cuda.synchronize()
    lam_g = lam.cpu().numpy()
    vg = v.cpu().numpy().T
    inf = info.cpu().numpy()
    assert bool(inf[0]) == info_ref.svqb and inf[1] == info_ref.rank and inf[2] == 0
    scale = max(1.0, np.abs(lam_ref).max())
    assert np.abs(lam_g - lam_ref).max() < 1e-9 * scale
    # S-orthonormal Ritz vectors that satisfy the pencil
    assert np.abs(vg.conj().T @ s @ vg - np.eye(n)).max() < 1e-8
    assert np.abs(a @ vg - (s @ vg) * lam_g[None, :]).max() < 1e-7 * scale * np.abs(s).max()


def test_rotate_and_residual_norms():
    torch = gpu()
    import paper_1211_1446_gb300 as P
    rows, nz, n = 4 * 1234, 50, 17
    z = _rand((nz, rows), 4)
    w = _rand((nz, n), 5)
    out = torch.empty((n, rows), dtype=torch.complex128, device="cuda")
    P.rotate(to_dev(z, torch.complex128), to_dev(w.T.copy(), torch.complex128), n, out)
    torch.cuda.synchronize()
    ref = (z.T @ w).T
    assert rel_err(out.cpu().numpy(), ref) < 1e-13
    x = _rand((n, rows), 6)
    hx = _rand((n, rows), 7)
    lam = np.linspace(-3, 3, n)
    nr = torch.empty(n, dtype=torch.float64, device="cuda")
    P.residual_norms(to_dev(x, torch.complex128), to_dev(hx, torch.complex128), to_dev(lam, torch.float64), nr)
    torch.cuda.synchronize()
    ref = np.linalg.norm(hx - lam[:, None] * x, axis=1)
    assert rel_err(nr.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("rows,nz", [(4 * 57419, 120), (1000, 33), (4 * 5, 1)])
def test_gram_double_float(rows, nz):
    """Double-float (FP32-pair) Gram on complex128 data: FP64-level accuracy (2^-48 per step)."""
    torch = gpu()
    import paper_1211_1446_gb300 as P
    z = _rand((nz, rows), 11)
    hz = _rand((nz, rows), 12)
    a = torch.empty((nz, nz), dtype=torch.complex128, device="cuda")
    s = torch.empty_like(a)
    P.gram(to_dev(z, torch.complex128), to_dev(hz, torch.complex128), a, s, emulated=True)
    torch.cuda.synchronize()
    assert rel_err(a.cpu().numpy().T, z.conj() @ hz.T) < 1e-12
    assert rel_err(s.cpu().numpy().T, z.conj() @ z.T) < 1e-12


@pytest.mark.parametrize("prec,rows,nz", [("fp32", 4 * 3001, 120), ("fp32", 1000, 33), ("fp32", 4 * 5, 1),
                                           ("fp32", 4 * 57419, 120), ("df", 4 * 3001, 120), ("df", 1000, 33),
                                           ("df", 4 * 5, 1), ("df", 4 * 57419, 97), ("fp64", 1000, 33),
                                           ("fp64", 4 * 3001, 120)])
def test_gram_hermitian(prec, rows, nz):
    """The solver's fused Gram (Algorithm 1's projected pencil): block lower triangles of A = Z^H HZ and
    S = Z^H Z in one pass, strict upper triangles the exact conjugate mirror of the lower ones."""
    torch = gpu()
    import paper_1211_1446_gb300 as P
    z = _rand((nz, rows), 21)
    hz = _rand((nz, rows), 22)
    if prec == "fp32":
        z, hz = (v.astype(np.complex64).astype(np.complex128) for v in (z, hz))
        dt, tol = torch.complex64, 1e-5
    else:
        dt, tol = torch.complex128, 1e-12
    a = torch.empty((nz, nz), dtype=torch.complex128, device="cuda")
    s = torch.empty_like(a)
    P.gram_hermitian(to_dev(z, dt), to_dev(hz, dt), a, s, emulated=(prec == "df"))
    torch.cuda.synchronize()
    low = np.tril(np.ones((nz, nz), dtype=bool))
    for got_t, ref in ((a, z.conj() @ hz.T), (s, z.conj() @ z.T)):
        got = got_t.cpu().numpy().T
        assert rel_err(np.where(low, got, 0), np.where(low, ref, 0)) < tol
        assert np.array_equal(got[~low], got.conj().T[~low])


def test_rotate_double_float():
    torch = gpu()
    import paper_1211_1446_gb300 as P
    rows, nz, n = 4 * 3001, 120, 40
    z = _rand((nz, rows), 13)
    w = _rand((nz, n), 14)
    out = torch.empty((n, rows), dtype=torch.complex128, device="cuda")
    P.rotate(to_dev(z, torch.complex128), to_dev(w.T.copy(), torch.complex128), n, out, emulated=True)
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), (z.T @ w).T) < 1e-13
