"""The allocation-free Rayleigh-Ritz entry point against the allocating one.

dks_rayleigh_ritz_static serves callers that may not allocate device memory when they need the
solve (their device memory belongs to an arena fixed at start-up, or their thread must not risk
the synchronisation an allocation can cause).  It must give the same Ritz pairs as
dks_rayleigh_ritz.  This file is collected last so that a failure here leaves every other test
already run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from ._helpers import gpu, to_dev

pytestmark = pytest.mark.gpu


def _pencil(nz, seed):
    rng = np.random.default_rng(seed)
    nn = 3 * nz + 17
    z = rng.standard_normal((nn, nz)) + 1j * rng.standard_normal((nn, nz))
    z *= rng.uniform(0.2, 5.0, nz)[None, :]
    h = rng.standard_normal((nn, nn)) + 1j * rng.standard_normal((nn, nn))
    h = h + h.conj().T
    return z.conj().T @ h @ z, z.conj().T @ z


def _solve(fn, a, s, n):
    import torch
    nz = a.shape[0]
    v = torch.full((n, nz), float("nan"), dtype=torch.complex128, device="cuda")
    lam = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    info = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    fn(to_dev(a.T.copy(), torch.complex128), to_dev(s.T.copy(), torch.complex128), n, v, lam, info)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), v.cpu().numpy().T, info.cpu().numpy()


@pytest.mark.parametrize("calls", [((96, 32, 1), (40, 12, 2)), ((128, 40, 3), (128, 40, 3))])
def test_static_matches_allocating_entry_point(calls):
    gpu()
    import paper_1211_1446_gb300 as P
    for nz, n, seed in calls:                  # two calls in a row on the shared array
        a, s = _pencil(nz, seed)
        lam_ref, v_ref, info_ref = _solve(P.rayleigh_ritz, a, s, n)
        lam, v, info = _solve(P.rayleigh_ritz_static, a, s, n)
        scale = max(1.0, np.abs(lam_ref).max())
        assert np.array_equal(info[:3], info_ref[:3])
        assert np.abs(lam - lam_ref).max() < 1e-9 * scale
        # same Ritz vectors up to a phase per column (both S-orthonormal)
        ov = np.abs(np.sum(v_ref.conj() * (s @ v), axis=0))
        assert np.abs(ov - 1.0).max() < 1e-8
        assert np.abs(a @ v - (s @ v) * lam[None, :]).max() < 1e-7 * scale * np.abs(s).max()


def test_static_rejects_oversized_pencil():
    torch = gpu()
    import paper_1211_1446_gb300 as P
    nz = 129
    a = torch.zeros((nz, nz), dtype=torch.complex128, device="cuda")
    v = torch.zeros((4, nz), dtype=torch.complex128, device="cuda")
    lam = torch.zeros(4, dtype=torch.float64, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(P.DKSError) as e:
        P.rayleigh_ritz_static(a, a, 4, v, lam, info)
    assert e.value.code == -9 and "128" in str(e.value)
