"""Pins for the SCF part of the oracle (density, Hartree, LDA, Kerker, Anderson, the loop).

What fixes each expected value: closed forms (uniform density of one planewave, the Hartree
potential of a single Fourier mode, Dirac exchange of the uniform gas, the Gell-Mann-Brueckner
high-density coefficient), brute-force sums without an FFT, identities (Parseval, the
thermodynamic relation v = d(rho eps)/d rho by finite differences), the finite termination of
Anderson mixing on a linear problem, self-consistency of the result, and the nonrelativistic
limit (DKS SCF -> two-component SCF as c -> oo).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import basis, scf


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- density, Eq. (density)

def test_density_single_planewave_is_uniform():
    wl = W.make("small", ecut=4.0)
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    x = np.zeros((1, 4, len(m)), dtype=np.complex128)
    x[0, 2, 17] = np.exp(0.3j)                      # a unit small-component planewave
    rho = scf.density(x, m, wl.grid, wl.volume, [1.0])
    assert np.abs(rho - 1.0 / wl.volume).max() < 1e-15 / wl.volume * 10


def test_density_brute_force_and_parseval():
    """Direct sum psi(r) = vol^-1/2 sum_G c_G exp(i (k+G).r) at sampled grid points, k != 0."""
    wl = W.make("small", ecut=4.0, kfrac=[[0.25, -0.1, 0.4]])
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    x = _rand((3, 4, len(m)), 5)
    x /= np.linalg.norm(x.reshape(3, -1), axis=1)[:, None, None]
    occ = np.array([1.0, 0.5, 2.0])
    rho = scf.density(x, m, wl.grid, wl.volume, occ)
    grid = np.asarray(wl.grid)
    rng = np.random.default_rng(1)
    for _ in range(6):
        n = rng.integers(0, grid)
        r = (n / grid) @ wl.lattice
        ph = np.exp(1j * (q @ r))                    # includes the k phase, which cancels in |psi|^2
        val = sum(occ[b] * np.sum(np.abs(x[b] @ ph) ** 2) for b in range(3)) / wl.volume
        assert abs(rho[tuple(n)] - val) < 1e-12 * val
    # Parseval: int rho = sum of the occupations of unit columns
    assert abs(rho.sum() * wl.volume / wl.ng - occ.sum()) < 1e-12


# ---------------------------------------------------------------- Hartree

def test_gvectors_signed_frequencies():
    lat = W.make("layered", ecut=2.0).lattice
    grid = (6, 5, 8)
    g = scf.gvectors(lat, grid)
    b = W.reciprocal_rows(lat)
    assert np.allclose(g[1, 0, 0], b[0]) and np.allclose(g[0, 4, 0], -b[1])
    assert np.allclose(g[3, 0, 0], -3 * b[0])         # Nyquist index -> -N/2
    assert np.allclose(g[0, 2, 7], 2 * b[1] - b[2])


def test_hartree_single_mode_closed_form():
    """rho = cos(G0.r) on a hexagonal (non-orthogonal) cell: V_H = 4 pi cos(G0.r) / |G0|^2."""
    wl = W.make("layered", ecut=2.0, grid=(12, 12, 20))
    b = W.reciprocal_rows(wl.lattice)
    g0 = 1 * b[0] + 2 * b[1] - 1 * b[2]
    n = np.stack(np.meshgrid(*[np.arange(k) for k in wl.grid], indexing="ij"), -1)
    r = (n / np.asarray(wl.grid)) @ wl.lattice
    rho = 0.3 + np.cos(r @ g0)                        # the constant part has no potential
    vh = scf.hartree(rho, wl.lattice)
    want = 4 * math.pi * np.cos(r @ g0) / (g0 @ g0)
    assert np.abs(vh - want).max() < 1e-12 * np.abs(want).max()


# ---------------------------------------------------------------- LDA (Perdew-Zunger fit)

def test_lda_exchange_is_dirac_exchange():
    """eps_x = -3 k_F / (4 pi) with k_F = (3 pi^2 rho)^(1/3), the exchange energy per electron of
    the uniform gas; the full LDA minus the correlation part gives it back."""
    rho = np.array([1e-4, 0.01, 0.3, 5.0])
    ex, vx = scf.lda_exchange(rho)
    kf = (3 * math.pi ** 2 * rho) ** (1.0 / 3.0)
    assert np.abs(ex + 3 * kf / (4 * math.pi)).max() < 1e-14 * np.abs(ex).max()
    eps, _ = scf.lda_pz81(rho)
    assert np.abs(eps - ex - scf.pz81_correlation(rho)[0]).max() < 1e-15


@pytest.mark.parametrize("rho", [1e-5, 3e-3, 0.05, 0.2387, 0.25, 2.0, 40.0])
def test_lda_potential_is_derivative_of_energy_density(rho):
    h = 1e-6 * rho
    e = lambda r: r * scf.lda_pz81(np.array([r]))[0][0]
    v = scf.lda_pz81(np.array([rho]))[1][0]
    fd = (e(rho + h) - e(rho - h)) / (2 * h)
    assert abs(v - fd) < 1e-7 * abs(v)


def test_lda_correlation_continuous_at_rs_one_and_high_density_limit():
    """The fit's two branches meet at r_s = 1 in energy and in potential (to the fit's 1e-4), and
    its r_s -> 0 branch carries the Gell-Mann-Brueckner coefficient (1 - ln 2) / pi^2."""
    rho1 = 3 / (4 * math.pi)                          # r_s = 1
    ec, vc = scf.pz81_correlation(np.array([rho1 * (1 + 1e-12), rho1 * (1 - 1e-12)]))
    assert abs(ec[0] - ec[1]) < 1e-4 and abs(vc[0] - vc[1]) < 1e-4
    assert abs(scf.PZ_A - (1 - math.log(2)) / math.pi ** 2) < 2e-5
    eps, v = scf.lda_pz81(np.array([-1.0, 0.0]))
    assert np.all(eps == 0) and np.all(v == 0)


# ---------------------------------------------------------------- Kerker and Anderson

def test_kerker_factor_on_single_modes():
    wl = W.make("small", ecut=4.0)
    b = W.reciprocal_rows(wl.lattice)
    n = np.stack(np.meshgrid(*[np.arange(k) for k in wl.grid], indexing="ij"), -1)
    r = (n / np.asarray(wl.grid)) @ wl.lattice
    for g0 in (b[0], 3 * b[1] + 2 * b[2]):
        f = 2.0 + np.sin(r @ g0)
        out = scf.kerker(f, wl.lattice, 0.7, 1.3)
        fac = 0.7 * (g0 @ g0) / (g0 @ g0 + 1.3 ** 2)
        assert np.abs(out - fac * np.sin(r @ g0)).max() < 1e-13


def test_anderson_terminates_on_linear_problem():
    """On rho_out = M rho_in + b, Anderson mixing with a full history reaches the fixed point in
    at most n + 1 steps (it then spans the Krylov space of M - I, as GMRES does)."""
    rng = np.random.default_rng(4)
    n = 5
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    m = q @ np.diag(rng.uniform(-0.9, 0.6, n)) @ q.T
    bvec = rng.standard_normal(n)
    xstar = np.linalg.solve(np.eye(n) - m, bvec)
    mix = scf.AndersonMixer(None, history=n + 2, precondition=lambda f: 0.4 * f)
    plain = scf.AndersonMixer(None, history=0, precondition=lambda f: 0.4 * f)
    x = y = np.zeros(n)
    for _ in range(n + 2):
        x = mix.step(x, m @ x + bvec)
        y = plain.step(y, m @ y + bvec)
    assert np.abs(x - xstar).max() < 1e-10
    assert np.abs(y - xstar).max() > 1e-3


# ---------------------------------------------------------------- the loop

def test_scf_is_self_consistent_and_conserves_charge():
    wl = W.make("small", ecut=4.0)
    res = scf.scf(wl, 4, nev=6, tol=1e-9)
    assert res.converged
    assert abs(res.rho.sum() * wl.volume / wl.ng - 4.0) < 1e-10
    # rebuild the potential from the returned density: its solve gives the same density back
    vhxc, _, _ = scf.hxc(res.rho, wl.lattice, wl.volume)
    assert np.abs(vhxc - res.v_hxc).max() < 1e-6
    assert np.abs(res.rho - res.rho_in).sum() * wl.volume / wl.ng < 1e-9
    lam = res.lam[0]
    assert np.all(lam > -wl.c ** 2) and lam[4] - lam[3] > 0.1   # the occupied set is gapped


def test_scf_nonrelativistic_limit():
    """c = 1e4: the DKS SCF (shifted) matches the two-component SCF without spin-orbit terms."""
    wl = W.make("cubic", ecut=4.0, c=1e4)
    d = scf.scf(wl, 2, nev=4, tol=1e-7)     # the dense solve spans 2c^2 = 2e8 Ha: ~1e-8 noise
    k = scf.scf(wl, 2, nev=4, tol=1e-7, model="ksso")
    assert d.converged and k.converged
    assert np.abs(d.lam[0] - k.lam[0]).max() < 1e-6
    assert np.abs(d.rho - k.rho).max() < 1e-6 * np.abs(k.rho).max()
