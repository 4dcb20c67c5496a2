"""Self-consistent field (SCF) loop around the DKS eigenproblem, plain FP64 numpy.

Test infrastructure (the oracle): plain, slow and written to be read against the paper; it
shares no code with the CUDA path.

What it computes (Sec. 2.1, DKS equations; Sec. 4.1, setup):
  * the electron density of the occupied four-spinors, Eq. (density) with B_xc = 0:
        rho(r) = sum_k w_k sum_{i occupied} psi_ik(r)^dag psi_ik(r),
        psi(r) = vol^-1/2 sum_G c_G exp(i (k+G).r)   (the phase exp(ik.r) drops out of |psi|^2);
  * V_hxc = Hartree + exchange-correlation (the unnumbered equation after Eq. DKS):
        V_H(G) = 4 pi rho(G) / |G|^2, V_H(G = 0) = 0 (neutralising background),
        v_xc from the LDA of Ceperley-Alder as parametrised by Perdew and Zunger (1981),
        spin-unpolarised (the magnetisation term is dropped, B_xc = 0 as in Eq. vDKS);
  * Anderson mixing of the density with the Kerker preconditioner (Sec. 4.1), in the
    residual-minimising form (readings below);
  * the loop itself: solve H'[V_loc + V_hxc(rho_in)] for the lowest nev positive-energy
    pairs, rho_out from the nocc lowest, stop when int |rho_out - rho_in| dr < tol, else mix.

Readings (the paper names the ingredients only):
  * signed grid frequencies follow the FFT convention m' = m - N for 2m >= N (the Nyquist index
    maps to -N/2), and every potential is the real part of its inverse transform;
  * density below zero (possible after Anderson extrapolation) counts as zero in the LDA;
  * Anderson step with history dR_j = rho_in^(j+1) - rho_in^(j), dF_j = F^(j+1) - F^(j)
    (F = rho_out - rho_in): gamma = argmin |F - dF gamma|_2 (plain sum over grid points;
    singular directions of dF below 1e-6 of the largest are left out, so that a history that
    has become nearly dependent does not amplify rounding),
    rho_bar = rho_in - dR gamma, F_bar = F - dF gamma, rho_next = rho_bar + P F_bar,
    with P the Kerker factor alpha |G|^2 / (|G|^2 + q0^2) applied in reciprocal space;
  * the first density comes from the operator with V_loc alone (no Hartree, no xc).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from workloads import reciprocal_rows

from .basis import grid_index, sphere
from .lobpcgf import dense_eigs
from .operator import dense_hamiltonian, dense_hamiltonian_ksso

# Perdew-Zunger (1981) fit of the Ceperley-Alder correlation energy, unpolarised gas (Ha)
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334          # r_s >= 1
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116          # r_s < 1


def density(x, miller, grid, volume, occ):
    """rho on the grid [N1, N2, N3] from x[band, comp, pw] with occupation occ[band]."""
    x = np.asarray(x, dtype=np.complex128)
    ng = int(np.prod(grid))
    gidx = grid_index(miller, grid)
    rho = np.zeros(tuple(grid))
    for b in range(x.shape[0]):
        for a in range(x.shape[1]):
            g = np.zeros(ng, dtype=np.complex128)
            g[gidx] = x[b, a]
            psi = np.fft.ifftn(g.reshape(grid)) * ng        # sum_G c_G e^{iG.r}
            rho += occ[b] * np.abs(psi) ** 2
    return rho / volume


def gvectors(lattice, grid):
    """Cartesian G of every grid frequency index, shape [N1, N2, N3, 3]."""
    brow = reciprocal_rows(np.asarray(lattice, dtype=np.float64))
    m = [np.fft.fftfreq(n, 1.0 / n) for n in grid]       # signed integers, Nyquist -> -N/2
    mm = np.stack(np.meshgrid(*m, indexing="ij"), axis=-1)
    return mm @ brow


def hartree(rho, lattice):
    """V_H on the grid: 4 pi rho(G) / |G|^2 for G != 0, nothing at G = 0."""
    g = gvectors(lattice, rho.shape)
    g2 = np.einsum("...i,...i->...", g, g)
    rg = np.fft.fftn(rho)
    vg = np.zeros_like(rg)
    nz = g2 > 0
    vg[nz] = 4.0 * math.pi * rg[nz] / g2[nz]
    return np.real(np.fft.ifftn(vg))


def _rs(rho):
    return (3.0 / (4.0 * math.pi * rho)) ** (1.0 / 3.0)


def lda_exchange(rho):
    """(eps_x, v_x) of the uniform gas for rho > 0: eps_x = -(3/4)(9/(4 pi^2))^(1/3) / r_s and
    v_x = d(rho eps_x)/d rho = (4/3) eps_x."""
    ex = -0.75 * (9.0 / (4.0 * math.pi ** 2)) ** (1.0 / 3.0) / _rs(rho)
    return ex, 4.0 / 3.0 * ex


def pz81_correlation(rho):
    """(eps_c, v_c) of the Perdew-Zunger fit for rho > 0, v_c = eps_c - (r_s / 3) d eps_c / d r_s."""
    rs = _rs(rho)
    ec = np.empty_like(rs)
    vc = np.empty_like(rs)
    lo = rs < 1.0
    r, lr = rs[lo], np.log(rs[lo])
    ec[lo] = PZ_A * lr + PZ_B + PZ_C * r * lr + PZ_D * r
    vc[lo] = ec[lo] - r / 3.0 * (PZ_A / r + PZ_C * lr + PZ_C + PZ_D)
    r = rs[~lo]
    sq = np.sqrt(r)
    den = 1.0 + PZ_BETA1 * sq + PZ_BETA2 * r
    ec[~lo] = PZ_GAMMA / den
    dden = 0.5 * PZ_BETA1 / sq + PZ_BETA2
    vc[~lo] = ec[~lo] - r / 3.0 * (-PZ_GAMMA * dden / den ** 2)
    return ec, vc


def lda_pz81(rho):
    """(eps_xc, v_xc) of the unpolarised LDA on a grid: Dirac exchange plus the Perdew-Zunger
    correlation; zero where rho <= 1e-30."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    on = rho > 1e-30
    ex, vx = lda_exchange(rho[on])
    ec, vc = pz81_correlation(rho[on])
    eps[on] = ex + ec
    v[on] = vx + vc
    return eps, v


def hxc(rho, lattice, volume):
    """V_hxc on the grid and the energies (E_H, E_xc)."""
    vh = hartree(rho, lattice)
    eps, vxc = lda_pz81(rho)
    dv = volume / rho.size
    return vh + vxc, 0.5 * dv * float(np.sum(rho * vh)), dv * float(np.sum(np.maximum(rho, 0.0) * eps))


def kerker(f, lattice, alpha, q0):
    """P f: the factor alpha |G|^2 / (|G|^2 + q0^2) on every Fourier component of f."""
    g = gvectors(lattice, f.shape)
    g2 = np.einsum("...i,...i->...", g, g)
    return np.real(np.fft.ifftn(np.fft.fftn(f) * (alpha * g2 / (g2 + q0 * q0))))


class AndersonMixer:
    """Anderson mixing with a preconditioner (Kerker by default), history of m differences."""

    def __init__(self, lattice, alpha=0.5, q0=1.0, history=8, precondition=None):
        self.lattice = lattice
        self.alpha, self.q0, self.m = alpha, q0, history
        self.pre = precondition if precondition is not None else (
            lambda f: kerker(f, self.lattice, self.alpha, self.q0))
        self.dr, self.df = [], []
        self.prev = None

    def step(self, rho_in, rho_out):
        f = rho_out - rho_in
        if self.prev is not None and self.m > 0:
            self.dr.append((rho_in - self.prev[0]).reshape(-1))
            self.df.append((f - self.prev[1]).reshape(-1))
            self.dr, self.df = self.dr[-self.m:], self.df[-self.m:]
        self.prev = (rho_in.copy(), f.copy())
        rbar, fbar = rho_in, f
        if self.df:
            dfm, drm = np.stack(self.df, axis=1), np.stack(self.dr, axis=1)
            gam = np.linalg.lstsq(dfm, f.reshape(-1), rcond=1e-6)[0]
            rbar = rho_in - (drm @ gam).reshape(rho_in.shape)
            fbar = f - (dfm @ gam).reshape(rho_in.shape)
        return rbar + self.pre(fbar)


@dataclasses.dataclass
class SCFResult:
    lam: list              # per k: the nev eigenvalues of the last solve (shifted units)
    x: list                # per k: eigenvectors [nev, ncomp, npw]
    rho: np.ndarray        # rho_out of the last solve
    rho_in: np.ndarray     # the density the last potential was built from
    v_hxc: np.ndarray
    iterations: int
    converged: bool
    history: list


def scf(wl, nocc, nev=None, tol=1e-8, max_iter=60, alpha=0.5, q0=1.0, history=8, model="dks"):
    """The SCF loop on the dense operator (small workloads).  nocc occupied states per k-point,
    each holding one electron, k-points weighted equally."""
    nev = nocc if nev is None else nev
    basis = [sphere(wl.lattice, wl.grid, wl.kfrac[ik], wl.ecut_k[ik]) for ik in range(wl.nk)]
    wk = 1.0 / wl.nk
    dense = dense_hamiltonian if model == "dks" else dense_hamiltonian_ksso
    nc = 4 if model == "dks" else 2
    v_loc = np.asarray(wl.v_r, dtype=np.float64)

    def solve(v):
        w = dataclasses.replace(wl, v_r=v)
        lam, xs = [], []
        for m, q in basis:
            h = dense(w, m, q)
            if model == "dks":
                l, u, _ = dense_eigs(h, wl.c, nev)
            else:
                ev, uu = np.linalg.eigh(h)
                l, u = ev[:nev], uu[:, :nev]
            lam.append(l)
            xs.append(u.T.reshape(-1, nc, q.shape[0]))
        return lam, xs

    def rho_of(xs):
        return sum(density(x[:nocc], m, wl.grid, wl.volume, np.full(nocc, wk))
                   for x, (m, _) in zip(xs, basis))

    lam, xs = solve(v_loc)
    rho_in = rho_of(xs)
    mixer = AndersonMixer(wl.lattice, alpha, q0, history)
    hist = []
    converged = False
    it = 0
    dv = wl.volume / wl.ng
    for it in range(1, max_iter + 1):
        vhxc, eh, exc = hxc(rho_in, wl.lattice, wl.volume)
        lam, xs = solve(v_loc + vhxc)
        rho_out = rho_of(xs)
        res = dv * float(np.abs(rho_out - rho_in).sum())
        hist.append(dict(it=it, residual=res, eh=eh, exc=exc, lam=[l.copy() for l in lam]))
        if res < tol:
            converged = True
            break
        rho_in = mixer.step(rho_in, rho_out)
    return SCFResult(lam=lam, x=xs, rho=rho_out, rho_in=rho_in, v_hxc=vhxc, iterations=it,
                     converged=converged, history=hist)
