"""Seeded synthetic inputs for the Dirac-Kohn-Sham eigenproblem.

This module is the only code shared by the CPU oracle and the CUDA path.  It
produces *inputs* -- cell, grid, cutoff, k-points, the local potential sampled
on the grid, projector parameters and the random start block -- and contains
none of the method's arithmetic (no Hamiltonian, no FFT-based operator, no
eigensolver).  Every number it returns is a pure function of the workload name,
its overrides and the seed.

The systems stand in for the paper's heavy-element dimers (Sec. 4.1: a dimer in
an orthorhombic box) and for the layered Bi2Se3 crystal (Sec. 4.1, Fig. 3),
whose HGH parameters are not available: the local part is a periodised
Gaussian-smeared Coulomb attraction per site and the nonlocal spin-orbit part
uses HGH-shaped Gaussian projectors with seeded strengths (Eq. 5 structure).

Conventions (both sides follow them):
  * lattice rows are a1, a2, a3 in bohr; reciprocal rows b_i = 2*pi*inv(A)^T.
  * the potential array v_r[i1, i2, i3] is V at r = sum_i (i_i/N_i) a_i, Ha.
  * projector strengths d[site, l, jj] in Ha, jj = 0 for j = l + 1/2 and
    jj = 1 for j = l - 1/2 (unused for l = 0).
  * the start block x0[band, comp, pw] is indexed by the canonical planewave
    order: Miller triples (m1, m2, m3) sorted lexicographically (signed).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DEFAULT_SEED = 20121106
C_LIGHT = 137.036  # a.u., Sec. 1


@dataclasses.dataclass
class Workload:
    name: str
    lattice: np.ndarray          # (3, 3) rows a1, a2, a3 (bohr)
    grid: tuple                  # (N1, N2, N3)
    c: float                     # speed of light (a.u.)
    kfrac: np.ndarray            # (nk, 3) fractional k
    ecut_k: np.ndarray           # (nk,) cutoff per k (Ha)
    v_r: np.ndarray              # (N1, N2, N3) real local potential (Ha)
    pos: np.ndarray              # (nsite, 3) cartesian (bohr)
    zion: np.ndarray             # (nsite,)
    sigma: np.ndarray            # (nsite,)
    lmax: np.ndarray             # (nsite,) int, -1 = no projector
    rl: np.ndarray               # (nsite, 3) Gaussian widths per l (bohr)
    d: np.ndarray                # (nsite, 3, 2) strengths (Ha)
    nev_k: np.ndarray            # (nk,) wanted eigenpairs per k
    nbuf: int
    seed: int

    @property
    def nk(self) -> int:
        return int(self.kfrac.shape[0])

    @property
    def nsite(self) -> int:
        return int(self.pos.shape[0])

    @property
    def ng(self) -> int:
        return int(np.prod(self.grid))

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))


def reciprocal_rows(lattice: np.ndarray) -> np.ndarray:
    """Rows b1, b2, b3 with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def smeared_coulomb_potential(lattice, grid, pos, zion, sigma) -> np.ndarray:
    """Periodised sum of -Z erf(r/sigma)/r, sampled on the grid (input data).

    Fourier coefficients V(G) = -(4 pi Z / vol) exp(-|G|^2 sigma^2 / 4) / |G|^2
    * exp(-i G.R) for G != 0 on the grid's centred Miller range, V(0) = 0;
    V(r_n) = Re sum_G V(G) exp(i G.r_n).
    """
    lattice = np.asarray(lattice, dtype=np.float64)
    n1, n2, n3 = grid
    brow = reciprocal_rows(lattice)
    vol = abs(np.linalg.det(lattice))
    f = [np.fft.fftfreq(n, 1.0 / n) for n in grid]          # centred integer Miller
    m1, m2, m3 = np.meshgrid(*f, indexing="ij")
    g = (m1[..., None] * brow[0] + m2[..., None] * brow[1] + m3[..., None] * brow[2])
    g2 = np.einsum("...i,...i->...", g, g)
    vg = np.zeros(grid, dtype=np.complex128)
    nz = g2 > 0
    for r, z, s in zip(pos, zion, sigma):
        phase = np.exp(-1j * (g @ np.asarray(r)))
        term = np.zeros(grid, dtype=np.complex128)
        term[nz] = -(4.0 * np.pi * z / vol) * np.exp(-g2[nz] * s * s / 4.0) / g2[nz]
        vg += term * phase
    # V(r_n) = sum_m V(G_m) exp(2 pi i m.n/N) = Ng * ifftn
    return np.ascontiguousarray(np.real(np.fft.ifftn(vg)) * (n1 * n2 * n3))


def _projector_params(rng, nsite, lmax, widths):
    """HGH-shaped strengths: D_{l,j=l+1/2} = h_l + k_l l/2, D_{l,j=l-1/2} = h_l - k_l (l+1)/2."""
    rl = np.zeros((nsite, 3))
    d = np.zeros((nsite, 3, 2))
    for s in range(nsite):
        for l in range(3):
            rl[s, l] = widths[s][l]
            if l <= lmax[s]:
                h = rng.uniform(-4.0, 4.0)
                kso = rng.uniform(-1.0, 1.0) if l > 0 else 0.0
                d[s, l, 0] = h + kso * l / 2.0
                d[s, l, 1] = h - kso * (l + 1) / 2.0 if l > 0 else 0.0
    return rl, d


def _finish(name, lattice, grid, c, kfrac, ecut_k, pos, zion, sigma, lmax, widths,
            nev_k, nbuf, seed, with_potential=True, with_projectors=True):
    rng = np.random.default_rng(seed)
    nsite = len(pos)
    lmax = np.asarray(lmax, dtype=np.int64)
    if not with_projectors:
        lmax = -np.ones(nsite, dtype=np.int64)
    rl, d = _projector_params(rng, nsite, lmax, widths)
    if with_potential and nsite:
        v = smeared_coulomb_potential(lattice, grid, pos, zion, sigma)
    else:
        v = np.zeros(grid)
    return Workload(name=name, lattice=np.asarray(lattice, dtype=np.float64), grid=tuple(grid),
                    c=float(c), kfrac=np.asarray(kfrac, dtype=np.float64).reshape(-1, 3),
                    ecut_k=np.asarray(ecut_k, dtype=np.float64), v_r=v,
                    pos=np.asarray(pos, dtype=np.float64).reshape(-1, 3),
                    zion=np.asarray(zion, dtype=np.float64), sigma=np.asarray(sigma, dtype=np.float64),
                    lmax=lmax, rl=rl, d=d, nev_k=np.asarray(nev_k, dtype=np.int64),
                    nbuf=int(nbuf), seed=int(seed))


def _hex_layer_sites(a, cz, nx, ny):
    """Three quintuple layers (species Z6, Z15, Z6, Z15, Z6 along c), ABC in-plane stacking."""
    a1 = np.array([a, 0.0, 0.0])
    a2 = np.array([-a / 2.0, a * math.sqrt(3.0) / 2.0, 0.0])
    abc = [(0.0, 0.0), (1.0 / 3.0, 2.0 / 3.0), (2.0 / 3.0, 1.0 / 3.0)]
    species = [6.0, 15.0, 6.0, 15.0, 6.0] * 3
    pos, zion, sigma = [], [], []
    for j in range(15):
        fx, fy = abc[j % 3]
        z = (j + 0.5) * cz / 15.0
        for ix in range(nx):
            for iy in range(ny):
                p = (fx + ix) * a1 + (fy + iy) * a2
                pos.append([p[0], p[1], z])
                zion.append(species[j])
                sigma.append(0.6 if species[j] == 6.0 else 0.8)
    return pos, zion, sigma


def make(name: str, seed: int = DEFAULT_SEED, **kw) -> Workload:
    """Build a named workload.  Overrides: c, ecut, grid, nev, potential, projectors.

    Names:
      cubic    -- cubic L=8, 12^3 grid, Ecut 8 Ha (515 planewaves), one site Z=10 sigma 0.5,
                  no projectors, Gamma, nev 8.
      dimer    -- 20x20x24 box, 48x48x56 grid, Ecut 25 Ha, two sites 4.5 bohr apart
                  (Z 18, sigma 0.8) with s/p/d spin-orbit projectors, Gamma, nev 32.
      layered  -- hexagonal a=7.8, c=28, 60x60x216 grid, Ecut 68 Ha with +-3% per-k jitter,
                  15 sites, 16 k-points (4x4x1), nev_k in {48,...,96}.
      supercell-- 2x2x1 of layered, 120x120x216 grid, 4 k-points, nev 480 + 64 buffer.
      small    -- a quick case with projectors: orthorhombic 7x7.5x8, 16x15x18 grid,
                  Ecut 6 Ha, two sites, Gamma, nev 6 (tests).
    """
    c = kw.pop("c", C_LIGHT)
    pot = kw.pop("potential", True)
    proj = kw.pop("projectors", True)
    if name == "cubic":
        lat = np.eye(3) * 8.0
        grid = kw.pop("grid", (12, 12, 12))
        ecut = kw.pop("ecut", 8.0)
        kfrac = kw.pop("kfrac", [[0.0, 0.0, 0.0]])
        nev = kw.pop("nev", 8)
        wl = _finish(name, lat, grid, c, kfrac, [ecut] * len(kfrac), [[4.0, 4.0, 4.0]], [10.0], [0.5],
                     [-1], [[0.5, 0.5, 0.5]], [nev] * len(kfrac), 0, seed, pot, False)
    elif name in ("dimer", "small"):
        if name == "dimer":
            lat = np.diag([20.0, 20.0, 24.0])
            grid = kw.pop("grid", (48, 48, 56))
            ecut = kw.pop("ecut", 25.0)
            nev = kw.pop("nev", 32)
            pos = [[10.0, 10.0, 12.0 - 2.25], [10.0, 10.0, 12.0 + 2.25]]
            zion, sig = [18.0, 18.0], [0.8, 0.8]
            widths = [[0.45, 0.55, 0.65]] * 2
        else:
            lat = np.diag([7.0, 7.5, 8.0])
            grid = kw.pop("grid", (16, 15, 18))
            ecut = kw.pop("ecut", 6.0)
            nev = kw.pop("nev", 6)
            pos = [[3.5, 3.7, 4.0 - 1.2], [3.4, 3.8, 4.0 + 1.2]]
            zion, sig = [8.0, 8.0], [0.7, 0.7]
            widths = [[0.6, 0.7, 0.8]] * 2
        kfrac = kw.pop("kfrac", [[0.0, 0.0, 0.0]])
        wl = _finish(name, lat, grid, c, kfrac, [ecut] * len(kfrac), pos, zion, sig, [2, 2],
                     widths, [nev] * len(kfrac), 0, seed, pot, proj)
    elif name in ("layered", "supercell"):
        a, cz = 7.8, 28.0
        rep = 1 if name == "layered" else 2
        lat = np.array([[a * rep, 0.0, 0.0], [-a * rep / 2.0, a * rep * math.sqrt(3.0) / 2.0, 0.0],
                        [0.0, 0.0, cz]])
        grid = kw.pop("grid", (60 * rep, 60 * rep, 216))
        ecut = kw.pop("ecut", 68.0)
        nkx = 4 if name == "layered" else 2
        kfrac = kw.pop("kfrac", [[i / nkx, j / nkx, 0.0] for i in range(nkx) for j in range(nkx)])
        rng = np.random.default_rng(seed + 7)
        if name == "layered":
            delta = rng.uniform(-0.03, 0.03, size=len(kfrac))
            ecut_k = ecut * (1.0 + delta) ** (2.0 / 3.0)
            nev_k = kw.pop("nev_k", rng.choice(np.arange(48, 97, 8), size=len(kfrac)))
            nbuf = 0
        else:
            ecut_k = np.full(len(kfrac), ecut)
            nev_k = kw.pop("nev_k", np.full(len(kfrac), 480))
            nbuf = 64
        pos, zion, sig = _hex_layer_sites(a, cz, rep, rep)
        widths = [[0.45, 0.55, 0.65] if z == 15.0 else [0.4, 0.5, 0.6] for z in zion]
        wl = _finish(name, lat, grid, c, kfrac, ecut_k, pos, zion, sig, [2] * len(pos), widths,
                     nev_k, nbuf, seed, pot, proj)
    else:
        raise ValueError(f"unknown workload {name!r}")
    if kw:
        raise TypeError(f"unused overrides {sorted(kw)}")
    return wl


def start_block(npw: int, nb: int, seed: int = DEFAULT_SEED, ik: int = 0, ncomp: int = 4) -> np.ndarray:
    """Seed-fixed complex normal start block x0[band, comp, pw] (canonical pw order); ncomp = 4 for
    four-spinors, 2 for two-spinors (the first two components of the same draw)."""
    rng = np.random.Generator(np.random.PCG64([seed, 1000 + ik, nb]))
    re = rng.standard_normal((nb, 4, npw))
    im = rng.standard_normal((nb, 4, npw))
    return ((re + 1j * im) / math.sqrt(2.0))[:, :ncomp].copy()


def random_block(npw: int, nb: int, seed: int, ncomp: int = 4) -> np.ndarray:
    """Generic seeded complex normal block [band, comp, pw] for operator tests."""
    rng = np.random.Generator(np.random.PCG64([seed, 77, nb, npw]))
    return (rng.standard_normal((nb, ncomp, npw)) + 1j * rng.standard_normal((nb, ncomp, npw))) / math.sqrt(2.0)


def save(wl: Workload, path: str) -> None:
    """Freeze a workload -- every generated number, the potential grid included -- into one .npz
    file that both sides can read back with load()."""
    fields = {f.name: getattr(wl, f.name) for f in dataclasses.fields(Workload)}
    arrays = {k: np.asarray(v) for k, v in fields.items()}
    np.savez_compressed(path, **arrays)


def load(path: str) -> Workload:
    """The workload frozen by save()."""
    with np.load(path, allow_pickle=False) as f:
        kw = {}
        for fld in dataclasses.fields(Workload):
            v = f[fld.name]
            if fld.name == "name":
                kw[fld.name] = str(v)
            elif fld.name == "grid":
                kw[fld.name] = tuple(int(x) for x in v)
            elif fld.name in ("c",):
                kw[fld.name] = float(v)
            elif fld.name in ("nbuf", "seed"):
                kw[fld.name] = int(v)
            else:
                kw[fld.name] = np.array(v)
    return Workload(**kw)
