"""The shifted DKS operator H' = H - c^2 on the planewave sphere, in FP64.

Vectors are stored as x[comp, pw] (or blocks x[band, comp, pw]); comp 0,1 are
the large two-spinor (spin up, down), comp 2,3 the small one.  A dense matrix
index is comp*npw + pw.  Energies are shifted by -mc^2 (Sec. 4), so the
positive band starts near 0 and the negative band near -2c^2.

Terms (Eq. vDKS with B_xc = 0):
  * free Dirac operator h_D of Eq. (2) with p -> q = k+G, shifted:
        [[0, c sigma.q], [c sigma.q, -2 c^2 I2]]  per planewave;
  * local potential V(r) I4: matrix element Vhat[(m_i - m_j) mod N] with
    Vhat = DFT(V)/Ng on the grid (the same discrete operator as the FFT route);
  * nonlocal spin-orbit projectors of Eq. (HGH): I2 (x) N acting identically on
    the large and small two-spinors (S = diag(sigma, sigma)/2), with
    N = sum_{site,l,j,mj} D beta beta^H and
    beta(q) = p_l(|q|) Omega_{j l mj}(qhat) exp(-i q.R) / sqrt(vol).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import eval_legendre, gamma

try:                                   # scipy >= 1.15
    from scipy.special import sph_harm_y
except ImportError:                    # older scipy: sph_harm(m, l, azimuth, polar)
    from scipy.special import sph_harm as _sph_harm_old

    def sph_harm_y(l, m, theta, phi):
        return _sph_harm_old(m, l, phi, theta)

from .basis import grid_index

# ---------------------------------------------------------------------------
# radial and angular parts of the projectors
# ---------------------------------------------------------------------------


def radial(l, r, q):
    """p_l(q) = A_l q^l exp(-q^2 r^2 / 2), A_l normalising p_l to unit L2 norm over d^3q/(2pi)^3."""
    a = math.sqrt(2.0 * (2.0 * math.pi) ** 3 * r ** (2 * l + 3) / gamma(l + 1.5))
    return a * q ** l * np.exp(-0.5 * (q * r) ** 2)


def _angles(q):
    qn = np.linalg.norm(q, axis=-1)
    safe = np.where(qn > 0, qn, 1.0)
    u = q / safe[..., None]
    u = np.where((qn > 0)[..., None], u, np.array([0.0, 0.0, 1.0]))
    theta = np.arccos(np.clip(u[..., 2], -1.0, 1.0))
    phi = np.arctan2(u[..., 1], u[..., 0])
    return qn, u, theta, phi


def _ylm(l, m, theta, phi):
    if abs(m) > l:
        return np.zeros_like(theta, dtype=np.complex128)
    return sph_harm_y(l, m, theta, phi)  # complex, Condon-Shortley phase


def spinor_harmonic(j2, l, mj2, theta, phi):
    """Omega_{j l mj}(theta, phi) as a (..., 2) array; j = j2/2, mj = mj2/2.

    Coupling of Y_lm with spin 1/2 by Clebsch-Gordan coefficients (standard
    closed form for s = 1/2).
    """
    mj = mj2 / 2.0
    m_up = (mj2 - 1) // 2   # mj - 1/2
    m_dn = (mj2 + 1) // 2   # mj + 1/2
    d = 2 * l + 1
    if j2 == 2 * l + 1:
        a_up = math.sqrt((l + mj + 0.5) / d)
        a_dn = math.sqrt((l - mj + 0.5) / d)
    elif j2 == 2 * l - 1:
        a_up = -math.sqrt((l - mj + 0.5) / d)
        a_dn = math.sqrt((l + mj + 0.5) / d)
    else:
        raise ValueError("j must be l +- 1/2")
    return np.stack([a_up * _ylm(l, m_up, theta, phi), a_dn * _ylm(l, m_dn, theta, phi)], axis=-1)


def projector_channels(wl):
    """List of (site, l, jj, j2, mj2) in the oracle's column order."""
    out = []
    for s in range(wl.nsite):
        for l in range(int(wl.lmax[s]) + 1):
            for jj, j2 in ((1, 2 * l - 1), (0, 2 * l + 1)):
                if j2 < 0:
                    continue
                for mj2 in range(-j2, j2 + 1, 2):
                    out.append((s, l, jj, j2, mj2))
    return out


def projector_matrix(wl, q):
    """B[(spin*npw + pw), channel] and the diagonal D[channel] (Ha).

    B's columns are the spinor projectors beta of Eq. (HGH) built from
    spinor spherical harmonics (scipy's Y_lm + Clebsch-Gordan).
    """
    npw = q.shape[0]
    qn, _, theta, phi = _angles(q)
    ch = projector_channels(wl)
    b = np.zeros((2 * npw, len(ch)), dtype=np.complex128)
    dvec = np.zeros(len(ch))
    vol = wl.volume
    for c, (s, l, jj, j2, mj2) in enumerate(ch):
        phase = np.exp(-1j * (q @ wl.pos[s]))
        rad = radial(l, wl.rl[s, l], qn) * phase / math.sqrt(vol)
        om = spinor_harmonic(j2, l, mj2, theta, phi)
        b[:npw, c] = rad * om[:, 0]
        b[npw:, c] = rad * om[:, 1]
        dvec[c] = wl.d[s, l, jj]
    return b, dvec


def _legendre_deriv(l, x):
    if l == 0:
        return np.zeros_like(x)
    if l == 1:
        return np.ones_like(x)
    if l == 2:
        return 3.0 * x
    raise ValueError("l <= 2 supported")


def spin_orbit_kernel(l, jj, u, v):
    """sum_mj Omega_{j l mj}(u) Omega_{j l mj}(v)^H as a closed form.

    With the addition theorem sum_m Y_lm(u) Y_lm(v)* = (2l+1)/(4 pi) P_l(u.v)
    and the j-projectors (l+1 + 2 L.S)/(2l+1), (l - 2 L.S)/(2l+1):
        j = l+1/2: [(l+1) P_l(u.v) I2 - i P_l'(u.v) sigma.(u x v)] / (4 pi)
        j = l-1/2: [ l    P_l(u.v) I2 + i P_l'(u.v) sigma.(u x v)] / (4 pi)
    (the kernel of 2 L.S is sigma.(L_u K) with L_u K = -i (2l+1)/(4 pi) P_l' u x v).
    u: (n,3), v: (m,3) unit vectors.  Returns (n, m, 2, 2).
    """
    x = np.clip(u @ v.T, -1.0, 1.0)
    w = np.cross(u[:, None, :], v[None, :, :])
    pl = eval_legendre(l, x)
    dpl = _legendre_deriv(l, x)
    sgn = -1.0 if jj == 0 else 1.0
    scal = (l + 1.0) if jj == 0 else float(l)
    k = np.zeros(x.shape + (2, 2), dtype=np.complex128)
    # sigma.w = [[wz, wx - i wy], [wx + i wy, -wz]]
    sw = np.zeros(x.shape + (2, 2), dtype=np.complex128)
    sw[..., 0, 0] = w[..., 2]
    sw[..., 0, 1] = w[..., 0] - 1j * w[..., 1]
    sw[..., 1, 0] = w[..., 0] + 1j * w[..., 1]
    sw[..., 1, 1] = -w[..., 2]
    k[..., 0, 0] = scal * pl
    k[..., 1, 1] = scal * pl
    k += sgn * 1j * dpl[..., None, None] * sw
    return k / (4.0 * math.pi)


def nonlocal_dense(wl, q):
    """N[(spin*npw+i), (spin'*npw+j)] from the Legendre closed form (no spherical harmonics)."""
    npw = q.shape[0]
    qn, u, _, _ = _angles(q)
    n = np.zeros((2 * npw, 2 * npw), dtype=np.complex128)
    vol = wl.volume
    for s in range(wl.nsite):
        phase = np.exp(-1j * (q @ wl.pos[s]))
        for l in range(int(wl.lmax[s]) + 1):
            pr = radial(l, wl.rl[s, l], qn) * phase
            outer = np.outer(pr, pr.conj()) / vol
            for jj in ((0,) if l == 0 else (0, 1)):
                k = spin_orbit_kernel(l, jj, u, u)
                blk = wl.d[s, l, jj] * outer[..., None, None] * k
                n[:npw, :npw] += blk[..., 0, 0]
                n[:npw, npw:] += blk[..., 0, 1]
                n[npw:, :npw] += blk[..., 1, 0]
                n[npw:, npw:] += blk[..., 1, 1]
    return n


# ---------------------------------------------------------------------------
# dense operator
# ---------------------------------------------------------------------------


def vhat(v_r):
    """Vhat = DFT(V)/Ng, so that <G_i|V|G_j> = Vhat[(m_i - m_j) mod N]."""
    return np.fft.fftn(v_r) / v_r.size


def dirac_block(qv, c):
    """Shifted free Dirac operator for one planewave q (Eq. 2 minus c^2)."""
    sq = np.array([[qv[2], qv[0] - 1j * qv[1]], [qv[0] + 1j * qv[1], -qv[2]]])
    h = np.zeros((4, 4), dtype=np.complex128)
    h[0:2, 2:4] = c * sq
    h[2:4, 0:2] = c * sq
    h[2:4, 2:4] = -2.0 * c * c * np.eye(2)
    return h


def dense_hamiltonian(wl, miller, q, with_local=True, with_nonlocal=True):
    """Dense 4npw x 4npw H' (index comp*npw + pw)."""
    npw = q.shape[0]
    h = np.zeros((4 * npw, 4 * npw), dtype=np.complex128)
    idx = np.arange(npw)
    for a in range(4):
        for b in range(4):
            blk = np.array([dirac_block(qv, wl.c)[a, b] for qv in q]) if npw else np.zeros(0)
            h[a * npw + idx, b * npw + idx] += blk
    if with_local:
        vh = vhat(wl.v_r)
        dm = np.mod(miller[:, None, :] - miller[None, :, :], np.asarray(wl.grid))
        vloc = vh[dm[..., 0], dm[..., 1], dm[..., 2]]
        for a in range(4):
            h[a * npw:(a + 1) * npw, a * npw:(a + 1) * npw] += vloc
    if with_nonlocal and int(np.max(wl.lmax, initial=-1)) >= 0:
        n = nonlocal_dense(wl, q)
        for big in (0, 2):
            h[big * npw:(big + 2) * npw, big * npw:(big + 2) * npw] += n
    return h


# ---------------------------------------------------------------------------
# matrix-free operator (numpy FFT), Sec. 3.1: Hx without forming H
# ---------------------------------------------------------------------------


class MatrixFreeH:
    """x[band, comp, pw] -> H'x using the FFT for V and B D B^H for the projectors."""

    def __init__(self, wl, miller, q, with_local=True, with_nonlocal=True):
        self.wl = wl
        self.q = q
        self.npw = q.shape[0]
        self.gidx = grid_index(miller, wl.grid)
        self.v = wl.v_r if with_local else None
        if with_nonlocal and int(np.max(wl.lmax, initial=-1)) >= 0:
            self.b, self.dvec = projector_matrix(wl, q)
        else:
            self.b, self.dvec = None, None
        self.count = 0  # number of single-band applications (Sec. 3.2 cost statement)

    def dirac(self, x):
        c, q = self.wl.c, self.q
        qx, qy, qz = q[:, 0], q[:, 1], q[:, 2]
        y = np.empty_like(x)
        y[:, 0] = c * (qz * x[:, 2] + (qx - 1j * qy) * x[:, 3])
        y[:, 1] = c * ((qx + 1j * qy) * x[:, 2] - qz * x[:, 3])
        y[:, 2] = c * (qz * x[:, 0] + (qx - 1j * qy) * x[:, 1]) - 2.0 * c * c * x[:, 2]
        y[:, 3] = c * ((qx + 1j * qy) * x[:, 0] - qz * x[:, 1]) - 2.0 * c * c * x[:, 3]
        return y

    def local(self, x):
        nb = x.shape[0]
        grid = self.wl.grid
        y = np.zeros_like(x)
        for b in range(nb):
            for a in range(4):
                g = np.zeros(int(np.prod(grid)), dtype=np.complex128)
                g[self.gidx] = x[b, a]
                psi = np.fft.ifftn(g.reshape(grid))            # (1/Ng) sum_G c_G e^{iG.r}
                y[b, a] = np.fft.fftn(self.v * psi).reshape(-1)[self.gidx]
        return y

    def nonlocal_(self, x):
        nb, npw = x.shape[0], self.npw
        xt = x.reshape(nb, 2, 2 * npw).reshape(2 * nb, 2 * npw).T   # columns: large_b, small_b
        z = self.b.conj().T @ xt
        yt = self.b @ (self.dvec[:, None] * z)
        return yt.T.reshape(nb, 2, 2 * npw).reshape(nb, 4, npw)

    def __call__(self, x):
        x = np.asarray(x, dtype=np.complex128)
        self.count += x.shape[0]
        y = self.dirac(x)
        if self.v is not None:
            y += self.local(x)
        if self.b is not None:
            y += self.nonlocal_(x)
        return y


# ---------------------------------------------------------------------------
# KSSO: two-component Kohn-Sham operator with spin-orbit coupling (Sec. 4, module KSSO)
# ---------------------------------------------------------------------------


def dense_hamiltonian_ksso(wl, miller, q, with_local=True, with_nonlocal=True):
    """Dense 2npw x 2npw KSSO operator on two-spinors (index comp*npw + pw): the kinetic energy
    |q|^2/2 on the diagonal, V as Vhat[(m_i - m_j) mod N] on each spin, and the spin-orbit
    projector operator N of Eq. (HGH) on the two-spinor.  Energies are not shifted."""
    npw = q.shape[0]
    h = np.zeros((2 * npw, 2 * npw), dtype=np.complex128)
    ek = 0.5 * np.einsum("ij,ij->i", q, q)
    h[np.arange(2 * npw), np.arange(2 * npw)] = np.concatenate([ek, ek])
    if with_local:
        vh = vhat(wl.v_r)
        dm = np.mod(miller[:, None, :] - miller[None, :, :], np.asarray(wl.grid))
        vloc = vh[dm[..., 0], dm[..., 1], dm[..., 2]]
        for a in range(2):
            h[a * npw:(a + 1) * npw, a * npw:(a + 1) * npw] += vloc
    if with_nonlocal and int(np.max(wl.lmax, initial=-1)) >= 0:
        h += nonlocal_dense(wl, q)
    return h


class MatrixFreeKSSO(MatrixFreeH):
    """x[band, comp, pw] (comp = spin up, down) -> H_KSSO x with numpy FFTs for V and B D B^H."""

    def kinetic(self, x):
        ek = 0.5 * np.einsum("ij,ij->i", self.q, self.q)
        return ek[None, None, :] * x

    def local(self, x):
        nb = x.shape[0]
        grid = self.wl.grid
        y = np.zeros_like(x)
        for b in range(nb):
            for a in range(2):
                g = np.zeros(int(np.prod(grid)), dtype=np.complex128)
                g[self.gidx] = x[b, a]
                psi = np.fft.ifftn(g.reshape(grid))
                y[b, a] = np.fft.fftn(self.v * psi).reshape(-1)[self.gidx]
        return y

    def nonlocal_(self, x):
        nb, npw = x.shape[0], self.npw
        xt = x.reshape(nb, 2 * npw).T                    # one two-spinor column per band
        yt = self.b @ (self.dvec[:, None] * (self.b.conj().T @ xt))
        return yt.T.reshape(nb, 2, npw)

    def __call__(self, x):
        x = np.asarray(x, dtype=np.complex128)
        self.count += x.shape[0]
        y = self.kinetic(x)
        if self.v is not None:
            y += self.local(x)
        if self.b is not None:
            y += self.nonlocal_(x)
        return y


# ---------------------------------------------------------------------------
# kinetic balance (Eq. RKB): start vectors from large components (Sec. 3.1)
# ---------------------------------------------------------------------------


def kinetic_balance(q, x, c):
    """Eq. (RKB) with p -> q = k+G and m = 1: for every column of x ([band, 4, npw] or
    [4, npw]) the small two-spinor becomes (sigma.q) phi / (2c), phi the large two-spinor
    (components 0, 1, unchanged).  Returns a new array."""
    y = np.array(x, dtype=np.complex128, copy=True)
    qx, qy, qz = q[:, 0], q[:, 1], q[:, 2]
    up, dn = y[..., 0, :], y[..., 1, :]
    y[..., 2, :] = (qz * up + (qx - 1j * qy) * dn) / (2.0 * c)
    y[..., 3, :] = ((qx + 1j * qy) * up - qz * dn) / (2.0 * c)
    return y


# ---------------------------------------------------------------------------
# filter (Eq. filter) and preconditioner (Sec. 4: Teter et al.)
# ---------------------------------------------------------------------------


def apply_filter(hop, y, cshift, omega):
    """f(H)y = (H - C)^2 y / Omega^2, as two applications of (H - C)/Omega."""
    t = (hop(y) - cshift * y) / omega
    return (hop(t) - cshift * t) / omega


def teter_factor(x):
    """Teter-Payne-Allan factor K(x) = P(x)/(P(x) + 16 x^4), P = 27 + 18x + 12x^2 + 8x^3."""
    p = 27.0 + 18.0 * x + 12.0 * x * x + 8.0 * x ** 3
    return p / (p + 16.0 * x ** 4)


def teter_precondition(q, x, r):
    """Y = K(x_G) R per band, x_G = (|q|^2/2) / T_band, T_band the kinetic energy of x."""
    ek = 0.5 * np.einsum("ij,ij->i", q, q)                   # (npw,)
    w = np.abs(x) ** 2                                        # (nb, 4, npw)
    tband = np.einsum("bap,p->b", w, ek) / np.maximum(w.sum(axis=(1, 2)), 1e-300)
    tband = np.maximum(tband, 1e-12)
    k = teter_factor(ek[None, :] / tband[:, None])            # (nb, npw)
    return k[:, None, :] * r


def filter_constants(wl, q):
    """Default shift C and scale Omega, shifted energies (readings of Sec. 3.1).

    C = midpoint of the free negative band; Omega = E_upper - C with
    E_upper = free positive maximum + max|V| + sum|D|, an upper estimate of the
    largest positive eigenvalue.
    """
    c = wl.c
    qmax = float(np.sqrt(np.einsum("ij,ij->i", q, q).max(initial=0.0)))
    emax = math.sqrt(c * c * qmax * qmax + c ** 4)
    cshift = -(3.0 * c * c + emax) / 2.0
    dsum = 0.0
    for s in range(wl.nsite):
        for l in range(int(wl.lmax[s]) + 1):
            dsum += abs(wl.d[s, l, 0]) + (abs(wl.d[s, l, 1]) if l > 0 else 0.0)
    eupper = (emax - c * c) + float(np.abs(wl.v_r).max(initial=0.0)) + dsum
    return cshift, eupper - cshift
