"""Pins for the FP64 CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a closed form of the paper
(Eq. 2 free Dirac spectrum), an invariant (Hermiticity, Kramers degeneracy,
E(k) = E(-k)), a library routine (sympy Clebsch-Gordan, scipy generalized
eigh, LAPACK zheevd), a brute-force sum, or a limit (nonrelativistic c -> oo).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import basis, davidson as dv, lobpcgf as lb, operator as op


def _setup(name, **kw):
    wl = W.make(name, **kw)
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    return wl, m, q


# ---------------------------------------------------------------- basis (Sec. 2.3)

def test_sphere_counts_brute_force():
    """Lattice-point counts by an explicit triple loop over integers (cubic: |m|^2 <= 25 -> 515)."""
    wl, m, q = _setup("cubic")
    cnt = sum(1 for a in range(-6, 7) for b in range(-6, 7) for c in range(-6, 7)
              if (2 * math.pi / 8) ** 2 * (a * a + b * b + c * c) / 2 <= 8.0)
    assert cnt == 515 == len(m)
    # canonical order: strictly increasing lexicographic Miller triples
    key = (m[:, 0] * 100 + m[:, 1]) * 100 + m[:, 2]
    assert np.all(np.diff(key) > 0)


def test_sphere_dimer_count_and_grid_fit():
    wl, m, q = _setup("dimer")
    # brute force over the box with integer arithmetic on (m/L)^2
    r, rz = np.arange(-24, 25), np.arange(-28, 29)
    a, b, c = np.meshgrid(r, r, rz, indexing="ij")
    e = 0.5 * (2 * math.pi) ** 2 * ((a / 20.0) ** 2 + (b / 20.0) ** 2 + (c / 24.0) ** 2)
    assert int((e <= 25.0).sum()) == len(m) == 57419
    with pytest.raises(ValueError):
        basis.sphere(wl.lattice, (40, 48, 56), wl.kfrac[0], 25.0)


# ---------------------------------------------------------------- free Dirac (Eq. 2)

def test_free_particle_closed_form():
    """V = 0, no projectors: spectrum is +-sqrt(c^2|q|^2 + c^4) - c^2, each twice."""
    wl, m, q = _setup("cubic", potential=False)
    h = op.dense_hamiltonian(wl, m, q)
    w = np.linalg.eigvalsh(h)
    c = wl.c
    e = np.sqrt(c * c * np.einsum("ij,ij->i", q, q) + c ** 4)
    ref = np.sort(np.concatenate([e - c * c, e - c * c, -e - c * c, -e - c * c]))
    assert np.allclose(w, ref, rtol=0, atol=1e-10 * c * c)
    # positive band relative accuracy (shifted energies are small)
    pos = w[w > -c * c]
    assert np.allclose(pos, np.sort(np.concatenate([e - c * c] * 2)), rtol=1e-10, atol=1e-9)


def test_free_particle_lobpcgf_shell():
    """LOBPCG-F on the free case returns the first closed shells: q=0 (2 states) then |q|=2pi/8 (12)."""
    wl, m, q = _setup("cubic", potential=False)
    hop = op.MatrixFreeH(wl, m, q)
    cs, om = op.filter_constants(wl, q)
    r = lb.lobpcgf(hop, q, W.start_block(len(q), 14, wl.seed), 14, cs, om, tol=1e-7)
    c = wl.c
    g = 2 * math.pi / 8
    ref = np.array([0.0] * 2 + [math.sqrt(c * c * g * g + c ** 4) - c * c] * 12)
    assert r.converged
    assert np.abs(r.lam - ref).max() < 1e-9


# ---------------------------------------------------------------- Hermiticity, equality of routes

def test_dense_hermitian_and_matrix_free_symmetric():
    wl, m, q = _setup("small")
    h = op.dense_hamiltonian(wl, m, q)
    assert np.abs(h - h.conj().T).max() < 1e-14 * np.abs(h).max()
    hop = op.MatrixFreeH(wl, m, q)
    x = W.random_block(len(q), 1, 3)
    y = W.random_block(len(q), 1, 4)
    lhs = np.vdot(y, hop(x))
    rhs = np.vdot(hop(y), x)
    assert abs(lhs - rhs) < 1e-13 * abs(np.vdot(hop(x), hop(x))) ** 0.5 * len(q)


def test_matrix_free_equals_dense_with_spin_orbit():
    """Two independent routes: dense N from the Legendre closed form, matrix-free N from
    spinor spherical harmonics (scipy Y_lm + Clebsch-Gordan); local part dense by Vhat
    wrap, matrix-free by numpy FFT."""
    for name, kf in (("small", [0.0, 0.0, 0.0]), ("small", [0.25, -0.125, 0.5])):
        wl = W.make(name, kfrac=[kf])
        m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
        h = op.dense_hamiltonian(wl, m, q)
        hop = op.MatrixFreeH(wl, m, q)
        x = W.random_block(len(q), 3, 5)
        y = hop(x)
        yd = (h @ x.reshape(3, -1).T).T.reshape(y.shape)
        assert np.abs(y - yd).max() < 1e-12 * np.abs(yd).max()


def test_local_matrix_element_brute_force():
    """<G_i|V|G_j> = (1/Ng) sum_n V(r_n) exp(-i (G_i - G_j).r_n) with explicit r_n."""
    wl, m, q = _setup("small")
    h = op.dense_hamiltonian(wl, m, q, with_nonlocal=False)
    npw = len(q)
    n1, n2, n3 = wl.grid
    fr = np.stack(np.meshgrid(np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3,
                              indexing="ij"), -1).reshape(-1, 3)
    r = fr @ wl.lattice
    brow = W.reciprocal_rows(wl.lattice)
    rng = np.random.default_rng(0)
    for _ in range(12):
        i, j = rng.integers(0, npw, 2)
        dg = (m[i] - m[j]) @ brow
        ref = np.sum(wl.v_r.reshape(-1) * np.exp(-1j * (r @ dg))) / wl.ng
        comp = rng.integers(0, 4)
        val = h[comp * npw + i, comp * npw + j]
        if i == j:
            val = val - op.dirac_block(q[i], wl.c)[comp, comp]
        assert abs(val - ref) < 1e-12


# ---------------------------------------------------------------- spin-orbit projectors (Eq. HGH)

def test_clebsch_gordan_vs_sympy():
    """Spinor harmonic coefficients against sympy's Clebsch-Gordan (library routine)."""
    from sympy import Rational, S
    from sympy.physics.quantum.cg import CG
    theta, phi = np.array([0.7]), np.array([1.3])
    for l in range(3):
        for j2 in (2 * l - 1, 2 * l + 1):
            if j2 < 0:
                continue
            for mj2 in range(-j2, j2 + 1, 2):
                om = op.spinor_harmonic(j2, l, mj2, theta, phi)[0]
                ref = np.zeros(2, complex)
                for k, ms2 in enumerate((1, -1)):
                    ml2 = mj2 - ms2
                    if abs(ml2) > 2 * l:
                        continue
                    cg = float(CG(S(l), Rational(ml2, 2), Rational(1, 2), Rational(ms2, 2),
                                  Rational(j2, 2), Rational(mj2, 2)).doit())
                    ref[k] = cg * op.sph_harm_y(l, ml2 // 2, theta, phi)[0]
                assert np.allclose(om, ref, atol=1e-14), (l, j2, mj2)


def test_spinor_harmonics_orthonormal():
    """Gauss-Legendre x uniform-phi quadrature (exact to degree 8) of Omega^H Omega'."""
    xg, wg = np.polynomial.legendre.leggauss(8)
    phis = np.arange(16) * 2 * np.pi / 16
    th, ph = np.meshgrid(np.arccos(xg), phis, indexing="ij")
    w = np.outer(wg, np.full(16, 2 * np.pi / 16)).reshape(-1)
    th, ph = th.reshape(-1), ph.reshape(-1)
    fs = []
    for l in range(3):
        for j2 in (2 * l - 1, 2 * l + 1):
            if j2 < 0:
                continue
            for mj2 in range(-j2, j2 + 1, 2):
                fs.append(op.spinor_harmonic(j2, l, mj2, th, ph))
    g = np.array([[np.sum(w * np.sum(a.conj() * b, axis=1)) for b in fs] for a in fs])
    assert np.allclose(g, np.eye(len(fs)), atol=1e-13)
    assert len(fs) == 18  # s: 2, p: 2 + 4, d: 4 + 6


def test_spin_orbit_kernel_two_routes():
    rng = np.random.default_rng(1)
    u = rng.normal(size=(6, 3))
    v = rng.normal(size=(5, 3))
    _, uu, tu, pu = op._angles(u)
    _, vv, tv, pv = op._angles(v)
    for l in range(3):
        for jj, j2 in ((0, 2 * l + 1), (1, 2 * l - 1)):
            if j2 < 0:
                continue
            s = np.zeros((6, 5, 2, 2), complex)
            for mj2 in range(-j2, j2 + 1, 2):
                a = op.spinor_harmonic(j2, l, mj2, tu, pu)
                b = op.spinor_harmonic(j2, l, mj2, tv, pv)
                s += a[:, None, :, None] * b[None, :, None, :].conj()
            assert np.abs(s - op.spin_orbit_kernel(l, jj, uu, vv)).max() < 1e-14


def test_spin_orbit_splitting_sign():
    """L.S eigenvalues: projecting the j=l+1/2 kernel onto itself gives trace 2j+1 (quadrature),
    and sum over j of kernels is (2l+1)/(4pi) P_l I2 (addition theorem)."""
    rng = np.random.default_rng(2)
    u = rng.normal(size=(4, 3))
    v = rng.normal(size=(3, 3))
    _, uu, _, _ = op._angles(u)
    _, vv, _, _ = op._angles(v)
    from scipy.special import eval_legendre
    for l in range(3):
        tot = op.spin_orbit_kernel(l, 0, uu, vv) + (op.spin_orbit_kernel(l, 1, uu, vv) if l else 0)
        ref = (2 * l + 1) / (4 * np.pi) * eval_legendre(l, np.clip(uu @ vv.T, -1, 1))
        assert np.allclose(tot[..., 0, 0], ref) and np.allclose(tot[..., 1, 1], ref)
        assert np.allclose(tot[..., 0, 1], 0) and np.allclose(tot[..., 1, 0], 0)
        # kernel at coincident points: trace = (2j+1)/(4pi)
        k = op.spin_orbit_kernel(l, 0, uu, uu)
        tr = np.einsum("iikk->i", k).real
        assert np.allclose(tr, (2 * l + 2) / (4 * np.pi))


def test_radial_normalisation():
    """sum_q |p_l(q) Y(qhat)|^2 / vol -> 1 on a fine reciprocal grid (continuum normalisation):
    with an angular factor of unit norm on the sphere, |Y|^2 averages to 1/(4 pi)."""
    for l in range(3):
        r = 0.6
        g = 2 * np.pi / 40.0
        k = np.arange(-60, 61) * g
        qx, qy, qz = np.meshgrid(k, k, k, indexing="ij")
        qn = np.sqrt(qx ** 2 + qy ** 2 + qz ** 2)
        s = np.sum(op.radial(l, r, qn) ** 2) / 40.0 ** 3
        assert abs(s / (4 * np.pi) - 1.0) < 1e-6


# ---------------------------------------------------------------- time reversal (Kramers)

def test_kramers_degeneracy_gamma():
    wl, m, q = _setup("small")
    w = np.linalg.eigvalsh(op.dense_hamiltonian(wl, m, q))
    pos = w[w > -wl.c ** 2][:40]
    assert np.abs(pos[0::2] - pos[1::2]).max() < 1e-9
    # and the spectrum is not trivially degenerate beyond pairs
    assert np.abs(pos[1:-1:2] - pos[2::2]).max() > 1e-4


def test_time_reversal_k_minus_k():
    k = [0.25, -0.125, 0.375]
    ws = []
    for kf in (k, [-x for x in k]):
        wl = W.make("small", kfrac=[kf])
        m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
        ws.append(np.linalg.eigvalsh(op.dense_hamiltonian(wl, m, q)))
    assert len(ws[0]) == len(ws[1])
    assert np.abs(ws[0] - ws[1]).max() < 1e-8
    # away from TRIM the SO coupling lifts the Kramers pairing
    pos = ws[0][ws[0] > -2e4][:20]
    assert np.abs(pos[0::2] - pos[1::2]).max() > 1e-6


# ---------------------------------------------------------------- nonrelativistic limit

def test_nonrelativistic_limit():
    """lambda(c) -> eigenvalues of |q|^2/2 + Vhat + N (2-spinor Schrodinger) with error ~ 1/c^2."""
    errs = []
    for c in (300.0, 1000.0, 3000.0):
        wl, m, q = _setup("small", c=c)
        npw = len(q)
        h = op.dense_hamiltonian(wl, m, q)
        lam = np.linalg.eigvalsh(h)
        lam = lam[lam > -c * c][:6]
        hd = op.dense_hamiltonian(wl, m, q, with_local=True, with_nonlocal=True)
        # Schrodinger 2-spinor operator built from the same pieces, independently of c
        hs = np.zeros((2 * npw, 2 * npw), complex)
        ek = 0.5 * np.einsum("ij,ij->i", q, q)
        hs[np.arange(2 * npw), np.arange(2 * npw)] = np.concatenate([ek, ek])
        hs += hd[:2 * npw, :2 * npw]          # large-large block: Vhat + N (Dirac part is 0 there)
        ls = np.linalg.eigvalsh(hs)[:6]
        errs.append(np.abs(lam - ls).max())
        # the KSSO oracle operator is this limit
        lk = np.linalg.eigvalsh(op.dense_hamiltonian_ksso(wl, m, q))[:6]
        assert np.abs(lk - ls).max() < 1e-10
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 8.0 < r1 < 13.0 and 7.0 < r2 < 11.0, errs   # (c ratio)^2 = 11.1, 9
    assert errs[2] < 1e-4


# ---------------------------------------------------------------- KSSO operator (Sec. 4)

def test_ksso_free_particle_closed_form():
    """V = 0, no projectors: the KSSO spectrum is |q|^2/2, each twice (spin)."""
    wl, m, q = _setup("cubic", potential=False)
    w = np.linalg.eigvalsh(op.dense_hamiltonian_ksso(wl, m, q))
    ek = 0.5 * np.einsum("ij,ij->i", q, q)
    assert np.allclose(w, np.sort(np.concatenate([ek, ek])), rtol=1e-13, atol=1e-13)


def test_ksso_matrix_free_equals_dense_and_hermitian():
    """Matrix-free KSSO (numpy FFT, spinor-harmonic projectors) against the dense matrix (Vhat
    wrap, Legendre closed form); the dense matrix is Hermitian and, at Gamma, Kramers-paired."""
    for kf in ([0.0, 0.0, 0.0], [0.25, -0.125, 0.5]):
        wl = W.make("small", kfrac=[kf])
        m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
        h = op.dense_hamiltonian_ksso(wl, m, q)
        assert np.abs(h - h.conj().T).max() < 1e-14 * np.abs(h).max()
        hop = op.MatrixFreeKSSO(wl, m, q)
        x = W.random_block(len(q), 3, 6, ncomp=2)
        y = hop(x)
        yd = (h @ x.reshape(3, -1).T).T.reshape(y.shape)
        assert np.abs(y - yd).max() < 1e-12 * np.abs(yd).max()
    wl, m, q = _setup("small")
    w = np.linalg.eigvalsh(op.dense_hamiltonian_ksso(wl, m, q))[:40]
    assert np.abs(w[0::2] - w[1::2]).max() < 1e-10
    assert np.abs(w[1:-1:2] - w[2::2]).max() > 1e-4


def test_ksso_lobpcg_matches_dense():
    """Algorithm 1 without the filter (standard LOBPCG, the KSSO module's solver) on the KSSO
    operator reaches the lowest dense eigenvalues."""
    wl, m, q = _setup("small")
    hop = op.MatrixFreeKSSO(wl, m, q)
    ref = np.linalg.eigvalsh(op.dense_hamiltonian_ksso(wl, m, q))[:8]
    x0 = W.start_block(len(q), 12, wl.seed, ncomp=2)
    res = lb.lobpcgf(hop, q, x0, 12, 0.0, 1.0, tol=1e-8, n_iter=300, nconv=8, use_filter=False)
    assert res.converged
    assert np.abs(res.lam[:8] - ref).max() < 1e-8


# ---------------------------------------------------------------- filter (Eq. filter) and Teter

def test_filter_identity_dense():
    wl, m, q = _setup("small")
    h = op.dense_hamiltonian(wl, m, q)
    hop = op.MatrixFreeH(wl, m, q)
    cs, om = op.filter_constants(wl, q)
    y = W.random_block(len(q), 2, 9)
    fy = op.apply_filter(hop, y, cs, om)
    hc = h - cs * np.eye(h.shape[0])
    ref = (hc @ (hc @ y.reshape(2, -1).T)).T.reshape(y.shape) / om ** 2
    assert np.abs(fy - ref).max() < 1e-12 * np.abs(ref).max()


def test_filter_suppression_ratio():
    """Sec. 3.1: f(E) = (E-C)^2/Omega^2 maps the positive band near 1 (<= 1 at the top) and the
    negative band to at most (w-/Omega)^2; relative suppression ~ (w/Delta)^2."""
    wl, m, q = _setup("cubic")
    w = np.linalg.eigvalsh(op.dense_hamiltonian(wl, m, q))
    cs, om = op.filter_constants(wl, q)
    f = (w - cs) ** 2 / om ** 2
    c2 = wl.c ** 2
    pos, neg = f[w > -c2], f[w < -c2]
    assert pos.max() <= 1.0 + 1e-12 and pos.min() > 0.99
    wneg = w[w < -c2].max() - w[w < -c2].min()
    assert w[w < -c2].min() < cs < w[w < -c2].max()      # C lies inside the negative band
    assert neg.max() <= (wneg / om) ** 2                  # so |E - C| <= w on that band
    assert neg.max() / pos.min() < 1e-6


def test_kinetic_balance_free_positive_eigenvector():
    """Eq. (RKB) against the exact positive-energy eigenvector of the free Dirac block: its small
    two-spinor is c (sigma.q) phi / (E + c^2), E = sqrt(c^2 q^2 + c^4), so the kinetic-balance
    vector differs from it by the factor 2c^2 / (E + c^2) = 1 - q^2/(4c^2) + O(q^4/c^4)."""
    rng = np.random.default_rng(11)
    for c in (137.036, 20.0):
        for _ in range(6):
            qv = rng.normal(size=3) * rng.uniform(0.2, 3.0)
            h = op.dirac_block(qv, c)
            lam, vec = np.linalg.eigh(h)
            for k in (2, 3):                                  # the two positive-energy states
                v = vec[:, k]
                x = np.zeros((4, 1), dtype=np.complex128)
                x[0:2, 0] = v[0:2]
                kb = op.kinetic_balance(qv[None, :], x, c)[2:4, 0]
                e = lam[k] + c * c                                 # unshifted energy
                assert math.isclose(e, math.sqrt(c * c * (qv @ qv) + c ** 4), rel_tol=1e-12)
                ratio = 2.0 * c * c / (e + c * c)
                assert np.allclose(v[2:4], ratio * kb, rtol=0, atol=1e-12 * np.abs(v).max())


def test_kinetic_balance_rayleigh_quotient_closed_form():
    """For psi = [phi, (sigma.q) phi/(2c)] the shifted free Dirac block gives the Rayleigh quotient
    (q^2/2) / (1 + q^2/(4c^2)) exactly ((sigma.q)^2 = q^2): the nonrelativistic kinetic energy
    in the limit.  Also |chi|^2 = q^2 |phi|^2 / (4c^2) per planewave."""
    rng = np.random.default_rng(12)
    c = 137.036
    q = rng.normal(size=(7, 3)) * 2.0
    x = rng.normal(size=(3, 4, 7)) + 1j * rng.normal(size=(3, 4, 7))
    y = op.kinetic_balance(q, x, c)
    assert np.array_equal(y[:, 0:2], x[:, 0:2])
    q2 = np.einsum("ij,ij->i", q, q)
    np.testing.assert_allclose((np.abs(y[:, 2:4]) ** 2).sum(axis=1),
                               q2 * (np.abs(x[:, 0:2]) ** 2).sum(axis=1) / (4 * c * c), rtol=1e-13)
    for b in range(3):
        for p in range(7):
            psi = y[b, :, p]
            rq = (psi.conj() @ op.dirac_block(q[p], c) @ psi).real / (psi.conj() @ psi).real
            assert math.isclose(rq, 0.5 * q2[p] / (1 + q2[p] / (4 * c * c)), rel_tol=1e-12)


def test_teter_factor_limits():
    """Teter-Payne-Allan design: K = 1 - O(x^4) near 0 (flat to third order) and K ~ 1/(2x)."""
    x = np.array([1e-3, 2e-3])
    k = op.teter_factor(x)
    assert np.allclose((1 - k) / x ** 4, 16.0 / 27.0, rtol=1e-2)
    big = np.array([1e4, 1e5])
    assert np.allclose(op.teter_factor(big) * 2 * big, 1.0, rtol=2e-3)
    xs = np.linspace(0, 50, 1001)
    assert np.all(np.diff(op.teter_factor(xs)) < 0)


def test_teter_factor_published_values():
    """K(x) at exact rational points worked out by hand from the Teter-Payne-Allan polynomial
    (tests/golden/teter_factor_values.txt): pins every coefficient, 18 and 12 included -- a
    changed coefficient moves K(1) = 65/81 or K(3/2) = 4/7."""
    path = os.path.join(os.path.dirname(__file__), "golden", "teter_factor_values.txt")
    vals = np.loadtxt(path, comments="#")
    assert vals.shape[0] >= 5
    for xn, xd, kn, kd in vals:
        assert abs(op.teter_factor(xn / xd) - kn / kd) < 1e-15


def test_teter_precondition_brute_force():
    wl, m, q = _setup("small")
    npw = len(q)
    x = W.random_block(npw, 2, 11)
    r = W.random_block(npw, 2, 12)
    y = op.teter_precondition(q, x, r)
    for b in range(2):
        num = sum(0.5 * float(q[p] @ q[p]) * abs(x[b, a, p]) ** 2 for a in range(4) for p in range(npw))
        den = sum(abs(x[b, a, p]) ** 2 for a in range(4) for p in range(npw))
        t = num / den
        for p in (0, 7, npw - 1):
            xx = 0.5 * float(q[p] @ q[p]) / t
            pp = 27 + 18 * xx + 12 * xx ** 2 + 8 * xx ** 3
            assert np.allclose(y[b, :, p], r[b, :, p] * pp / (pp + 16 * xx ** 4))


# ---------------------------------------------------------------- Rayleigh-Ritz and Algorithm 1

def test_rayleigh_ritz_vs_scipy():
    rng = np.random.default_rng(5)
    n = 24
    b = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    s = b.conj().T @ b + 0.1 * np.eye(n)
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    a = a + a.conj().T
    lam, v, info = lb.rayleigh_ritz(a, s, 7)
    ref = sla.eigh(a, s, eigvals_only=True)[:7]
    assert not info.svqb
    assert np.allclose(lam, ref, atol=1e-10)
    assert np.allclose(v.conj().T @ s @ v, np.eye(7), atol=1e-10)
    assert np.abs(a @ v - s @ v * lam).max() < 1e-9


def test_rayleigh_ritz_svqb_rank_deficient():
    """S singular (a repeated column): SVQB drops the null direction; the result is the pencil on range(S)."""
    rng = np.random.default_rng(6)
    nn, k = 200, 12
    z = rng.normal(size=(nn, k)) + 1j * rng.normal(size=(nn, k))
    z[:, 5] = z[:, 2] * 2.0
    hm = rng.normal(size=(nn, nn)) + 1j * rng.normal(size=(nn, nn))
    hm = hm + hm.conj().T
    lam, v, info = lb.rayleigh_ritz(z.conj().T @ hm @ z, z.conj().T @ z, 4)
    assert info.svqb and info.rank == k - 1
    zq = np.delete(z, 5, axis=1)
    ref = sla.eigh(zq.conj().T @ hm @ zq, zq.conj().T @ zq, eigvals_only=True)[:4]
    assert np.allclose(lam, ref, atol=1e-8)


def test_lobpcgf_matches_dense_definition():
    """Algorithm 1 result == lowest nev dense eigenvalues above the gap midpoint (no negative state)."""
    wl, m, q = _setup("cubic")
    h = op.dense_hamiltonian(wl, m, q)
    lam_ref, u, w = lb.dense_eigs(h, wl.c, 8)
    hop = op.MatrixFreeH(wl, m, q)
    cs, om = op.filter_constants(wl, q)
    r = lb.lobpcgf(hop, q, W.start_block(len(q), 8, wl.seed), 8, cs, om, tol=1e-6)
    assert r.converged and np.all(r.resnorms < 1e-6)
    assert np.all(r.lam > -wl.c ** 2)
    assert np.abs(r.lam - lam_ref).max() < 1e-8
    # 3 H applications per active column per iteration (Sec. 3.2) + 3 initial filters (2 each) + 1
    assert r.h_applications == 8 * (3 * 2 + 1) + 3 * sum(h["nact"] for h in r.history)
    # eigenvectors: subspace of each degenerate cluster
    x = r.x.reshape(8, -1).T
    x = x / np.linalg.norm(x, axis=0)
    sv = np.linalg.svd(u.conj().T @ x, compute_uv=False)
    assert sv.min() > 1 - 1e-9


@pytest.mark.parametrize("c", [39.0, 137.036])
def test_standard_lobpcg_collapses_lobpcgf_does_not(c):
    """Sec. 3.1: without the filter, negative-band error grows ~Delta/w per iteration and LOBPCG
    collapses into the negative band; LOBPCG-F returns the positive-band states."""
    wl, m, q = _setup("cubic", c=c)
    hop = op.MatrixFreeH(wl, m, q)
    cs, om = op.filter_constants(wl, q)
    x0 = W.start_block(len(q), 8, wl.seed)
    lam_ref, _, _ = lb.dense_eigs(op.dense_hamiltonian(wl, m, q), c, 8)
    plain = lb.lobpcgf(hop, q, x0, 8, cs, om, tol=1e-6, n_iter=60, use_filter=False, precond="identity")
    assert plain.lam.min() < -c * c          # collapsed below the gap midpoint
    filt = lb.lobpcgf(hop, q, x0, 8, cs, om, tol=1e-6, n_iter=60, precond="identity")
    assert filt.converged and np.abs(filt.lam - lam_ref).max() < 1e-8


# ---------------------------------------------------------------- Davidson-F (Sec. 3: filter in other solvers)

def test_davidson_f_orthonormal_basis():
    """SVQB basis: orthonormal, same span, dependent columns dropped."""
    rng = np.random.default_rng(5)
    t = rng.normal(size=(50, 6)) + 1j * rng.normal(size=(50, 6))
    t[:, 5] = 2.0 * t[:, 0] - 1j * t[:, 3]
    b = dv.orthonormal_basis(t)
    assert b.shape[1] == 5
    assert np.abs(b.conj().T @ b - np.eye(5)).max() < 1e-13
    proj = b @ (b.conj().T @ t)
    assert np.abs(proj - t).max() < 1e-12 * np.abs(t).max()


def test_davidson_f_matches_dense_definition():
    """Davidson-F reaches the lowest nev dense eigenvalues above the gap midpoint, on the local-only
    cubic case and on the spin-orbit case, with three H applications per active column per
    iteration."""
    for name, nev in (("cubic", 8), ("small", 6)):
        wl, m, q = _setup(name)
        lam_ref, _, _ = lb.dense_eigs(op.dense_hamiltonian(wl, m, q), wl.c, nev)
        hop = op.MatrixFreeH(wl, m, q)
        cs, om = op.filter_constants(wl, q)
        r = dv.davidson_f(hop, q, W.start_block(len(q), nev + 2, wl.seed), nev + 2, cs, om, tol=1e-7,
                          nconv=nev, n_iter=300)
        assert r.converged and np.all(r.lam > -wl.c ** 2)
        assert np.abs(r.lam[:nev] - lam_ref).max() < 1e-8


def test_davidson_f_h_count():
    """Like LOBPCG-F (Sec. 3.2), Davidson-F applies H' three times per new direction: twice in the
    filter and once to extend HV; plus 2 n N_init for the initial filtering and n for HV0."""
    wl, m, q = _setup("cubic")
    hop = op.MatrixFreeH(wl, m, q)
    cs, om = op.filter_constants(wl, q)
    r = dv.davidson_f(hop, q, W.start_block(len(q), 8, wl.seed), 8, cs, om, tol=1e-6)
    assert r.converged
    filt = sum(2 * h["nact"] for h in r.history if "added" in h)
    ext = sum(h["added"] for h in r.history if "added" in h)
    assert r.h_applications == 2 * 8 * 3 + 8 + filt + ext
    assert ext == sum(h["nact"] for h in r.history if "added" in h)   # no direction dropped here


@pytest.mark.parametrize("c", [39.0, 137.036])
def test_davidson_without_filter_collapses(c):
    """The filter protects Davidson as it protects LOBPCG (Sec. 3.1 mechanism): without it the
    basis picks up negative-band directions and the iteration returns states below the gap."""
    wl, m, q = _setup("cubic", c=c)
    hop = op.MatrixFreeH(wl, m, q)
    cs, om = op.filter_constants(wl, q)
    x0 = W.start_block(len(q), 8, wl.seed)
    lam_ref, _, _ = lb.dense_eigs(op.dense_hamiltonian(wl, m, q), c, 8)
    plain = dv.davidson_f(hop, q, x0, 8, cs, om, tol=1e-6, n_iter=60, use_filter=False, precond="identity")
    assert plain.lam.min() < -c * c
    filt = dv.davidson_f(hop, q, x0, 8, cs, om, tol=1e-6, n_iter=120, precond="identity")
    assert filt.converged and np.abs(filt.lam - lam_ref).max() < 1e-8


def test_golden_cubic_dense_eigs():
    """Stored dense eigenvalues (tests/golden/make_golden.py, oracle only) still reproduce."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "cubic_dense_eigs.txt")
    ref = np.loadtxt(path)
    wl, m, q = _setup("cubic")
    lam, _, _ = lb.dense_eigs(op.dense_hamiltonian(wl, m, q), wl.c, 8)
    assert np.abs(lam - ref).max() < 1e-10


# ---------------------------------------------------------------- band blocks with deflation

@pytest.mark.parametrize("n,block,nbuf", [(20, 8, 4), (14, 7, 2)])
def test_blocked_lobpcgf_matches_dense(n, block, nbuf):
    """Algorithm 1 on band blocks deflated against the earlier blocks gives the n lowest dense
    eigenvalues above the gap (block 7 puts a block edge inside a Kramers pair), with orthonormal
    vectors that satisfy the eigen-equation of the dense matrix."""
    wl, m, q = _setup("small", ecut=4.0)
    hop = op.MatrixFreeH(wl, m, q)
    cs, om = op.filter_constants(wl, q)
    x0 = W.start_block(len(m), n + 3 * nbuf + block, wl.seed)
    res = lb.lobpcgf_blocked(hop, q, x0, n, block, cs, om, nbuf=nbuf, tol=1e-8)
    h = op.dense_hamiltonian(wl, m, q)
    ref, _, _ = lb.dense_eigs(h, wl.c, n)
    assert res.converged and np.abs(res.lam - ref).max() < 1e-9
    x = res.x.reshape(n, -1).T
    assert np.abs(x.conj().T @ x - np.eye(n)).max() < 1e-12
    assert np.abs(h @ x - x * res.lam[None, :]).max() < 1e-7


def test_blocked_lobpcgf_one_block_is_algorithm_1():
    """With one block holding every wanted pair, the blocked form is lobpcgf() itself."""
    wl, m, q = _setup("small", ecut=4.0)
    cs, om = op.filter_constants(wl, q)
    x0 = W.start_block(len(m), 8, wl.seed)
    a = lb.lobpcgf(op.MatrixFreeH(wl, m, q), q, x0, 8, cs, om, tol=1e-8)
    b = lb.lobpcgf_blocked(op.MatrixFreeH(wl, m, q), q, x0, 8, 8, cs, om, tol=1e-8)
    assert a.iterations == b.iterations and np.abs(a.lam - b.lam).max() < 1e-13


def test_blocked_lobpcg_ksso_matches_dense():
    """Band blocks on the two-component KSSO operator (standard LOBPCG, no filter): the lowest
    dense eigenvalues of the KSSO matrix."""
    wl, m, q = _setup("small", ecut=4.0)
    hop = op.MatrixFreeKSSO(wl, m, q)
    x0 = W.start_block(len(m), 30, wl.seed, ncomp=2)
    res = lb.lobpcgf_blocked(hop, q, x0, 16, 6, 0.0, 1.0, nbuf=2, tol=1e-8, use_filter=False)
    ref = np.linalg.eigvalsh(op.dense_hamiltonian_ksso(wl, m, q))[:16]
    assert res.converged and np.abs(res.lam - ref).max() < 1e-9


def test_lobpcgf_eigenvectors_match_dense_subspaces():
    """Eigenvectors of Algorithm 1 against the dense ones, compared per cluster as subspaces
    (largest principal-angle sine): at residual tol the sines are of order tol / gap."""
    from tests._helpers import cluster_sines
    wl, m, q = _setup("cubic", ecut=4.0)
    h = op.dense_hamiltonian(wl, m, q)
    lam, u, _ = lb.dense_eigs(h, wl.c, 8)
    cs, om = op.filter_constants(wl, q)
    res = lb.lobpcgf(op.MatrixFreeH(wl, m, q), q, W.start_block(len(m), 10, wl.seed), 10, cs, om, tol=1e-8, nconv=8)
    x = res.x.reshape(10, -1).T[:, :8]
    assert np.abs(res.lam[:8] - lam).max() < 1e-9
    assert cluster_sines(lam, u, x) < 1e-4          # tol / gap with the 2.3e-4 Ha p-level splitting
    # a wrong vector in a cluster is seen: swap in a vector of another cluster
    xb = x.copy()
    xb[:, 0] = u[:, 5]
    assert cluster_sines(lam, u, xb) > 0.5


def test_davidson_ksso_matches_dense():
    """The oracle's block Davidson on the two-component KSSO operator (no filter, as the KSSO
    module has no negative continuum) gives its lowest dense eigenvalues."""
    wl, m, q = _setup("small", ecut=4.0)
    hop = op.MatrixFreeKSSO(wl, m, q)
    x0 = W.start_block(len(m), 8, wl.seed, ncomp=2)
    res = dv.davidson_f(hop, q, x0, 8, 0.0, 1.0, tol=1e-8, use_filter=False, nconv=6)
    ref = np.linalg.eigvalsh(op.dense_hamiltonian_ksso(wl, m, q))[:6]
    assert res.converged and np.abs(res.lam[:6] - ref).max() < 1e-9
