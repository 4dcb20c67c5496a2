"""Algorithm 1 (LOBPCG-F) in plain FP64 numpy, and the dense-matrix definition.

The iteration follows Algorithm 1 step by step with X^T -> X^H (complex data):

  1. X0 <- f(H) X0, N_init times (the underlined initial filtering).
  2. Rayleigh-Ritz on X0: (X0^H H X0) V = (X0^H X0) V Lambda, ascending.
  3. X <- X0 V, R <- H X - X Lambda, P <- [].
  4. loop: Y from T Y = R (Teter factor), Y <- f(H) Y (underlined filter),
     Z = [X, Y, P], Rayleigh-Ritz on Z keeping the first n Ritz pairs,
     X <- Z V, R <- H X - X Lambda, stop when every column norm < eps,
     keep only the columns of R (and V) with norm > eps, P <- [0, Y, P] V.

H X is carried by the same rotation as X (H Z V), so each iteration applies H
three times (two for the filter, one for H Y), as Sec. 3.2 states.

The generalized eigenproblems are solved after the diagonal scaling of S
(reading of the Rayleigh-Ritz steps, where the paper gives no orthonormalisation detail):
Cholesky of the scaled S when its smallest pivot is safely positive, otherwise
SVQB (eigen-decomposition of S, directions with eigenvalue below drop_tol times
the largest are discarded).

``dense_eigs`` is the plain definition of the result: all eigenvalues of the
dense H' (zheevd), keeping the nev lowest above the gap midpoint (-c^2 in the
shifted units, E = 0 unshifted).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from .operator import apply_filter, teter_precondition


@dataclasses.dataclass
class RRInfo:
    svqb: bool
    rank: int


def rayleigh_ritz(a, s, n, drop_tol=1e-12, chol_tol=1e-12):
    """Lowest n pairs of A v = lambda S v (A, S Hermitian, S PSD). Returns (lam, V, info)."""
    a = 0.5 * (a + a.conj().T)
    s = 0.5 * (s + s.conj().T)
    d = 1.0 / np.sqrt(np.real(np.diag(s)))
    a1 = d[:, None] * a * d[None, :]
    s1 = d[:, None] * s * d[None, :]
    use_svqb = False
    try:
        l = np.linalg.cholesky(s1)
        if np.min(np.real(np.diag(l))) ** 2 < chol_tol:
            use_svqb = True
    except np.linalg.LinAlgError:
        use_svqb = True
    if not use_svqb:
        t = sla.solve_triangular(l, a1, lower=True)                      # L^-1 A
        c = sla.solve_triangular(l, t.conj().T, lower=True).conj().T       # L^-1 A L^-H
        c = 0.5 * (c + c.conj().T)
        lam, u = np.linalg.eigh(c)
        v = sla.solve_triangular(l.conj().T, u, lower=False)              # L^-H U
        rank = s.shape[0]
    else:
        w, u = np.linalg.eigh(s1)
        keep = w > drop_tol * w.max()
        qm = u[:, keep] / np.sqrt(w[keep])[None, :]
        c = qm.conj().T @ a1 @ qm
        c = 0.5 * (c + c.conj().T)
        lam, u2 = np.linalg.eigh(c)
        v = qm @ u2
        rank = int(keep.sum())
    if v.shape[1] < n:
        raise np.linalg.LinAlgError("subspace rank below the block size")
    v = d[:, None] * v
    return lam[:n], v[:, :n], RRInfo(use_svqb, rank)


@dataclasses.dataclass
class SolveResult:
    lam: np.ndarray
    x: np.ndarray
    iterations: int
    converged: bool
    resnorms: np.ndarray
    history: list
    h_applications: int


def _cols(blk):
    """[band, comp, pw] -> (4 npw, nb) column matrix."""
    return blk.reshape(blk.shape[0], -1).T


def _blk(mat, npw, ncomp=4):
    return mat.T.reshape(mat.shape[1], ncomp, npw)


def lobpcgf(hop, q, x0, n, cshift, omega, n_init=3, n_iter=200, tol=1e-6, nconv=None,
            use_filter=True, precond="teter", callback=None):
    """Algorithm 1.  hop: x[nb,ncomp,npw] -> H'x (ncomp = 4 four-spinors; 2 for the KSSO operator,
    run with use_filter=False).  Returns SolveResult (lam ascending, x[n,ncomp,npw])."""
    npw = q.shape[0]
    nc = np.asarray(x0).shape[1]
    nconv = n if nconv is None else nconv
    start = hop.count if hasattr(hop, "count") else 0

    def fh(y):
        return apply_filter(hop, y, cshift, omega) if use_filter else y

    def tinv(xb, rb):
        if precond == "teter":
            return teter_precondition(q, xb, rb)
        return rb.copy()

    x = np.array(x0, dtype=np.complex128)
    for _ in range(n_init if use_filter else 0):          # initial filtering
        x = fh(x)
    hx = hop(x)
    xm, hxm = _cols(x), _cols(hx)
    lam, v, _ = rayleigh_ritz(xm.conj().T @ hxm, xm.conj().T @ xm, n)   # first Rayleigh-Ritz
    xm, hxm = xm @ v, hxm @ v                                           # X, HX rotated
    rm = hxm - xm * lam[None, :]                                        # residual
    act = np.arange(n)
    pm = hpm = None                                                     # no search block yet
    history = []
    norms = np.linalg.norm(rm, axis=0)
    converged = False
    it = 0
    for it in range(1, n_iter + 1):                                     # iteration
        yb = tinv(_blk(xm[:, act], npw, nc), _blk(rm, npw, nc))         # preconditioned residual
        yb = fh(yb)                                                     # filter
        ym = _cols(yb)
        hym = _cols(hop(yb))
        zm = np.hstack([xm, ym] + ([pm] if pm is not None else []))     # subspace Z
        hzm = np.hstack([hxm, hym] + ([hpm] if hpm is not None else []))
        lam, v, info = rayleigh_ritz(zm.conj().T @ hzm, zm.conj().T @ zm, n)   # Rayleigh-Ritz
        xm, hxm = zm @ v, hzm @ v                                       # X, HX rotated
        rm = hxm - xm * lam[None, :]                                    # residual
        norms = np.linalg.norm(rm, axis=0)
        history.append(dict(it=it, max_res=float(norms[:nconv].max()), nz=zm.shape[1],
                            nact=len(act), svqb=info.svqb, lam=lam.copy()))
        if callback is not None:
            callback(it, lam, norms)
        if np.all(norms[:nconv] < tol):                                 # convergence test
            converged = True
            break
        act = np.nonzero(norms > tol)[0]                                # soft locking
        rm = rm[:, act]
        va = v[n:, act]                                                 # coefficients of the active columns
        pm, hpm = zm[:, n:] @ va, hzm[:, n:] @ va                       # P <- [0, Y, P] V
    used = (hop.count - start) if hasattr(hop, "count") else -1
    return SolveResult(lam=lam, x=_blk(xm, npw, nc), iterations=it, converged=converged,
                       resnorms=norms, history=history, h_applications=used)


def dense_eigs(h, c, nev):
    """Lowest nev eigenpairs of the dense shifted H' above the gap midpoint -c^2."""
    w, u = np.linalg.eigh(h)
    pos = np.nonzero(w > -c * c)[0]
    sel = pos[:nev]
    return w[sel], u[:, sel], w


def _project_out(qm, ym):
    """Y <- Y - Q (Q^H Y), twice (classical Gram-Schmidt with one reorthogonalisation)."""
    if qm is None or qm.shape[1] == 0:
        return ym
    for _ in range(2):
        ym = ym - qm @ (qm.conj().T @ ym)
    return ym


def lobpcgf_blocked(hop, q, x0, n, block, cshift, omega, nbuf=0, n_init=3, n_iter=200, tol=1e-6,
                    use_filter=True, precond="teter"):
    """Algorithm 1 on band blocks, for more wanted pairs than one block can hold (reading of a
    large-cell configuration: bands of at most `block` wanted columns, each block deflated
    against the converged earlier ones).

    Block b wants the pairs b*block .. min(n, (b+1)*block) - 1 and iterates them with nbuf
    buffer columns above them (not convergence-checked).  Its start block is the previous
    block's buffer columns followed by unused columns of x0; every block that enters the
    subspace -- the filtered start block and every filtered correction Y -- has the span of
    the locked vectors Q (all earlier blocks' converged columns) projected out, so the block
    converges to the next pairs above them.  Each block is otherwise Algorithm 1 as in
    lobpcgf().  Returns SolveResult with the n eigenvalues in ascending block order."""
    npw = q.shape[0]
    x0 = np.array(x0, dtype=np.complex128)
    nc = x0.shape[1]
    start = hop.count if hasattr(hop, "count") else 0

    def fh(y):
        return apply_filter(hop, y, cshift, omega) if use_filter else y

    def tinv(xb, rb):
        if precond == "teter":
            return teter_precondition(q, xb, rb)
        return rb.copy()

    qm = None                                   # locked vectors, columns
    lams, history = [], []
    pool = [x0[j] for j in range(x0.shape[0])]  # unused start columns
    carry = []                                  # buffer columns of the previous block
    iterations, converged = 0, True
    nblk = (n + block - 1) // block
    for b in range(nblk):
        nw = min(block, n - b * block)
        m = nw + nbuf
        cols = carry[:m]
        while len(cols) < m:
            if not pool:
                raise ValueError("x0 has too few columns for the blocks")
            cols.append(pool.pop(0))
        x = np.stack(cols)
        for _ in range(n_init if use_filter else 0):
            x = fh(x)
        xm = _project_out(qm, _cols(x))
        hxm = _cols(hop(_blk(xm, npw, nc)))
        lam, v, _ = rayleigh_ritz(xm.conj().T @ hxm, xm.conj().T @ xm, m)
        xm, hxm = xm @ v, hxm @ v
        rm = hxm - xm * lam[None, :]
        act = np.arange(m)
        pm = hpm = None
        norms = np.linalg.norm(rm, axis=0)
        ok = False
        for it in range(1, n_iter + 1):
            yb = fh(tinv(_blk(xm[:, act], npw, nc), _blk(rm, npw, nc)))
            ym = _project_out(qm, _cols(yb))
            hym = _cols(hop(_blk(ym, npw, nc)))
            zm = np.hstack([xm, ym] + ([pm] if pm is not None else []))
            hzm = np.hstack([hxm, hym] + ([hpm] if hpm is not None else []))
            lam, v, info = rayleigh_ritz(zm.conj().T @ hzm, zm.conj().T @ zm, m)
            xm, hxm = zm @ v, hzm @ v
            rm = hxm - xm * lam[None, :]
            norms = np.linalg.norm(rm, axis=0)
            history.append(dict(block=b, it=it, max_res=float(norms[:nw].max()), nz=zm.shape[1]))
            if np.all(norms[:nw] < tol):
                ok = True
                break
            act = np.nonzero(norms > tol)[0]
            rm = rm[:, act]
            va = v[m:, act]
            pm, hpm = zm[:, m:] @ va, hzm[:, m:] @ va
        iterations += it
        converged = converged and ok
        lams.append(lam[:nw])
        qm = xm[:, :nw] if qm is None else np.hstack([qm, xm[:, :nw]])
        carry = [c for c in _blk(xm[:, nw:], npw, nc)]
    used = (hop.count - start) if hasattr(hop, "count") else -1
    return SolveResult(lam=np.concatenate(lams), x=_blk(qm, npw, nc), iterations=iterations,
                       converged=converged, resnorms=None, history=history, h_applications=used)
