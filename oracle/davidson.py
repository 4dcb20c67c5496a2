"""Block Davidson with the filter step of LOBPCG-F ("Davidson-F"), plain FP64 numpy.

Test infrastructure (the oracle): plain, slow and written to be read against the reading below;
it shares no code with the CUDA path.

The paper remarks (Sec. 3, where LOBPCG-F is introduced, and again in the conclusion) that the
filtering step applies to other preconditioned iterative solvers such as Davidson-type methods,
without giving such an algorithm.  The reading implemented here keeps everything of Algorithm 1
that is not specific to LOBPCG -- the N_init initial filter steps, the Teter factor on the
residuals of the active columns, the filter f(H) = (H - C)^2 / Omega^2 on every new direction,
the Rayleigh-Ritz selection of the first n pairs, the soft-locking test -- and replaces the
three-block subspace [X, Y, P] by a growing orthonormal basis V:

  1. X0 <- f(H) X0, N_init times; V <- an orthonormal basis of X0; HV <- H V.
  2. loop:
       Rayleigh-Ritz on V (the pencil (V^H H V, V^H V)), first n pairs: X <- V C, HX <- HV C,
       R <- HX - X Theta; stop when the first nconv column norms are below eps;
       T <- K(R) on the columns with norm above eps (Teter factor), T <- f(H) T;
       restart when V would exceed m_max columns: V <- X, HV <- HX;
       T <- T - V (V^H T), twice (classical Gram-Schmidt with one reorthogonalisation);
       T <- an orthonormal basis of T; V <- [V, T], HV <- [HV, H T].
Each iteration applies H three times per active column (two for the filter), as LOBPCG-F does.
"""
from __future__ import annotations

import numpy as np

from .lobpcgf import SolveResult, _blk, _cols, rayleigh_ritz
from .operator import apply_filter, teter_precondition


def orthonormal_basis(t, drop_tol=1e-12):
    """Columns spanning the same space as t, orthonormal: SVQB (eigen-decomposition of the
    diagonally scaled Gram matrix; directions below drop_tol times the largest are dropped)."""
    g = t.conj().T @ t
    g = 0.5 * (g + g.conj().T)
    d = 1.0 / np.sqrt(np.maximum(np.real(np.diag(g)), 1e-300))
    w, u = np.linalg.eigh(d[:, None] * g * d[None, :])
    keep = w > drop_tol * w.max()
    return t @ (d[:, None] * u[:, keep] / np.sqrt(w[keep])[None, :])


def davidson_f(hop, q, x0, n, cshift, omega, n_init=3, n_iter=200, tol=1e-6, nconv=None,
               use_filter=True, precond="teter", m_max=None):
    """Davidson-F as read above.  hop: x[nb, ncomp, npw] -> Hx.  m_max: largest basis (default 4n)."""
    npw = q.shape[0]
    nc = np.asarray(x0).shape[1]
    nconv = n if nconv is None else nconv
    m_max = 4 * n if m_max is None else m_max
    start = hop.count if hasattr(hop, "count") else 0

    def fh(y):
        return apply_filter(hop, y, cshift, omega) if use_filter else y

    x = np.array(x0, dtype=np.complex128)
    for _ in range(n_init if use_filter else 0):
        x = fh(x)
    v = orthonormal_basis(_cols(x))
    hv = _cols(hop(_blk(v, npw, nc)))
    history = []
    converged = False
    it = 0
    lam = norms = xm = None
    for it in range(1, n_iter + 1):
        lam, cm, info = rayleigh_ritz(v.conj().T @ hv, v.conj().T @ v, n)
        xm, hxm = v @ cm, hv @ cm
        rm = hxm - xm * lam[None, :]
        norms = np.linalg.norm(rm, axis=0)
        act = np.nonzero(norms > tol)[0]
        history.append(dict(it=it, max_res=float(norms[:nconv].max()), m=v.shape[1], lam=lam.copy(),
                            nact=len(act)))
        if np.all(norms[:nconv] < tol):
            converged = True
            break
        xb, rb = _blk(xm[:, act], npw, nc), _blk(rm[:, act], npw, nc)
        t = _cols(fh(teter_precondition(q, xb, rb) if precond == "teter" else rb.copy()))
        if v.shape[1] + t.shape[1] > m_max:
            v, hv = xm, hxm
        for _ in range(2):
            t = t - v @ (v.conj().T @ t)
        t = orthonormal_basis(t)
        history[-1]["added"] = t.shape[1]
        v = np.hstack([v, t])
        hv = np.hstack([hv, _cols(hop(_blk(t, npw, nc)))])
    used = (hop.count - start) if hasattr(hop, "count") else -1
    return SolveResult(lam=lam, x=_blk(xm, npw, nc), iterations=it, converged=converged,
                       resnorms=norms, history=history, h_applications=used)
