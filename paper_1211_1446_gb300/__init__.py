"""Python binding of libdks.so (GB300 LOBPCG-F for the Dirac-Kohn-Sham operator).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in include/dks.h.  PyTorch provides device
memory and streams.  If the shared library is missing or fails to load, every
entry point raises -- there is no CPU fallback.

Layouts follow include/dks.h: vector blocks are complex tensors of shape
[nb, ncomp, npw] (ncomp = 4 for the DKS model, 2 for KSSO; complex128 for FP64,
complex64 for FP32), planewaves in the canonical (lexicographic Miller) order
returned by Context.basis(ik).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdks.so")
DEBUG_LIB_PATH = os.path.join(HERE, "libdks_debug.so")   # index-checked build (build --debug)

PREC_FP64, PREC_FP32, PREC_FP64_EMULATED = 0, 1, 2
MODE_FP64, MODE_MIXED = 0, 1
PRECOND_TETER, PRECOND_IDENTITY = 0, 1

ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_NEG_STATE, ERR_RANK, ERR_TIMEOUT = -1, -2, -3, -4, -5, -6, -7
ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "NOT_CONVERGED", -5: "NEG_STATE",
          -6: "RANK", -7: "TIMEOUT", -8: "GRID", -9: "UNSUPPORTED"}


class DKSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Cell(C.Structure):
    _fields_ = [("lattice", C.c_double * 9), ("grid", C.c_int * 3), ("c", C.c_double), ("nk", C.c_int),
                ("kfrac", C.POINTER(C.c_double)), ("ecut_k", C.POINTER(C.c_double))]


class _Pot(C.Structure):
    _fields_ = [("v_r", C.POINTER(C.c_double))]


class _Proj(C.Structure):
    _fields_ = [("nsite", C.c_int), ("pos", C.POINTER(C.c_double)), ("lmax", C.POINTER(C.c_int)),
                ("rl", C.POINTER(C.c_double)), ("d", C.POINTER(C.c_double))]


class SolveOpts(C.Structure):
    _fields_ = [("n_init", C.c_int), ("n_iter", C.c_int), ("nbuf", C.c_int), ("C", C.c_double),
                ("Omega", C.c_double), ("mode", C.c_int), ("refine_tol", C.c_double), ("precond", C.c_int),
                ("use_filter", C.c_int), ("nev_k", C.POINTER(C.c_int)), ("stream", C.c_void_p),
                ("chol_tol", C.c_double), ("drop_tol", C.c_double), ("emulate_fp64", C.c_int),
                ("concurrency", C.c_int), ("solver", C.c_int), ("m_max", C.c_int), ("block", C.c_int)]


class SolveReport(C.Structure):
    _fields_ = [("iterations", C.c_int * 64), ("fp64_iterations", C.c_int * 64),
                ("max_residual", C.c_double * 64), ("h_applications", C.c_longlong), ("shift", C.c_double),
                ("seconds", C.c_double), ("status", C.c_int), ("hist_len", C.c_int),
                ("res_history", C.c_double * 512)]


class ScfOpts(C.Structure):
    _fields_ = [("nocc", C.c_int), ("max_iter", C.c_int), ("tol", C.c_double), ("alpha", C.c_double),
                ("kerker_q0", C.c_double), ("history", C.c_int), ("n_init_warm", C.c_int),
                ("solve_tol", C.c_double), ("solve", SolveOpts)]


class ScfReport(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("residual", C.c_double), ("e_h", C.c_double),
                ("e_xc", C.c_double), ("solve_iterations", C.c_longlong), ("h_applications", C.c_longlong),
                ("seconds", C.c_double), ("status", C.c_int), ("hist_len", C.c_int),
                ("res_history", C.c_double * 128)]


class TuneReport(C.Structure):
    _fields_ = [("ncand", C.c_int), ("best", C.c_int), ("chunk_bytes", C.c_longlong * 32),
                ("plane_threads", C.c_int * 32), ("plane_split", C.c_int * 32), ("ms", C.c_double * 32),
                ("proj_tc", C.c_int), ("proj_ms", C.c_double * 2)]


EXPORTS = ["dks_create", "dks_destroy", "dks_npw", "dks_basis", "dks_nproj", "dks_filter_constants",
           "dks_apply_H", "dks_filter", "dks_solve_opts_default", "dks_lobpcgf_solve", "dks_precond",
           "dks_gram", "dks_rayleigh_ritz", "dks_rotate", "dks_residual_norms", "dks_strerror",
           "dks_last_error", "dks_profile_ncat", "dks_profile_name", "dks_profile_enable", "dks_profile_read",
           "dks_rayleigh_ritz_static", "dks_gram_hermitian", "dks_kinetic_balance", "dks_create_model",
           "dks_ncomp", "dks_density", "dks_hxc", "dks_set_potential", "dks_mixer_create", "dks_mix",
           "dks_mixer_destroy", "dks_scf_opts_default", "dks_scf", "dks_update_potential",
           "dks_density_residual", "dks_autotune", "dks_tune_get", "dks_tune_set", "dks_fft_plan",
           "dks_debug_check", "dks_tensor_cores", "dks_tensor_cores_get", "dks_debug_rr_wait",
           "dks_tune_contractions_get", "dks_tune_contractions_set"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdks.so (raises if it is missing: build it with paper_1211_1446_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libdks.so not found at {path}; run `python -m paper_1211_1446_gb300.build`")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    lib.dks_create.argtypes = [C.POINTER(_Cell), d, C.POINTER(_Pot), C.POINTER(_Proj), C.POINTER(vp)]
    lib.dks_destroy.argtypes = [vp]
    lib.dks_destroy.restype = None
    lib.dks_npw.argtypes = [vp, i, C.POINTER(i)]
    lib.dks_create_model.argtypes = [C.POINTER(_Cell), d, C.POINTER(_Pot), C.POINTER(_Proj), i, C.POINTER(vp)]
    lib.dks_ncomp.argtypes = [vp, C.POINTER(i)]
    lib.dks_basis.argtypes = [vp, i, C.POINTER(i)]
    lib.dks_nproj.argtypes = [vp, C.POINTER(i)]
    lib.dks_filter_constants.argtypes = [vp, i, C.POINTER(d), C.POINTER(d)]
    lib.dks_apply_H.argtypes = [vp, i, vp, vp, i, i, vp]
    lib.dks_filter.argtypes = [vp, i, vp, vp, i, d, d, i, vp]
    lib.dks_solve_opts_default.argtypes = [C.POINTER(SolveOpts)]
    lib.dks_solve_opts_default.restype = None
    lib.dks_lobpcgf_solve.argtypes = [vp, i, d, C.POINTER(SolveOpts), C.POINTER(d), C.POINTER(vp),
                                      C.POINTER(SolveReport)]
    lib.dks_precond.argtypes = [vp, i, vp, vp, vp, vp, i, vp, i, i, vp]
    lib.dks_gram.argtypes = [vp, vp, i, i, vp, vp, i, vp]
    lib.dks_gram_hermitian.argtypes = [vp, vp, i, i, vp, vp, i, vp]
    lib.dks_kinetic_balance.argtypes = [vp, i, vp, i, i, vp]
    lib.dks_rayleigh_ritz.argtypes = [vp, vp, i, i, vp, vp, vp, vp]
    lib.dks_rayleigh_ritz_static.argtypes = [vp, vp, i, i, vp, vp, vp, vp]
    lib.dks_rotate.argtypes = [vp, i, i, vp, i, i, vp, d, i, vp]
    lib.dks_residual_norms.argtypes = [vp, vp, vp, i, i, vp, i, vp]
    lib.dks_density.argtypes = [vp, i, vp, i, C.POINTER(d), vp, vp]
    lib.dks_hxc.argtypes = [vp, vp, vp, C.POINTER(d), vp]
    lib.dks_set_potential.argtypes = [vp, vp, vp]
    lib.dks_update_potential.argtypes = [vp, vp, C.POINTER(d), vp]
    lib.dks_density_residual.argtypes = [vp, vp, vp, C.POINTER(d), vp]
    lib.dks_mixer_create.argtypes = [vp, i, d, d, C.POINTER(vp)]
    lib.dks_mix.argtypes = [vp, vp, vp, vp, vp]
    lib.dks_mixer_destroy.argtypes = [vp]
    lib.dks_mixer_destroy.restype = None
    lib.dks_scf_opts_default.argtypes = [C.POINTER(ScfOpts)]
    lib.dks_scf_opts_default.restype = None
    lib.dks_scf.argtypes = [vp, i, C.POINTER(ScfOpts), C.POINTER(d), C.POINTER(vp), vp, C.POINTER(ScfReport)]
    lib.dks_autotune.argtypes = [vp, i, i, i, vp, C.POINTER(TuneReport)]
    lib.dks_tune_get.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(i), C.POINTER(i)]
    lib.dks_tune_set.argtypes = [vp, C.c_longlong, i, i]
    lib.dks_fft_plan.argtypes = [i, C.POINTER(i), C.POINTER(i), C.POINTER(i)]
    lib.dks_debug_check.argtypes = [C.POINTER(i), C.POINTER(C.c_uint)]
    lib.dks_strerror.argtypes = [i]
    lib.dks_strerror.restype = C.c_char_p
    lib.dks_last_error.argtypes = []
    lib.dks_last_error.restype = C.c_char_p
    lib.dks_profile_ncat.argtypes = []
    lib.dks_profile_name.argtypes = [i]
    lib.dks_profile_name.restype = C.c_char_p
    lib.dks_profile_enable.argtypes = [i]
    lib.dks_profile_read.argtypes = [i, vp, vp, vp, vp]
    lib.dks_tensor_cores.argtypes = [i, i]
    lib.dks_tune_contractions_get.argtypes = [vp, C.POINTER(i)]
    lib.dks_tune_contractions_set.argtypes = [vp, i]
    lib.dks_debug_rr_wait.argtypes = [C.c_uint, C.POINTER(C.c_uint)]
    lib.dks_tensor_cores_get.argtypes = [C.POINTER(i), C.POINTER(i)]
    _lib = lib
    return lib


def _check(rc):
    if rc != 0:
        raise DKSError(rc, _lib.dks_last_error().decode())


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _complex128():
    import torch
    return torch.complex128


def _prec_of(t):
    import torch
    if t.dtype == torch.complex128:
        return PREC_FP64
    if t.dtype == torch.complex64:
        return PREC_FP32
    raise TypeError("blocks must be complex128 or complex64")


MODELS = {"dks": 0, "ksso": 1}
SOLVERS = {"lobpcg": 0, "davidson": 1}


class Context:
    """Owns a dks_ctx: planewave spheres, FFT plans, V(r) and projector tables on the GPU."""

    def __init__(self, lattice, grid, c, kfrac, ecut, v_r=None, pos=None, lmax=None, rl=None, d=None,
                 ecut_k=None, model="dks"):
        """model "dks": four-component H' (columns [4, npw]); "ksso": the two-component KSSO
        operator (columns [2, npw]) solved by Algorithm 1 without the filter."""
        lib = load_library()
        self._keep = []
        cell = _Cell()
        cell.lattice[:] = [float(x) for x in np.asarray(lattice, dtype=np.float64).reshape(9)]
        cell.grid[:] = [int(x) for x in grid]
        cell.c = float(c)
        kf = np.ascontiguousarray(np.asarray(kfrac, dtype=np.float64).reshape(-1, 3))
        cell.nk = kf.shape[0]
        cell.kfrac = self._arr(kf, C.c_double)
        if ecut_k is not None:
            cell.ecut_k = self._arr(np.ascontiguousarray(ecut_k, dtype=np.float64), C.c_double)
        pot = _Pot()
        if v_r is not None:
            pot.v_r = self._arr(np.ascontiguousarray(v_r, dtype=np.float64).reshape(-1), C.c_double)
        proj = _Proj()
        if pos is not None and len(pos) and lmax is not None and int(np.max(lmax)) >= 0:
            proj.nsite = len(pos)
            proj.pos = self._arr(np.ascontiguousarray(pos, dtype=np.float64).reshape(-1), C.c_double)
            proj.lmax = self._arr(np.ascontiguousarray(lmax, dtype=np.int32).reshape(-1), C.c_int)
            proj.rl = self._arr(np.ascontiguousarray(rl, dtype=np.float64).reshape(-1), C.c_double)
            proj.d = self._arr(np.ascontiguousarray(d, dtype=np.float64).reshape(-1), C.c_double)
        self._h = C.c_void_p()
        if model not in MODELS:
            raise ValueError(f"model must be one of {sorted(MODELS)}")
        _check(lib.dks_create_model(C.byref(cell), float(ecut if ecut is not None else 0.0), C.byref(pot),
                                    C.byref(proj), MODELS[model], C.byref(self._h)))
        nc = C.c_int()
        _check(lib.dks_ncomp(self._h, C.byref(nc)))
        self.ncomp = nc.value
        self.model = model
        self.grid = tuple(int(x) for x in grid)
        self.nk = cell.nk
        self.c = float(c)
        self._keep = []

    def _arr(self, a, ctype):
        self._keep.append(a)
        return a.ctypes.data_as(C.POINTER(ctype))

    @classmethod
    def from_workload(cls, wl, model="dks"):
        """Build from any object with the attributes of workloads.Workload (duck-typed)."""
        return cls(wl.lattice, wl.grid, wl.c, wl.kfrac, None, v_r=wl.v_r, pos=wl.pos, lmax=wl.lmax,
                   rl=wl.rl, d=wl.d, ecut_k=wl.ecut_k, model=model)

    def close(self):
        if getattr(self, "_h", None):
            _lib.dks_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- queries
    def npw(self, ik=0):
        n = C.c_int()
        _check(_lib.dks_npw(self._h, ik, C.byref(n)))
        return n.value

    def basis(self, ik=0):
        m = np.zeros((self.npw(ik), 3), dtype=np.int32)
        _check(_lib.dks_basis(self._h, ik, m.ctypes.data_as(C.POINTER(C.c_int))))
        return m

    def nproj(self):
        n = C.c_int()
        _check(_lib.dks_nproj(self._h, C.byref(n)))
        return n.value

    def filter_constants(self, ik=0):
        cs, om = C.c_double(), C.c_double()
        _check(_lib.dks_filter_constants(self._h, ik, C.byref(cs), C.byref(om)))
        return cs.value, om.value

    # ---- operator
    def _block(self, ik, *ts, nb=None):
        """Shape check of device blocks before their pointers cross the ABI (which cannot check):
        [nb, ncomp, npw], contiguous, one dtype; returns nb."""
        npw = self.npw(ik)
        nb = ts[0].shape[0] if nb is None else nb
        for t in ts:
            if t.dim() != 3 or t.shape[1] != self.ncomp or t.shape[2] != npw or t.shape[0] < nb:
                raise ValueError(f"block of shape {tuple(t.shape)}: need [{nb}, {self.ncomp}, {npw}]")
            if not t.is_contiguous() or t.dtype != ts[0].dtype:
                raise ValueError("blocks must be contiguous and of one dtype")
        return nb

    def apply_H(self, ik, x, hx, stream=None, emulated=False):
        nb = self._block(ik, x, hx)
        prec = PREC_FP64_EMULATED if (emulated and _prec_of(x) == PREC_FP64) else _prec_of(x)
        _check(_lib.dks_apply_H(self._h, ik, _dptr(x), _dptr(hx), nb, prec, _stream(stream)))
        return hx

    def kinetic_balance(self, ik, x, stream=None):
        """dks_kinetic_balance: small components of x ([nb, 4, npw], in place) from its large ones."""
        nb = self._block(ik, x)
        _check(_lib.dks_kinetic_balance(self._h, ik, _dptr(x), nb, _prec_of(x), _stream(stream)))
        return x

    def filter(self, ik, y, fy, cshift, omega, stream=None):
        nb = self._block(ik, y, fy)
        _check(_lib.dks_filter(self._h, ik, _dptr(y), _dptr(fy), nb, float(cshift), float(omega),
                               _prec_of(y), _stream(stream)))
        return fy

    def precond(self, ik, x, hx, lam, act, y, precond=PRECOND_TETER, stream=None):
        self._block(ik, x, hx)
        self._block(ik, y, nb=act.shape[0])
        _check(_lib.dks_precond(self._h, ik, _dptr(x), _dptr(hx), _dptr(lam), _dptr(act), act.shape[0],
                                _dptr(y), precond, _prec_of(x), _stream(stream)))
        return y

    # ---- launch-parameter tuning (results never depend on it, only the time)
    def tuning(self):
        """The context's launch parameters and projector contraction schedule."""
        chunk, threads, split, ptc = C.c_longlong(), C.c_int(), C.c_int(), C.c_int()
        _check(_lib.dks_tune_get(self._h, C.byref(chunk), C.byref(threads), C.byref(split)))
        _check(_lib.dks_tune_contractions_get(self._h, C.byref(ptc)))
        return dict(chunk_bytes=chunk.value, plane_threads=threads.value, plane_split=split.value,
                    proj_tc=ptc.value)

    def set_tuning(self, chunk_bytes, plane_threads=0, plane_split=0, proj_tc=None):
        _check(_lib.dks_tune_set(self._h, int(chunk_bytes), int(plane_threads), int(plane_split)))
        if proj_tc is not None:
            _check(_lib.dks_tune_contractions_set(self._h, int(proj_tc)))

    def autotune(self, ik=0, nb=40, prec=PREC_FP32, cache=None, stream=None):
        """dks_autotune on an nb-column block of k-point ik; with `cache` (a JSON file path) a stored
        choice for the same grid, basis size, model, block width, precision and device is applied
        instead, and a new choice is stored.  Returns the chosen parameters (and, when timed, the
        candidates' times)."""
        import torch
        key = tuning_key(self.grid, self.npw(ik), self.ncomp, nb, prec, torch.cuda.get_device_name())
        if cache:
            hit = tuning_cache_lookup(cache, key)
            if hit is not None:
                self.set_tuning(hit["chunk_bytes"], hit["plane_threads"], hit["plane_split"], hit.get("proj_tc"))
                return dict(hit, cached=True)
        rep = TuneReport()
        _check(_lib.dks_autotune(self._h, int(ik), int(nb), int(prec), _stream(stream), C.byref(rep)))
        choice = dict(chunk_bytes=int(rep.chunk_bytes[rep.best]), plane_threads=int(rep.plane_threads[rep.best]),
                      plane_split=int(rep.plane_split[rep.best]))
        if rep.proj_tc >= 0:
            choice.update(proj_tc=int(rep.proj_tc), proj_ms=[float(rep.proj_ms[0]), float(rep.proj_ms[1])])
        if cache:
            tuning_cache_store(cache, key, choice)
        cands = [dict(chunk_bytes=int(rep.chunk_bytes[i]), plane_threads=int(rep.plane_threads[i]),
                      plane_split=int(rep.plane_split[i]), ms=float(rep.ms[i])) for i in range(rep.ncand)]
        return dict(choice, cached=False, candidates=cands)

    # ---- SCF pieces (grids: float64 device tensors of shape grid, natural order)
    def _grid(self, *ts):
        import torch
        for t in ts:
            if t is None:
                continue
            if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != int(np.prod(self.grid)):
                raise ValueError(f"grid arrays are contiguous float64 with {int(np.prod(self.grid))} values")

    def density(self, ik, x, occ, rho, stream=None):
        """dks_density: rho += sum_j occ[j] |psi_j(r)|^2 for the columns of x (complex128)."""
        nb = self._block(ik, x, nb=len(occ))
        if x.dtype != _complex128():
            raise ValueError("density blocks are complex128")
        self._grid(rho)
        o = np.ascontiguousarray(occ, dtype=np.float64)
        _check(_lib.dks_density(self._h, ik, _dptr(x), nb, o.ctypes.data_as(C.POINTER(C.c_double)), _dptr(rho),
                                _stream(stream)))
        return rho

    def hxc(self, rho, vhxc, stream=None):
        """dks_hxc: vhxc = V_H + v_xc of rho; returns (E_H, E_xc) (synchronises the stream)."""
        self._grid(rho, vhxc)
        e = (C.c_double * 2)()
        _check(_lib.dks_hxc(self._h, _dptr(rho), _dptr(vhxc), e, _stream(stream)))
        return e[0], e[1]

    def set_potential(self, v, stream=None):
        """dks_set_potential: V(r) of the operator becomes v (synchronous)."""
        self._grid(v)
        _check(_lib.dks_set_potential(self._h, _dptr(v), _stream(stream)))

    def update_potential(self, rho=None, stream=None):
        """dks_update_potential: V = V_loc + V_hxc(rho) (V_loc alone for rho None); returns
        (E_H, E_xc) of rho (synchronous)."""
        self._grid(rho)
        e = (C.c_double * 2)()
        _check(_lib.dks_update_potential(self._h, _dptr(rho), e, _stream(stream)))
        return e[0], e[1]

    def density_residual(self, a, b, stream=None):
        """dks_density_residual: int |a - b| dr over the grid (synchronous)."""
        self._grid(a, b)
        out = C.c_double()
        _check(_lib.dks_density_residual(self._h, _dptr(a), _dptr(b), C.byref(out), _stream(stream)))
        return out.value

    def mixer(self, history=8, alpha=0.5, q0=1.0):
        return Mixer(self, history, alpha, q0)

    def scf(self, x_list, nev, nocc, tol=1e-8, max_iter=60, alpha=0.5, q0=1.0, history=8, n_init_warm=1,
            solve_tol=1e-8, rho=None, n_init=3, mode=MODE_FP64, nbuf=0, n_iter=200, precond=PRECOND_TETER,
            stream=None, check=True, block=0):
        """dks_scf: the SCF loop (solve, density, V_hxc, Kerker-Anderson mixing) from the potential
        given at creation; block > 0 solves in band blocks (see solve).  Returns (eigenvalues per
        k, report dict, status code)."""
        o = ScfOpts()
        _lib.dks_scf_opts_default(C.byref(o))
        o.nocc, o.max_iter, o.tol, o.alpha, o.kerker_q0 = int(nocc), int(max_iter), float(tol), float(alpha), float(q0)
        o.history, o.n_init_warm, o.solve_tol = int(history), int(n_init_warm), float(solve_tol)
        o.solve.n_init, o.solve.n_iter, o.solve.nbuf = int(n_init), int(n_iter), int(nbuf)
        o.solve.mode, o.solve.precond, o.solve.block = int(mode), int(precond), int(block)
        o.solve.stream = _stream(stream)
        if len(x_list) != self.nk:
            raise ValueError(f"need one block per k-point ({self.nk})")
        for ik, t in enumerate(x_list):
            self._block(ik, t, nb=int(nev) + int(nbuf))
            if t.dtype != _complex128():
                raise ValueError("SCF blocks are complex128")
        self._grid(rho)
        eig = np.zeros(int(nev) * self.nk, dtype=np.float64)
        ptrs = (C.c_void_p * self.nk)(*[t.data_ptr() for t in x_list])
        rep = ScfReport()
        rc = _lib.dks_scf(self._h, int(nev), C.byref(o), eig.ctypes.data_as(C.POINTER(C.c_double)), ptrs,
                          _dptr(rho), C.byref(rep))
        if check and rc != 0:
            _check(rc)
        report = dict(iterations=rep.iterations, converged=bool(rep.converged), residual=rep.residual,
                      e_h=rep.e_h, e_xc=rep.e_xc, solve_iterations=int(rep.solve_iterations),
                      h_applications=int(rep.h_applications), seconds=rep.seconds, status=rep.status,
                      history=list(rep.res_history[:rep.hist_len]),
                      message=_lib.dks_last_error().decode() if rc else "")
        return [eig[i * nev:(i + 1) * nev].copy() for i in range(self.nk)], report, rc

    # ---- solver
    def solve(self, x_list, nev, tol=1e-6, n_init=3, n_iter=200, mode=MODE_FP64, refine_tol=1e-5,
              precond=PRECOND_TETER, use_filter=True, cshift=None, omega=None, nev_k=None, nbuf=0,
              stream=None, check=True, chol_tol=None, drop_tol=None, emulate_fp64=True, concurrency=0,
              solver="lobpcg", m_max=0, block=0):
        """Algorithm 1 on every k-point (solver="davidson": block Davidson with the same filter, basis
        of at most m_max columns).  x_list[ik]: complex128 [nev_k+nbuf, ncomp, npw] (X0 in, X out).
        block > 0: the pairs are found in band blocks of `block` wanted columns (plus nbuf buffer
        columns each), every block deflated against the converged earlier ones.
        Returns (eigenvalues per k as numpy arrays, report dict, status code)."""
        opts = SolveOpts()
        _lib.dks_solve_opts_default(C.byref(opts))
        opts.n_init, opts.n_iter, opts.nbuf = int(n_init), int(n_iter), int(nbuf)
        opts.C = float("nan") if cshift is None else float(cshift)
        opts.Omega = float("nan") if omega is None else float(omega)
        opts.mode, opts.refine_tol, opts.precond = int(mode), float(refine_tol), int(precond)
        opts.use_filter = 1 if use_filter else 0
        if chol_tol is not None:
            opts.chol_tol = float(chol_tol)
        if drop_tol is not None:
            opts.drop_tol = float(drop_tol)
        opts.emulate_fp64 = 1 if emulate_fp64 else 0
        opts.concurrency = int(concurrency)
        if solver not in SOLVERS:
            raise ValueError(f"solver must be one of {sorted(SOLVERS)}")
        opts.solver, opts.m_max, opts.block = SOLVERS[solver], int(m_max), int(block)
        nevs = [int(nev)] * self.nk if nev_k is None else [int(v) for v in nev_k]
        if nev_k is not None:
            arr = np.ascontiguousarray(nevs, dtype=np.int32)
            self._keep.append(arr)
            opts.nev_k = arr.ctypes.data_as(C.POINTER(C.c_int))
        opts.stream = _stream(stream)
        if len(x_list) != self.nk:
            raise ValueError(f"need one block per k-point ({self.nk})")
        for ik, t in enumerate(x_list):
            self._block(ik, t, nb=nevs[ik] + int(nbuf))
            if t.dtype != _complex128():
                raise ValueError("solve blocks are complex128")
        eig = np.zeros(sum(nevs), dtype=np.float64)
        ptrs = (C.c_void_p * self.nk)(*[t.data_ptr() for t in x_list])
        rep = SolveReport()
        rc = _lib.dks_lobpcgf_solve(self._h, int(nev), float(tol), C.byref(opts),
                                    eig.ctypes.data_as(C.POINTER(C.c_double)), ptrs, C.byref(rep))
        self._keep = []
        if check and rc not in (0,):
            _check(rc)
        out, o = [], 0
        for v in nevs:
            out.append(eig[o:o + v].copy())
            o += v
        nk = min(self.nk, 64)
        report = dict(iterations=list(rep.iterations[:nk]), fp64_iterations=list(rep.fp64_iterations[:nk]),
                      max_residual=list(rep.max_residual[:nk]), h_applications=int(rep.h_applications),
                      shift=rep.shift, seconds=rep.seconds, status=rep.status,
                      history=list(rep.res_history[:rep.hist_len]),
                      message=_lib.dks_last_error().decode() if rc else "")
        return out, report, rc


def debug_check():
    """dks_debug_check: (checks compiled in, first failed check code or 0)."""
    lib = load_library()
    compiled, code = C.c_int(), C.c_uint()
    _check(lib.dks_debug_check(C.byref(compiled), C.byref(code)))
    return bool(compiled.value), int(code.value)


def fft_plan(n):
    """dks_fft_plan: (radices of the passes, DIF position of every frequency) of an axis of length n."""
    lib = load_library()
    nst = C.c_int()
    radix = (C.c_int * 8)()
    pos = (C.c_int * max(1, int(n)))()
    _check(lib.dks_fft_plan(int(n), C.byref(nst), radix, pos))
    return [int(radix[i]) for i in range(nst.value)], [int(pos[k]) for k in range(int(n))]


def tuning_key(grid, npw, ncomp, nb, prec, device):
    """Cache key of one tuning problem."""
    return "grid=%dx%dx%d npw=%d ncomp=%d nb=%d prec=%d device=%s" % (tuple(int(g) for g in grid) +
                                                                      (int(npw), int(ncomp), int(nb), int(prec),
                                                                       str(device)))


def tuning_cache_lookup(path, key):
    """The stored choice for key in the JSON cache at path, or None (missing or unreadable file)."""
    import json
    try:
        with open(path) as f:
            entry = json.load(f).get(key)
    except (OSError, ValueError, AttributeError):
        return None
    if not isinstance(entry, dict) or any(k not in entry for k in ("chunk_bytes", "plane_threads", "plane_split")):
        return None
    out = dict(chunk_bytes=int(entry["chunk_bytes"]), plane_threads=int(entry["plane_threads"]),
               plane_split=int(entry["plane_split"]))
    if "proj_tc" in entry:                     # the projector contraction schedule, when it was tuned
        out["proj_tc"] = int(entry["proj_tc"])
    return out


def tuning_cache_store(path, key, choice):
    """Adds (or replaces) key in the JSON cache at path, written atomically."""
    import json
    data = {}
    try:
        with open(path) as f:
            data = json.load(f)
        if not isinstance(data, dict):
            data = {}
    except (OSError, ValueError):
        data = {}
    data[key] = dict(chunk_bytes=int(choice["chunk_bytes"]), plane_threads=int(choice["plane_threads"]),
                     plane_split=int(choice["plane_split"]))
    if "proj_tc" in choice:
        data[key]["proj_tc"] = int(choice["proj_tc"])
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Mixer:
    """dks_mixer: Anderson mixing of densities with the Kerker preconditioner (device history)."""

    def __init__(self, ctx, history=8, alpha=0.5, q0=1.0):
        self._ctx = ctx
        self._h = C.c_void_p()
        _check(_lib.dks_mixer_create(ctx._h, int(history), float(alpha), float(q0), C.byref(self._h)))

    def step(self, rho_in, rho_out, rho_next, stream=None):
        self._ctx._grid(rho_in, rho_out, rho_next)
        _check(_lib.dks_mix(self._h, _dptr(rho_in), _dptr(rho_out), _dptr(rho_next), _stream(stream)))
        return rho_next

    def close(self):
        if getattr(self, "_h", None):
            _lib.dks_mixer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TC_ROTATE, TC_GRAM, TC_PROJ_HN, TC_PROJ_NN, TC_FP64, TC_ALL = 1, 2, 4, 8, 16, 31


def tensor_cores(mask=None, kchunk=0):
    """dks_tensor_cores: select which contractions run on the tcgen05 tensor cores (TC_* bits;
    TC_FP64: the complex128 Gram matrices and rotations of the double-float refinement phase
    from exact integer slices; None leaves the mask) and the longest FP32 accumulation of the
    complex64 Gram forms (kchunk rows, 0 = unchanged).  Returns the previous (mask, kchunk)."""
    lib = load_library()
    m, k = C.c_int(), C.c_int()
    _check(lib.dks_tensor_cores_get(C.byref(m), C.byref(k)))
    _check(lib.dks_tensor_cores(int(m.value if mask is None else mask), int(kchunk)))
    return m.value, k.value


def debug_rr_wait(first_wait_polls=1 << 24):
    """dks_debug_rr_wait: set the polls of the first staging wait of the Rayleigh-Ritz per-column
    kernels (0: every such wait gives up at once and the single-CTA kernel redoes the step) and
    return the number of steps redone that way since the previous call."""
    lib = load_library()
    n = C.c_uint()
    _check(lib.dks_debug_rr_wait(int(first_wait_polls), C.byref(n)))
    return n.value


def profile_enable(on=True):
    """Start (or stop) per-launch CUDA-event timing inside the library; clears counters."""
    _check(load_library().dks_profile_enable(1 if on else 0))


def profile_read():
    """Synchronise and return {category: dict(ms, launches, bytes, flops)}; clears the records."""
    lib = load_library()
    n = lib.dks_profile_ncat()
    ms = np.zeros(n)
    la = np.zeros(n, dtype=np.int64)
    by = np.zeros(n)
    fl = np.zeros(n)
    _check(lib.dks_profile_read(n, ms.ctypes.data_as(C.c_void_p), la.ctypes.data_as(C.c_void_p),
                                by.ctypes.data_as(C.c_void_p), fl.ctypes.data_as(C.c_void_p)))
    return {lib.dks_profile_name(c).decode(): dict(ms=float(ms[c]), launches=int(la[c]), bytes=float(by[c]),
                                                   flops=float(fl[c])) for c in range(n)}


# ---- single steps of Algorithm 1 (blocks are [ncol, rows] complex tensors)

def gram(z, hz, a_out, s_out, stream=None, emulated=False):
    load_library()
    nz, rows = z.shape[0], z[0].numel()
    prec = PREC_FP64_EMULATED if (emulated and _prec_of(z) == PREC_FP64) else _prec_of(z)
    _check(_lib.dks_gram(_dptr(z), _dptr(hz), rows, nz, _dptr(a_out), _dptr(s_out), prec, _stream(stream)))


def gram_hermitian(z, hz, a_out, s_out, stream=None, emulated=False):
    """dks_gram_hermitian: the solver's fused lower-triangle Gram, upper triangles mirrored."""
    load_library()
    nz, rows = z.shape[0], z[0].numel()
    prec = PREC_FP64_EMULATED if (emulated and _prec_of(z) == PREC_FP64) else _prec_of(z)
    _check(_lib.dks_gram_hermitian(_dptr(z), _dptr(hz), rows, nz, _dptr(a_out), _dptr(s_out), prec,
                                   _stream(stream)))


def _rr_args(a, s, n, v_out, lam_out, info_out):
    """Shapes, dtypes, device and contiguity of a Rayleigh-Ritz call, checked before any pointer
    reaches the library: A, S complex128 nz x nz, V complex128 with room for n x nz, lam float64
    with room for n, info int32 with room for 3 (every call writes info[0..2])."""
    import torch
    nz = a.shape[0]
    if a.dim() != 2 or tuple(a.shape) != (nz, nz) or tuple(s.shape) != (nz, nz):
        raise ValueError("A and S must be nz x nz")
    if not 0 < int(n) <= nz:
        raise ValueError("need 0 < n <= nz")
    args = (("A", a, torch.complex128, nz * nz), ("S", s, torch.complex128, nz * nz),
            ("V", v_out, torch.complex128, int(n) * nz), ("lam", lam_out, torch.float64, int(n)),
            ("info", info_out, torch.int32, 3))
    for name, t, dt, need in args:
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}")
        if t.numel() < need:
            raise ValueError(f"{name} needs at least {need} elements")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    for name, t, _, _ in args:
        if not t.is_cuda or t.device != a.device:
            raise ValueError(f"{name} must be on the device of A")
    return nz


def rayleigh_ritz(a, s, n, v_out, lam_out, info_out, stream=None):
    """dks_rayleigh_ritz: the n lowest pairs of A v = lam S v on the device (info: int32[>= 3])."""
    load_library()
    _rr_args(a, s, n, v_out, lam_out, info_out)
    _check(_lib.dks_rayleigh_ritz(_dptr(a), _dptr(s), a.shape[0], int(n), _dptr(v_out), _dptr(lam_out),
                                  _dptr(info_out), _stream(stream)))


def rayleigh_ritz_static(a, s, n, v_out, lam_out, info_out, stream=None):
    """dks_rayleigh_ritz_static: same solve with the library's fixed device scratch array (no
    allocation; nz <= 128; calls that overlap on the GPU race on the shared array)."""
    load_library()
    _rr_args(a, s, n, v_out, lam_out, info_out)
    _check(_lib.dks_rayleigh_ritz_static(_dptr(a), _dptr(s), a.shape[0], int(n), _dptr(v_out), _dptr(lam_out),
                                         _dptr(info_out), _stream(stream)))


def rotate(z, w, n, out, beta=0.0, stream=None, emulated=False):
    """out[j] = sum_i z[i] w[i, j] (+ beta out[j]); w: complex128 tensor [n, nz] holding the columns of W."""
    load_library()
    nz, rows = z.shape[0], z[0].numel()
    ldw = w.shape[-1] if w.dim() == 2 else nz
    prec = PREC_FP64_EMULATED if (emulated and _prec_of(z) == PREC_FP64) else _prec_of(z)
    _check(_lib.dks_rotate(_dptr(z), rows, nz, _dptr(w), ldw, int(n), _dptr(out), float(beta), prec,
                           _stream(stream)))


def residual_norms(x, hx, lam, norms_out, stream=None):
    load_library()
    n, rows = x.shape[0], x[0].numel()
    _check(_lib.dks_residual_norms(_dptr(x), _dptr(hx), _dptr(lam), rows, n, _dptr(norms_out), _prec_of(x),
                                   _stream(stream)))
