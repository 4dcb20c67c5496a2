"""The C-ABI library builds for sm_103a, loads, and exports every function include/dks.h declares
(no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|void|const char\s*\*)\s*(dks_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1211_1446_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    import paper_1211_1446_gb300 as P
    assert set(P.EXPORTS) == set(_declared())


def test_strerror_without_gpu():
    import paper_1211_1446_gb300 as P
    lib = P.load_library()
    assert lib.dks_strerror(-8).decode().startswith("planewave sphere")
    assert lib.dks_strerror(0).decode() == "ok"


def test_scf_entry_points_validate_arguments_without_gpu():
    """The SCF entry points reject bad arguments before touching the device: every call below
    returns DKS_ERR_INVALID_ARG and leaves a message; the option defaults are host-only."""
    import ctypes as C
    import paper_1211_1446_gb300 as P
    lib = P.load_library()
    bad = -1
    out = C.c_void_p()
    assert lib.dks_mixer_create(None, 8, 0.5, 1.0, C.byref(out)) == bad and not out.value
    assert lib.dks_mixer_create(None, 8, 0.5, 1.0, None) == bad
    assert lib.dks_density(None, 0, None, 1, None, None, None) == bad
    assert lib.dks_hxc(None, None, None, None, None) == bad
    assert lib.dks_set_potential(None, None, None) == bad
    assert lib.dks_mix(None, None, None, None, None) == bad
    assert "dks_mix" in lib.dks_last_error().decode()
    o = P.ScfOpts()
    lib.dks_scf_opts_default(C.byref(o))
    assert (o.nocc, o.max_iter, o.history, o.n_init_warm) == (0, 60, 8, 1)
    assert (o.tol, o.alpha, o.kerker_q0, o.solve_tol) == (1e-8, 0.5, 1.0, 1e-8)
    assert o.solve.n_init == 3 and o.solve.n_iter == 200          # the solver's own defaults
    eig = (C.c_double * 4)()
    assert lib.dks_scf(None, 4, C.byref(o), eig, None, None, None) == bad
    lib.dks_mixer_destroy(None)                                    # no-op on NULL
    assert lib.dks_update_potential(None, None, None, None) == bad
    res = C.c_double(-1.0)
    assert lib.dks_density_residual(None, None, None, C.byref(res), None) == bad and res.value == -1.0


def test_solve_opts_layout_matches_the_library():
    """dks_solve_opts_default writes every field at the offset the binding reads it from: fill the
    ctypes structure with sentinels, let the library write its defaults, read them back."""
    import ctypes as C
    import math
    import paper_1211_1446_gb300 as P
    lib = P.load_library()
    o = P.SolveOpts()
    C.memset(C.byref(o), 0x7f, C.sizeof(o))
    lib.dks_solve_opts_default(C.byref(o))
    assert (o.n_init, o.n_iter, o.nbuf, o.mode, o.precond, o.use_filter) == (3, 200, 0, 0, 0, 1)
    assert math.isnan(o.C) and math.isnan(o.Omega) and o.refine_tol == 1e-5
    assert (o.chol_tol, o.drop_tol, o.emulate_fp64, o.concurrency) == (1e-12, 1e-12, 1, 0)
    assert (o.solver, o.m_max, o.block) == (0, 0, 0) and not o.nev_k and not o.stream
    s = P.ScfOpts()
    C.memset(C.byref(s), 0x7f, C.sizeof(s))
    lib.dks_scf_opts_default(C.byref(s))
    assert (s.nocc, s.history, s.n_init_warm, s.solve.block, s.solve.n_iter) == (0, 8, 1, 0, 200)


def test_tuning_entry_points_and_cache_without_gpu(tmp_path):
    """The tuning entry points reject bad arguments before touching the device; the JSON cache
    of tuning choices round-trips, keeps other keys and ignores unreadable files."""
    import ctypes as C
    import paper_1211_1446_gb300 as P
    lib = P.load_library()
    assert lib.dks_autotune(None, 0, 8, 1, None, None) == -1
    assert lib.dks_tune_set(None, 64 << 20, 0, 0) == -1
    chunk, thr, spl = C.c_longlong(), C.c_int(), C.c_int()
    assert lib.dks_tune_get(None, C.byref(chunk), C.byref(thr), C.byref(spl)) == -1
    rep = P.TuneReport()
    # ncand, best, the 32 candidates, then proj_tc (padded to 8 bytes) and proj_ms[2]
    assert C.sizeof(rep) == 8 + 32 * 8 + 32 * 4 + 32 * 4 + 32 * 8 + 8 + 2 * 8
    assert lib.dks_tune_contractions_set(None, 1) == -1
    assert lib.dks_tune_contractions_get(None, C.byref(thr)) == -1
    path = str(tmp_path / "tune.json")
    k1 = P.tuning_key((48, 48, 56), 57419, 4, 40, 1, "GB300")
    k2 = P.tuning_key((48, 48, 56), 57419, 4, 40, 0, "GB300")
    assert k1 != k2 and P.tuning_cache_lookup(path, k1) is None
    P.tuning_cache_store(path, k1, dict(chunk_bytes=32 << 20, plane_threads=256, plane_split=0))
    P.tuning_cache_store(path, k2, dict(chunk_bytes=64 << 20, plane_threads=0, plane_split=1))
    assert P.tuning_cache_lookup(path, k1) == dict(chunk_bytes=32 << 20, plane_threads=256, plane_split=0)
    assert P.tuning_cache_lookup(path, k2) == dict(chunk_bytes=64 << 20, plane_threads=0, plane_split=1)
    open(path, "w").write("{not json")
    assert P.tuning_cache_lookup(path, k1) is None
    P.tuning_cache_store(path, k1, dict(chunk_bytes=16 << 20, plane_threads=128, plane_split=0))
    assert P.tuning_cache_lookup(path, k1) == dict(chunk_bytes=16 << 20, plane_threads=128, plane_split=0)
    # the projector contraction schedule round-trips when present
    P.tuning_cache_store(path, k2, dict(chunk_bytes=32 << 20, plane_threads=0, plane_split=0, proj_tc=1, proj_ms=[1, 2]))
    assert P.tuning_cache_lookup(path, k2) == dict(chunk_bytes=32 << 20, plane_threads=0, plane_split=0, proj_tc=1)


def _min_passes(n, memo={1: 0}):
    if n not in memo:
        memo[n] = min([1 + _min_passes(n // r) for r in (2, 3, 4, 5, 6, 7, 8) if n % r == 0] or [10 ** 6])
    return memo[n]


def _dif_inverse(x, radices):
    """Mixed-radix decimation-in-frequency passes in the given order (inverse sign): pass s
    combines elements j + r S (r < R) of every block of length L_s, S = L_s / R, with a size-R
    DFT and then multiplies output m by exp(+2 pi i j m / L_s)."""
    x = np.array(x, dtype=np.complex128)
    n, blk = len(x), len(x)
    for r in radices:
        sub = blk // r
        out = x.copy()
        w = np.exp(2j * np.pi * np.outer(np.arange(r), np.arange(r)) / r)
        for b in range(0, n, blk):
            for j in range(sub):
                v = w @ x[b + j + sub * np.arange(r)]
                out[b + j + sub * np.arange(r)] = v * np.exp(2j * np.pi * j * np.arange(r) / blk)
        x, blk = out, sub
    return x


def test_fft_plans_without_gpu():
    """Every axis length 1..256 with prime factors 2, 3, 5, 7 gets a plan whose radices multiply to
    n in the fewest passes (brute force over factorisations), and running its DIF passes leaves
    frequency k of the inverse DFT at the reported position pos[k]; other lengths are refused."""
    import paper_1211_1446_gb300 as P
    rng = np.random.default_rng(3)
    for n in range(1, 257):
        m = n
        for p in (2, 3, 5, 7):
            while m % p == 0:
                m //= p
        if m != 1:
            with pytest.raises(P.DKSError) as e:
                P.fft_plan(n)
            assert e.value.code == -9
            continue
        radices, pos = P.fft_plan(n)
        assert all(r in (2, 3, 4, 5, 6, 7, 8) for r in radices)
        assert int(np.prod(radices)) == n and len(radices) == _min_passes(n)
        assert sorted(pos) == list(range(n))
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        want = np.fft.ifft(x) * n                                   # sum_t x_t exp(+2 pi i k t / n)
        got = _dif_inverse(x, radices)
        assert np.abs(got[pos] - want).max() < 1e-9 * max(1.0, np.abs(want).max())
    with pytest.raises(P.DKSError):
        P.fft_plan(257)


def test_debug_build_and_check_entry_without_gpu():
    """The index-checked debug library builds and exports dks_debug_check; the product library
    reports that its checks are compiled out (without any device call)."""
    import paper_1211_1446_gb300 as P
    from paper_1211_1446_gb300 import build
    assert P.debug_check() == (False, 0)
    path = build.build(debug=True)
    assert path.endswith("libdks_debug.so")
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_rayleigh_ritz_binding_rejects_short_info_and_bad_shapes():
    """The Rayleigh-Ritz entry points write info[0..2]: the binding refuses an info of two ints, a
    non-square S and a V with room for fewer than n x nz values before any pointer reaches the
    library (checked on CPU tensors, so no GPU call is made)."""
    import torch

    import paper_1211_1446_gb300 as P
    nz, n = 6, 3
    a = torch.zeros((nz, nz), dtype=torch.complex128)
    v = torch.zeros((n, nz), dtype=torch.complex128)
    lam = torch.zeros(n, dtype=torch.float64)
    for fn in (P.rayleigh_ritz, P.rayleigh_ritz_static):
        with pytest.raises(ValueError, match="info needs at least 3"):
            fn(a, a, n, v, lam, torch.zeros(2, dtype=torch.int32))
        with pytest.raises(ValueError, match="nz x nz"):
            fn(a, a[:, :4], n, v, lam, torch.zeros(3, dtype=torch.int32))
        with pytest.raises(ValueError, match="V needs"):
            fn(a, a, n, v[:2], lam, torch.zeros(3, dtype=torch.int32))
        with pytest.raises(ValueError, match="device of A"):
            fn(a, a, n, v, lam, torch.zeros(3, dtype=torch.int32))


def test_tensor_core_mask_without_gpu():
    """The TC_* bits match include/dks.h, the default mask holds the projector contractions and
    the refinement phase's exact slices, DKS_TC_ALL is accepted and a bit above it rejected."""
    import paper_1211_1446_gb300 as P
    src = open(os.path.join(ROOT, "include", "dks.h")).read()
    bits = {k: int(v) for k, v in re.findall(r"#define DKS_TC_(\w+)\s+(\d+)", src)}
    assert bits["ROTATE"] == P.TC_ROTATE and bits["GRAM"] == P.TC_GRAM
    assert bits["PROJ_HN"] == P.TC_PROJ_HN and bits["PROJ_NN"] == P.TC_PROJ_NN
    assert bits["FP64"] == P.TC_FP64 and bits["ALL"] == P.TC_ALL
    assert P.TC_ALL == P.TC_ROTATE | P.TC_GRAM | P.TC_PROJ_HN | P.TC_PROJ_NN | P.TC_FP64
    old = P.tensor_cores()
    try:
        P.tensor_cores(P.TC_ALL)
        assert P.tensor_cores()[0] == P.TC_ALL
        with pytest.raises(Exception):
            P.tensor_cores(P.TC_ALL + 1)
        assert P.tensor_cores()[0] == P.TC_ALL
    finally:
        P.tensor_cores(old[0])
    assert P.tensor_cores()[0] == old[0]
