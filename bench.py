#!/usr/bin/env python
"""Benchmark: time to the nev lowest positive-energy DKS eigenpairs with LOBPCG-F on one GB300.

One step = one full solve of Algorithm 1 (N_init = 3 filter steps on a seed-fixed start
block, then iterations until every residual norm ||H'x - lambda x|| < 1e-6, eigenvalues
copied to the host) on the dimer workload: 20x20x24 bohr box, 48x48x56 FFT grid,
Ecut 25 Ha (57,419 planewaves, dimension 229,676), two Gaussian-smeared sites 4.5 bohr
apart with 36 spin-orbit projector channels, Gamma point, nev = 32, c = 137.036.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode mixed|fp64] [--impl ours|reference]

value  = converged eigenpairs per second over all ranks (nev * ranks / step time);
e2e    = the same through the public C ABI with the start block in pinned host memory and
         the eigenvectors returned to host memory inside the timed region;
roofline = the kernel category with the largest device time inside the timed region, its
         algorithmic bytes (or flops) per launch divided by its mean CUDA-event duration.
Multi-GPU (torchrun): every rank solves its own replica of the single-k-point dimer (weak
scaling, no collective in the solve); the only collectives are the timing barrier and max.  The
layered-crystal section then splits its 16 k-points into contiguous cost-balanced shards, one per
rank (no collective in the solve, one gather of the eigenvalues at the end).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "time to nev DKS eigenpairs at 1e-8 Ha (mixed+batched vs FP64); H·X GB/s vs peak"
WORKLOAD = ("dimer: 20x20x24 bohr, 48x48x56 grid, Ecut 25 Ha (npw 57419, dim 229676), 2 sites Z=18 "
            "sigma 0.8, 36 SO projector channels, Gamma, nev 32 (+8 buffer columns), c 137.036, "
            "residual tol 1e-6, N_init 3")
NEV = 32
NBUF = 8
# profile categories whose complex128 work runs in double-float arithmetic in the mixed mode
DF_CATEGORIES = ("gram", "rotate", "proj_bh_x", "proj_b_dz")
TOL = 1e-6


def _peaks():
    path = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names[1:], p[5:9]):
                if val.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_sample(wl, nev, n_iter_ref, budget_s=20.0):
    """Time the FP64 CPU oracle (as it stands) on a bounded sample of the workload: N_init filter
    steps + the first Rayleigh-Ritz + as many Algorithm 1 iterations as fit in about budget_s;
    scaled to a full solve of n_iter_ref iterations.  Returns (eigenpairs/s, cores, sample text)."""
    import numpy as np

    from oracle import basis, lobpcgf, operator
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    hop = operator.MatrixFreeH(wl, m, q)
    cs, om = operator.filter_constants(wl, q)
    import workloads as W
    x0 = W.start_block(len(q), nev + NBUF, wl.seed)
    t_it = []
    t0 = time.perf_counter()
    marks = [t0]

    class Stop(Exception):
        pass

    def cb(it, lam, norms):
        marks.append(time.perf_counter())
        if marks[-1] - t0 > budget_s:
            raise Stop()

    try:
        lobpcgf.lobpcgf(hop, q, x0, nev + NBUF, cs, om, tol=TOL, n_iter=1000, nconv=nev, callback=cb)
    except Stop:
        pass
    t_init = marks[1] - marks[0] - ((marks[2] - marks[1]) if len(marks) > 2 else 0.0)
    t_it = np.diff(marks[1:]) if len(marks) > 2 else np.array([marks[1] - marks[0]])
    per_it = float(np.mean(t_it))
    full = max(t_init, 0.0) + per_it * n_iter_ref
    cores = len(os.sched_getaffinity(0))
    sample = (f"oracle Algorithm 1 on the same dimer: initial filtering + {len(marks) - 2} iterations "
              f"({marks[-1] - t0:.1f} s), extrapolated to {n_iter_ref} iterations")
    return nev / full, cores, sample, full


def cpu_configs_section(n_iter_ref, gpu_layered_happ=None):
    """The CPU baselines of the other configurations, oracle as it stands, on the host cores:
    dense zheevd of the cubic cell (515 planewaves) and of the dimer at Ecut 2 Ha (1295
    planewaves); the oracle's Algorithm 1 on the cubic cell; and, for one k-point of the layered
    crystal (about 40,000 planewaves), the time of one H' application per column, extrapolated to
    a solve by 3 applications per column and iteration over n_iter_ref iterations (marked as
    extrapolated).  About a minute; the dense dimer step is skipped (and said so) when the cubic
    cell's time predicts more than 90 s for it."""
    import numpy as np

    import workloads as W
    from oracle import basis, lobpcgf, operator
    out = {"cores": len(os.sched_getaffinity(0))}
    wl = W.make("cubic")
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    h = operator.dense_hamiltonian(wl, m, q)
    t0 = time.perf_counter()
    lobpcgf.dense_eigs(h, wl.c, 8)
    out["cubic_dense_zheevd_s"] = time.perf_counter() - t0
    out["cubic_dense_dim"] = int(h.shape[0])
    cs, om = operator.filter_constants(wl, q)
    t0 = time.perf_counter()
    r = lobpcgf.lobpcgf(operator.MatrixFreeH(wl, m, q), q, W.start_block(len(q), 8, wl.seed), 8, cs, om, tol=TOL)
    dt = time.perf_counter() - t0
    out["cubic_lobpcgf_s"] = dt
    out["cubic_lobpcgf_iterations"] = r.iterations
    out["cubic_lobpcgf_eigenpairs_per_s"] = 8 / dt
    wl = W.make("dimer", ecut=2.0)
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    # dense cost grows as the cube of the dimension: skip when the cubic cell predicts over 90 s
    predicted = out["cubic_dense_zheevd_s"] * (4.0 * len(q) / out["cubic_dense_dim"]) ** 3
    out["dimer_ecut2_dense_dim"] = 4 * len(q)
    if predicted > 90.0:
        out["dimer_ecut2_dense_zheevd_s"] = None
        out["dimer_ecut2_note"] = f"skipped: predicted {predicted:.0f} s from the cubic cell's time"
    else:
        h = operator.dense_hamiltonian(wl, m, q)
        t0 = time.perf_counter()
        lobpcgf.dense_eigs(h, wl.c, 32)
        out["dimer_ecut2_dense_zheevd_s"] = time.perf_counter() - t0
        del h
    wl = W.make("layered")
    m, q = basis.sphere(wl.lattice, wl.grid, wl.kfrac[0], wl.ecut_k[0])
    hop = operator.MatrixFreeH(wl, m, q)
    x = W.random_block(len(q), 4, wl.seed)
    hop(x[:1])                                                      # first-call setup
    t0 = time.perf_counter()
    hop(x)
    per_col = (time.perf_counter() - t0) / 4
    nev0 = int(wl.nev_k[0])
    out["layered_k0_npw"] = len(q)
    out["layered_k0_hx_s_per_column"] = per_col
    out["layered_k0_solve_s_extrapolated"] = per_col * 3 * nev0 * n_iter_ref
    out["layered_k0_note"] = (f"extrapolated: {per_col:.3f} s per column x 3 applications x {nev0} columns x "
                              f"{n_iter_ref} iterations (every column active)")
    return out


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import workloads as W
    wl = W.make("dimer")
    n_iter_ref = args.ref_iterations
    vals = []
    for i in range(args.warmup + args.steps):
        v, cores, sample, full = cpu_oracle_sample(wl, NEV, n_iter_ref, budget_s=args.ref_budget)
        if i >= args.warmup:
            vals.append(v)
    value = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * NEV / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "mode": "fp64 oracle (numpy/scipy)"},
            "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "extrapolated": True},
            "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per kernel launch from ncu captures of
# the current kernels at the dimer's sizes, one kernel and one launch per capture, e.g.
#   ncu --set full --clock-control none -k regex:k_oz_gram -c 1 -o prof python bench.py --kernel-case gramdf
NCU_TRAFFIC = {
    "rayleigh_ritz": {"bytes_per_launch": (526.3e3 + 2 * 469.2e3 + 425.5e3 + 539.9e3) / 5,
                      "note": "kernel case rr (m = 120, n = 40): mean over the five kernels of a step, "
                              "each captured cold (the pencil is 537 KB)"},
    "gram": {"bytes_per_launch": 1561.8e6 + 20.7e6,
             "note": "kernel case gramdf (k_oz_gram, exact integer slices of 120 columns of 229,676 rows: "
                     "one DRAM pass over the Z and HZ slices)"},
}


def kernel_case(case):
    """One hot step of the solve at the bench's dimer size, three launches (ncu --set full target).
    hx64/hx32/hxdf: H' on 40 columns; gram64/gram32/gramdf: the solver's fused lower-triangle
    A = Z^H HZ, S = Z^H Z with 120 columns (gramdf includes the split into double-float copies);
    rotate64/rotate32/rotatedf: X = Z V with Z of 120 columns and V 120 x 40; rr: the 120 x 120 pencil.
    The *df cases run the complex128 arithmetic in double-float form."""
    import numpy as np
    import torch

    import paper_1211_1446_gb300 as P
    import workloads as W
    wl = W.make("dimer")
    ctx = P.Context.from_workload(wl)
    npw = ctx.npw(0)
    n, m = NEV + NBUF, 3 * (NEV + NBUF)
    rows = 4 * npw
    cdt = torch.complex64 if case.endswith("32") else torch.complex128
    df = case.endswith("df")
    g = torch.Generator(device="cuda").manual_seed(1)
    if case.startswith("hx"):
        x = torch.randn((n, 4, npw), dtype=cdt, device="cuda", generator=g)
        hx = torch.empty_like(x)
        for _ in range(3):
            ctx.apply_H(0, x, hx, emulated=df)
    elif case.startswith("gram"):
        z = torch.randn((m, rows), dtype=cdt, device="cuda", generator=g)
        a = torch.empty((m, m), dtype=torch.complex128, device="cuda")
        s = torch.empty_like(a)
        for _ in range(3):
            P.gram_hermitian(z, z, a, s, emulated=df)
    elif case.startswith("rotate"):
        z = torch.randn((m, rows), dtype=cdt, device="cuda", generator=g)
        w = torch.randn((n, m), dtype=torch.complex128, device="cuda", generator=g)
        out = torch.empty((n, rows), dtype=cdt, device="cuda")
        for _ in range(3):
            P.rotate(z, w, n, out, emulated=df)
    else:
        rng = np.random.default_rng(2)
        zz = rng.standard_normal((3 * m, m)) + 1j * rng.standard_normal((3 * m, m))
        hh = rng.standard_normal((3 * m, 3 * m)) + 1j * rng.standard_normal((3 * m, 3 * m))
        hh = hh + hh.conj().T
        a = torch.from_numpy((zz.conj().T @ hh @ zz).T.copy()).cuda()
        s = torch.from_numpy((zz.conj().T @ zz).T.copy()).cuda()
        v = torch.empty((n, m), dtype=torch.complex128, device="cuda")
        lam = torch.empty(n, dtype=torch.float64, device="cuda")
        info = torch.zeros(4, dtype=torch.int32, device="cuda")
        for _ in range(3):
            P.rayleigh_ritz(a, s, n, v, lam, info)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": case, "ok": True}))
    return 0


def warm_start(P, W, wl, ctx, x_conv, x0, mode, stream):
    """Start vectors for a consecutive solve (Sec. 3.1): the operator of the next step of an outer
    (SCF-like) loop is stood in for by the dimer with its local potential scaled by 1.01.  Three
    starts on that operator, one solve each (after one untimed solve for its workspace):
      cold     the seeded random X0 with N_init = 3 (the default solve);
      previous X0 = the converged X of the unperturbed dimer, N_init = 1;
      balance  X0 = the large components of that X with the small ones rebuilt by the kinetic-balance
               prescription Eq. (RKB) (dks_kinetic_balance), N_init = 1 -- the start a two-component
               (KS/KSSO) calculation would give."""
    import dataclasses

    import numpy as np
    import torch
    wl2 = dataclasses.replace(wl, v_r=wl.v_r * 1.01)
    ctx2 = P.Context.from_workload(wl2)
    xs = torch.empty_like(x0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(start, n_init, kb=False):
        xs.copy_(start)
        torch.cuda.synchronize()
        e0.record(stream)
        if kb:
            ctx2.kinetic_balance(0, xs)
        lam, rep, rc = ctx2.solve([xs], NEV, tol=TOL, n_init=n_init, mode=mode, nbuf=NBUF, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError(f"warm-start solve failed: {P.ERRORS.get(rc, rc)}")
        return lam[0], {"ms": e0.elapsed_time(e1), "iterations": rep["iterations"][0],
                        "fp64_iterations": rep["fp64_iterations"][0], "n_init": n_init}

    run(x0, 3)
    lam_c, cold = run(x0, 3)
    prev = x_conv.clone()
    lam_p, warm_p = run(prev, 1)
    lam_k, warm_k = run(prev, 1, kb=True)
    warm_p["max_eig_diff_vs_cold"] = float(np.abs(lam_p - lam_c).max())
    warm_k["max_eig_diff_vs_cold"] = float(np.abs(lam_k - lam_c).max())
    return {"operator": "dimer with V scaled by 1.01", "cold": cold, "previous": warm_p, "balance": warm_k}


def ksso_section(P, W, wl, ctx, x0, lam_dks, ms_dks, mode, stream):
    """The paper's KSSO module (Sec. 4) on the same dimer: the two-component operator with
    spin-orbit coupling, solved by Algorithm 1 without the filter (standard LOBPCG), one warm-up and
    one timed solve; the DKS/KSSO time ratio (the paper reports about 4); and the start recipe of
    Sec. 3.1: the KSSO vectors as large components, small components by kinetic balance (Eq. RKB),
    then the DKS solve with N_init = 1."""
    import numpy as np
    import torch
    ctxk = P.Context.from_workload(wl, model="ksso")
    npw = ctxk.npw(0)
    xk0 = torch.from_numpy(W.start_block(npw, NEV + NBUF, wl.seed, ncomp=2)).cuda()
    xk = torch.empty_like(xk0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def solve_k():
        xk.copy_(xk0)
        torch.cuda.synchronize()
        e0.record(stream)
        lam, rep, rc = ctxk.solve([xk], NEV, tol=TOL, mode=mode, nbuf=NBUF, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError(f"KSSO solve failed: {P.ERRORS.get(rc, rc)}")
        return lam[0], rep, e0.elapsed_time(e1)

    solve_k()
    lam_k, rep_k, ms_k = solve_k()
    xs = torch.zeros_like(x0)
    xs[:, 0:2] = xk
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.kinetic_balance(0, xs)
    lam_p, rep_p, rc = ctx.solve([xs], NEV, tol=TOL, n_init=1, mode=mode, nbuf=NBUF, check=False)
    e1.record(stream)
    torch.cuda.synchronize()
    if rc != 0:
        raise RuntimeError(f"DKS solve from the KSSO start failed: {P.ERRORS.get(rc, rc)}")
    return {"ms_per_solve": ms_k, "iterations": rep_k["iterations"][0],
            "fp64_iterations": rep_k["fp64_iterations"][0], "dks_over_ksso_time": ms_dks / ms_k,
            "lowest_eig": float(lam_k[0]),
            "dks_from_ksso_start": {"ms": e0.elapsed_time(e1), "n_init": 1, "iterations": rep_p["iterations"][0],
                                    "fp64_iterations": rep_p["fp64_iterations"][0],
                                    "max_eig_diff_vs_cold": float(np.abs(lam_p[0] - lam_dks).max())}}


def davidson_section(P, ctx, x0, lam_dks, ms_dks, mode, stream, m_max=160):
    """Davidson-F: block Davidson with the filter of Algorithm 1 (the paper's remark that the
    filter carries over to Davidson-type solvers), on the same dimer and start block, basis of at
    most m_max columns; one warm-up and one timed solve, against the LOBPCG-F solve."""
    import numpy as np
    import torch
    x = torch.empty_like(x0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = None
    for _ in range(2):
        x.copy_(x0)
        torch.cuda.synchronize()
        e0.record(stream)
        lam, rep, rc = ctx.solve([x], NEV, tol=TOL, mode=mode, nbuf=NBUF, check=False, solver="davidson",
                                 m_max=m_max)
        e1.record(stream)
        torch.cuda.synchronize()
        out = {"ms_per_solve": e0.elapsed_time(e1), "status": int(rc), "m_max": m_max,
               "iterations": rep["iterations"][0], "fp64_iterations": rep["fp64_iterations"][0],
               "h_applications": rep["h_applications"]}
        if rc == 0:
            out["max_eig_diff_vs_lobpcgf"] = float(np.abs(lam[0] - lam_dks).max())
            out["time_vs_lobpcgf"] = out["ms_per_solve"] / ms_dks
    return out


def scf_section(P, W, wl, ctx, mode, stream, nocc=20, tol=1e-4, solve_tol=1e-7, max_iter=40):
    """The SCF loop around the solver (Sec. 2.1 density and V_hxc, Sec. 4.1 Kerker-Anderson
    mixing) on the dimer: nocc = 20 occupied states (the first 20 eigenpairs are separated from
    the rest by 1.3 Ha), the workload's 32 + 8 columns per solve, warm starts with N_init = 1.
    One timed run from the seeded start block; then the grid steps of one SCF iteration
    (density of nocc states, V_hxc, mixing, potential update) timed on their own."""
    import numpy as np
    import torch
    x = torch.from_numpy(W.start_block(ctx.npw(0), NEV + NBUF, wl.seed)).cuda()
    rho = torch.zeros(wl.grid, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lam, rep, rc = ctx.scf([x], NEV, nocc, tol=tol, solve_tol=solve_tol, max_iter=max_iter, nbuf=NBUF, mode=mode,
                           rho=rho, check=False, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1)
    its = rep["iterations"]
    out = {"status": int(rc), "converged": rep["converged"], "nocc": nocc, "scf_iterations": its,
           "tol_electrons": tol, "solve_tol": solve_tol, "residual": rep["residual"], "ms_total": total,
           "ms_per_solve_and_update": total / (its + 1), "solve_iterations": rep["solve_iterations"],
           "h_applications": rep["h_applications"], "e_h": rep["e_h"], "e_xc": rep["e_xc"],
           "electrons": float(rho.sum().item() * wl.volume / wl.ng),
           "residual_history": [float("%.3e" % r) for r in rep["history"]]}
    if rc == 0:
        out["eig_lowest"] = [float(v) for v in lam[0][:4]]
    # grid steps of one SCF iteration, each timed alone (3 repetitions after one warm-up)
    occ = [1.0] * nocc
    rout = torch.zeros_like(rho)
    vh = torch.empty_like(rho)
    mx = ctx.mixer()
    steps = {"density": lambda: ctx.density(0, x, occ, rout, stream=stream),
             "hxc": lambda: ctx.hxc(rho, vh, stream=stream),
             "mix": lambda: mx.step(rho, rout, vh, stream=stream),
             "set_potential": lambda: ctx.set_potential(vh, stream=stream)}
    grid = {}
    for name, fn in steps.items():
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        grid[name] = e0.elapsed_time(e1) / 3
    mx.close()
    out["grid_steps_ms"] = grid
    out["grid_share"] = sum(grid.values()) / out["ms_per_solve_and_update"]
    # restore the creation potential for whatever runs after
    ctx.set_potential(torch.from_numpy(np.ascontiguousarray(wl.v_r)).cuda())
    return out


def hx_rate(P, ctx, ik, nb, npw, nproj, ng, dtype, emulated, stream, hbm, reps=5):
    """H' on nb columns of k-point ik: mean CUDA-event time and the effective bandwidth of the
    sphere-only algorithmic bytes (read X, write HX, V once, B twice), with its fraction of the
    measured HBM copy bandwidth."""
    import torch
    es = 8 if dtype == torch.complex64 else 16
    g = torch.Generator(device="cuda").manual_seed(11)
    x = torch.randn((nb, 4, npw), dtype=dtype, device="cuda", generator=g)
    hx = torch.empty_like(x)
    for _ in range(2):
        ctx.apply_H(ik, x, hx, emulated=emulated)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.apply_H(ik, x, hx, emulated=emulated)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / reps / 1e3
    alg = 2 * 4 * npw * es * nb + ng * es / 2 + 2 * (2 * npw * nproj * es)
    return {"ms": t * 1e3, "columns": nb, "algorithmic_bytes": alg, "achieved_gbs": alg / t / 1e9,
            "frac_of_hbm": alg / t / 1e9 / hbm}


def layered_sharded(P, W, mode, stream, ws, rank, nbuf=8):
    """The layered crystal on ws GPUs, one process each: the 16 k-points are split into contiguous
    blocks balanced by (nev_k + nbuf) npw_k (paper_1211_1446_gb300.shard; npw_k taken as
    proportional to Ecut_k^(3/2)), every rank solves its own k-points with no collective, and the
    eigenvalues are gathered once at the end.  Time = the slowest rank's (max over ranks, after
    a barrier); eigenpairs/s counts every rank's pairs."""
    import dataclasses

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1211_1446_gb300 import shard
    wl = W.make("layered")
    nev_all = [int(v) for v in wl.nev_k]
    costs = [(nev_all[ik] + nbuf) * float(wl.ecut_k[ik]) ** 1.5 for ik in range(wl.nk)]
    mine = shard.kpoint_shards(costs, ws)[rank]
    out = {"ranks": ws, "kpoints_per_rank": [len(b) for b in shard.kpoint_shards(costs, ws)]}
    lam, ms = {}, 0.0
    if mine:
        wk = dataclasses.replace(wl, kfrac=wl.kfrac[mine], ecut_k=wl.ecut_k[mine], nev_k=wl.nev_k[mine])
        ctx = P.Context.from_workload(wk)
        nev_k = [nev_all[ik] for ik in mine]
        x0 = [torch.from_numpy(W.start_block(ctx.npw(i), nev_k[i] + nbuf, wl.seed, ik)).cuda()
              for i, ik in enumerate(mine)]
        xs = [t.clone() for t in x0]
        ctx.solve(xs, 0, nev_k=nev_k, nbuf=nbuf, tol=TOL, mode=mode, n_iter=1, check=False)   # workspaces
        for a, b in zip(xs, x0):
            a.copy_(b)
    torch.cuda.synchronize()
    dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc = 0
    if mine:
        lk, rep, rc = ctx.solve(xs, 0, nev_k=nev_k, nbuf=nbuf, tol=TOL, mode=mode, check=False, stream=stream)
        lam = {ik: lk[i] for i, ik in enumerate(mine)}
    e1.record(stream)
    torch.cuda.synchronize()
    ms = shard.max_over_ranks(e0.elapsed_time(e1))
    allk = shard.gather_eigenvalues(lam)
    worst = shard.max_over_ranks(float(-rc))                    # status codes are <= 0
    out.update({"status": -int(worst), "ms": ms, "eigenpairs": sum(nev_all),
                "eigenpairs_per_s": sum(nev_all) / (ms / 1e3), "kpoints_gathered": len(allk)})
    gold = os.path.join(HERE, "tests", "golden", "layered_k0_eigs.txt")
    if 0 in allk and os.path.exists(gold):
        g = np.loadtxt(gold)
        out["max_eig_err_vs_oracle_k0"] = float(np.abs(allk[0][:len(g)] - g).max())
    return out


def layered_section(P, W, mode, stream, hbm, nbuf=8, sample=(4, 9)):
    """The layered crystal (hexagonal a = 7.8, c = 28 bohr, 15 sites, 270 spin-orbit projector
    channels, 60 x 60 x 216 grid, 16 k-points with their own spheres of about 39,000-41,000
    planewaves and nev_k of 48-96): all 16 k-points in one call (concurrent solve workers), mixed
    precision, one timed solve after a one-iteration call that sizes the workspaces.  Beside it,
    for a sample of k-points each solved alone, the mixed and the plain FP64 GPU forms (the
    speedup denominator), H' bandwidth at k = 0, and the eigenvalue error at k = 0 against the
    oracle's Algorithm 1 (tests/golden/layered_k0_eigs.txt)."""
    import dataclasses

    import numpy as np
    import torch
    wl = W.make("layered")
    ctx = P.Context.from_workload(wl)
    nev_k = [int(v) for v in wl.nev_k]
    x0 = [torch.from_numpy(W.start_block(ctx.npw(ik), nev_k[ik] + nbuf, wl.seed, ik)).cuda() for ik in range(wl.nk)]
    xs = [t.clone() for t in x0]
    ctx.solve(xs, 0, nev_k=nev_k, nbuf=nbuf, tol=TOL, mode=mode, n_iter=1, check=False)   # workspaces
    for a, b in zip(xs, x0):
        a.copy_(b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lam, rep, rc = ctx.solve(xs, 0, nev_k=nev_k, nbuf=nbuf, tol=TOL, mode=mode, check=False, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"workload": "layered crystal: hexagonal a 7.8 c 28 bohr, 15 sites, 270 SO projector channels, "
                       "60x60x216 grid, 16 k-points (4x4x1), npw 39000-41000 per k, nev_k 48-96 + 8 buffer",
           "status": int(rc), "ms": ms, "eigenpairs": sum(nev_k), "eigenpairs_per_s": sum(nev_k) / (ms / 1e3),
           "iterations": rep["iterations"][:wl.nk], "fp64_iterations": rep["fp64_iterations"][:wl.nk],
           "max_residual": max(rep["max_residual"][:wl.nk])}
    gold = os.path.join(HERE, "tests", "golden", "layered_k0_eigs.txt")
    if rc == 0 and os.path.exists(gold):
        g = np.loadtxt(gold)
        out["max_eig_err_vs_oracle_k0"] = float(np.abs(lam[0][:len(g)] - g).max())
    # mixed vs plain FP64 on sampled k-points, each alone (one k-point per context)
    per = []
    for ik in sample:
        wk = dataclasses.replace(wl, kfrac=wl.kfrac[ik:ik + 1], ecut_k=wl.ecut_k[ik:ik + 1], nev_k=wl.nev_k[ik:ik + 1])
        ck = P.Context.from_workload(wk)
        row = {"k": ik, "nev": nev_k[ik], "npw": ck.npw(0)}
        for tag, md in (("mixed", mode), ("fp64", P.MODE_FP64)):
            xk = torch.from_numpy(W.start_block(ck.npw(0), nev_k[ik] + nbuf, wl.seed, ik)).cuda()
            torch.cuda.synchronize()
            e0.record(stream)
            lk, rk, rck = ck.solve([xk], nev_k[ik], nbuf=nbuf, tol=TOL, mode=md, check=False, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            row[tag + "_ms"] = e0.elapsed_time(e1)
            row[tag + "_status"] = int(rck)
            row[tag + "_iterations"] = rk["iterations"][0]
            row[tag + "_eig"] = lk[0]
        row["speedup_mixed_vs_fp64"] = row["fp64_ms"] / row["mixed_ms"]
        row["max_eig_diff"] = float(np.abs(row.pop("mixed_eig") - row.pop("fp64_eig")).max())
        per.append(row)
        ck.close()
    out["per_k_sample"] = per
    out["speedup_mixed_vs_fp64_sample"] = sum(r["fp64_ms"] for r in per) / sum(r["mixed_ms"] for r in per)
    nproj = ctx.nproj()
    out["hx_k0"] = {"fp32": hx_rate(P, ctx, 0, 104, ctx.npw(0), nproj, wl.ng, torch.complex64, False, stream, hbm),
                    "fp64_double_float": hx_rate(P, ctx, 0, 104, ctx.npw(0), nproj, wl.ng, torch.complex128, True,
                                                 stream, hbm)}
    ctx.close()
    return out


def supercell_hx_section(P, W, stream, hbm, nb=160):
    """H' bandwidth at the large-cell size (2 x 2 x 1 supercell of the layered crystal: 120 x 120 x
    216 grid, about 158,000 planewaves at Gamma, 1080 spin-orbit projector channels) on a block of
    nb columns, FP32 and double-float; one k-point is enough for the operator's rate."""
    import dataclasses
    import torch
    wl = W.make("supercell")
    wk = dataclasses.replace(wl, kfrac=wl.kfrac[:1], ecut_k=wl.ecut_k[:1], nev_k=wl.nev_k[:1])
    ctx = P.Context.from_workload(wk)
    npw, nproj = ctx.npw(0), ctx.nproj()
    out = {"workload": "supercell 2x2x1 of the layered crystal: 120x120x216 grid, Gamma, 1080 SO projector channels",
           "npw": npw, "fp32": hx_rate(P, ctx, 0, nb, npw, nproj, wl.ng, torch.complex64, False, stream, hbm, reps=3),
           "fp64_double_float": hx_rate(P, ctx, 0, nb // 4, npw, nproj, wl.ng, torch.complex128, True, stream, hbm,
                                        reps=2)}
    ctx.close()
    return out


def supercell_section(P, W, mode, stream, kpoints=4, block=128, nbuf=32, tol=1e-6, nev=None, fp64=False):
    """The large-cell configuration (2 x 2 x 1 supercell of the layered crystal: 120 x 120 x 216
    grid, about 158,000 planewaves per k, 1080 projector channels, 480 pairs per k-point), solved
    in band blocks of `block` wanted + nbuf buffer columns with deflation, k-point by k-point
    (the first `kpoints` of the 2 x 2 x 1 mesh), each k-point's result printed to stderr as soon
    as it is known.  Opt-in (--supercell): it holds most of the GPU's memory and runs for minutes
    per k-point.  fp64: each k-point is solved again from the same start block in the plain FP64
    form, for the speedup and the eigenvalue difference."""
    import dataclasses

    import torch
    wl = W.make("supercell")
    out = {"workload": "supercell 2x2x1 of the layered crystal: 120x120x216 grid, 1080 SO projector channels, "
                       f"480 pairs per k in band blocks of {block} + {nbuf} buffer columns",
           "kpoints": []}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for ik in range(min(kpoints, wl.nk)):
        wk = dataclasses.replace(wl, kfrac=wl.kfrac[ik:ik + 1], ecut_k=wl.ecut_k[ik:ik + 1], nev_k=wl.nev_k[ik:ik + 1])
        ctx = P.Context.from_workload(wk)
        nv = int(wl.nev_k[ik]) if nev is None else int(nev)
        x = torch.from_numpy(W.start_block(ctx.npw(0), nv + nbuf, wl.seed, ik)).cuda()
        torch.cuda.synchronize()
        e0.record(stream)
        lam, rep, rc = ctx.solve([x], nv, nbuf=nbuf, tol=tol, mode=mode, block=block if nv > block else 0,
                                 check=False, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        row = {"k": ik, "status": int(rc), "message": rep["message"], "ms": ms, "eigenpairs": nv,
               "eigenpairs_per_s": nv / (ms / 1e3), "npw": ctx.npw(0), "iterations": rep["iterations"][0],
               "fp64_iterations": rep["fp64_iterations"][0], "max_residual": rep["max_residual"][0],
               "h_applications": rep["h_applications"], "lowest_eigs": [float(v) for v in lam[0][:4]],
               "residual_history": [float(f"{v:.3g}") for v in rep["history"]]}
        if rc == 0:
            row["kramers_max_split"] = float(abs(lam[0][0::2] - lam[0][1::2]).max()) if ik == 0 else None
        if fp64 and mode != P.MODE_FP64:
            x.copy_(torch.from_numpy(W.start_block(ctx.npw(0), nv + nbuf, wl.seed, ik)))
            torch.cuda.synchronize()
            e0.record(stream)
            lam64, rep64, rc64 = ctx.solve([x], nv, nbuf=nbuf, tol=tol, mode=P.MODE_FP64,
                                           block=block if nv > block else 0, check=False, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1)
            row.update({"fp64_form_status": int(rc64), "fp64_form_ms": ms64,
                        "fp64_form_iterations": rep64["iterations"][0],
                        "speedup_mixed_vs_fp64": ms64 / ms,
                        "max_eig_diff_vs_fp64": float(abs(lam64[0] - lam[0]).max()) if rc == 0 and rc64 == 0 else None})
        out["kpoints"].append(row)
        print(json.dumps({"supercell_kpoint": row}), file=sys.stderr, flush=True)
        ctx.close()
        del x
        torch.cuda.empty_cache()
    done = [r for r in out["kpoints"] if r["status"] == 0]
    out["eigenpairs_per_s"] = (sum(r["eigenpairs"] for r in out["kpoints"]) /
                               (sum(r["ms"] for r in out["kpoints"]) / 1e3)) if out["kpoints"] else None
    out["all_converged"] = len(done) == len(out["kpoints"])
    return out


def tc_study(masks, reps):
    """The tensor-core study of the complex64 contractions: the dimer solve (mixed precision, the
    bench configuration) reps times for each DKS_TC_* mask, recording the FP32 phase's residual
    floor (lowest residual before the hand-off), the FP64-phase iterations and the solve time.
    The FP32 floor sets how many FP64 iterations remain, so a contraction belongs on the tensor
    cores only if it leaves the floor where the CUDA-core kernels put it.  Repeat r starts from
    the seeded block of seed + r, the same starts for every mask (a deterministic path gives the
    same trajectory every time from one start)."""
    import numpy as np
    import torch

    import paper_1211_1446_gb300 as P
    import workloads as W
    wl = W.make("dimer")
    ctx = P.Context.from_workload(wl)
    x0s = [torch.from_numpy(W.start_block(ctx.npw(0), NEV + NBUF, wl.seed + r)).cuda() for r in range(reps)]
    x = torch.empty_like(x0s[0])
    gold = np.loadtxt(os.path.join(HERE, "tests", "golden", "dimer_lobpcgf_eigs.txt"))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    old = P.tensor_cores()
    out = {}
    for mask in masks:
        P.tensor_cores(mask)
        rows = []
        for r in range(reps):
            x.copy_(x0s[r])
            torch.cuda.synchronize()
            e0.record()
            lam, rep, rc = ctx.solve([x], NEV, tol=TOL, mode=P.MODE_MIXED, nbuf=NBUF, check=False)
            e1.record()
            torch.cuda.synchronize()
            it32 = rep["iterations"][0] - rep["fp64_iterations"][0]
            rows.append({"status": int(rc), "ms": e0.elapsed_time(e1), "iterations": rep["iterations"][0],
                         "fp64_iterations": rep["fp64_iterations"][0],
                         "fp32_floor": min(rep["history"][:it32]) if it32 > 0 else None,
                         "max_eig_err_vs_oracle": float(np.abs(lam[0] - gold).max()) if rc == 0 else None})
        out[str(mask)] = {"runs": rows, "median_ms": float(np.median([r["ms"] for r in rows])),
                          "median_fp32_floor": float(np.median([r["fp32_floor"] for r in rows])),
                          "median_fp64_iterations": float(np.median([r["fp64_iterations"] for r in rows]))}
    P.tensor_cores(*old)
    print(json.dumps({"tc_study": out, "workload": WORKLOAD}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true")
    ap.add_argument("--no-ksso", action="store_true")
    ap.add_argument("--no-davidson", action="store_true")
    ap.add_argument("--no-scf", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch parameters instead of running dks_autotune before the timed solves")
    ap.add_argument("--no-layered", action="store_true", help="skip the layered-crystal (16 k-point) section")
    ap.add_argument("--no-supercell-hx", action="store_true", help="skip H' bandwidth at the supercell size")
    ap.add_argument("--supercell-kpoints", type=int, default=4, help="k-points of the supercell solve (1-4)")
    ap.add_argument("--supercell-nev", type=int, default=None, help="pairs per k-point of the supercell solve (480)")
    ap.add_argument("--supercell-nbuf", type=int, default=32, help="buffer columns of the supercell solves")
    ap.add_argument("--supercell-fp64", action="store_true",
                    help="also solve each supercell k-point in the plain FP64 form (speedup)")
    ap.add_argument("--supercell", action="store_true",
                    help="also solve the large-cell configuration in band blocks (minutes, most of the GPU memory)")
    ap.add_argument("--ref-iterations", type=int, default=60)
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--tc-study", default=None,
                    help="comma-separated DKS_TC_* masks: FP32-phase floor, FP64 iterations and time per mask "
                         "(--steps solves each)")
    ap.add_argument("--tc", type=int, default=None,
                    help="DKS_TC_* mask: complex64 contractions on the tcgen05 tensor cores (default: library default)")
    ap.add_argument("--kernel-case", default=None,
                    choices=["hx64", "hx32", "hxdf", "gram64", "gram32", "gramdf", "rotate64", "rotate32", "rotatedf",
                             "rr"],
                    help="run one hot step a few times at the dimer's bench size (for ncu captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.tc is not None:
        import paper_1211_1446_gb300 as P
        P.tensor_cores(args.tc)
    if args.kernel_case:
        return kernel_case(args.kernel_case)
    if args.tc_study:
        return tc_study([int(v) for v in args.tc_study.split(",")], args.steps)

    import numpy as np
    import torch

    import paper_1211_1446_gb300 as P
    import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = W.make("dimer")
    ctx = P.Context.from_workload(wl)
    npw = ctx.npw(0)
    mode = P.MODE_MIXED if args.mode == "mixed" else P.MODE_FP64
    # launch parameters and the projector contraction schedule from the autotuner (H' on the
    # solve's block width, FP32: the phase that applies H' most often), before anything is timed
    tune = None
    if not args.no_tune:
        tune = ctx.autotune(0, nb=NEV + NBUF, prec=P.PREC_FP32)
        tune.pop("candidates", None)
    x0 = torch.from_numpy(W.start_block(npw, NEV + NBUF, wl.seed)).cuda()
    x = torch.empty_like(x0)
    stream = torch.cuda.current_stream()

    def step(m=mode):
        x.copy_(x0)
        lam, rep, rc = ctx.solve([x], NEV, tol=TOL, mode=m, nbuf=NBUF, check=False)
        if rc != 0:
            raise RuntimeError(f"solve failed: {P.ERRORS.get(rc, rc)} {rep}")
        return lam[0], rep

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    P.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = []
    for _ in range(args.steps):
        lam, rep = step()
        reps.append(rep)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = P.profile_read()
    P.profile_enable(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        from paper_1211_1446_gb300 import shard
        ms = shard.max_over_ranks(ms)
        dist.barrier()
    value = NEV * ws / (ms / 1e3)

    # end to end through the public ABI: start block from pinned host memory, vectors back to host
    xh = x0.cpu().pin_memory()
    xo = torch.empty_like(xh).pin_memory()
    step()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        x.copy_(xh, non_blocking=True)
        lam_e, rep_e, rc = ctx.solve([x], NEV, tol=TOL, mode=mode, nbuf=NBUF, check=False)
        xo.copy_(x, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    bytes_vec = x0.numel() * x0.element_size()

    # the plain FP64 GPU form of the same solve (speedup denominator)
    fp64 = None
    if mode == P.MODE_MIXED and args.fp64_steps > 0:
        step(P.MODE_FP64)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.fp64_steps):
            lam64, rep64 = step(P.MODE_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        fp64 = {"ms_per_step": ms64, "iterations": rep64["iterations"][0], "speedup_mixed_vs_fp64": ms64 / ms,
                "max_eig_diff_vs_mixed": float(np.abs(lam64 - lam).max())}

    # accuracy against the oracle's stored eigenvalues (written by tests/golden/make_golden.py)
    acc = {"max_residual": max(r["max_residual"][0] for r in reps), "iterations": reps[-1]["iterations"][0],
           "fp64_iterations": reps[-1]["fp64_iterations"][0], "h_applications": reps[-1]["h_applications"],
           "iterations_per_step": [r["iterations"][0] for r in reps],
           "fp64_iterations_per_step": [r["fp64_iterations"][0] for r in reps],
           "residual_history_last_step": [float(f"{v:.3g}") for v in reps[-1]["history"]]}
    gold = os.path.join(HERE, "tests", "golden", "dimer_lobpcgf_eigs.txt")
    if os.path.exists(gold):
        acc["max_eig_err_vs_oracle"] = float(np.abs(lam - np.loadtxt(gold)).max())

    # roofline of the dominant kernel category
    hbm, bf16, src = _peaks()
    fp64_peak = 1250.0           # GFLOP/s, nominal GB300 FP64 (no measured FP64 peak is available)
    fp32_peak = 152 * 128 * 2 * 2.07   # GFLOP/s, FP32 CUDA cores x max SM clock (unit count derivation)
    df_peak = 152 * 128 * 2.07 * 2 / 15    # GFLOP/s of FP64-equivalent flops in double-float arithmetic
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    per_launch_s = d["ms"] / max(d["launches"], 1) / 1e3
    launches = int(sum(v["launches"] for v in prof.values()))
    if dom.startswith(("stick", "plane", "dirac", "col_stats", "precond", "convert")):
        ach = d["bytes"] / max(d["launches"], 1) / per_launch_s / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "peak_source": f"{src} HBM copy bandwidth"}
    else:
        if dom.endswith("fp32"):
            pk, psrc = fp32_peak, "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz"
        elif dom in DF_CATEGORIES and mode == P.MODE_MIXED:
            # complex128 contractions of the refinement phase run in double-float arithmetic on the
            # FP32 lanes: one real multiply-add of the algorithm costs 15 FP32 instructions
            pk, psrc = df_peak, ("derived: FP64-equivalent rate of the double-float multiply-add "
                                 "(15 FP32 instructions) on 152 SMs x 128 FP32 lanes x 2070 MHz")
        else:
            pk, psrc = fp64_peak, "nominal GB300 FP64 1.25 TFLOP/s (recipe table)"
        ach = d["flops"] / max(d["launches"], 1) / per_launch_s / 1e9
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk, "unit": "GFLOP/s", "frac": ach / pk,
                "peak_source": psrc}
    # the refinement phase's Gram matrices and rotations: with DKS_TC_FP64 (default) on the tcgen05
    # tensor cores from exact integer slices (28 BF16 slice products per real multiply-add, so the
    # FP64-equivalent ceiling is the BF16 tensor peak / 28), else double-float on the FP32 lanes
    if mode == P.MODE_MIXED:
        slices = bool(P.tensor_cores()[0] & P.TC_FP64)
        cats = [c for c in ("gram", "rotate") if prof.get(c, {}).get("launches")]
        if cats:
            f = sum(prof[c]["flops"] for c in cats)
            t = sum(prof[c]["ms"] for c in cats) / 1e3
            pk = bf16 * 1e3 / 28.0 if slices else df_peak
            roof.update({"top_kernel": ("k_oz_gram + k_oz_rot (refinement-phase Gram matrices and rotations, "
                                        "tcgen05, exact integer slices)" if slices else
                                        "k_gram_df + k_gemm_nn_df4 (refinement-phase Gram matrices and rotations, "
                                        "double-float)"),
                         "top_kernel_share_of_step": t * 1e3 / (ms * args.steps),
                         "top_kernel_gflops": f / t / 1e9, "top_kernel_peak_gflops": pk,
                         "top_kernel_frac": f / t / 1e9 / pk,
                         "top_kernel_peak_source": (f"{src} BF16 tensor peak / 28 slice products per multiply-add"
                                                    if slices else
                                                    "derived: FP64-equivalent rate of the double-float multiply-add "
                                                    "(15 FP32 instructions) on 152 SMs x 128 FP32 lanes x 2070 MHz")})
            if slices and prof.get("rotate", {}).get("launches"):
                r = prof["rotate"]
                roof["top_kernel_rotate_gbs"] = r["bytes"] / (r["ms"] / 1e3) / 1e9
                roof["top_kernel_rotate_frac_hbm"] = roof["top_kernel_rotate_gbs"] / hbm
    tr = NCU_TRAFFIC.get(dom)
    roof.update({"traffic": tr["bytes_per_launch"] if tr else None,
                 "traffic_note": tr["note"] if tr else "no ncu DRAM capture of this category's kernels",
                 "share_of_step": d["ms"] / (ms * args.steps),
                 "per_category_ms": {k: round(v["ms"] / args.steps, 3) for k, v in prof.items() if v["launches"]}})

    # H' x effective bandwidth (sphere-only algorithmic bytes) on the bench block width, outside the
    # timed region: FP32 (the first phase), double-float (the refinement) and native FP64
    nproj = ctx.nproj()
    hx_line = {tag: hx_rate(P, ctx, 0, NEV + NBUF, npw, nproj, wl.ng, dt, emu, stream, hbm)
               for tag, dt, emu in (("fp32", torch.complex64, False), ("fp64_double_float", torch.complex128, True),
                                    ("fp64", torch.complex128, False))}
    # FP32 H' flops per column (FFT 8 transforms of 5 Ng log2 Ng, projectors 2 x 8 (2 npw) nproj x 2
    # spinor columns, 4 x 4 term) against the FP32 CUDA-core peak
    import math
    fl = (8 * 5 * wl.ng * math.log2(wl.ng) + 2 * 8 * (2 * npw) * nproj * 2 + 4 * 32 * npw) * (NEV + NBUF)
    hx_line["fp32"]["gflops"] = fl / (hx_line["fp32"]["ms"] / 1e3) / 1e9
    hx_line["fp32"]["frac_of_fp32_alu"] = hx_line["fp32"]["gflops"] / fp32_peak
    # flat copies, so that records which keep only scalars of the roofline object keep these too
    roof.update({"hx_fp32_gbs": hx_line["fp32"]["achieved_gbs"], "hx_fp32_frac_hbm": hx_line["fp32"]["frac_of_hbm"],
                 "hx_fp32_frac_fp32_alu": hx_line["fp32"]["frac_of_fp32_alu"],
                 "hx_df_gbs": hx_line["fp64_double_float"]["achieved_gbs"],
                 "hx_df_frac_hbm": hx_line["fp64_double_float"]["frac_of_hbm"]})

    warm = None if args.no_warm_start else warm_start(P, W, wl, ctx, x, x0, mode, stream)
    ksso = None if args.no_ksso else ksso_section(P, W, wl, ctx, x0, lam, ms, mode, stream)
    dav = None if args.no_davidson else davidson_section(P, ctx, x0, lam, ms, mode, stream)
    scf = None if args.no_scf else scf_section(P, W, wl, ctx, mode, stream)
    sup = (supercell_section(P, W, mode, stream, kpoints=args.supercell_kpoints, nev=args.supercell_nev,
                             nbuf=args.supercell_nbuf, fp64=args.supercell_fp64)
           if args.supercell else None)
    if args.no_layered:
        lay = None
    elif ws > 1:
        lay = layered_sharded(P, W, mode, stream, ws, rank)     # k-point shards, one per GPU
    else:
        lay = layered_section(P, W, mode, stream, hbm)
    sup_hx = None if (args.no_supercell_hx or ws > 1) else supercell_hx_section(P, W, stream, hbm)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, cores, sample, full = cpu_oracle_sample(wl, NEV, acc["iterations"])
        cpu = {"value": v, "unit": "eigenpairs/s", "cores": cores, "kind": "oracle", "sample": sample,
               "extrapolated": True}
        try:
            cpu["other_configs"] = cpu_configs_section(acc["iterations"])
        except Exception as exc:                                  # a baseline must not cost the bench line
            cpu["other_configs"] = {"error": f"{type(exc).__name__}: {exc}"}

    line = {"metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+df64" if mode == P.MODE_MIXED else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": args.mode, "parallelism": f"replicas x{ws}",
                       "l2": "working set (>1 GB of blocks per solve) exceeds the 129 MB L2",
                       "dtype_note": (("FP32 phase (complex64; projector contractions on tcgen05 tensor cores "
                                       "with three BF16 slices per FP32 value), then the FP64 refinement with "
                                       "complex128 storage: Gram matrices and rotations on tcgen05 tensor cores "
                                       "from exact integer slices (seven 8-bit digits per value, exact FP32 "
                                       "level sums), projector contractions and FFTs in double-float arithmetic "
                                       "(about 2^-48 per operation); Rayleigh-Ritz in FP64"
                                       if P.tensor_cores()[0] & P.TC_FP64 else
                                       "FP32 phase (complex64; projector contractions on tcgen05 tensor cores "
                                       "with three BF16 slices per FP32 value), then the FP64 refinement with "
                                       "complex128 storage whose contractions and FFTs run in double-float "
                                       "arithmetic (about 2^-48 per operation); Rayleigh-Ritz in FP64")
                                      if mode == P.MODE_MIXED else "FP64"),
                       "tensor_cores_mask": P.tensor_cores()[0], "tuning": tune or "defaults"},
            "e2e": {"value": NEV * ws / (ms_e2e / 1e3), "unit": "eigenpairs/s",
                    "h2d_bytes_per_step": bytes_vec, "d2h_bytes_per_step": bytes_vec + 8 * NEV},
            "gpu_launches": launches, "clocks": clk, "roofline": roof,
            "cpu_baseline": cpu, "hx": hx_line, "layered": lay, "supercell_hx": sup_hx, "fp64_form": fp64,
            "warm_start": warm, "ksso": ksso, "davidson_f": dav, "scf": scf, "supercell": sup, "accuracy": acc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
