#!/usr/bin/env python
"""Benchmark: converged frequency solves per second of the EWM elastodynamic BEM sweep.

Workload (default ``cavity5120``): spherical cavity of radius 1 in an infinite
solid (E = 1, nu = 0.25, rho = 1), geodesic sphere with 5,120 flat triangles
(15,360 unknowns), uniform Heaviside pressure, 256 samples at dt = 0.25 (the
sampling step of the 320-triangle case), i.e. T = 64 and 129 complex
frequencies s_k = 5/T + i k 2 pi / T up to omega = 4 pi, all resolved by the
mesh (about 4 elements per shear wavelength), Hanning window, hierarchical
operator (leaf 64 elements, ACA tolerance 1e-5), complex64 mixed precision
with FP64 singular integrals and FP64 true-residual refinement, GMRES to a
true relative residual of 1e-5, solution extrapolation with K = 4.

One step = the whole hot path on that input: geometry and cluster tree,
static singular parts, for every frequency the right-hand side, operator
assembly (near blocks + ACA), initial guess and GMRES, then the windowed
inverse DFT of the full field (every unknown, 256 time samples).

``value``: solves/s with the inputs already in device memory (CUDA events on
the library's stream). ``e2e``: the same through the host-pointer API (mesh,
load and pattern copied in, the full time response copied out, every step).
``plain``: the same sweep in the plain form (complex128 operator, FP64
everywhere), timed once. ``cpu_baseline`` and ``--impl reference``: the CPU
oracle, one complete frequency of the same workload (every row on all host
cores, then the LU of the full system), measured.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the 5,120-triangle cavity sweep: the metric's configuration
    "cavity5120": dict(n=16, T=64.0, n_omega=256, eta=5.0 / 64.0, aca_tol=1e-5, leaf=64, tol=1e-5),
    # same with T = 8 (dt = 1/32): the upper frequencies are not resolved by the mesh
    "cavity5120_T8": dict(n=16, T=8.0, n_omega=256, eta=5.0 / 8.0, aca_tol=1e-5, leaf=64, tol=1e-5),
    # small case (320 triangles, 32 samples) for quick runs
    "cavity320": dict(n=4, T=8.0, n_omega=32, eta=5.0 / 8.0, aca_tol=1e-5, leaf=64, tol=1e-5),
}
MAT = dict(E=1.0, nu=0.25, rho=1.0)


# DRAM read + write of one H-matrix product (k_hmv_fused) at k = n_omega / 4
# of cavity5120, from the ncu capture of `bench.py --profile-case`
# (profiles/k_hmv_fused_cavity5120.md: 888.0 MB read, 3.9 MB written); the
# same product's algorithmic bytes are 887.3 MB (counted by the library), so
# the kernel streams every operator entry once.
HMV_TRAFFIC_K64 = 891_946_752


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over the ranks of the default process group (x without one).

    The replicas share no data: the timing maximum is the only collective."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, t_max_ms: float) -> float:
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / (t_max_ms / 1e3)


def _lu_seconds(n):
    """Seconds of one dense complex LU solve of size n in this process."""
    rng = np.random.default_rng(0)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)) + n * np.eye(n)
    b = rng.normal(size=n) + 0j
    t0 = time.perf_counter()
    np.linalg.solve(A, b)
    return time.perf_counter() - t0


def _lu_seconds_one_thread(n):
    """The same in a fresh process whose BLAS runs one thread."""
    import multiprocessing as mp

    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(1) as p:
            return p.apply(_lu_seconds, (n,))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cpu_oracle_measure(cfg, single_core_rows=48, single_core_lu=3072):
    """Times the CPU oracle on one complete frequency of the workload.

    All cores (the reported value): the oracle's dense collocation rows
    (Eq. Aa_b) of every element at s_1, computed by one worker process per
    core (``oracle.pool``), then the direct solve of the full system (LAPACK
    LU, all cores). Before the timed frequency the workers assemble s_0,
    which fills their caches of frequency-independent static parts, as in a
    sweep. solves/s = 1 / (t_rows + t_solve), measured, not scaled.

    One core (reported beside it): rows of ``single_core_rows`` elements in
    one worker, scaled by Ne / rows, plus an LU of size ``single_core_lu``
    with one BLAS thread, scaled by (N / n)^3.
    """
    from oracle import kernels, pool, solvers
    from paper_1212_3032_gb300 import inputs

    mesh = inputs.cavity_problem(cfg["n"])
    mat = kernels.Material(**MAT)
    ne, N = mesh.ne, 3 * mesh.ne
    s0 = cfg["eta"]
    s1 = cfg["eta"] + 1j * 2 * math.pi / cfg["T"]
    known = mesh.pattern.astype(complex)
    cores = os.cpu_count() or 1
    t_start = time.perf_counter()
    with pool.RowPool(mesh, mat, workers=cores) as P:
        P.rows(known, s0)
        t0 = time.perf_counter()
        A, b = P.rows(known, s1)
        t_rows = time.perf_counter() - t0
    t0 = time.perf_counter()
    solvers.direct_solve(A, b)
    t_solve = time.perf_counter() - t0
    del A
    rows = np.linspace(0, ne - 1, single_core_rows).astype(np.int64)
    with pool.RowPool(mesh, mat, workers=1) as P:
        P.rows(known, s0, rows=rows)
        t0 = time.perf_counter()
        P.rows(known, s1, rows=rows)
        t1_rows = (time.perf_counter() - t0) * ne / single_core_rows
    t1_lu = _lu_seconds_one_thread(single_core_lu) * (N / single_core_lu) ** 3
    t_freq = t_rows + t_solve
    return {"value": 1.0 / t_freq, "unit": "solves/s", "cores": cores, "kind": "oracle", "measured": True,
            "sample": (f"one complete frequency (k = 1) of the {ne}-triangle sweep: every oracle row "
                       f"({N} x {N}, complex128) in {cores} worker processes, then LU of the full system "
                       f"(LAPACK, {cores} threads); static parts cached by a preceding k = 0 assembly"),
            "seconds": {"rows": t_rows, "solve": t_solve, "total_with_warmup": time.perf_counter() - t_start},
            "one_core": {"value": 1.0 / (t1_rows + t1_lu), "unit": "solves/s", "cores": 1,
                         "sample": (f"rows of {single_core_rows} elements scaled by {ne}/{single_core_rows}, "
                                    f"LU of {single_core_lu} scaled by (N/{single_core_lu})^3"),
                         "seconds": {"rows": t1_rows, "solve": t1_lu}}}


METRIC = "converged frequency solves/s (GMRES true residual <= 1e-5)"


def workload_config(args, cfg):
    """The config object of the JSON line (both arms)."""
    ne = 20 * cfg["n"] ** 2  # geodesic sphere with 20 n^2 triangles
    return {"workload": args.workload, "triangles": ne, "unknowns": 3 * ne, "n_omega": cfg["n_omega"],
            "solves_per_step": cfg["n_omega"] // 2 + 1, "T": cfg["T"], "eta": cfg["eta"], "window": "hanning",
            "aca_tol": cfg["aca_tol"], "leaf": cfg["leaf"], "gmres_tol": cfg["tol"],
            "guess": GUESS_LABEL[args.guess], "precond": getattr(args, "precond", "block3"),
            "l2": "flushed (256 MB write) before every timed step"}


def run_reference(args, cfg):
    """The CPU oracle as the reference arm: one complete frequency solve of the
    workload (every row on all cores, then LU), timed once. A step here is
    that one solve; the line declares the one timed step it ran."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    t0 = time.perf_counter()
    cb = cpu_oracle_measure(cfg)
    wall = time.perf_counter() - t0
    v = cb["value"]
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s",
           "n_gpus": ws, "steps": 1, "warmup": 1, "requested": {"steps": args.steps, "warmup": args.warmup},
           "ms_per_step": 1e3 / v, "wall_s": wall,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic", "config": workload_config(args, cfg),
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


GUESS_LABEL = {
    "sem": "SEM K=4",
    "zero": "zero",
    "mlp": "SEM K=4 + learned column (online Adam, 4 steps/frequency; weights carried over from earlier sweeps)",
}


def profile_case(ctx, binding, mesh, cfg, opts):
    """Two neighbouring frequencies of the workload (k = n_omega / 4 - 1, then
    k = n_omega / 4, whose assembly reuses the first one's ACA pivots), then
    the right-hand side and one GMRES solve at the second, for profiler
    captures of single launches."""
    k = cfg["n_omega"] // 4
    ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, opts)
    ctx.assemble(cfg["eta"] + 1j * (k - 1) * 2 * math.pi / cfg["T"], opts)
    s = cfg["eta"] + 1j * k * 2 * math.pi / cfg["T"]
    ctx.assemble(s, opts)
    b = ctx.rhs(1.0, mesh.pattern)
    ctx.set_profiling(True)
    _, st = ctx.solve_assembled(b, opts=opts)
    prof = ctx.get_profile()
    ctx.set_profiling(False)
    print(json.dumps({"profile_case": True, "s": [s.real, s.imag], "iters": st["iters"],
                      "rel_residual": st["rel_residual"],
                      "hmv_algorithmic_bytes_per_product": prof["hmv_bytes"] / max(1, prof["hmv_launches"]),
                      "hmv_us_per_product": 1e3 * prof["hmv_ms"] / max(1, prof["hmv_launches"])}))


def run_ours(args, cfg):
    import torch

    from paper_1212_3032_gb300 import binding, build, inputs

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    stream = torch.cuda.current_stream(dev)
    ctx = binding.Context(local, stream=stream.cuda_stream)
    ctx.set_material(**MAT)
    ctx.set_window(cfg["eta"], binding.WIN_HANNING)
    ctx.set_aca_reuse(not args.no_aca_reuse)
    mesh = inputs.cavity_problem(cfg["n"])
    N = 3 * mesh.ne
    n_omega = cfg["n_omega"]
    nf = n_omega // 2 + 1
    load = inputs.heaviside_history(n_omega)
    guess = {"sem": binding.GUESS_SEM, "mlp": binding.GUESS_MLP, "zero": binding.GUESS_ZERO}[args.guess]
    precond = {"block3": binding.PRECOND_BLOCK3, "leaf": binding.PRECOND_LEAF,
               "auto": binding.PRECOND_AUTO}[args.precond]
    opts = binding.default_opts(leaf_size=cfg["leaf"], aca_tol=cfg["aca_tol"], tol=cfg["tol"],
                                precision=binding.PREC_C64_MIXED, guess=guess, sem_k=4, precond=precond)
    if args.profile_case:
        return profile_case(ctx, binding, mesh, cfg, opts)
    # device-resident inputs
    xyz_t = torch.tensor(mesh.xyz, dtype=torch.float64, device=dev)
    tri_t = torch.tensor(mesh.tri, dtype=torch.int32, device=dev)
    bc_t = torch.tensor(mesh.bc_type, dtype=torch.int8, device=dev)
    load_t = torch.tensor(load, dtype=torch.float64, device=dev)
    pat_t = torch.tensor(mesh.pattern, dtype=torch.float64, device=dev)
    dofs_t = torch.arange(N, dtype=torch.int64, device=dev)
    out_t = torch.empty((n_omega, N), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def step(o=opts):
        ctx.mesh_dev(xyz_t, tri_t, bc_t, o)
        st = ctx.solve_sweep_dev(cfg["T"], n_omega, load_t, pat_t, o, allow_unconverged=True)
        ctx.time_response_dev(dofs_t, out_t)
        return st

    for _ in range(args.warmup):
        stats = step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ctx.set_profiling(True)
    total_ms = 0.0
    unconverged = 0
    iters = 0
    cycles = 0
    phase_ms = {"assemble_ms": 0.0, "guess_ms": 0.0, "solve_ms": 0.0}
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats = step()
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            unconverged += sum(1 for s in stats if not s["converged"])
            iters += sum(s["iters"] for s in stats)
            cycles += sum(s["cycles"] for s in stats)
            for key in ("assemble_ms", "guess_ms", "solve_ms"):
                phase_ms[key] += sum(s[key] for s in stats)
        torch.cuda.synchronize()
    prof = ctx.get_profile()
    ctx.set_profiling(False)
    clocks = clk.summary()
    t_max = max_over_ranks(total_ms, dev)
    value = replica_throughput(nf * args.steps, ws, t_max)

    # end to end through the host-pointer API
    h2d = mesh.xyz.nbytes + mesh.tri.astype(np.int32).nbytes + mesh.bc_type.nbytes + load.nbytes + \
        mesh.pattern.nbytes
    d2h = n_omega * N * 8
    dofs = np.arange(N, dtype=np.int64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, opts)
        ctx.solve_sweep(cfg["T"], n_omega, load, mesh.pattern, opts, allow_unconverged=True)
        tr = ctx.time_response(dofs)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = nf * args.steps / e2e_s

    # the plain form (complex128 operator and FP64 everywhere), one timed sweep
    plain = None
    if not args.no_plain:
        popts = binding.default_opts(leaf_size=cfg["leaf"], aca_tol=cfg["aca_tol"], tol=cfg["tol"],
                                     precision=binding.PREC_C128, guess=binding.GUESS_SEM, sem_k=4)
        step(popts)
        torch.cuda.synchronize()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pst = step(popts)
        e1.record(stream)
        e1.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"value": nf / (pms / 1e3), "unit": "solves/s", "ms_per_step": pms,
                 "iters": sum(s["iters"] for s in pst), "speedup": value / ws / (nf / (pms / 1e3))}

    # the H-matrix product alone (no assembly sharing the GPU): one solve at
    # k = n_omega / 4, as in --profile-case
    kq = n_omega // 4
    ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, opts)
    ctx.assemble(cfg["eta"] + 1j * (kq - 1) * 2 * math.pi / cfg["T"], opts)
    ctx.assemble(cfg["eta"] + 1j * kq * 2 * math.pi / cfg["T"], opts)
    bq = ctx.rhs(1.0, mesh.pattern)
    ctx.set_profiling(True)
    ctx.solve_assembled(bq, opts=opts)
    iprof = ctx.get_profile()
    ctx.set_profiling(False)
    iso_gbs = iprof["hmv_bytes"] / (iprof["hmv_ms"] / 1e3) / 1e9 if iprof["hmv_ms"] > 0 else None

    if rank != 0:
        return
    peak, peak_kind = _peaks()
    hmv_gbs = prof["hmv_bytes"] / (prof["hmv_ms"] / 1e3) / 1e9 if prof["hmv_ms"] > 0 else None
    out = {
        "metric": METRIC,
        "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 (FP32 kernel evaluation; FP64 singular, Arnoldi, refinement)", "data": "synthetic",
        "config": workload_config(args, cfg),
        "gmres_iters_per_step": iters / args.steps, "gmres_cycles_per_step": cycles / args.steps,
        "unconverged": unconverged,
        "guess_residual_mean": statistics.fmean(s["guess_residual"] for s in stats[1:]),
        "sem_residual_mean": statistics.fmean(s["sem_residual"] for s in stats[1:]),
        "roofline": {"kernel": "H-matrix product (k_hmv_fused, one launch)", "bound": "hbm", "achieved": hmv_gbs,
                     "peak": peak, "unit": "GB/s", "frac": (hmv_gbs / peak) if hmv_gbs else None,
                     "peak_source": peak_kind, "traffic": HMV_TRAFFIC_K64,
                     "traffic_note": "DRAM read + write of one product at k = n_omega/4 (ncu capture of the current "
                                     "kernel, profiles/k_hmv_fused_cavity5120.md); algorithmic 887.3 MB there",
                     "launches": prof["hmv_launches"], "ms_total": prof["hmv_ms"],
                     "note": "timed inside the sweep, where the next frequency's assembly shares the GPU",
                     "isolated": {"achieved": iso_gbs, "frac": (iso_gbs / peak) if iso_gbs else None,
                                  "launches": iprof["hmv_launches"],
                                  "case": "one solve at k = n_omega/4 with nothing else running"}},
        "phases_ms_per_step": {"assembly": phase_ms["assemble_ms"] / args.steps,
                               "initial_guess": phase_ms["guess_ms"] / args.steps,
                               "gmres": phase_ms["solve_ms"] / args.steps,
                               "gmres_hmatvec": prof["hmv_ms"] / args.steps},
        "aca": {"pivot_reuse": not args.no_aca_reuse, "blocks": prof["aca_blocks"],
                "stepped": prof["aca_stepped"]},
        "gpu_launches": prof["kernel_launches"],
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "plain": plain,
    }
    if ws == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_oracle_measure(cfg)
    print(json.dumps(out))


def run_batched(args):
    """Sixteen uneven meshes (closed boxes and ellipsoids of 2k-37k triangles,
    cavity problems, T = 64, 128 samples): converged solves/s of one batched
    sweep (bem_add_mesh + bem_solve_sweep_batched, compact far-field storage)
    against the same meshes swept one after another through single-mesh
    contexts (default storage, assembly overlapped with the solve). Wall time
    around each complete call (both calls return after the GPU work)."""
    import torch

    from paper_1212_3032_gb300 import binding, build, inputs

    build.build()
    torch.cuda.set_device(0)
    meshes = inputs.batched_meshes()
    T, n_omega = 64.0, 128
    eta = 5.0 / T
    nf = n_omega // 2 + 1
    load = inputs.heaviside_history(n_omega)
    opts = binding.default_opts(leaf_size=64, aca_tol=1e-5, tol=1e-5, precision=binding.PREC_C64_MIXED,
                                guess=binding.GUESS_SEM, sem_k=4, precond=binding.PRECOND_AUTO)
    out = {"metric": "converged frequency solves/s, 16 uneven meshes swept on one GPU", "unit": "solves/s",
           "config": {"workload": "batched16", "triangles": [m.ne for m in meshes], "n_omega": n_omega, "T": T,
                      "aca_tol": 1e-5, "gmres_tol": 1e-5, "guess": "SEM K=4",
                      "precond": "per mesh: 3x3 or leaf blocks, chosen at its first k > 0"}}
    c = binding.Context(0)
    try:
        c.set_material(**MAT)
        c.set_window(eta, binding.WIN_HANNING)
        c.set_far_storage(binding.FAR_COMPACT)
        for m in meshes:
            c.add_mesh(m.xyz, m.tri, m.bc_type, opts)
        pats = [m.pattern for m in meshes]
        times = []
        for _ in range(2):  # the first sweep is the warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = c.solve_sweep_batched(T, n_omega, load, pats, opts, allow_unconverged=True)
            times.append(time.perf_counter() - t0)
        t_b = statistics.median(times[1:])
        out["batched"] = {"value": len(meshes) * nf / t_b, "seconds": t_b,
                          "unconverged": sum(1 for per in st for s in per if not s["converged"]),
                          "iters": sum(s["iters"] for per in st for s in per)}
    finally:
        c.close()
    ctxs = []
    try:
        for m in meshes:
            one = binding.Context(0)
            ctxs.append(one)
            one.set_material(**MAT)
            one.set_window(eta, binding.WIN_HANNING)
            one.mesh(m.xyz, m.tri, m.bc_type, opts)
        times = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            iters = 0
            for one, m in zip(ctxs, meshes):
                st = one.solve_sweep(T, n_omega, load, m.pattern, opts, allow_unconverged=True)
                iters += sum(s["iters"] for s in st)
            times.append(time.perf_counter() - t0)
        t_s = statistics.median(times[1:])
        out["sequential"] = {"value": len(meshes) * nf / t_s, "seconds": t_s, "iters": iters}
    finally:
        for one in ctxs:
            one.close()
    out["value"] = out["batched"]["value"]
    out["speedup_vs_sequential"] = out["batched"]["value"] / out["sequential"]["value"]
    print(json.dumps(out))


def run_large(args):
    """The 231,088-triangle cube with 8 spherical cavities (693,264 unknowns):
    bottom face fixed, top face under a step traction, the rest free; E = 1,
    nu = 0.3, rho = 1; 128 samples (65 solves), T = 8 (--large-T), eta = 5/T; complex64
    operator with ACA tolerance 1e-4, compact far-field storage, leaf-block
    preconditioner, extrapolated guesses, GMRES 1e-5. One sweep, timed with
    CUDA events on the library's stream; device memory in use sampled after
    it. A separate line (not the benchmark's step)."""
    import torch

    from paper_1212_3032_gb300 import binding, build, inputs

    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    mesh = inputs.cube_with_cavities()
    T, n_omega = float(args.large_T), 128
    eta = 5.0 / T
    nf = n_omega // 2 + 1
    stream = torch.cuda.current_stream(dev)
    ctx = binding.Context(0, stream=stream.cuda_stream)
    try:
        ctx.set_material(1.0, 0.3, 1.0)
        ctx.set_window(eta, binding.WIN_HANNING)
        opts = binding.default_opts(leaf_size=64, aca_tol=1e-4, tol=1e-5, precision=binding.PREC_C64_MIXED,
                                    guess=binding.GUESS_SEM, sem_k=4, precond=binding.PRECOND_LEAF)
        t0 = time.perf_counter()
        ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, opts)
        t_mesh = time.perf_counter() - t0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ctx.solve_sweep(T, n_omega, inputs.heaviside_history(n_omega), mesh.pattern, opts,
                             allow_unconverged=True)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        free, total = torch.cuda.mem_get_info()
        fs = ctx.far_storage()
    finally:
        ctx.close()
    out = {"metric": "converged frequency solves/s, 231,088-triangle cube with 8 cavities (one sweep)",
           "value": nf / (ms / 1e3), "unit": "solves/s", "seconds": ms / 1e3, "mesh_setup_s": t_mesh,
           "solves": nf, "converged": sum(1 for s in st if s["converged"]),
           "gmres_iters": sum(s["iters"] for s in st), "max_iters_one_frequency": max(s["iters"] for s in st),
           "assembly_ms_mean": statistics.fmean(s["assemble_ms"] for s in st),
           "device_memory_in_use_gb": (total - free) / 1e9, "far_storage": fs,
           "config": {"workload": "cube231k", "triangles": mesh.ne, "unknowns": 3 * mesh.ne, "n_omega": n_omega,
                      "T": T, "eta": eta, "aca_tol": 1e-4, "gmres_tol": 1e-5, "precond": "leaf blocks",
                      "guess": "SEM K=4", "material": {"E": 1.0, "nu": 0.3, "rho": 1.0}}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cavity5120", choices=sorted(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--guess", default="sem", choices=["sem", "mlp", "zero"])
    ap.add_argument("--precond", default="block3", choices=["block3", "leaf", "auto"],
                    help="GMRES preconditioner: 3x3 element blocks (default), leaf blocks, or chosen by the sweep")
    ap.add_argument("--no-aca-reuse", action="store_true",
                    help="assemble every frequency with a fresh ACA (no reuse of the previous pivots)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one frequency (assembly + one solve) and exit; for profiler captures")
    ap.add_argument("--batched", action="store_true",
                    help="the 16-mesh batched sweep against the same meshes one after another (separate line)")
    ap.add_argument("--large", action="store_true",
                    help="one sweep of the 231,088-triangle cube with cavities (separate line)")
    ap.add_argument("--large-T", type=float, default=8.0, help="time window of the --large sweep")
    args = ap.parse_args()
    cfg = WORKLOADS[args.workload]
    if args.large:
        run_large(args)
    elif args.batched:
        run_batched(args)
    elif args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
