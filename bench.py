#!/usr/bin/env python
"""Benchmark: preconditioned-OMM solves per second on one GB300 (replicas on N GPUs).

One step = one whole solve of the 2D 128^2 smooth-field workload (n = 16384, N = 128
states, 16 conformal poles, GMRES(15) x 5 at rtol 1e-5 with the sparsifying
preconditioner, mixed precision): set the starting block, filter it with the pole
expansion, run the preconditioned CG with the exact quartic line search, filter once
more with GMRES at rtol 1e-6 and run the CG to convergence again (so that the result
meets both accuracy targets against the FP64 form: energy 1e-8, subspace angle 1e-6),
and evaluate the energy and residuals in FP64.  Inputs are resident in HBM when the
timed region starts; the GMRES working set (~5 GB) is far larger than L2.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead (a bounded
sample of the same workload, scaled to solves/s).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "OMM solves/sec and H-apply GB/s at E err≤1e-8 vs FP64 form; p50/p99 latency"


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="smooth2d-128",
                    help="smooth2d-128 (the default line), wells2d-32, lattice3d-48")
    ap.add_argument("--gram-tensor", type=int, default=1,
                    help="1: complex64 Grams on the tcgen05 tensor cores (TF32 x 3); 0: FP32 CUDA cores")
    ap.add_argument("--precond", default="pole", choices=["pole", "projector", "gtpa"],
                    help="pole: the pole expansion every iteration (Sec. 3.1); projector: U U^* precomputed by "
                         "Algorithm 2 inside each timed solve (Sec. 3.3); gtpa: the Fourier-diagonal TPA-type "
                         "comparison preconditioner of Sec. 2.2 (no filter, tau from the exact eigenvectors)")
    ap.add_argument("--gtpa-t", type=int, default=3, help="gtpa: polynomial degree t (3 = eq. TPA; the paper's gTPA runs use 5)")
    ap.add_argument("--maxit", type=int, default=0, help="CG iteration cap (0: 40, or 4000 with gtpa as in Sec. 4)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer pass (profiler runs)")
    ap.add_argument("--inner", default="auto", choices=["auto", "spp", "kinetic"],
                    help="GMRES inner preconditioner; auto: sparsifying in 2D and up to 16^3, kinetic above")
    ap.add_argument("--iters", type=int, default=0, help="fixed CG iterations (0: energy criterion)")
    ap.add_argument("--no-fp64-check", action="store_true", help="skip the untimed FP64-form comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", type=int, default=0,
                    help="1: per-class CUDA events inside the timed region (perturbs it); 0: counters only there")
    ap.add_argument("--no-profile-pass", dest="profile_pass", action="store_false",
                    help="skip the untimed per-class profile solve after the timed region")
    ap.add_argument("--refilter", type=int, default=1,
                    help="extra filter + CG rounds after convergence (1: the default line meets the 1e-6 angle)")
    ap.add_argument("--rtol", type=float, default=1e-5, help="GMRES relative tolerance (paper: 1e-5)")
    ap.add_argument("--refilter-rtol", type=float, default=1e-6,
                    help="GMRES tolerance of the refilter rounds (0: --rtol)")
    ap.add_argument("--N", type=int, default=0, help="override N (reduced case for profiler captures only)")
    ap.add_argument("--P", type=int, default=0, help="override P (reduced case for profiler captures only)")
    ap.add_argument("--mode", default="solve", choices=["solve", "batch", "serve", "graph"],
                    help="solve: the default line; batch: 64 uneven Hamiltonians at once; serve: Poisson arrivals")
    ap.add_argument("--requests", type=int, default=120, help="serve mode: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serve mode: arrivals per second")
    ap.add_argument("--slots", type=int, default=8, help="batch/serve: concurrent solves")
    ap.add_argument("--mix", default="2d", choices=["2d", "full"],
                    help="serve: '2d' the twelve 2D well Hamiltonians; 'full' adds four 2D ones with N in "
                         "[129, 256] and the 3D lattice on 32^3 (N = 64) and 48^3 (N = 64, 256)")
    ap.add_argument("--trsv-streams", type=int, default=0,
                    help="omm_params.trsv_streams: streams of the triangular solves (0: one per pole)")
    ap.add_argument("--overlap", type=int, default=1, choices=[0, 1],
                    help="omm_params.launch_overlap: programmatic dependent launches in the triangular solves")
    ap.add_argument("--orbitals", default="real", choices=["real", "complex"],
                    help="real: real X (eq. lst writes Y real), conjugate pole pairs folded (P/2 solves); complex: P solves")
    return ap.parse_args()


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------------------ workload
def load_workload(name):
    from workloads import WORKLOADS
    wl = WORKLOADS[name]
    spectra = json.load(open(os.path.join(ROOT, "workloads", "spectra.json")))[name]
    return wl, spectra


def inner_choice(wl, inner="auto"):
    if inner == "auto":
        return "spp" if (wl.dim == 2 or wl.m <= 16) else "kinetic"
    return inner


def workload_config(wl, spectra, iters, precision="mixed", refilter=0, rtol=1e-5, orbitals="real", inner="auto",
                    refilter_rtol=0.0):
    return {"workload": f"{wl.name}: {wl.dim}D {wl.m}^{wl.dim} periodic grid (n={wl.n}), N={wl.N} states, "
                        f"P={wl.P} conformal poles, {wl.potential} potential, {precision}",
            "orbitals": ("real X, conjugate pole pairs folded (P/2 GMRES solves per application)"
                         if orbitals == "real" else "complex X, P GMRES solves per application"),
            "grid": [wl.m] * wl.dim, "box_len": wl.L, "N": wl.N, "P": wl.P, "precision": precision,
            "inner_preconditioner": ("sparsifying (nested-dissection multifrontal LU)"
                                     if inner_choice(wl, inner) == "spp" else
                                     "kinetic (T + <V> - sigma - z)^-1 (the sparsifying factor is not built above 16^3)"),
            "gmres": f"restart 15, <=5 cycles, rtol {rtol:g}", "cg_iters": iters if iters else "energy criterion",
            "refilter": refilter, **({"refilter_rtol": refilter_rtol} if refilter and refilter_rtol else {}),
            "l2": "inputs/working set larger than L2 (GMRES basis ~GBs)", "parallelism": "replicas",
            "spectral_interval": "stored exact [lam_1, lam_N], lam_{N+1} (workloads/spectra.json)"}


# ------------------------------------------------------------------------------ CPU oracle timing
def oracle_setup(wl, spectra, rtol=1e-5):
    """The FP64 oracle's pole-expansion preconditioner for the workload: all P poles, each
    with its own sparsifying factor (SuperLU) or Green symbol, GMRES to relative tolerance
    rtol; built once, outside any timed sample."""
    from oracle import poles as opoles
    from oracle.precond import PolePreconditioner
    V = wl.potential_values()
    z, w = opoles.poles_conformal(spectra["lam1"], spectra["lamN"], spectra["lamN1"], wl.P)
    return PolePreconditioner(wl.shape, wl.L, V, spectra["sigma"], z, w, mode="gmres",
                              inner="spp" if inner_choice(wl) == "spp" else "lap", rtol=rtol)


def oracle_unit(pc, X0, rep, cols):
    """One sample unit of the oracle's dominant work: the whole pole expansion (every pole's
    GMRES + sparsifying solve) applied to `cols` columns of the starting block.  Returns
    (wall seconds, CPU seconds, mean GMRES steps per system of the unit)."""
    import numpy as np
    nblk = X0.shape[0] // cols
    k = rep % nblk
    n0 = len(pc.stats)
    t0, c0 = time.perf_counter(), time.process_time()
    pc(X0[k * cols:(k + 1) * cols])
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    its = [float(np.mean(st["iters"])) for st in pc.stats[n0:] if "iters" in st]
    return wall, cpu, (float(np.mean(its)) if its else float("nan"))


def oracle_sample(wl, spectra, budget_s=12.0, pc=None):
    """Time the oracle's pole expansion (all P poles, 2 columns per unit) for about
    budget_s seconds; returns (seconds per unit, columns per unit, host cores used, mean
    GMRES steps per system, units)."""
    import numpy as np
    pc = pc or oracle_setup(wl, spectra)
    X0 = wl.initial_block(np.complex128, real=True)
    cols, walls, cpus, its = 2, [], [], []
    while True:
        wall, cpu, it = oracle_unit(pc, X0, len(walls), cols)
        walls.append(wall)
        cpus.append(cpu)
        its.append(it)
        if sum(walls) > budget_s:
            break
    t = sum(walls) / len(walls)
    cores = round(max(sum(cpus) / sum(walls), 1.0), 1)   # host threads the oracle kept busy
    return t, cols, cores, float(np.nanmean(its)), len(walls)


def threads_used():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return 1


def cpu_baseline_record(wl, spectra, applications, gpu_gmres_mean=None):
    t, cols, cores, its, units = oracle_sample(wl, spectra)
    per_solve = t * (wl.N / cols) * applications
    gpu = f"; the GPU solve's largest GMRES step count per application averages {gpu_gmres_mean:.1f}" \
        if gpu_gmres_mean else ""
    return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": (f"{units} units of the oracle's pole expansion, each all {wl.P} poles (GMRES + "
                       f"{'sparsifying' if inner_choice(wl) == 'spp' else 'kinetic'} preconditioner, no conjugate "
                       f"folding) on {cols} starting columns ({t:.2f} s per unit); scaled by N/{cols} column pairs x "
                       f"{applications} applications per solve; the oracle's GMRES took {its:.1f} steps per system "
                       f"on average{gpu}; pocketfft and SuperLU, BLAS pool {threads_used()} threads; "
                       f"cores = CPU time / wall time of the sample")}


# Workloads whose whole oracle solve takes seconds (wells2d-32: about 20 s on 8 host cores):
# the CPU baseline times one whole solve there instead of scaling a sample.
WHOLE_ORACLE_SOLVE = {"wells2d-32"}


def cpu_baseline_whole(wl, spectra, refilter, maxit, tol):
    """One whole oracle solve of the workload (the filter, then Algorithm 1 with the pole
    expansion, refilter rounds as the GPU arm runs them), timed; the P sparsifying factors
    are built before the timed region, as the GPU arm's omm_set_poles is."""
    import numpy as np
    from oracle import solve as osolve
    pc = oracle_setup(wl, spectra)
    X0 = wl.initial_block(np.complex128, real=True)
    t0, c0 = time.perf_counter(), time.process_time()
    _, info = osolve.solve(wl.shape, wl.L, wl.potential_values(), spectra["sigma"], X0, pc.z, pc.w, maxit=maxit,
                           tol=tol, refilter=refilter, precond=pc)
    wall = time.perf_counter() - t0
    cores = round(max((time.process_time() - c0) / wall, 1.0), 1)
    iters = sum(len(h) - 1 for h in info["history"])
    err = abs(info["E"] - spectra["E_ref"]) / abs(spectra["E_ref"])
    return {"value": 1.0 / wall, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": (f"one whole oracle solve ({wall:.1f} s): the filter and {iters} CG iterations of Algorithm 1 "
                       f"over {refilter + 1} round(s), every application the pole expansion with all {wl.P} poles "
                       f"(GMRES + {'sparsifying' if inner_choice(wl) == 'spp' else 'kinetic'} preconditioner, no "
                       f"conjugate folding), FP64; the {wl.P} factorisations built before the timed region; "
                       f"E error {err:.1e}; pocketfft and SuperLU, BLAS pool {threads_used()} threads; "
                       f"cores = CPU time / wall time")}


def cpu_baseline_gtpa(wl, spectra, t, iters, real=True, sample_iters=8):
    """The oracle's OMM with the same gTPA preconditioner (Algorithm 1, FP64, pocketfft)
    for a bounded number of iterations on the whole workload, scaled to the GPU solve's
    iteration count."""
    import numpy as np
    from oracle import gtpa as ogtpa, hamiltonian as ham, omm as oomm
    V = wl.potential_values()
    pc = ogtpa.GtpaPreconditioner(wl.shape, ogtpa.default_coefficients(t), spectra["gtpa_tau"])
    X0 = wl.initial_block(np.complex128, real=real)
    t0, c0 = time.perf_counter(), time.process_time()
    oomm.nlcg(lambda Y: ham.apply_h_fft(Y, wl.shape, wl.L, V, spectra["sigma"]), pc, X0, maxit=sample_iters, tol=0.0)
    wall = time.perf_counter() - t0
    cores = round(max((time.process_time() - c0) / wall, 1.0), 1)
    per_solve = wall / sample_iters * max(iters, 1)
    return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": (f"oracle OMM with gTPA t = {t}: {sample_iters} iterations of Algorithm 1 on the whole "
                       f"workload ({wall:.1f} s), scaled to the GPU solve's {iters} iterations; cores = CPU time / "
                       f"wall time of the sample")}


def run_reference(a):
    """The oracle as it stands, on the host cores: each step is one bounded sample unit of
    the workload (the whole pole expansion, all P poles, on two starting columns), timed;
    the line's value scales the median unit to one whole solve."""
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, spectra = load_workload(a.workload)
    # CG iterations of one solve of this workload, as the GPU arm measured them (smooth2d-128
    # at the default settings: 22 iterations over the two rounds; the others without the
    # refilter): the sample is scaled to the filters (1 + refilter) plus that many
    # preconditioner applications, the count the GPU arm's own cpu_baseline uses
    cg_iters = {"smooth2d-128": 22, "wells2d-32": 13, "lattice3d-48": 21}.get(wl.name, 12)
    applications = 1 + a.refilter + (a.iters or cg_iters)
    pc = oracle_setup(wl, spectra, a.rtol)          # untimed: SuperLU factors of every pole
    X0 = wl.initial_block(np.complex128, real=True)
    cols = 2
    walls, cpus, its = [], [], []
    for s_ in range(a.warmup + a.steps):
        wall, cpu, it = oracle_unit(pc, X0, s_, cols)
        if s_ >= a.warmup:
            walls.append(wall)
            cpus.append(cpu)
            its.append(it)
    t = statistics.median(walls)
    v = 1.0 / (t * (wl.N / cols) * applications)
    cores = round(max(sum(cpus) / sum(walls), 1.0), 1)
    rec = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * sum(walls) / len(walls),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           # refilter: the applications the sample is scaled to; every sampled unit runs the
           # oracle's GMRES at its own rtol, so no separate refilter tolerance is claimed
           "config": dict(workload_config(wl, spectra, a.iters, "fp64 oracle", a.refilter, a.rtol, orbitals="complex",
                                          inner=a.inner),
                          orbitals="complex X: the oracle solves every pole (no conjugate folding)"),
           "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                            "sample": f"each step: the oracle's whole pole expansion (all {wl.P} poles, GMRES + "
                                      f"sparsifying preconditioner) on {cols} starting columns, "
                                      f"{statistics.median(walls):.2f} s median; value = 1 / (that x N/{cols} x "
                                      f"{applications} applications per solve); oracle GMRES {np.nanmean(its):.1f} "
                                      f"steps per system on average"},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(rec))


# ------------------------------------------------------------------------------ replicas
def aggregate_ranks(ms_local, steps, world, device="cpu"):
    """Whole-job throughput of independent replicas: the slowest rank's timed region
    (MAX over ranks) and value = world * steps / that time (solves/s)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    ms_max = float(t.item())
    return ms_max, world * steps / (ms_max / 1000.0)


# ------------------------------------------------------------------------------ GPU arm
def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_1603_09724_gb300 as omm

    wl, spectra = load_workload(a.workload)
    if a.N or a.P:
        import dataclasses
        wl = dataclasses.replace(wl, N=a.N or wl.N, P=a.P or wl.P)
    V = wl.potential_values()
    mixed = wl.precision == "mixed"
    prec = omm.OMM_MIXED if mixed else omm.OMM_FP64
    cdt = torch.complex64 if mixed else torch.complex128
    z, w = omm.poles_fermi(spectra["lam1"], spectra["lamN"], spectra["lamN1"], wl.P)
    tol = 0.0 if a.iters else (1e-10 if mixed else 1e-13)
    maxit = a.iters if a.iters else (a.maxit or (4000 if a.precond == "gtpa" else 40))
    real = a.orbitals == "real"
    inner = omm.OMM_INNER_SPARSIFY if inner_choice(wl, a.inner) == "spp" else omm.OMM_INNER_KINETIC
    prm = omm.default_params(precision=prec, maxit=maxit, tol=tol, refilter=a.refilter, gmres_rtol=a.rtol,
                             real_orbitals=int(real), inner=inner, gram_tensor=a.gram_tensor,
                             refilter_rtol=a.refilter_rtol, gap=spectra["lamN1"] - spectra["lamN"],
                             launch_overlap=a.overlap, trsv_streams=a.trsv_streams)
    s = omm.Solver(wl.dim, wl.m, wl.L, V, wl.N, shift=spectra["sigma"], params=prm)
    t_setup = time.perf_counter()
    if a.precond == "gtpa":
        if "gtpa_tau" not in spectra:
            raise SystemExit(f"no stored tau for {a.workload} (2D workloads only)")
        s.set_gtpa(a.gtpa_t, spectra["gtpa_tau"])
    else:
        s.set_poles(z, w)
    t_setup = time.perf_counter() - t_setup
    X0h = torch.from_numpy(wl.initial_block(np.complex64 if mixed else np.complex128, real=real)).pin_memory()
    X0 = X0h.to("cuda")
    stream = torch.cuda.current_stream()
    B0 = None
    if a.precond == "projector":
        from workloads import gaussian_block, gaussian_block_real
        gen = gaussian_block_real if real else gaussian_block
        # k = N extra columns: 2N Gaussian columns, N kept by the rank-revealing step
        B0 = torch.from_numpy(gen(wl.n, 2 * wl.N, seed=2000 + wl.seed,
                                  dtype=np.complex64 if mixed else np.complex128)).to("cuda")

    # gTPA has no GMRES basis: its working set (six n x N blocks) fits in L2, so L2 is
    # flushed by a write larger than it before every solve (timed, ~0.1 ms)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda") if a.precond == "gtpa" else None

    def step():
        if flush is not None:
            flush.zero_()
        if B0 is not None:
            s.build_projector(B0)   # Algorithm 2: the pole solves on B0 and the QR, every solve
        s.set_orbitals(X0)
        return s.solve()

    for _ in range(a.warmup):
        st = step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    # the timed region runs with the kernel counters only (no per-class CUDA events); the
    # per-class profile comes from a separate untimed solve below
    s.profile(True if a.profile else "count")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat = []
    for _ in range(a.steps):
        ls = torch.cuda.Event(enable_timing=True)
        le = torch.cuda.Event(enable_timing=True)
        ls.record(stream)
        st = step()
        le.record(stream)
        lat.append((ls, le))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    counts = s.profile_read()
    s.profile(False)
    clk = clocks.stop()
    lat_ms = sorted(x.elapsed_time(y) for x, y in lat)
    ms_max, value = aggregate_ranks(ms, a.steps, world, "cuda")

    # end to end through the public API with host buffers (pinned), copies in the timed region
    Xout = torch.empty_like(X0h).pin_memory()
    Xdev = torch.empty_like(X0)
    e2e_ms = None
    if not a.no_e2e:
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(a.steps):
            if flush is not None:
                flush.zero_()
            Xdev.copy_(X0h, non_blocking=True)
            if B0 is not None:
                s.build_projector(B0)
            s.set_orbitals(Xdev)
            s.solve()
            s.get_orbitals(Xdev)
            Xout.copy_(Xdev, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1)
    nbytes = X0h.numel() * X0h.element_size()

    # per-class profile: one more solve (untimed) with CUDA events around every kernel class
    prof = None
    if a.profile_pass and not a.profile:
        s.profile(True)
        st_p = step()
        torch.cuda.synchronize()
        prof = s.profile_read()
        prof_ms = sum(v["ms"] for v in prof.values())
        s.profile(False)
    elif a.profile:
        prof, prof_ms = counts, ms

    if rank != 0:
        return
    peaks = measured_peaks()
    apps = st["filters"] + st["iters"]
    rec = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c64" if mixed else "c128", "data": "synthetic",
           "gpu_launches": int(sum(v["kernels"] for v in counts.values())),
           "config": dict(workload_config(wl, spectra, a.iters, "mixed" if mixed else "fp64", a.refilter, a.rtol,
                                          a.orbitals, a.inner, a.refilter_rtol),
                          preconditioner=precond_text(a, spectra),
                          timing=("CUDA events on the handle's stream around the whole timed region; kernel "
                                  "counters on, per-class events off" if not a.profile else
                                  "per-class CUDA events on inside the timed region (--profile 1)"),
                          **({"l2": "working set (six n x N blocks, ~100 MB) fits in L2: a 512 MB write flushes "
                                    "L2 before every timed solve"} if a.precond == "gtpa" else {})),
           "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1, int(0.99 * len(lat_ms)))]},
           "solve": {"iters": st["iters"], "filters": st["filters"], "converged": st["converged"],
                     "energy_fp64": st["energy_fp64"], "resid_fp64": st["resid_fp64"],
                     "E_rel_err_vs_exact": abs(st["energy_fp64"] - spectra["E_ref"]) / abs(spectra["E_ref"]),
                     "gmres_iters_max": st["gmres_iters_max"], "gmres_iters_total": st["gmres_iters_total"],
                     "grad_norm": st["grad_norm"], "resid_orth": st["resid_orth"], "angle_bound": st["angle_bound"],
                     "setup_s_all_poles": t_setup},
           "clocks": clk,
           "e2e": ({"value": world * a.steps / (e2e_ms / 1000.0), "unit": "solves/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes} if e2e_ms else None)}
    if prof:
        dom = max(prof, key=lambda k: prof[k]["ms"])
        kern = {}
        for k, v in prof.items():
            if v["calls"]:
                kern[k] = {"calls": v["calls"], "kernels": v["kernels"], "ms": round(v["ms"], 3),
                           "share": round(v["ms"] / max(prof_ms, 1e-9), 4),
                           "GB_s": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1) if v["bytes"] else None,
                           **({"impl_GB_s": round(v["impl_bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                              if v.get("impl_bytes") and abs(v["impl_bytes"] - v["bytes"]) > 1e-6 * v["bytes"]
                              else {})}
        rec["kernels"] = {"pass": ("one untimed solve with per-class CUDA events after the timed region"
                                   if not a.profile else "the timed region"), "classes": kern}
        rec["roofline"] = roofline_record(prof, dom, wl, peaks, clk.get("sm_mhz"), a.gram_tensor, apps)
        ha = prof["happly"]
        rec["happly_GB_s"] = ha["bytes"] / max(ha["ms"], 1e-9) / 1e6
    if not a.no_fp64_check and world == 1:
        acc = fp64_compare(a, wl, spectra, s, omm, torch, V, z, w)
        rec["accuracy_vs_fp64"] = acc
        if "sin_angle" in acc:
            rec["accuracy_gates"] = {"E_rel_diff_vs_fp64_form": acc["E_rel_diff"], "E_gate": 1e-8,
                                     "sin_angle_vs_fp64_form": acc["sin_angle"], "sin_gate": 1e-6,
                                     "pass": bool(acc["E_rel_diff"] <= 1e-8 and acc["sin_angle"] <= 1e-6)}
    if not a.no_cpu_baseline:
        if a.precond == "gtpa":
            rec["cpu_baseline"] = cpu_baseline_gtpa(wl, spectra, a.gtpa_t, st["iters"], real)
        elif wl.name in WHOLE_ORACLE_SOLVE and not (a.N or a.P or a.iters):
            rec["cpu_baseline"] = cpu_baseline_whole(wl, spectra, a.refilter, maxit, 1e-13)
        else:
            rec["cpu_baseline"] = cpu_baseline_record(wl, spectra, apps, st["gmres_iters_total"] / max(apps, 1))
    print(json.dumps(rec))


# DRAM bytes one call of a kernel class moved in an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum summed over the class's kernels for one call, scaled to the bench
# workload's systems), keyed by (workload, N, class); absent until captured for the class's
# current kernels.
TRAFFIC_PER_CALL = {
    # profiles/traffic_trsv_smooth2d-128_N64.md: 192.8 MB read per call at N = 64 (S = 512),
    # the vector part scaled to S = 1024, the factor part (66.1 MB) as measured; writes stay
    # in L2 and are not attributed to these kernels
    ("smooth2d-128", 128, "trsv_levels"): 319.5e6,
}


SMS, FP32_LANES_PER_SM = 152, 128          # GB300: 152 SMs x 4 partitions x 32 FP32 lanes
TF32_PER_BF16 = 1.1 / 2.25                 # nominal dense tensor-core rates, TF32 / BF16


def roofline_record(prof, dom, wl, peaks, sm_mhz, gram_tensor, apps):
    """Roofline of the dominant kernel class `dom` from the untimed per-class profile.

    HBM-bound classes: the class's algorithmic bytes (the library's count: H-apply 2v plus V,
    Green 2v plus the symbol tables, CGS2 k+3 vectors (basis and w read once, the new vector written), triangular solves 4 per
    unknown and active system plus the factor) / its CUDA-event time, against the measured
    copy bandwidth.  The Gram class (it dominates only when the preconditioner is cheap,
    e.g. gTPA) is compute-bound: 48 n N^2 algorithmic real flops per fused Gram [X D]^*
    [X D HX HD] (its 6 N^2 distinct complex entries, 8 flops per complex multiply-add),
    every call counted as one such Gram; against FP32 FMA on the CUDA cores (SMs x 128 lanes
    x 2 flops x the median SM clock of the timed region), or, on tcgen05, the measured bf16
    rate x the nominal TF32 / BF16 ratio."""
    d = prof[dom]
    ms = max(d["ms"], 1e-9)
    N, n = wl.N, wl.n
    if dom == "gram":
        flops = d["calls"] * 48.0 * n * N * N
        ach = flops / ms / 1e9                                  # TFLOP/s
        if gram_tensor:
            peak = peaks.get("bf16_tflops", 1900.0) * TF32_PER_BF16
            bound, how = "tensor", "measured bf16 GEMM rate x nominal TF32/BF16 ratio (of measured)"
        else:
            mhz = sm_mhz or peaks.get("sm_max_mhz", 2070.0)
            peak = SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
            bound, how = "alu", f"FP32 FMA on the CUDA cores at {mhz:.0f} MHz"
        return {"kernel": dom, "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None,
                "note": f"achieved = 48 n N^2 flops per Gram call / CUDA-event time of the profile solve; peak = {how}"}
    hbm = peaks.get("hbm_gbs", 6800.0)
    ach = d["bytes"] / ms / 1e6
    per_call = d["bytes"] / max(d["calls"], 1)
    formula = {
        "trsv_levels": "per application: 4 x n_sep x 8 B per active system (rhs in, y out, y in, x out) + the "
                       "separator blocks W_f, W_b of every pole once",
        "trsv_leaf": "per application: 4 x n_leaf x 8 B per active system + the leaf factor values of every pole once",
        "happly": "2 x n x 8 B per column (X in, Y out) + V",
        "greenq": "2 x n x 8 B per column + the Green symbol of each pole",
        "orth": "(k + 3) x n x 8 B per active system at Arnoldi step k (V_0..V_k and w read once, V_k+1 written)",
    }.get(dom, "the library's algorithmic byte count")
    tr = TRAFFIC_PER_CALL.get((getattr(wl, "name", None), N, dom))
    rec = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
           "traffic": tr,
           "algorithmic_bytes_per_call": per_call,
           "impl_bytes_per_call": d.get("impl_bytes", d["bytes"]) / max(d["calls"], 1),
           "note": (f"achieved = algorithmic bytes / CUDA-event time summed over the class's launches in one "
                    f"untimed profile solve ({formula}); a call is one application of the class to all "
                    f"systems (one GMRES step's triangular solves, H-apply, ...); peak = measured copy bandwidth "
                    f"(of measured); traffic = DRAM bytes per call from ncu, or null")}
    if d.get("flops", 0.0) > 0.0:
        # the same class against FP32 FMA: its dense supernode products carry about 128 flops
        # per byte of W, so the arithmetic bound lies far below the byte bound
        mhz = sm_mhz or peaks.get("sm_max_mhz", 2070.0)
        fpk = SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        fach = d["flops"] / ms / 1e9
        rec["alu"] = {"achieved": fach, "peak": fpk, "unit": "TFLOP/s", "frac": fach / fpk,
                      "flops_per_call": d["flops"] / max(d["calls"], 1),
                      "note": f"8 real flops per W_f / W_b entry and active system of its pole; peak = FP32 FMA "
                              f"on the CUDA cores at {mhz:.0f} MHz ({SMS} SMs x {FP32_LANES_PER_SM} lanes x 2)"}
    return rec


def precond_text(a, spectra):
    if a.precond == "pole":
        return "pole expansion every iteration (Sec. 3.1)"
    if a.precond == "projector":
        return "U U^* from Algorithm 2 (k = N, rank-revealing column choice), built inside each timed solve"
    return (f"gTPA t = {a.gtpa_t} (Sec. 2.2; t = 3 is eq. TPA), tau = {spectra.get('gtpa_tau', 0):.6g} from the exact "
            "eigenvectors (Sec. 4); CG from the unfiltered start")


def fp64_compare(a, wl, spectra, s, omm, torch, V, z, w, timed=2):
    """The same solve in the plain FP64 form (its own handle, poles set outside the timing):
    energy and subspace agreement, and its solve time measured like the mixed line's
    (CUDA events around `timed` solves after one untimed solve)."""
    import numpy as np
    try:
        Xm = s.get_orbitals().cpu().numpy().astype(np.complex128)
        real = a.orbitals == "real"
        prm = omm.default_params(precision=omm.OMM_FP64, maxit=a.iters if a.iters else 40,
                                 tol=0.0 if a.iters else 1e-13, refilter=a.refilter, gmres_rtol=a.rtol,
                                 refilter_rtol=a.refilter_rtol, real_orbitals=int(real),
                                 inner=omm.OMM_INNER_SPARSIFY if inner_choice(wl, a.inner) == "spp"
                                 else omm.OMM_INNER_KINETIC, launch_overlap=a.overlap)
        t0 = time.perf_counter()
        s64 = omm.Solver(wl.dim, wl.m, wl.L, V, wl.N, shift=spectra["sigma"], params=prm)
        s64.set_poles(z, w)
        X0 = torch.from_numpy(wl.initial_block(np.complex128, real=real)).to("cuda")
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        s64.set_orbitals(X0)
        st = s64.solve()                               # untimed first solve
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(timed):
            s64.set_orbitals(X0)
            st = s64.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1000.0 / timed
        X64 = s64.get_orbitals().cpu().numpy()
        Q1, _ = np.linalg.qr(Xm.T)
        Q2, _ = np.linalg.qr(X64.T)
        sin = float(np.linalg.norm(Q1 - Q2 @ (Q2.conj().T @ Q1), 2))
        Em = s.energy()
        s64.close()
        return {"E_rel_diff": abs(Em - st["energy_fp64"]) / abs(st["energy_fp64"]), "sin_angle": sin,
                "fp64_form_iters": st["iters"], "fp64_form_E_rel_err_vs_exact":
                    abs(st["energy_fp64"] - spectra["E_ref"]) / abs(spectra["E_ref"]),
                "fp64_form_solve_s": t64, "fp64_form_solves_per_s": 1.0 / t64, "fp64_form_setup_s": setup_s,
                "fp64_form_timing": f"CUDA events around {timed} solves after one untimed solve; handle creation "
                                    "and pole set-up outside"}
    except Exception as e:   # report, never hide
        return {"error": repr(e)}


def run_many(a):
    """Batched (all requests at t = 0) or served (Poisson arrivals) solves of many uneven
    Hamiltonians through the continuous-batching server; one JSON line."""
    import numpy as np
    import torch
    from paper_1603_09724_gb300.serve import OmmServer, Request, latency_summary
    from workloads import batch_mix, serving_mix, serving_mix_3d, serving_mix_wide, poisson_arrivals
    import paper_1603_09724_gb300 as omm
    spectra = json.load(open(os.path.join(ROOT, "workloads", "spectra.json")))
    specs = batch_mix() if a.mode == "batch" else serving_mix()
    if a.mode == "serve" and a.mix == "full":
        specs = specs + serving_mix_wide() + serving_mix_3d()

    def request(h):
        sp = spectra[h.key]
        dim = getattr(h, "dim", 2)
        # the sparsifying factor is built up to 16^3 in 3D; larger 3D grids take the kinetic inner preconditioner
        params = {"inner": omm.OMM_INNER_KINETIC} if dim == 3 and h.m > 16 else None
        return Request(h.key, dim, h.m, h.L, h.potential_values(), sp["N"], sp["lam1"], sp["lamN"], sp["lamN1"],
                       sigma=sp["sigma"], P=16, params=params)

    free, total = torch.cuda.mem_get_info()
    srv = OmmServer(hbm_budget=int(0.85 * free), slots=a.slots, gmres_rtol=a.rtol,
                    real_orbitals=int(a.orbitals == "real"))
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    if a.mode == "batch":
        reqs = [request(h) for h in specs]
        for r in reqs:
            srv.submit(r)
        res = srv.drain(len(reqs))
        wall = time.perf_counter() - t0
        # the same Hamiltonians again: resident handles warm-start from their last solution
        t1 = time.perf_counter()
        for r in reqs:
            srv.submit(request(next(h for h in specs if h.key == r.key)))
        res2 = srv.drain(len(reqs))
        wall2 = time.perf_counter() - t1
        extra = {"warm_pass": latency_summary(res2, wall2)}
        cfg = "64 independent 2D Hamiltonians, grids from {32,64,96,128}^2, N in [16,128], smooth random V"
    else:
        times, keys = poisson_arrivals(a.requests, a.rate, len(specs))
        base = [request(h) for h in specs]
        for t, k in zip(times, keys):
            delay = t - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            h = specs[int(k)]
            srv.submit(request(h))
        res = srv.drain(a.requests)
        wall = time.perf_counter() - t0
        extra = {"arrival_rate_per_s": a.rate}
        cfg = (f"Poisson arrivals ({a.rate:g}/s) over {len(specs)} Hamiltonians: 2D Gaussian wells on "
               f"{{64,72,96,128}}^2 with N in [32,128]" +
               (", four more 2D ones with N in [129,256], and the 3D well lattice on 32^3 (N = 64) and "
                "48^3 (N = 64 and 256), with the kinetic inner preconditioner above 16^3" if a.mix == "full" else ""))
    clk = clocks.stop()
    summ = latency_summary(res, wall)
    failed = [r.error for r in res if r.error is not None]
    res = [r for r in res if r.error is None]
    errs = [abs(r.stats["energy_fp64"] - spectra[r.key]["E_ref"]) / abs(spectra[r.key]["E_ref"]) for r in res]
    srv.close()
    rec = {"mode": a.mode, "metric": METRIC, "value": summ["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
           "higher_is_better": True, "data": "synthetic", "dtype": "c64",
           "config": {"workload": cfg, "slots": a.slots, "hbm_budget_GB": round(0.85 * free / 2**30, 1),
                      "gmres_rtol": a.rtol, "orbitals": a.orbitals},
           "latency_ms": {"p50": summ["p50_ms"], "p99": summ["p99_ms"]}, "requests": summ["requests"],
           "failed": summ["failed"], **({"first_error": failed[0]} if failed else {}),
           "warm_fraction": summ["warm_fraction"], "wall_s": wall,
           "E_rel_err_vs_exact": {"max": max(errs), "median": float(np.median(errs))} if errs else None,
           "converged": int(sum(r.stats["converged"] for r in res)), "clocks": clk}
    rec.update(extra)
    print(json.dumps(rec))


def run_graph(a):
    """The 64-Hamiltonian batch mix solved by one CUDA-graph launch (paper_1603_09724_gb300.
    batch): fixed CG schedule (20 iterations), one GMRES cycle of 12 steps with the systems
    that meet rtol 1e-5 masked on the device, real orbitals, mixed; the launch schedule of
    every shape chosen by the autotuner; the timed region is `steps` replays of the graph;
    one JSON line."""
    import tempfile
    import numpy as np
    import torch
    from paper_1603_09724_gb300 import batch
    from workloads import batch_mix
    spectra = json.load(open(os.path.join(ROOT, "workloads", "spectra.json")))
    insts = []
    for i, h in enumerate(batch_mix()):
        sp = spectra[h.key]
        insts.append(batch.Instance(h.key, 2, h.m, h.L, h.potential_values(), sp["N"], sp["lam1"], sp["lamN"],
                                    sp["lamN1"], sigma=sp["sigma"], seed=i))
    schedule = dict(precision=1, real_orbitals=1, fixed_iters=20, gmres_m=12, gmres_cycles=1, tol=1e-10)
    tune_path = os.path.join(tempfile.mkdtemp(), "omm_tune.json")
    tuner = batch.Autotuner(tune_path)
    t0 = time.perf_counter()
    gb = batch.GraphBatch(insts, schedule, autotuner=tuner)
    gb.setup()
    gb.capture()
    setup_s = time.perf_counter() - t0
    for _ in range(max(a.warmup, 1)):
        res = gb.run()
    clocks = ClockSampler(0)
    clocks.start()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(a.steps):
        gb.graph.replay()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    res = [s.read_result() for _, s, _, _ in gb.items]
    errs = [abs(r["energy_fp64"] - spectra[i.key]["E_ref"]) / abs(spectra[i.key]["E_ref"]) for i, r in zip(insts, res)]
    rec = {"mode": "graph", "metric": METRIC, "value": len(insts) * a.steps / (ms / 1000.0), "unit": "solves/s",
           "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
           "config": {"workload": f"{len(insts)} independent 2D Hamiltonians, grids from {{32,64,96,128}}^2, N in "
                                  "[16,128], smooth random V; one CUDA-graph launch per step solves all of them",
                      "schedule": schedule, "autotuned": {k: v["params"] for k, v in tuner.table.items()},
                      "l2": "working set (all instances' GMRES bases) far larger than L2"},
           "gpu_launches": 1, "graph_launches_per_step": 1,
           "setup_s": setup_s, "E_rel_err_vs_exact": {"max": max(errs), "median": float(np.median(errs))},
           "clocks": clk}
    gb.close()
    print(json.dumps(rec))


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "graph":
        run_graph(a)
    elif a.mode != "solve":
        run_many(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
