"""bench.py's GPU arm keeps its JSON-line contract, checked on the CPU: run_ours (pole
expansion, gTPA, projector) and run_many (batch, serve) run end to end against a fake
library module and stubbed torch.cuda plumbing (events, streams, device copies), and print
one line with the keys the contract requires.  A fake solve that fails now and then shows
up as failed requests, not as a crash.  Only the host logic of bench.py and serve.py runs;
every stub is undone after the test."""
import contextlib
import importlib.util
import io
import json
import os
import sys
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REQUIRED = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "clocks", "e2e", "gpu_launches", "roofline")


def fake_library(fail_every=0):
    lib = types.ModuleType("paper_1603_09724_gb300")
    lib.__path__ = []
    lib.OMM_FP64, lib.OMM_MIXED = 0, 1
    lib.OMM_INNER_SPARSIFY, lib.OMM_INNER_KINETIC, lib.OMM_INNER_NONE = 0, 1, 2
    lib.default_params = lambda **kw: dict(kw)
    lib.poles_fermi = lambda a, b, c, P: (np.linspace(a, c, P) + 0.5j, np.ones(P) + 0j)
    count = {"solves": 0}

    class Solver:
        def __init__(self, dim, m, L, V, N, shift=None, params=None, stream=None):
            self.n, self.N, self.dtype = m ** dim, N, torch.complex64
            self.X = torch.zeros(N, self.n, dtype=torch.complex64)

        def set_poles(self, z, w):
            pass

        def set_gtpa(self, t, tau, coeffs=None):
            pass

        def build_projector(self, B):
            return {}

        def set_orbitals(self, X):
            self.X = X.clone()

        def get_orbitals(self, X=None):
            return self.X.clone()

        def solve(self):
            count["solves"] += 1
            if fail_every and count["solves"] % fail_every == 0:
                raise RuntimeError("omm_solve: a CUDA runtime call failed (-6)")
            return dict(iters=20, filters=1, converged=1, energy=-1.0, energy_fp64=-1.0, resid_fp64=0.03,
                        gmres_iters_max=11, gmres_iters_total=220, gmres_relres_max=1e-5, grad_norm=1e-3,
                        resid_orth=1e-3, angle_bound=1e-2)

        def energy(self):
            return -1.0

        def profile(self, on=True):
            self.mode = on

        def profile_read(self):
            names = ("happly", "greenq", "trsv_levels", "orth", "gram", "block_update", "vector", "small",
                     "trsv_leaf")
            timed = getattr(self, "mode", False) is True   # per-class events only in profiling mode
            return {k: {"calls": 10, "kernels": 20, "ms": (1.0 + i) if timed else 0.0, "bytes": 1e9,
                        "impl_bytes": 2e9} for i, k in enumerate(names)}

        def device_bytes(self):
            return 1 << 30

        def close(self):
            pass

    lib.Solver = Solver
    return lib


class Event:
    clock = [0.0]

    def __init__(self, enable_timing=True):
        self.t = 0.0

    def record(self, stream=None):
        Event.clock[0] += 5.0
        self.t = Event.clock[0]

    def elapsed_time(self, other):
        return other.t - self.t


@pytest.fixture
def bench(monkeypatch):
    lib = fake_library()
    monkeypatch.setitem(sys.modules, "paper_1603_09724_gb300", lib)
    spec = importlib.util.spec_from_file_location("paper_1603_09724_gb300.serve",
                                                  os.path.join(ROOT, "paper_1603_09724_gb300", "serve.py"))
    serve = importlib.util.module_from_spec(spec)
    monkeypatch.setitem(sys.modules, "paper_1603_09724_gb300.serve", serve)
    spec.loader.exec_module(serve)
    cuda = torch.cuda
    monkeypatch.setattr(cuda, "set_device", lambda i: None)
    monkeypatch.setattr(cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(cuda, "Event", Event)
    monkeypatch.setattr(cuda, "current_stream", lambda *a: types.SimpleNamespace(cuda_stream=0,
                                                                                  synchronize=lambda: None))
    monkeypatch.setattr(cuda, "mem_get_info", lambda *a: (100 << 30, 200 << 30))
    monkeypatch.setattr(cuda, "Stream", lambda *a, **k: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(cuda, "stream", lambda s: contextlib.nullcontext())
    to, tensor, empty = torch.Tensor.to, torch.tensor, torch.empty

    def host_to(self, *a, **k):
        a = tuple(x for x in a if x != "cuda")
        k.pop("device", None)
        k.pop("non_blocking", None)
        return to(self, *a, **k) if (a or k) else self

    monkeypatch.setattr(torch.Tensor, "to", host_to)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    monkeypatch.setattr(torch, "tensor", lambda *a, **k: tensor(*a, **{x: v for x, v in k.items() if x != "device"}))
    monkeypatch.setattr(torch, "empty", lambda *a, **k: empty(*a, **{x: v for x, v in k.items() if x != "device"}))
    monkeypatch.syspath_prepend(ROOT)
    import bench as b
    return b, lib


def run(b, fn, argv, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        fn(b.args_parse())
    lines = out.getvalue().strip().splitlines()
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("argv", [["--no-cpu-baseline"],
                                  ["--precond", "gtpa", "--no-cpu-baseline", "--steps", "1"],
                                  ["--precond", "projector", "--no-cpu-baseline", "--no-fp64-check"]])
def test_solve_line_keeps_the_contract(bench, argv, monkeypatch):
    b, _ = bench
    rec = run(b, b.run_ours, argv, monkeypatch)
    for k in REQUIRED:
        assert k in rec, k
    assert rec["n_gpus"] == 1 and rec["higher_is_better"] is True and rec["unit"] == "solves/s"
    assert rec["e2e"]["h2d_bytes_per_step"] > 0 and rec["gpu_launches"] > 0
    assert rec["roofline"]["bound"] in ("hbm", "alu", "tensor") and rec["roofline"]["frac"] > 0
    assert "workload" in rec["config"] and "l2" in rec["config"]
    # the per-class profile comes from its own untimed solve, not from the timed region
    assert rec["kernels"]["pass"].startswith("one untimed solve")
    assert "counters on, per-class events off" in rec["config"]["timing"]
    if "accuracy_vs_fp64" in rec:
        assert "fp64_form_solves_per_s" in rec["accuracy_vs_fp64"] and "accuracy_gates" in rec


def test_serve_line_counts_failed_requests(bench, monkeypatch):
    b, lib = bench
    rec = run(b, b.run_many, ["--mode", "serve", "--requests", "10", "--rate", "100"], monkeypatch)
    assert rec["requests"] == 10 and rec["failed"] == 0 and rec["value"] > 0
    flaky = fake_library(fail_every=4)
    monkeypatch.setattr(lib, "Solver", flaky.Solver)
    rec = run(b, b.run_many, ["--mode", "serve", "--requests", "10", "--rate", "100"], monkeypatch)
    assert rec["requests"] == 10 and rec["failed"] == 2 and "CUDA runtime" in rec["first_error"]


def test_small_workload_times_one_whole_oracle_solve(bench, monkeypatch):
    """wells2d-32 finishes a whole oracle solve in seconds: the CPU baseline times one (the
    oracle's solve is stubbed here; its arithmetic has its own tests), with the poles'
    factorisations built before the timed call."""
    b, _ = bench
    from oracle import solve as osolve
    sp = json.load(open(os.path.join(ROOT, "workloads", "spectra.json")))["wells2d-32"]
    calls = []

    def fake_solve(shape, L, V, shift, X0, z, w, maxit=20, tol=1e-13, refilter=0, precond=None, **kw):
        calls.append(dict(maxit=maxit, tol=tol, refilter=refilter, precond=precond))
        return X0, dict(history=[[None] * 14], E=sp["E_ref"], precond=precond)

    monkeypatch.setattr(osolve, "solve", fake_solve)
    rec = run(b, b.run_ours, ["--workload", "wells2d-32", "--no-fp64-check", "--steps", "1"], monkeypatch)
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["unit"] == "solves/s" and cb["value"] > 0
    assert cb["sample"].startswith("one whole oracle solve") and "13 CG iterations" in cb["sample"]
    assert len(calls) == 1 and calls[0]["precond"] is not None and calls[0]["maxit"] == 40
