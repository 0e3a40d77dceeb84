"""Many independent Hamiltonians solved by one CUDA-graph launch, with a measured
autotuner for the per-shape launch schedule.

Each instance (a Hamiltonian: grid, box, potential, N, spectral interval for the pole
rule) gets its own handle on its own CUDA stream.  Its solve runs a fixed schedule
(fixed_iters CG iterations per round, all gmres_m GMRES steps of each cycle, the systems
that meet the GMRES tolerance masked on the device), which omm_solve_enqueue enqueues
without any host synchronisation.  One warm-up solve
per handle allocates its work space; then the starting blocks and every instance's
enqueued solve are captured into one CUDA graph, the instances on parallel branches
(each stream forked from and joined back to the capturing stream), so that one
cudaGraphLaunch runs all of them and their kernels overlap on the device.

The autotuner picks, per shape (dim, m, N up to a multiple of 32, precision), the launch
schedule that gives
the shortest solve among candidates (complex64 Grams on tensor cores or CUDA cores; the
triangular solves on one stream or four), timing one fixed-schedule solve of each
candidate with CUDA events on the shape's first instance, and keeps the choices in a
JSON file keyed by the shape so that later batches reuse them.

All device work is the library's (libomm.so); this module only schedules it.
"""
from __future__ import annotations

import dataclasses
import json
import os
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Instance:
    key: str
    dim: int
    m: int
    L: float
    V: np.ndarray
    N: int
    lam1: float
    lamN: float
    lamN1: float
    sigma: Optional[float] = None
    P: int = 16
    X0: Optional[np.ndarray] = None    # host (N, n) starting block; a seeded real Gaussian if None
    seed: int = 0


# launch-schedule candidates of the autotuner (omm_params fields)
CANDIDATES = ({"gram_tensor": 1, "trsv_streams": 1}, {"gram_tensor": 0, "trsv_streams": 1},
              {"gram_tensor": 1, "trsv_streams": 4})


def shape_key(inst: Instance, precision: int) -> str:
    """Grid, precision and N rounded up to a multiple of 32: instances of one key share a
    schedule choice."""
    nb = 32 * ((inst.N + 31) // 32)
    return f"d{inst.dim}-m{inst.m}-N{nb}-p{precision}"


class Autotuner:
    """Per-shape choice among CANDIDATES by timed fixed-schedule solves; the table is kept
    in `path` (JSON, shape key -> chosen overrides and the measured milliseconds)."""

    def __init__(self, path: Optional[str] = None, candidates=CANDIDATES):
        self.path = path
        self.candidates = [dict(c) for c in candidates]
        self.table = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    def save(self):
        if self.path:
            with open(self.path, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)

    def choose(self, key: str, timer) -> dict:
        """timer(overrides) -> milliseconds of one solve with those overrides."""
        if key in self.table:
            return dict(self.table[key]["params"])
        best, best_ms, tried = None, None, {}
        for c in self.candidates:
            ms = float(timer(c))
            tried[json.dumps(c, sort_keys=True)] = ms
            if best_ms is None or ms < best_ms:
                best, best_ms = c, ms
        self.table[key] = {"params": best, "ms": best_ms, "tried": tried}
        self.save()
        return dict(best)


class GraphBatch:
    """instances: list of Instance; schedule: omm_params overrides shared by all (must
    include fixed_iters > 0); autotuner: an Autotuner or None (then
    `schedule` alone decides).  backend: this package by default."""

    def __init__(self, instances, schedule: dict, autotuner: Optional[Autotuner] = None, backend=None):
        import torch
        if backend is None:
            import paper_1603_09724_gb300 as backend
        self.torch = torch
        self.omm = backend
        self.instances = list(instances)
        self.schedule = dict(schedule)
        self.autotuner = autotuner
        self.precision = self.schedule.get("precision", backend.OMM_MIXED)
        self.dtype = torch.complex64 if self.precision == backend.OMM_MIXED else torch.complex128
        self.items = []
        self.graph = None
        self.chosen = {}

    # ---------------------------------------------------------------- set-up
    def _start_block(self, inst):
        if inst.X0 is not None:
            X0 = np.asarray(inst.X0)
        else:
            n = inst.m ** inst.dim
            rng = np.random.default_rng(1000 + inst.seed)
            X0 = np.sqrt(1.0 / n) * rng.standard_normal((inst.N, n))
        return self.torch.from_numpy(np.ascontiguousarray(X0)).to(device="cuda", dtype=self.dtype)

    def _solver(self, inst, stream, overrides):
        prm = self.omm.default_params(**{**self.schedule, **overrides})
        s = self.omm.Solver(inst.dim, inst.m, inst.L, inst.V, inst.N, shift=inst.sigma, params=prm,
                            stream=stream.cuda_stream)
        z, w = self.omm.poles_fermi(inst.lam1, inst.lamN, inst.lamN1, inst.P)
        s.set_poles(z, w)
        return s

    def _time(self, inst, overrides, X0):
        torch = self.torch
        st = torch.cuda.Stream()
        s = self._solver(inst, st, overrides)
        with torch.cuda.stream(st):
            s.set_orbitals(X0)
            s.solve()                         # allocates the work space
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.set_orbitals(X0)
            e0.record(st)
            s.solve_enqueue()
            e1.record(st)
        s.read_result()
        ms = e0.elapsed_time(e1)
        s.close()
        return ms

    def setup(self):
        """Handles, poles, starting blocks, one warm-up solve each (work space allocated)."""
        torch = self.torch
        for inst in self.instances:
            X0 = self._start_block(inst)
            key = shape_key(inst, self.precision)
            if self.autotuner is not None and key not in self.chosen:
                self.chosen[key] = self.autotuner.choose(key, lambda c: self._time(inst, c, X0))
            overrides = self.chosen.get(key, {})
            st = torch.cuda.Stream()
            s = self._solver(inst, st, overrides)
            with torch.cuda.stream(st):
                s.set_orbitals(X0)
                s.solve()
            self.items.append((inst, s, st, X0))
        torch.cuda.synchronize()

    def capture(self):
        """One CUDA graph: every instance's starting block and fixed-schedule solve on its
        own branch."""
        torch = self.torch
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=cap):
            for inst, s, st, X0 in self.items:
                st.wait_stream(cap)
                with torch.cuda.stream(st):
                    s.set_orbitals(X0)
                    s.solve_enqueue()
                cap.wait_stream(st)
        self.graph = g
        return g

    def run(self):
        """Replay the graph (one launch for all instances) and read every result."""
        self.graph.replay()
        self.torch.cuda.synchronize()
        return [s.read_result() for _, s, _, _ in self.items]

    def solve_alone(self, i):
        """The same fixed-schedule solve of instance i outside the graph (for comparison)."""
        inst, s, st, X0 = self.items[i]
        with self.torch.cuda.stream(st):
            s.set_orbitals(X0)
            s.solve_enqueue()
        st.synchronize()
        return s.read_result()

    def orbitals(self, i):
        inst, s, st, X0 = self.items[i]
        with self.torch.cuda.stream(st):
            X = s.get_orbitals()
        return X

    def close(self):
        self.graph = None
        for _, s, _, _ in self.items:
            s.close()
        self.items = []
