"""Continuous-batching request loop for OMM solves on one GPU.

Requests (a Hamiltonian: grid, box, potential, N, its spectral interval for the pole rule)
arrive over time.  The server keeps, per Hamiltonian key, a resident handle: the device
copy of V, the FFT twiddles, the per-pole sparsifying factors and the last orbitals, so
that a repeated request skips the setup and warm-starts from the previous solution.
Admission is by device-memory footprint: a request waits until its handle fits the HBM
budget, evicting idle resident handles (least recently used) when needed.  Up to
`slots` solves run at the same time, each on its own CUDA stream and host thread (the
library's calls release the GIL), so their kernels overlap on the device; a new request
is admitted as soon as a slot and memory free up.  Latency = completion - arrival.  A
request that fails (a library error) comes back as a Result with `error` set.

All device work is the library's (libomm.so); this module only schedules it.
"""
from __future__ import annotations

import dataclasses
import queue
import threading
import time
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Request:
    key: str                      # Hamiltonian identity (same key = same H, warm start allowed)
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
    X0: Optional[np.ndarray] = None   # host (N, n) starting block; random if None and cold
    arrival: float = 0.0              # seconds (time.perf_counter scale), set by submit()
    rid: int = -1
    params: Optional[dict] = None     # omm_params overrides for this Hamiltonian's handle
                                      # (e.g. the inner preconditioner of a large 3D grid)


@dataclasses.dataclass
class Result:
    rid: int
    key: str
    X: Optional[np.ndarray]
    stats: dict
    latency_s: float
    queue_s: float
    warm: bool
    error: Optional[str] = None       # set (and X None) when the request failed


class _Resident:
    def __init__(self, solver, bytes_, stream):
        self.solver = solver
        self.bytes = bytes_
        self.stream = stream
        self.busy = False
        self.last_used = time.perf_counter()
        self.X = None      # device tensor of the last solution


class TorchDevice:
    """Device plumbing of the server (streams and host<->device copies) through PyTorch."""

    def __init__(self):
        import torch
        self.torch = torch

    def set_device(self, i):
        self.torch.cuda.set_device(i)

    def new_stream(self):
        return self.torch.cuda.Stream()

    def stream_ctx(self, stream):
        return self.torch.cuda.stream(stream)

    def stream_handle(self, stream):
        return stream.cuda_stream

    def upload(self, arr, dtype):
        return self.torch.from_numpy(np.ascontiguousarray(arr)).to(device="cuda", dtype=dtype, non_blocking=False)

    def download(self, t):
        return t.cpu().numpy()


class OmmServer:
    """slots: concurrent solves; hbm_budget: bytes the resident handles may hold;
    params: keyword overrides of omm_params (precision, tolerances ...).
    backend (default: this package) supplies Solver, default_params, poles_fermi and the
    precision constants; device (default: TorchDevice) the streams and copies."""

    def __init__(self, hbm_budget: int, slots: int = 4, device: int = 0, backend=None, device_api=None,
                 **params):
        if backend is None:
            import paper_1603_09724_gb300 as backend
        self.omm = backend
        self.dev = device_api if device_api is not None else TorchDevice()
        self.device = device
        self.budget = int(hbm_budget)
        self.slots = slots
        # one triangular-solve stream per handle: the server already overlaps handles
        self.params = dict(precision=backend.OMM_MIXED, maxit=40, tol=1e-10, trsv_streams=1, trsv_persistent=0)
        self.params.update(params)
        self.resident: dict[str, _Resident] = {}
        self.shape_bytes: dict[tuple, int] = {}
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.pending: list[Request] = []
        self.creating: set[str] = set()   # keys whose handle is being built
        self.reserved: dict[str, int] = {}   # estimated bytes held for handles being built
        self.results: "queue.Queue[Result]" = queue.Queue()
        self.active = 0
        self.next_id = 0
        self.stop = False
        self.sched = threading.Thread(target=self._scheduler, daemon=True)
        self.sched.start()

    # ---------------------------------------------------------------- public
    def submit(self, req: Request) -> int:
        if self._estimate(req) > self.budget:   # would wait forever for room
            raise ValueError("request needs more device memory than the server's budget")
        with self.cv:
            req.rid = self.next_id
            self.next_id += 1
            req.arrival = time.perf_counter()
            self.pending.append(req)
            self.cv.notify_all()
            return req.rid

    def drain(self, count: int, timeout: float = 3600.0) -> list[Result]:
        out = []
        t0 = time.perf_counter()
        while len(out) < count:
            out.append(self.results.get(timeout=max(1.0, timeout - (time.perf_counter() - t0))))
        return out

    def close(self, timeout: float = 600.0):
        """Stop admitting, wait (up to timeout) for the solves in flight, then free every
        resident handle."""
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        self.sched.join(timeout=10)
        t_end = time.perf_counter() + timeout
        with self.cv:
            while self.active > 0 and time.perf_counter() < t_end:
                self.cv.wait(timeout=0.05)
            for r in list(self.resident.values()):
                if not r.busy:
                    r.solver.close()
            self.resident.clear()

    def resident_bytes(self) -> int:
        return sum(r.bytes for r in self.resident.values())

    def _held(self) -> int:
        """Resident handles plus the reservations of handles being built."""
        return self.resident_bytes() + sum(self.reserved.values())

    # ---------------------------------------------------------------- internals
    def _shape(self, req: Request):
        return (req.dim, req.m, req.N, req.P, self.params.get("precision"),
                tuple(sorted((req.params or {}).items())))

    def _estimate(self, req: Request) -> int:
        """Footprint of a handle: measured for a shape seen before, else the GMRES work
        space (2m+4 vectors per system), the factors and the CG blocks."""
        shape = self._shape(req)
        if shape in self.shape_bytes:
            return self.shape_bytes[shape]
        n = req.m ** req.dim
        csz = 16 if self.params.get("precision") == self.omm.OMM_FP64 else 8
        gm = self.params.get("gmres_m", 15)
        S = req.P * req.N
        return int(((2 * gm + 5) * S * n + 8 * req.N * n) * csz + req.P * 400 * n * csz)

    def _admissible(self, req: Request) -> bool:
        if req.key in self.creating:
            return False
        if req.key in self.resident:
            return not self.resident[req.key].busy
        need = self._estimate(req)
        have = self.budget - self._held()
        if need <= have:
            return True
        # evict idle handles, least recently used first, while that helps
        idle = sorted((r for r in self.resident.values() if not r.busy), key=lambda r: r.last_used)
        freeable = sum(r.bytes for r in idle)
        return need <= have + freeable

    def _evict_for(self, need: int):
        idle = sorted(((k, r) for k, r in self.resident.items() if not r.busy), key=lambda kr: kr[1].last_used)
        for k, r in idle:
            if self.budget - self._held() >= need:
                break
            r.solver.close()
            del self.resident[k]

    def _scheduler(self):
        while True:
            with self.cv:
                while not self.stop and (self.active >= self.slots or
                                         not any(self._admissible(r) for r in self.pending)):
                    self.cv.wait(timeout=0.05)
                if self.stop:
                    return
                req = next(r for r in self.pending if self._admissible(r))
                self.pending.remove(req)
                self.active += 1
                if req.key not in self.resident:
                    need = self._estimate(req)
                    self._evict_for(need)
                    self.creating.add(req.key)
                    self.reserved[req.key] = need
                res = self.resident.get(req.key)
                if res is not None:
                    res.busy = True
            threading.Thread(target=self._run, args=(req,), daemon=True).start()

    def _run(self, req: Request):
        omm, dev = self.omm, self.dev
        t_start = time.perf_counter()
        res = self.resident.get(req.key)
        warm = res is not None and res.X is not None
        try:
            dev.set_device(self.device)
            if res is None:
                stream = dev.new_stream()
                s = None
                try:
                    with dev.stream_ctx(stream):
                        prm = omm.default_params(**{**self.params, **(req.params or {})})
                        s = omm.Solver(req.dim, req.m, req.L, req.V, req.N, shift=req.sigma, params=prm,
                                       stream=dev.stream_handle(stream))
                        z, w = omm.poles_fermi(req.lam1, req.lamN, req.lamN1, req.P)
                        s.set_poles(z, w)
                except BaseException:
                    if s is not None:      # created but not set up: never becomes resident
                        s.close()
                    raise
                res = _Resident(s, s.device_bytes(), stream)
                res.busy = True
                with self.cv:
                    self.resident[req.key] = res
                    self.creating.discard(req.key)
                    self.reserved.pop(req.key, None)
                    self.shape_bytes[self._shape(req)] = res.bytes
            s = res.solver
            with dev.stream_ctx(res.stream):
                if warm:
                    s.set_orbitals(res.X)
                else:
                    X0 = req.X0
                    if X0 is None:
                        from workloads import gaussian_block   # seeded synthetic start
                        X0 = gaussian_block(s.n, s.N, seed=1000 + req.rid)
                    s.set_orbitals(dev.upload(X0, s.dtype))
                st = s.solve()
                X = s.get_orbitals()
                res.X = X
                Xh = dev.download(X)
            done = time.perf_counter()
            self.results.put(Result(req.rid, req.key, Xh, st, done - req.arrival, t_start - req.arrival, warm))
        except Exception as e:   # the caller gets a failed result instead of waiting for one
            done = time.perf_counter()
            self.results.put(Result(req.rid, req.key, None, {}, done - req.arrival, t_start - req.arrival, warm,
                                    error=repr(e)))
        finally:
            with self.cv:
                self.creating.discard(req.key)
                self.reserved.pop(req.key, None)
                res = self.resident.get(req.key)
                if res is not None:
                    res.busy = False
                    res.last_used = time.perf_counter()
                self.active -= 1
                self.cv.notify_all()


def latency_summary(results: list[Result], wall_s: float) -> dict:
    """Throughput and latency of the completed solves; failed requests are counted apart."""
    ok = [r for r in results if r.error is None]
    lat = np.array([r.latency_s for r in ok]) if ok else np.zeros(1)
    return {"requests": len(results), "failed": len(results) - len(ok), "solves_per_s": len(ok) / wall_s,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "warm_fraction": float(np.mean([r.warm for r in ok])) if ok else 0.0}
