"""Host logic of the continuous-batching server (paper_1603_09724_gb300.serve) with a fake
solver and fake device plumbing, so that it runs without a GPU: the resident handles and
the reservations of handles being built never exceed the memory budget, idle handles are
evicted least recently used first, a repeated Hamiltonian warm-starts, no more than
`slots` solves run at once, and a request larger than the budget is refused."""
import contextlib
import threading
import time

import numpy as np
import pytest

from paper_1603_09724_gb300.serve import OmmServer, Request


class Ledger:
    def __init__(self):
        self.lock = threading.Lock()
        self.live = 0          # bytes of open fake handles
        self.peak = 0
        self.running = 0
        self.peak_running = 0
        self.created = []
        self.closed = []


class FakeBackend:
    OMM_FP64, OMM_MIXED = 0, 1

    def __init__(self, ledger, handle_bytes, solve_s=0.02):
        self.ledger, self.handle_bytes, self.solve_s = ledger, handle_bytes, solve_s
        backend = self

        class Solver:
            def __init__(self, dim, m, L, V, N, shift=None, params=None, stream=None):
                self.key = float(V[0])
                self.n, self.N = m ** dim, N
                self.dtype = np.complex64
                self.bytes = backend.handle_bytes
                self.X = None
                with backend.ledger.lock:
                    backend.ledger.live += self.bytes
                    backend.ledger.peak = max(backend.ledger.peak, backend.ledger.live)
                    backend.ledger.created.append(self.key)

            def set_poles(self, z, w):
                pass

            def device_bytes(self):
                return self.bytes

            def set_orbitals(self, X):
                self.warm = self.X is not None and X is self.X
                self.X = X

            def solve(self):
                lg = backend.ledger
                with lg.lock:
                    lg.running += 1
                    lg.peak_running = max(lg.peak_running, lg.running)
                time.sleep(backend.solve_s)
                with lg.lock:
                    lg.running -= 1
                return {"converged": 1, "iters": 3 if self.warm else 9, "energy_fp64": -1.0}

            def get_orbitals(self):
                return self.X

            def close(self):
                with backend.ledger.lock:
                    backend.ledger.live -= self.bytes
                    backend.ledger.closed.append(self.key)

        self.Solver = Solver

    @staticmethod
    def default_params(**kw):
        return dict(kw)

    @staticmethod
    def poles_fermi(a, b, c, P):
        return np.zeros(P), np.zeros(P)


class FakeDevice:
    def set_device(self, i):
        pass

    def new_stream(self):
        return None

    def stream_ctx(self, stream):
        return contextlib.nullcontext()

    def stream_handle(self, stream):
        return None

    def upload(self, arr, dtype):
        return np.asarray(arr, dtype=dtype)

    def download(self, t):
        return t


def request(key, m=16, N=4):
    return Request(str(key), 2, m, 10.0, np.full(m * m, float(key)), N, -3.0, -2.0, -1.0, sigma=5.0,
                   X0=np.zeros((N, m * m), dtype=np.complex64))


def handle_bytes():
    """A fake handle holds 90% of the server's a-priori estimate (measured handles come in
    below it on the GPU too)."""
    probe = OmmServer(hbm_budget=1 << 40, slots=1, backend=FakeBackend(Ledger(), 0), device_api=FakeDevice(),
                      precision=1)
    est = probe._estimate(request(0))
    probe.close()
    return int(0.9 * est)


def server(ledger, budget, slots, **kw):
    return OmmServer(hbm_budget=budget, slots=slots, backend=FakeBackend(ledger, handle_bytes(), **kw),
                     device_api=FakeDevice(), precision=1)


def test_budget_slots_and_warm_starts():
    lg = Ledger()
    one = handle_bytes()
    srv = server(lg, budget=int(2.5 * one), slots=3)
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 5, size=40)
    for k in keys:
        srv.submit(request(int(k)))
    res = srv.drain(len(keys), timeout=60)
    srv.close()
    assert len(res) == len(keys) and all(r.stats["converged"] == 1 for r in res)
    assert lg.peak <= 2.5 * one               # never more than two handles alive
    assert lg.peak_running <= 3
    assert lg.live == 0                        # close() released every handle
    assert any(r.warm for r in res) and all(r.stats["iters"] == (3 if r.warm else 9) for r in res)


def test_least_recently_used_idle_handle_is_evicted():
    lg = Ledger()
    one = handle_bytes()
    srv = server(lg, budget=int(2.5 * one), slots=1)
    for k in (1, 2):
        srv.submit(request(k))
        srv.drain(1)
    srv.submit(request(1))                     # touch 1: now 2 is the least recently used
    srv.drain(1)
    srv.submit(request(3))                     # needs room: evicts 2
    srv.drain(1)
    assert lg.closed == [2.0]
    assert sorted(srv.resident) == ["1", "3"]
    srv.close()


def test_request_larger_than_the_budget_is_refused():
    lg = Ledger()
    srv = server(lg, budget=1000, slots=1)
    with pytest.raises(ValueError):
        srv.submit(request(1, m=32, N=16))
    srv.close()
