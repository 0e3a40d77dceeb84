"""Host logic of the continuous-batching server (paper_1603_09724_gb300.serve) with a fake
solver and fake device plumbing, so that it runs without a GPU: the resident handles and
the reservations of handles being built never exceed the memory budget, idle handles are
evicted least recently used first, a repeated Hamiltonian warm-starts, no more than
`slots` solves run at once, and a request larger than the budget is refused.  Failures are
made on the host by the fake: a handle that cannot be built or set up, a solve that
raises; each comes back as a Result with `error`, leaks no handle or reservation, and the
server keeps serving.  close() waits for the solves in flight."""
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
        self.solves_done = 0
        self.closed_while_running = 0


class FakeBackend:
    OMM_FP64, OMM_MIXED = 0, 1

    def __init__(self, ledger, handle_bytes, solve_s=0.02, fail_create=(), fail_poles=(), fail_solve=()):
        self.ledger, self.handle_bytes, self.solve_s = ledger, handle_bytes, solve_s
        backend = self

        class Solver:
            def __init__(self, dim, m, L, V, N, shift=None, params=None, stream=None):
                if float(V[0]) in fail_create:
                    raise RuntimeError("omm_create: out of device memory (-2)")
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
                if self.key in fail_poles:
                    raise RuntimeError("omm_set_poles: out of device memory (-2)")

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
                    lg.solves_done += 1
                if self.key in fail_solve:
                    raise RuntimeError("omm_solve: a CUDA runtime call failed (-6)")
                return {"converged": 1, "iters": 3 if self.warm else 9, "energy_fp64": -1.0}

            def get_orbitals(self):
                return self.X

            def close(self):
                with backend.ledger.lock:
                    backend.ledger.live -= self.bytes
                    backend.ledger.closed.append(self.key)
                    backend.ledger.closed_while_running += backend.ledger.running

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


def test_failures_come_back_as_results_and_leak_nothing():
    lg = Ledger()
    one = handle_bytes()
    srv = server(lg, budget=int(2.5 * one), slots=2, fail_create=(1.0,), fail_poles=(2.0,), fail_solve=(3.0,))
    for k in (1, 2, 3, 4, 4):
        srv.submit(request(k))
    res = {r.rid: r for r in srv.drain(5, timeout=30)}
    t0 = time.perf_counter()                     # the last worker's bookkeeping follows its result
    while srv.active and time.perf_counter() - t0 < 10:
        time.sleep(0.01)
    assert "out of device memory" in res[0].error and res[0].X is None
    assert "out of device memory" in res[1].error
    assert "CUDA runtime" in res[2].error
    assert res[3].error is None and res[4].error is None and res[4].warm
    assert 2.0 in lg.closed                      # built, not set up: closed, never resident
    assert sorted(srv.resident) == ["3", "4"]    # a handle whose solve failed stays usable
    assert not srv.reserved and not srv.creating and srv.active == 0
    srv.submit(request(5))                       # still serving
    assert srv.drain(1, timeout=30)[0].error is None
    srv.close()
    assert lg.live == 0


def test_close_waits_for_solves_in_flight():
    lg = Ledger()
    one = handle_bytes()
    srv = server(lg, budget=int(4.5 * one), slots=3, solve_s=0.3)
    for k in (1, 2, 3):
        srv.submit(request(k))
    t0 = time.perf_counter()
    while lg.running < 3 and time.perf_counter() - t0 < 10:
        time.sleep(0.01)
    srv.close()
    assert lg.solves_done == 3 and lg.closed_while_running == 0 and lg.live == 0
