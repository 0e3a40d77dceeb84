"""Continuous-batching server (paper_1603_09724_gb300.serve): a request gives the same
orbitals alone and when its solve overlaps other requests on the device, a repeated
Hamiltonian warm-starts from its resident previous solution, and admission keeps the
resident handles within the HBM budget."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from workloads import wells_2d, smooth_field_2d, gaussian_block

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def spectrum(m, V, N, L=10.0):
    sig = ham.default_shift((m, m), L, V)
    lam = np.linalg.eigvalsh(ham.dense_h((m, m), L, V, sig))
    return sig, lam[0], lam[N - 1], lam[N]


@pytest.fixture(scope="module")
def reqs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09724_gb300.serve import Request
    out = {}
    for key, m, N, V in (("A", 32, 16, wells_2d(32, 10.0, seed=0)), ("B", 48, 24, smooth_field_2d(48, 10.0, seed=2)),
                         ("C", 32, 8, wells_2d(32, 10.0, seed=5)), ("D", 32, 16, wells_2d(32, 10.0, seed=9))):
        sig, l1, lN, lN1 = spectrum(m, V, N)
        X0 = gaussian_block(m * m, N, seed=7, dtype=np.complex64)
        out[key] = lambda key=key, m=m, N=N, V=V, sig=sig, l1=l1, lN=lN, lN1=lN1, X0=X0: Request(
            key, 2, m, 10.0, V, N, l1, lN, lN1, sigma=sig, X0=X0)
    return out


def test_alone_and_in_the_mix_agree_and_warm_start(reqs):
    from paper_1603_09724_gb300.serve import OmmServer, latency_summary
    solo = OmmServer(hbm_budget=8 << 30, slots=1)
    solo.submit(reqs["A"]())
    a_alone = solo.drain(1)[0]
    solo.close()

    mix = OmmServer(hbm_budget=8 << 30, slots=4)
    for key in ("B", "A", "C", "B"):
        mix.submit(reqs[key]())
    res = mix.drain(4)
    mix.submit(reqs["A"]())            # same Hamiltonian again: warm start from the resident X
    res += mix.drain(1)
    summ = latency_summary(res, wall_s=sum(r.latency_s for r in res))
    mix.close()

    a_mix = [r for r in res if r.key == "A" and not r.warm][0]
    assert a_alone.stats["converged"] == 1 and a_mix.stats["converged"] == 1
    assert np.array_equal(a_alone.X, a_mix.X)              # bit for bit
    warm = [r for r in res if r.key == "A" and r.warm]
    assert len(warm) == 1 and warm[0].stats["iters"] < a_mix.stats["iters"]
    assert abs(warm[0].stats["energy_fp64"] - a_mix.stats["energy_fp64"]) <= 1e-9 * abs(a_mix.stats["energy_fp64"])
    assert summ["p99_ms"] >= summ["p50_ms"] > 0


def test_admission_respects_the_memory_budget(reqs):
    from paper_1603_09724_gb300.serve import OmmServer
    probe = OmmServer(hbm_budget=8 << 30, slots=1)
    probe.submit(reqs["A"]())
    probe.drain(1)
    one = probe.resident_bytes()
    probe.close()
    # room for one resident handle only: a second Hamiltonian of the same shape evicts the first
    srv = OmmServer(hbm_budget=int(one * 1.5), slots=2)
    srv.submit(reqs["A"]())
    srv.submit(reqs["D"]())
    out = srv.drain(2)
    assert all(r.stats["converged"] == 1 for r in out)
    assert srv.resident_bytes() <= int(one * 1.5)
    assert len(srv.resident) == 1
    srv.close()
