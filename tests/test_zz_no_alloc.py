"""omm_gram_noalloc: the Gram A^* B computed with a fixed device array instead of
allocated work memory, for callers that cannot call cudaMalloc (for example code running
inside another framework's memory manager, or on paths where the synchronisation of
cudaMalloc is not acceptable).  Its output must match omm_gram, the allocating entry
point, on consecutive calls that share the array.  This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

from workloads import gaussian_block

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as m
    return m


def noalloc(omm, prec, A, B, n):
    na, nb = A.shape[0], B.shape[0]
    C = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
    st = omm.lib.omm_gram_noalloc(prec, ctypes.c_void_p(A.data_ptr()), na, ctypes.c_void_p(B.data_ptr()), nb, n,
                                  ctypes.c_void_p(C.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    omm.check(st, "omm_gram_noalloc")
    torch.cuda.synchronize()
    return C.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_gram_matches_allocating_gram_on_consecutive_calls(omm, prec):
    m = 64
    n = m * m
    dt = torch.complex128 if prec == 0 else torch.complex64
    s = omm.Solver(2, m, 10.0, np.zeros(n), 8, params=omm.default_params(precision=prec))
    tol = 1e-13 if prec == 0 else 2e-6
    # two calls in a row with different shapes: the second reuses the array the first filled
    for seed, (na, nb) in enumerate([(40, 96), (17, 5)]):
        A = torch.from_numpy(gaussian_block(n, na, seed=10 + seed)).to(device="cuda", dtype=dt)
        B = torch.from_numpy(gaussian_block(n, nb, seed=20 + seed)).to(device="cuda", dtype=dt)
        ref = s.gram(A, B).cpu().numpy()
        got = noalloc(omm, prec, A, B, n)
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_gram_with_fewer_splits_matches_allocating_gram(omm, prec):
    """Shapes whose partials do not fit the array at the allocating Gram's split count: at
    724 x 724 (n = 16384) the array holds one split where omm_gram uses three; at 256 x 256 it
    holds eight where omm_gram uses nineteen.  Two calls in a row, each against omm_gram."""
    m = 128
    n = m * m
    dt = torch.complex128 if prec == 0 else torch.complex64
    s = omm.Solver(2, m, 10.0, np.zeros(n), 8, params=omm.default_params(precision=prec))
    tol = 1e-13 if prec == 0 else 2e-6
    for seed, (na, nb) in enumerate([(724, 724), (256, 256)]):
        A = torch.from_numpy(gaussian_block(n, na, seed=30 + seed)).to(device="cuda", dtype=dt)
        B = A if seed == 0 else torch.from_numpy(gaussian_block(n, nb, seed=40 + seed)).to(device="cuda", dtype=dt)
        got = noalloc(omm, prec, A, B, n)
        ref = s.gram(A, B).cpu().numpy()
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
        del A, B
    s.close()


def test_noalloc_gram_rejects_sizes_beyond_its_array(omm):
    n = 256
    A = torch.zeros((1024, n), dtype=torch.complex64, device="cuda")
    C = torch.empty(1, dtype=torch.complex128, device="cuda")
    st = omm.lib.omm_gram_noalloc(1, ctypes.c_void_p(A.data_ptr()), 1024, ctypes.c_void_p(A.data_ptr()), 1024, n,
                                  ctypes.c_void_p(C.data_ptr()), None)
    assert st == omm.OMM_EINVAL
    assert "static capacity" in omm.lib.omm_last_error_message().decode()
