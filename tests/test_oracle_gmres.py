"""Pins for oracle.gmres (Sec. 3.1 eq. lst; Sec. 4 GMRES parameters) and the
sparsifying preconditioner's effect (Sec. 3.2, Tests 2-3)."""
import numpy as np
import pytest

from oracle import gmres
from oracle import hamiltonian as ham
from oracle import poles
from oracle.precond import PolePreconditioner
from workloads import wells_2d, gaussian_block


def test_full_gmres_equals_direct_solve():
    """Without restart and with m = n steps GMRES is the exact solve (tiny system)."""
    rng = np.random.default_rng(0)
    n = 24
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 6 * np.eye(n)
    b = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    Mi = np.diag(1.0 / np.diag(A))
    x, info = gmres.gmres(lambda v: (A @ v.T).T, lambda v: (Mi @ v.T).T, b, np.zeros_like(b),
                          m=n, rtol=0.0, max_cycles=1, fixed=True)
    np.testing.assert_allclose(x, np.linalg.solve(A, b.T).T, atol=1e-10)


def test_gmres_meets_tolerance_and_restarts():
    rng = np.random.default_rng(1)
    n = 60
    A = np.diag(np.linspace(1, 30, n)) + 0.3 * rng.standard_normal((n, n))
    b = rng.standard_normal((4, n)) + 0j
    x, info = gmres.gmres(lambda v: (A @ v.T).T, lambda v: v, b, b, m=8, rtol=1e-6, max_cycles=20)
    assert np.all(info["relres"] <= 1e-6)
    assert np.all(info["iters"] > 8)          # needed restarts
    res = np.linalg.norm(b - (A @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)
    assert np.all(res <= 1e-6)


def test_fixed_schedule_residual_never_increases():
    rng = np.random.default_rng(2)
    n = 40
    A = np.diag(np.linspace(1, 10, n)) + 0.2 * rng.standard_normal((n, n))
    b = rng.standard_normal((2, n)) + 0j
    prev = np.full(2, np.inf)
    for k in range(1, 12):
        _, info = gmres.gmres(lambda v: (A @ v.T).T, lambda v: v, b, b, m=k, rtol=0.0,
                              max_cycles=1, fixed=True)
        assert np.all(info["relres"] <= prev * (1 + 1e-12))
        prev = info["relres"]


def test_sparsifying_preconditioner_makes_gmres_converge_fast():
    """Tests 2-3: with the sparsifying preconditioner the rough (1e-5) pole solves
    need only a few GMRES steps, while the shifted kinetic inverse alone (PP) needs far
    more for the poles near the gap."""
    shape, L = (32, 32), 10.0
    V = wells_2d(32, L, seed=0)
    sig = ham.default_shift(shape, L, V)
    lam = np.linalg.eigvalsh(ham.dense_h(shape, L, V, sig))
    N = 16
    z, w = poles.poles_conformal(lam[0], lam[N - 1], lam[N], 16)
    near = np.argsort(np.abs(z - 0.5 * (lam[N - 1] + lam[N])))[:2]
    b = gaussian_block(1024, 4, seed=3)
    spp = PolePreconditioner(shape, L, V, sig, z[near], w[near], inner="spp")
    lap = PolePreconditioner(shape, L, V, sig, z[near], w[near], inner="lap")
    for j in range(2):
        spp.solve_pole(j, b)
        lap.solve_pole(j, b)
    it_spp = max(int(s["iters"].max()) for s in spp.stats)
    it_lap = max(int(s["iters"].max()) for s in lap.stats)
    assert all(np.all(s["relres"] <= 1e-5) for s in spp.stats)
    assert it_spp <= 10
    assert it_lap > 3 * it_spp
