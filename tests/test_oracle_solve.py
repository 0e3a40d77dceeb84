"""Pins for the whole oracle solve (Sec. 4 procedure; Algorithm 1) and oracle.metrics."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import metrics, poles, solve
from workloads import wells_2d, gaussian_block


def test_metrics_invariances():
    rng = np.random.default_rng(0)
    X = gaussian_block(50, 4, seed=1)
    A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    Y = A.T @ X                                        # same span, other basis
    assert metrics.max_angle_sine(X, Y) < 1e-12
    assert metrics.d_metric(X, Y) < 1e-12
    Z = gaussian_block(50, 4, seed=2)
    assert metrics.max_angle_sine(X, Z) > 0.1
    assert metrics.cond_number([1.0, 2.0, 4.0, 11.0], 2) == pytest.approx(10.0 / 2.0)


def test_metrics_closed_form_for_two_lines():
    """Two lines of R^2 at angle theta: the largest principal angle has sine |sin theta|,
    and the projector difference [[-s^2, cs], [cs, s^2]] has largest entry max(s^2, |cs|)
    (d is the entrywise-max ratio, the projector of the reference line has entry 1)."""
    for th in (0.1, 0.7, 1.3):
        c, s_ = np.cos(th), np.sin(th)
        X0 = np.array([[1.0, 0.0]])
        X = np.array([[c, s_]]) * 3.0                    # any scale: the span is what counts
        assert metrics.max_angle_sine(X, X0) == pytest.approx(abs(s_), abs=1e-14)
        assert metrics.d_metric(X, X0) == pytest.approx(max(s_ * s_, abs(c * s_)), abs=1e-14)


def test_small_solve_reaches_the_eigenspace():
    """Filter + preconditioned CG with exact pole solves: E = 1/2 sum lam_i and the
    subspace angle to the eigh subspace below 1e-10 (one refilter removes the filter
    leakage floor)."""
    shape, L, N = (16, 16), 10.0, 8
    V = wells_2d(16, L, seed=0)
    sig = ham.default_shift(shape, L, V)
    lamN, U, lam = solve.reference_eigs(shape, L, V, sig, N)
    z, w = poles.poles_conformal(lam[0], lam[N - 1], lam[N], 16)
    X0 = gaussian_block(256, N, seed=5)
    X, info = solve.solve(shape, L, V, sig, X0, z, w, maxit=40, tol=1e-14, mode="exact", refilter=1)
    assert info["E"] == pytest.approx(0.5 * lamN.sum(), rel=1e-12)
    assert metrics.max_angle_sine(X, U) < 1e-10


@pytest.mark.slow
def test_small_solve_with_gmres_and_sparsifying_preconditioner():
    """The paper's configuration (GMRES rtol 1e-5, restart 15, 5 cycles, sparsifying
    preconditioner): energy to 1e-10 and the subspace to the GMRES roughness."""
    shape, L, N = (16, 16), 10.0, 8
    V = wells_2d(16, L, seed=0)
    sig = ham.default_shift(shape, L, V)
    lamN, U, lam = solve.reference_eigs(shape, L, V, sig, N)
    z, w = poles.poles_conformal(lam[0], lam[N - 1], lam[N], 16)
    X0 = gaussian_block(256, N, seed=5)
    X, info = solve.solve(shape, L, V, sig, X0, z, w, maxit=30, tol=1e-13, mode="gmres", inner="spp")
    assert info["E"] == pytest.approx(0.5 * lamN.sum(), rel=1e-10)
    assert metrics.max_angle_sine(X, U) < 1e-5
