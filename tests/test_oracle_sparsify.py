"""Pins for oracle.sparsify (Sec. 3.2, eqs. GLu, QG, P)."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import sparsify
from workloads import wells_2d, gaussian_block


def dense_green(shape, L, V, shift, z):
    n = int(np.prod(shape))
    l = np.mean(V)
    A0 = ham.dense_kinetic(shape, L) + (l - shift - z) * np.eye(n)
    return np.linalg.inv(A0)


def brute_stencil(shape, r=1):
    """Stencil sets a(j) built directly from grid coordinates."""
    d = len(shape)
    pts = [p[::-1] for p in np.ndindex(*shape[::-1])]
    index = {p: i for i, p in enumerate(pts)}
    offs = sparsify.stencil_offsets(d, r)
    return [[index[tuple((p[a] + o[a]) % shape[a] for a in range(d))] for o in offs] for p in pts]


@pytest.mark.parametrize("shape", [(8, 8), (6, 6, 6)])
def test_q_is_the_minimal_row_and_p_matches_dense_definition(shape):
    """q minimises ||q G(a,a^c)|| over unit rows (checked against the smallest eigenvalue
    of the Hermitian G(a,a^c) G(a,a^c)^*), and P equals Q + QG(V - l) restricted to the
    stencil pattern, built with dense Q and G."""
    L = 5.0
    n = int(np.prod(shape))
    V = np.random.default_rng(1).uniform(-3, 1, n)
    shift, z = 40.0, 0.3 + 0.7j
    st = sparsify.setup(shape, L, V, shift, z)
    G = dense_green(shape, L, V, shift, z)
    a = brute_stencil(shape)
    comp = [i for i in range(n) if i not in set(a[0])]
    M = G[np.ix_(a[0], comp)]
    ev = np.linalg.eigvalsh(M @ M.conj().T)
    qM = st["q"] @ M
    assert np.linalg.norm(st["q"]) == pytest.approx(1.0, rel=1e-14)
    assert np.linalg.norm(qM) ** 2 == pytest.approx(ev[0], rel=1e-6, abs=1e-14 * ev[-1])
    # dense Q, then P restricted to the pattern
    Q = np.zeros((n, n), dtype=complex)
    for j in range(n):
        Q[j, a[j]] = st["q"]
    l = np.mean(V)
    full = Q + Q @ G @ np.diag(V - l)
    Pd = np.zeros_like(full)
    for j in range(n):
        Pd[j, a[j]] = full[j, a[j]]
    np.testing.assert_allclose(st["P"].toarray(), Pd, atol=1e-12 * np.max(np.abs(Pd)))
    # the preconditioner output equals P^-1 Q G b done densely
    b = gaussian_block(n, 3, seed=9)
    ref = np.linalg.solve(Pd, Q @ G @ b.T).T
    np.testing.assert_allclose(sparsify.apply(st, b), ref, atol=1e-10 * np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(16, 16), (6, 6, 6)])
def test_constant_potential_makes_preconditioner_exact(shape):
    """V = const => V - l = 0 => P = Q => P^-1 Q G b = G b = (H - sigma - z)^-1 b exactly."""
    L = 6.0
    n = int(np.prod(shape))
    V = np.full(n, -2.5)
    shift, z = 30.0, -1.0 + 0.4j
    st = sparsify.setup(shape, L, V, shift, z)
    b = gaussian_block(n, 2, seed=5)
    Hz = ham.dense_h(shape, L, V, shift) - z * np.eye(n)
    ref = np.linalg.solve(Hz, b.T).T
    np.testing.assert_allclose(sparsify.apply(st, b), ref, atol=1e-10 * np.max(np.abs(ref)))


def test_green_symbol_matches_dense_inverse():
    shape, L = (8, 8), 4.0
    V = wells_2d(8, L, seed=2)
    st = sparsify.setup(shape, L, V, 50.0, 0.2j)
    b = gaussian_block(64, 2, seed=3)
    G = dense_green(shape, L, V, 50.0, 0.2j)
    np.testing.assert_allclose(sparsify.apply_green(st, b), (G @ b.T).T, atol=1e-13)
