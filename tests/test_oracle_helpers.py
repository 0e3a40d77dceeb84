"""Direct pins for the oracle's helpers (each is also exercised through the functions built on
it): wave-number order and the Nyquist reading, the kinetic symbol's axis order, the explicit
DFT matrices against numpy's FFT (a library routine as the special case), the circulant
Green kernel of Sec. 3.2 against its dense definition, the periodic stencil apply Q of eq. QG
against an explicit loop, and the orthonormal basis behind the subspace metrics."""
import numpy as np
import pytest

from oracle import gtpa, hamiltonian as ham, metrics, sparsify


def test_wave_numbers_order_and_nyquist():
    assert list(ham.wave_numbers(8)) == [0, 1, 2, 3, -4, -3, -2, -1]      # K = [-m/2, m/2)
    assert list(ham.wave_numbers(6)) == [0, 1, 2, -3, -2, -1]
    assert list(ham.wave_numbers(1)) == [0]


@pytest.mark.parametrize("shape", [(6, 4), (4, 6, 2)])
def test_kinetic_symbol_axis_order_and_maximum(shape):
    L = 7.0
    T = ham.kinetic_symbol(shape, L)
    ks = [ham.wave_numbers(mi) for mi in shape]
    n = int(np.prod(shape))
    for i in range(n):
        idx, r = [], i
        for mi in shape:                       # x fastest
            idx.append(r % mi)
            r //= mi
        k2 = sum(int(ks[a][idx[a]]) ** 2 for a in range(len(shape)))
        assert T[i] == pytest.approx(2 * np.pi ** 2 / L ** 2 * k2, rel=1e-15)
    assert ham.kinetic_max(shape, L) == pytest.approx(T.max(), rel=1e-15)
    k2 = gtpa.integer_k2(shape)
    np.testing.assert_allclose(k2 * 2 * np.pi ** 2 / L ** 2, T, rtol=1e-15)


def test_dft_matrices_against_numpy_fft():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    F1 = ham.dft_matrix_1d(6)
    np.testing.assert_allclose(F1 @ x, np.fft.fft(x), atol=1e-12)
    np.testing.assert_allclose(F1 @ F1.conj().T, 6 * np.eye(6), atol=1e-12)
    shape = (6, 4)                             # x extent 6, y extent 4, x fastest
    g = rng.standard_normal(24) + 1j * rng.standard_normal(24)
    ref = np.fft.fftn(g.reshape(4, 6)).ravel()
    np.testing.assert_allclose(ham.dft_matrix(shape) @ g, ref, atol=1e-12)


def test_green_kernel_is_the_column_of_the_dense_circulant():
    """G = F^-1 diag(Ghat) F (explicit DFT matrices) is circulant with G(i, j) = g[i - j]
    taken component-wise modulo the grid."""
    shape, L = (6, 4), 10.0
    V = np.linspace(-1.0, 1.0, 24)
    Ghat = sparsify.green_symbol(shape, L, V, 30.0, -2.0 + 0.5j)
    g = sparsify.green_kernel(shape, Ghat)
    F = ham.dft_matrix(shape)
    G = (F.conj().T * Ghat) @ F / 24
    for i in range(24):
        for j in range(24):
            d = ((i % 6 - j % 6) % 6) + 6 * ((i // 6 - j // 6) % 4)
            assert abs(G[i, j] - g[d]) < 1e-13


def test_apply_q_is_the_periodic_stencil():
    shape = (5, 3)
    rng = np.random.default_rng(1)
    offs = sparsify.stencil_offsets(2)
    q = rng.standard_normal(len(offs)) + 1j * rng.standard_normal(len(offs))
    st = dict(shape=shape, q=q, offsets=offs)
    v = rng.standard_normal(15) + 1j * rng.standard_normal(15)
    out = sparsify.apply_q(st, v[None, :])[0]
    for j in range(15):
        x, y = j % 5, j // 5
        ref = sum(qi * v[(x + o[0]) % 5 + 5 * ((y + o[1]) % 3)] for qi, o in zip(q, offs))
        assert abs(out[j] - ref) < 1e-13


def test_orthonormal_basis_spans_the_rows():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((3, 10)) + 1j * rng.standard_normal((3, 10))
    Q = metrics.orthonormal_basis(X)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(3), atol=1e-13)
    np.testing.assert_allclose(Q @ (Q.conj().T @ X.T), X.T, atol=1e-12)
