"""Pins for oracle.hamiltonian (Sec. 4 Test 1, eq. ex1mat; Sec. 1 shift)."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from workloads import wells_2d, lattice_wells_3d, gaussian_block


def brute_force_kinetic(shape, L):
    """Kernel of F^-1 diag(T) F written entry by entry: (1/n) sum_k T(k) e^{2 pi i k.(x-y)/m}
    with k in [-m/2, m/2)^d -- no Kronecker products, no DFT matrices."""
    d = len(shape)
    pts = list(np.ndindex(*shape[::-1]))            # (z, y, x) tuples in flat order
    pts = [p[::-1] for p in pts]                    # -> (x, y, z)
    ks = list(np.ndindex(*shape))
    ks = [tuple(kk - (shape[a] if kk >= shape[a] // 2 else 0) for a, kk in enumerate(k)) for k in ks]
    n = len(pts)
    T = np.zeros((n, n), dtype=complex)
    for i, x in enumerate(pts):
        for j, y in enumerate(pts):
            s = 0.0
            for k in ks:
                k2 = sum(kk * kk for kk in k)
                ph = sum(k[a] * (x[a] - y[a]) / shape[a] for a in range(d))
                s += 2 * np.pi ** 2 / L ** 2 * k2 * np.exp(2j * np.pi * ph)
            T[i, j] = s / n
    return T


@pytest.mark.parametrize("shape", [(4, 4), (6, 4), (2, 4, 2)])
def test_dense_kinetic_matches_entrywise_definition(shape):
    L = 3.0
    np.testing.assert_allclose(ham.dense_kinetic(shape, L), brute_force_kinetic(shape, L),
                               atol=1e-12, rtol=0)


def test_h_is_real_symmetric():
    shape, L = (12, 12), 10.0
    V = wells_2d(12, L, seed=3)
    H = ham.dense_h(shape, L, V, 0.0)
    scale = np.max(np.abs(H))
    assert np.max(np.abs(H.imag)) <= 1e-13 * scale
    assert np.max(np.abs(H - H.T)) <= 1e-13 * scale
    assert np.max(np.abs(H - H.conj().T)) <= 1e-13 * scale


@pytest.mark.parametrize("shape,L", [((16, 16), 10.0), ((8, 8, 8), 4.0), ((12, 6), 2.0)])
def test_free_particle_closed_form_spectrum(shape, L):
    """V = 0: eigenvalues are (2 pi^2/L^2)|k|^2 - sigma over k in [-m/2,m/2)^d with the
    exact multiplicities (closed form, incl. the Nyquist shell)."""
    n = int(np.prod(shape))
    sigma = 7.25
    H = ham.dense_h(shape, L, np.zeros(n), sigma)
    ev = np.linalg.eigvalsh(H)
    closed = []
    for k in np.ndindex(*shape):
        kk = [k[a] - shape[a] if k[a] >= shape[a] // 2 else k[a] for a in range(len(shape))]
        closed.append(2 * np.pi ** 2 / L ** 2 * sum(x * x for x in kk) - sigma)
    np.testing.assert_allclose(ev, np.sort(closed), atol=1e-10 * max(1, np.max(np.abs(closed))))


def test_free_particle_2d_multiplicities():
    """2D shells |k|^2 = 0,1,2,4,5 have multiplicities 1,4,4,4,8 (lattice point counts)."""
    shape, L = (16, 16), 2.0
    H = ham.dense_h(shape, L, np.zeros(256), 0.0)
    ev = np.sort(np.linalg.eigvalsh(H)) / (2 * np.pi ** 2 / L ** 2)
    vals, counts = np.unique(np.round(ev, 8), return_counts=True)
    assert list(vals[:5]) == [0, 1, 2, 4, 5]
    assert list(counts[:5]) == [1, 4, 4, 4, 8]


@pytest.mark.parametrize("shape", [(16, 16), (6, 4, 8)])
def test_fft_apply_equals_dense(shape):
    L = 7.0
    n = int(np.prod(shape))
    V = np.random.default_rng(0).standard_normal(n)
    sigma = 3.0
    z = 0.5 + 0.25j
    X = gaussian_block(n, 5, seed=2)
    Hd = ham.dense_h(shape, L, V, sigma) - z * np.eye(n)
    ref = (Hd @ X.T).T
    got = ham.apply_h_fft(X, shape, L, V, sigma + z)
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.max(np.abs(ref)))


@pytest.mark.parametrize("shape,V", [((16, 16), wells_2d(16, 10.0, seed=1)),
                                     ((8, 8, 8), lattice_wells_3d(8, 40.0))])
def test_default_shift_makes_h_negative_definite(shape, V):
    L = 10.0 if len(shape) == 2 else 40.0
    sig = ham.default_shift(shape, L, V)
    ev = np.linalg.eigvalsh(ham.dense_h(shape, L, V, sig))
    lo, hi = ham.weyl_bounds(shape, L, V, sig)
    assert ev.max() < 0.0
    assert lo <= ev.min() + 1e-9 and ev.max() <= hi + 1e-9
