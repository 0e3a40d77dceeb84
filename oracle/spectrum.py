"""Lowest eigenvalues of the grid Hamiltonian from a truncated plane-wave basis (oracle;
test infrastructure only).

On the grid, H = F^-1 diag(T) F + diag(V) (Sec. 4, eq. ex1mat).  In the DFT basis the
potential acts as the circular convolution with Vh = DFT(V)/n, so
    H(k, k') = T(k) delta_{kk'} + Vh(k - k')   (k - k' taken modulo the grid).
Restricting k, k' to the box |k|_inf <= kc gives a Hermitian matrix whose lowest
eigenvalues are those of the grid H whenever the low eigenvectors have no weight
outside the box (a smooth, band-limited V).  With kc >= m/2 the box is the whole grid
and the result is the dense eigh of H.  Used for the 128^2 smooth-field workload,
whose dense H (16384^2) is too large to diagonalise here.
"""
from __future__ import annotations

import itertools

import numpy as np

from .hamiltonian import kinetic_symbol


def lowest_eigs_kspace(shape, L, V, shift, count, kc):
    K, Hk = _kspace_matrix(shape, L, V, shift, kc)
    lam = np.linalg.eigvalsh(Hk)
    return lam[:count]


def kinetic_tau_kspace(shape, L, V, shift, N, kc):
    """tau of the TPA-type preconditioners (Sec. 4, Test 1): the largest (1/2) sum_k |k|^2
    |xhat_j(k)|^2 over the N lowest eigenvectors, here taken in the plane-wave box (whose
    eigenvectors are the Fourier coefficients xhat_j themselves, unit norm)."""
    K, Hk = _kspace_matrix(shape, L, V, shift, kc)
    _, C = np.linalg.eigh(Hk)
    k2 = np.sum(K.astype(np.float64) ** 2, axis=1)
    return float(np.max(0.5 * (k2 @ (np.abs(C[:, :N]) ** 2))))


def _kspace_matrix(shape, L, V, shift, kc):
    """Integer wave vectors K of the box |k|_inf <= kc and H(k, k') restricted to it."""
    d = len(shape)
    m = shape[0]
    n = int(np.prod(shape))
    Vh = np.fft.fftn(np.asarray(V).reshape(tuple(shape[::-1]))) / n       # axes (z, y, x)
    T = kinetic_symbol(shape, L).reshape(tuple(shape[::-1]))
    kc = min(kc, m // 2)
    rng = range(-kc, kc) if kc == m // 2 else range(-kc, kc + 1)
    ks = [tuple(reversed(t)) for t in itertools.product(*([rng] * d))]   # (kx, ky[, kz])
    K = np.array(ks)
    idx = tuple((K[:, a] % shape[a]) for a in range(d))[::-1]             # index tuple in (z, y, x)
    Tk = T[idx]
    diff = (K[:, None, :] - K[None, :, :])
    didx = tuple((diff[..., a] % shape[a]) for a in range(d))[::-1]
    Hk = Vh[didx] + np.diag(Tk) - shift * np.eye(len(ks))
    return K, Hk


def lowest_eigs_bloch(shape, L, V, shift, cells, count):
    """Exact lowest eigenvalues of the grid H for a potential periodic on a lattice of
    `cells` cells per axis (each cell mc = m / cells grid points wide).

    V(x + mc e_a) = V(x) makes Vh(q) vanish unless every component of q is a multiple of
    `cells`, so H(k, k') (above) couples k and k' only when k = k' (mod cells) in every
    component.  The DFT grid splits into cells^d Bloch sectors r (k = r + cells * j,
    j in [0, mc)^d), each a dense mc^d x mc^d Hermitian block; the union of the blocks'
    spectra is the spectrum of H, with no truncation.  Used for the 48^3 lattice workload
    (64 blocks of 1728)."""
    d = len(shape)
    m = shape[0]
    assert all(mi == m for mi in shape) and m % cells == 0
    mc = m // cells
    n = m ** d
    Vg = np.asarray(V).reshape((m,) * d)                                  # axes (z, y, x)
    Vh = np.fft.fftn(Vg) / n
    T = kinetic_symbol(shape, L).reshape((m,) * d)
    J = np.array([tuple(reversed(t)) for t in itertools.product(range(mc), repeat=d)])   # (jx, jy[, jz])
    lams = []
    for r in itertools.product(range(cells), repeat=d):
        K = np.asarray(r[::-1])[None, :] + cells * J                     # DFT indices (kx, ky[, kz]) in [0, m)
        Tk = T[tuple(K[:, a] for a in range(d))[::-1]]
        diff = (K[:, None, :] - K[None, :, :]) % m
        Hr = Vh[tuple(diff[..., a] for a in range(d))[::-1]] + np.diag(Tk - shift)
        lams.append(np.linalg.eigvalsh(Hr))
    lam = np.sort(np.concatenate(lams))
    return lam[:count]
