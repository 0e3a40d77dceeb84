"""Pseudospectral Hamiltonian on a periodic box (oracle; test infrastructure only).

Sec. 4, Test 1 (eq. ex1mat): H = -Delta/2 + V with -Delta/2 = F^-1 diag(2 pi^2 |k|^2) F
on the unit box and k in K = [-m/2, m/2)^d.  On a box of side L the kinetic symbol is
(2 pi^2 / L^2) |k|^2 (rescaling x = r/L).  Sec. 1: the diagonal is shifted by sigma so
that H - sigma I is negative definite (needed for E_omm to have the eigenspace as its
minimiser); the shift does not change the eigenvectors.

A grid function is a flat vector of n = prod(m) values, x index fastest.
"""
from __future__ import annotations

import numpy as np


def wave_numbers(m: int) -> np.ndarray:
    """Integer wave numbers in DFT order: 0..m/2-1, then -m/2..-1 (K = [-m/2, m/2))."""
    k = np.arange(m)
    return np.where(k < (m + 1) // 2 if m % 2 else k < m // 2, k, k - m)


def kinetic_symbol(shape, L: float) -> np.ndarray:
    """T(k) = (2 pi^2 / L^2) |k|^2 on the DFT grid, flat in the same (x fastest) order."""
    d = len(shape)
    ks = [wave_numbers(mi).astype(np.float64) for mi in shape]
    mesh = np.meshgrid(*ks[::-1], indexing="ij")[::-1]   # mesh[0] = k_x (fastest)
    k2 = sum(mesh[a] ** 2 for a in range(d))
    return (2.0 * np.pi ** 2 / L ** 2 * k2).ravel()


def dft_matrix_1d(m: int) -> np.ndarray:
    """F_1[k, j] = exp(-2 pi i k j / m) (unnormalised forward DFT), written out."""
    j = np.arange(m)
    return np.exp(-2j * np.pi * np.outer(j, j) / m)


def dft_matrix(shape) -> np.ndarray:
    """Forward DFT of a flat grid function with x fastest: F = F_z (x) F_y (x) F_x."""
    F = np.ones((1, 1), dtype=complex)
    for mi in shape[::-1]:            # slowest axis first in the Kronecker product
        F = np.kron(F, dft_matrix_1d(mi))
    return F


def dense_kinetic(shape, L: float) -> np.ndarray:
    """-Delta/2 = F^-1 diag(T) F as a dense n x n matrix (Sec. 4, eq. ex1mat)."""
    F = dft_matrix(shape)
    n = F.shape[0]
    T = kinetic_symbol(shape, L)
    return (F.conj().T * T) @ F / n


def dense_h(shape, L: float, V: np.ndarray, shift: float) -> np.ndarray:
    """Dense H_sigma = -Delta/2 + diag(V) - sigma I."""
    H = dense_kinetic(shape, L)
    H = H + np.diag(np.asarray(V, dtype=np.float64) - shift)
    return H


def apply_h_fft(X: np.ndarray, shape, L: float, V: np.ndarray, shift: complex) -> np.ndarray:
    """(H - shift) X for a block X given as (ncols, n) rows = columns, via the DFT
    (numpy pocketfft as the transform):  F^-1 (T . F x) + (V - shift) . x."""
    X = np.asarray(X)
    lead = X.shape[:-1]
    g = X.reshape(lead + tuple(shape[::-1]))
    axes = tuple(range(len(lead), len(lead) + len(shape)))
    T = kinetic_symbol(shape, L).reshape(tuple(shape[::-1]))
    Y = np.fft.ifftn(T * np.fft.fftn(g, axes=axes), axes=axes)
    Y = Y.reshape(lead + (-1,)) + (np.asarray(V) - shift) * X
    return Y


def kinetic_max(shape, L: float) -> float:
    """Largest kinetic symbol: (2 pi^2/L^2) * sum_a (m_a/2)^2 (Nyquist corner)."""
    return 2.0 * np.pi ** 2 / L ** 2 * sum((mi // 2) ** 2 for mi in shape)


def default_shift(shape, L: float, V: np.ndarray) -> float:
    """sigma = T_max + max(max V, 0) + delta, delta = 1e-3 * (T_max + max V - min V).

    By Weyl's inequality every eigenvalue of -Delta/2 + V is <= T_max + max V, so
    H - sigma is negative definite (Sec. 1: shift the diagonal so that H < 0)."""
    V = np.asarray(V, dtype=np.float64)
    tmax = kinetic_max(shape, L)
    width = tmax + V.max() - V.min()
    return float(tmax + max(V.max(), 0.0) + 1e-3 * width)


def weyl_bounds(shape, L: float, V: np.ndarray, shift: float) -> tuple[float, float]:
    """Spectral enclosure of H - sigma: [min V - sigma, T_max + max V - sigma]."""
    V = np.asarray(V, dtype=np.float64)
    return float(V.min() - shift), float(kinetic_max(shape, L) + V.max() - shift)
