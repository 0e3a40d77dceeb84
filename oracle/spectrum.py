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
    lam = np.linalg.eigvalsh(Hk)
    return lam[:count]
