"""Fourier-diagonal preconditioners of Sec. 2.2 -- shifted Laplacian (eq. Lap), TPA (eq.
TPA) and generalised TPA (eq. gTPA) -- the comparison preconditioners of the experiments
in Sec. 4 (oracle; test infrastructure only).

P_t is diagonal in the plane-wave basis: the component of wave vector k is multiplied by

    g_t(s) = p_t(s) / (p_t(s) + c_{t+1} s^{t+1}),   p_t(s) = c_0 + c_1 s + ... + c_t s^t,

with s = |k|^2 / tau, k the integer wave vector in K = [-m/2, m/2)^d.  t = 0 with
c = (1, 1) is eq. Lap, (1 + |k|^2 / tau)^-1; t = 3 with c = (27, 18, 12, 8, 16) is eq. TPA.
For other t the paper names the family but takes the coefficients from its reference;
default_coefficients states the reading used here.

tau (Sec. 4, Test 1): the largest kinetic energy (1/2) sum_k |k|^2 |xhat_j(k)|^2 over
the columns xhat_j of F X_0, where X_0 holds the exact eigenvectors (orthonormal) and F
is the unitary DFT; kinetic_tau computes it from a block of eigenvectors.
"""
from __future__ import annotations

import numpy as np

from .hamiltonian import wave_numbers


def default_coefficients(t: int) -> list:
    """c_0, ..., c_{t+1} of the gTPA family used when the caller gives none.

    Reading: the printed TPA coefficients are a geometric progression, 27, 18, 12, 8 =
    27 (2/3)^k for k = 0..3, and the tail 16 = 3 * 27 (2/3)^4.  The same pattern for any t,
    c_k = 27 (2/3)^k (k <= t) and c_{t+1} = 3 * 27 (2/3)^{t+1}, reproduces eq. TPA at t = 3
    and keeps TPA's large-s behaviour g_t(s) ~ c_t / (c_{t+1} s) = 1 / (2 s) for every t
    (so at t = 0 it is eq. Lap with tau halved)."""
    if t < 0:
        raise ValueError("t must be >= 0")
    c = [27.0 * (2.0 / 3.0) ** k for k in range(t + 1)]
    c.append(3.0 * 27.0 * (2.0 / 3.0) ** (t + 1))
    return c


def symbol(s, c):
    """g_t(s) (eq. gTPA) for s an array, a float or a fractions.Fraction; t = len(c) - 2."""
    t = len(c) - 2
    p = c[0] + 0 * s
    sk = 1 + 0 * s
    for k in range(1, t + 1):
        sk = sk * s
        p = p + c[k] * sk
    return p / (p + c[t + 1] * (sk * s))


def integer_k2(shape) -> np.ndarray:
    """|k|^2 of the integer wave vector at every DFT index, flat with x fastest."""
    d = len(shape)
    ks = [wave_numbers(mi).astype(np.float64) for mi in shape]
    mesh = np.meshgrid(*ks[::-1], indexing="ij")[::-1]   # mesh[0] = k_x (fastest)
    return sum(mesh[a] ** 2 for a in range(d)).ravel()


class GtpaPreconditioner:
    """R -> F^-1 diag(g_t(|k|^2 / tau)) F R for a row-stored block R (row j = column j)."""

    def __init__(self, shape, c, tau: float):
        if tau <= 0:
            raise ValueError("tau must be positive")
        self.shape, self.c, self.tau = tuple(shape), list(c), float(tau)
        self.g = symbol(integer_k2(self.shape) / self.tau, self.c)

    def __call__(self, R):
        R = np.atleast_2d(np.asarray(R, dtype=np.complex128))
        lead = R.shape[:-1]
        grid = R.reshape(lead + self.shape[::-1])
        axes = tuple(range(len(lead), len(lead) + len(self.shape)))
        gk = self.g.reshape(self.shape[::-1])
        return np.fft.ifftn(gk * np.fft.fftn(grid, axes=axes), axes=axes).reshape(R.shape)


def kinetic_tau(X0, shape) -> float:
    """tau = max_j (1/2) sum_k |k|^2 |xhat_j(k)|^2 / sum_k |xhat_j(k)|^2 over the rows x_j of
    X0 (row-stored eigenvectors; for orthonormal rows the denominator is 1)."""
    X0 = np.atleast_2d(X0)
    Xh = np.fft.fftn(X0.reshape((X0.shape[0],) + tuple(shape)[::-1]), axes=tuple(range(1, len(shape) + 1)))
    Xh = Xh.reshape(X0.shape[0], -1)
    w = np.abs(Xh) ** 2
    return float(np.max(0.5 * (w @ integer_k2(shape)) / w.sum(axis=1)))
