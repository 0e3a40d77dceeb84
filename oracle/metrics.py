"""Accuracy metrics (oracle; test infrastructure only).

  principal angles between span(X) and span(X0) (largest one reported as its sine);
  d(X, X0) of Sec. 4: entrywise max-norm of X(X^*X)^-1X^* - X0(X0^*X0)^-1X0^* divided by
  the entrywise max-norm of the second projector;
  cond = (lam_n - lam_1) / (lam_{N+1} - lam_N) (Sec. 2.3, the lower bound on the
  condition number of the OMM Hessian, reported as "cond" in Tables 1-3).
Blocks are row-stored (N, n).
"""
from __future__ import annotations

import numpy as np


def orthonormal_basis(X):
    """Orthonormal basis of the row space of a row-stored block (via QR)."""
    Q, _ = np.linalg.qr(np.asarray(X).T)
    return Q                                            # n x N, orthonormal columns


def max_angle_sine(X, X0) -> float:
    """sin of the largest principal angle = ||(I - Q0 Q0^*) Q||_2."""
    Q = orthonormal_basis(X)
    Q0 = orthonormal_basis(X0)
    R = Q - Q0 @ (Q0.conj().T @ Q)
    return float(np.linalg.norm(R, 2))


def projector(X):
    Xc = np.asarray(X).T                                # n x N
    S = Xc.conj().T @ Xc
    return Xc @ np.linalg.solve(S, Xc.conj().T)


def d_metric(X, X0) -> float:
    P = projector(X)
    P0 = projector(X0)
    return float(np.max(np.abs(P - P0)) / np.max(np.abs(P0)))


def cond_number(eigs, N) -> float:
    e = np.sort(np.asarray(eigs))
    return float((e[-1] - e[0]) / (e[N] - e[N - 1]))
