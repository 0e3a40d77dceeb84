"""Restarted, right-preconditioned GMRES (oracle; test infrastructure only).

Sec. 3.1 (eq. lst and the text after it) solves (H - z_j) Y = G(X) roughly by GMRES with
the right-hand side as the initial guess; Sec. 4 fixes relative tolerance 1e-5, restart
15 and at most 5 restarts (75 iterations).  The right preconditioner is the sparsifying
preconditioner of Sec. 3.2 (or, for the PP variant of Test 1, the shifted kinetic
inverse G).

Textbook GMRES (Saad & Schultz): Arnoldi with modified Gram-Schmidt on the
preconditioned operator A M^-1, least-squares solve of the small Hessenberg system, and
the update x = x0 + M^-1 V_k y.  The preconditioned basis Z_i = M^-1 v_i is kept
(flexible form), which is the same update in exact arithmetic.  Columns are independent
systems; they run side by side, and a column that meets the tolerance stops changing.
The tolerance is on the true relative residual ||b - A x|| / ||b|| per column; within a
cycle the small least-squares residual is used as its estimate.

With fixed=True the tolerance test is skipped and every cycle runs exactly m steps
(the fixed-step schedule used for bit-for-bit comparable runs).
"""
from __future__ import annotations

import numpy as np


def _norms(B):
    return np.sqrt(np.sum(np.abs(B) ** 2, axis=-1))


def gmres(apply_a, apply_m, b, x0, m: int = 15, rtol: float = 1e-5, max_cycles: int = 5,
          fixed: bool = False):
    """Solve A x = b for a row-stored block b (ncols, n).  Returns x, info dict."""
    b = np.atleast_2d(b)
    x = np.array(np.atleast_2d(x0), dtype=np.complex128, copy=True)
    ncols, n = b.shape
    nb = _norms(b)
    nb = np.where(nb == 0.0, 1.0, nb)
    active = np.ones(ncols, dtype=bool)
    iters = np.zeros(ncols, dtype=np.int64)
    relres = np.zeros(ncols)
    for cycle in range(max_cycles):
        r = b - apply_a(x)
        beta = _norms(r)
        relres = beta / nb
        if not fixed:
            active &= relres > rtol
        if not active.any():
            break
        V = np.zeros((m + 1, ncols, n), dtype=np.complex128)
        Z = np.zeros((m, ncols, n), dtype=np.complex128)
        Hh = np.zeros((ncols, m + 1, m), dtype=np.complex128)
        safe = np.where(beta == 0.0, 1.0, beta)
        V[0] = r / safe[:, None]
        steps = np.zeros(ncols, dtype=np.int64)
        live = active & (beta > 0.0)
        for k in range(m):
            if not live.any():
                break
            Z[k] = apply_m(V[k])
            w = apply_a(Z[k])
            for i in range(k + 1):                      # modified Gram-Schmidt
                hik = np.sum(V[i].conj() * w, axis=-1)
                Hh[:, i, k] = hik
                w = w - hik[:, None] * V[i]
            hk1 = _norms(w)
            Hh[:, k + 1, k] = hk1
            steps = np.where(live, k + 1, steps)
            V[k + 1] = w / np.where(hk1 == 0.0, 1.0, hk1)[:, None]
            # residual estimate of the small least-squares problem, per live column
            for col in np.nonzero(live)[0]:
                kk = k + 1
                e1 = np.zeros(kk + 1, dtype=np.complex128)
                e1[0] = beta[col]
                y, *_ = np.linalg.lstsq(Hh[col, :kk + 1, :kk], e1, rcond=None)
                est = np.linalg.norm(Hh[col, :kk + 1, :kk] @ y - e1) / nb[col]
                if hk1[col] == 0.0 or (not fixed and est <= rtol):
                    live[col] = False
        for col in np.nonzero(active & (steps > 0))[0]:
            kk = steps[col]
            e1 = np.zeros(kk + 1, dtype=np.complex128)
            e1[0] = beta[col]
            y, *_ = np.linalg.lstsq(Hh[col, :kk + 1, :kk], e1, rcond=None)
            x[col] = x[col] + np.tensordot(y, Z[:kk, col, :], axes=(0, 0))
            iters[col] += kk
    r = b - apply_a(x)
    relres = _norms(r) / nb
    return x, dict(iters=iters, relres=relres)
