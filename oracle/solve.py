"""Whole preconditioned OMM solve (oracle; test infrastructure only).

Sec. 4: filter the starting guess with the preconditioner (X_1 = P X_0), then run the
preconditioned nonlinear CG of Algorithm 1 with the exact quartic line search.  The
reference answer of Sec. 1 (eq. tracemin): the span of the N lowest eigenvectors of
H - sigma, and the minimum E_omm = 1/2 sum_{i<=N} lam_i (the minimiser of E_omm spans
that eigenspace when H - sigma < 0).

refilter: if > 0, after the CG the filter is applied again and the CG restarted, that
many times (one more application of the same operators; used when the filter leakage
r(lam_{N+1}) exceeds the target subspace accuracy).
"""
from __future__ import annotations

import numpy as np

from . import omm
from .hamiltonian import apply_h_fft, dense_h
from .precond import PolePreconditioner


def reference_eigs(shape, L, V, shift, N):
    """Dense eigh of H - sigma: lowest N eigenvalues, eigenvectors (row-stored), all eigs."""
    H = dense_h(shape, L, V, shift)
    lam, U = np.linalg.eigh(H)
    return lam[:N], U[:, :N].T, lam


def solve(shape, L, V, shift, X0, z, w, maxit=20, tol=1e-13, mode="gmres", inner="spp",
          gmres_m=15, rtol=1e-5, cycles=5, fixed=False, refilter=0, min_iters=1, precond=None):
    """precond: a PolePreconditioner already built for these poles and options (its setup,
    the per-pole factorisations, then stays outside a caller's timing); None builds one."""
    Pc = precond if precond is not None else PolePreconditioner(shape, L, V, shift, z, w, mode=mode, inner=inner,
                                                                gmres_m=gmres_m, rtol=rtol, cycles=cycles,
                                                                fixed=fixed)
    apply_h = lambda X: apply_h_fft(X, shape, L, V, shift)
    X = Pc(X0)
    hist_all = []
    for rep in range(refilter + 1):
        if rep > 0:
            X = Pc(X)
        X, hist = omm.nlcg(apply_h, Pc, X, maxit=maxit, tol=tol, min_iters=min_iters)
        hist_all.append(hist)
    HX = apply_h(X)
    return X, dict(history=hist_all, E=omm.energy(X, HX), precond=Pc)
