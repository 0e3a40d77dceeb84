"""The Fermi-projection preconditioner P R = sum_j w_j (H - z_j)^-1 R (oracle; test
infrastructure only).

Sec. 3.1 eqs. direct and lst: G_m = -sum_j w_j Y_{m,j}, (H - z_j) Y_{m,j} = G(X_m), each
Y_{m,j} a rough GMRES solution started from the right-hand side.  Sec. 4: the same
operator filters the starting guess once (X_1 = P X_0) before the CG.

ProjectorPreconditioner: the precomputed U U^* of Sec. 3.3 (Algorithm 2).

Modes
  'exact'  dense LU solve of every shifted system (n small): the projector r(H) itself
  'gmres'  GMRES per pole, inner right preconditioner 'spp' (sparsifying, Sec. 3.2),
           'lap' (shifted kinetic inverse G, the PP variant of Test 1) or 'none'
"""
from __future__ import annotations

import numpy as np

from . import gmres as _gmres
from . import sparsify
from .hamiltonian import apply_h_fft, dense_h


class PolePreconditioner:
    def __init__(self, shape, L, V, shift, z, w, mode="gmres", inner="spp", gmres_m=15,
                 rtol=1e-5, cycles=5, fixed=False, r=1):
        self.shape, self.L, self.V, self.shift = tuple(shape), L, np.asarray(V), shift
        self.z, self.w = np.asarray(z), np.asarray(w)
        self.mode, self.inner = mode, inner
        self.gmres_m, self.rtol, self.cycles, self.fixed = gmres_m, rtol, cycles, fixed
        self.stats = []
        if mode == "exact":
            H = dense_h(self.shape, L, self.V, shift)
            n = H.shape[0]
            self.lus = [np.linalg.inv(H - zj * np.eye(n)) for zj in self.z]
        else:
            self.spp = None
            if inner == "spp":
                self.spp = [sparsify.setup(self.shape, L, self.V, shift, zj, r) for zj in self.z]
            elif inner == "lap":
                self.spp = [dict(shape=self.shape,
                                 Ghat=sparsify.green_symbol(self.shape, L, self.V, shift, zj))
                            for zj in self.z]

    def solve_pole(self, j, R):
        """Y_j ~ (H - sigma - z_j)^-1 R for a row-stored block R."""
        if self.mode == "exact":
            return (self.lus[j] @ R.T).T
        zj = self.z[j]
        A = lambda x: apply_h_fft(x, self.shape, self.L, self.V, self.shift + zj)
        if self.inner == "spp":
            M = lambda v: sparsify.apply(self.spp[j], v)
        elif self.inner == "lap":
            M = lambda v: sparsify.apply_green(self.spp[j], v)
        else:
            M = lambda v: v
        Y, info = _gmres.gmres(A, M, R, R, m=self.gmres_m, rtol=self.rtol,
                               max_cycles=self.cycles, fixed=self.fixed)
        self.stats.append(info)
        return Y

    def __call__(self, R):
        R = np.atleast_2d(R)
        out = np.zeros(R.shape, dtype=np.complex128)
        for j in range(len(self.z)):
            out += self.w[j] * self.solve_pole(j, R)
        return out


class ProjectorPreconditioner:
    """The precomputed preconditioner U U^* of Sec. 3.3 (Algorithm 2), B with N + k columns
    (the paper's experiments use k = 0, B of size n x N):
      1. Y = sum_j w_j Y_j with (H - z_j) Y_j = B (pole: a PolePreconditioner, any mode);
      2. rank-revealing QR of Y (column pivoting), U = its first N orthonormal columns;
      3. the preconditioner is R -> U U^* R.
    Blocks are row-stored (N, n) like everywhere in the oracle: row j is column j."""

    def __init__(self, pole, B, N=None):
        """B: (N + k, n) Gaussian block; N: the number of columns kept (default: all of B,
        k = 0)."""
        import scipy.linalg as sla
        Y = pole(np.atleast_2d(B))
        N = Y.shape[0] if N is None else N
        Q, _, _ = sla.qr(Y.T, mode="economic", pivoting=True)
        self.U = np.ascontiguousarray(Q[:, :N].T)          # row-stored, orthonormal rows

    def __call__(self, R):
        R = np.atleast_2d(R)
        return (R @ self.U.conj().T) @ self.U               # columns: U (U^* R)
