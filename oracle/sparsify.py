"""Sparsifying preconditioner for (H - sigma - z) u = b (oracle; test infrastructure only).

Sec. 3.2 of arXiv:1603.09724, written for the operator A = T + V - sigma - z where
T = -Delta/2 (kinetic symbol (2 pi^2/L^2)|k|^2):
  l = <V> (spatial average)                                  (text before eq. GLu)
  G = (T + l - sigma - z)^-1, diagonal in k                  (eq. GLu)
  (I + G (V - l)) u = G b                                    (eq. GLu)
  Q: row j supported on the stencil a(j), chosen so that Q(j,a(j)) G(a(j), a(j)^c) ~ 0
                                                             (eq. QG)
  P_{ji} = (Q + Q G (V - l))_{ji} for i in a(j), 0 elsewhere (eq. P)
  preconditioner: u~ = P^-1 Q (G b)                          (text after eq. P)

Readings (the paper defers details to the sparsifying-preconditioner papers):
  * a(j) is the (2r+1)^d box of grid points around j (periodic), r = 1 by default;
  * G is a circulant, so G(a(j), a(j)^c) is the same matrix for every j and one SVD
    gives one row q (unit norm) used for every j: q = conj(u_min)^T, u_min the left
    singular vector of G(a(0), a(0)^c) for its smallest singular value;
  * P is solved with a sparse direct LU (SuperLU here; the paper names nested
    dissection; any exact sparse solve gives the same u~ up to rounding).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from .hamiltonian import kinetic_symbol


def stencil_offsets(dim: int, r: int = 1):
    """Offsets of the (2r+1)^d box, x offset fastest (same flat order as the grid)."""
    rng = range(-r, r + 1)
    offs = []
    for tup in itertools.product(*([rng] * dim)):
        offs.append(tuple(reversed(tup)))            # tup = (dz, dy, dx) -> (dx, dy, dz)
    return offs


def _flat(shape, coords):
    idx = 0
    stride = 1
    for a, mi in enumerate(shape):
        idx = idx + (coords[a] % mi) * stride
        stride *= mi
    return idx


def green_symbol(shape, L, V, shift, z):
    """G(k) = 1 / (T(k) + l - sigma - z), l = mean(V)."""
    l = float(np.mean(V))
    return 1.0 / (kinetic_symbol(shape, L) + l - shift - z)


def green_kernel(shape, Ghat):
    """g[x] with G(i, j) = g[(i - j) mod m]: g = inverse DFT of G(k) (1/n included)."""
    g = np.fft.ifftn(Ghat.reshape(tuple(shape[::-1])))
    return g.ravel()


def setup(shape, L, V, shift, z, r: int = 1):
    """Build q, P and its sparse LU for one pole z.  Returns a dict."""
    dim = len(shape)
    n = int(np.prod(shape))
    V = np.asarray(V, dtype=np.float64)
    l = float(np.mean(V))
    Ghat = green_symbol(shape, L, V, shift, z)
    g = green_kernel(shape, Ghat)
    offs = stencil_offsets(dim, r)
    a0 = [_flat(shape, o) for o in offs]
    in_a = np.zeros(n, dtype=bool)
    in_a[a0] = True
    comp = np.nonzero(~in_a)[0]
    # coordinates of every grid point, to form (i - j) mod m in flat form
    coords = np.unravel_index(np.arange(n), tuple(shape[::-1]))[::-1]   # x, y, z arrays

    def diff_index(i_list, j_arr):
        out = np.empty((len(i_list), len(j_arr)), dtype=np.int64)
        for row, o in enumerate(i_list):
            dc = [(o[a] - coords[a][j_arr]) for a in range(dim)]
            out[row] = _flat(shape, dc)
        return out

    M = g[diff_index(offs, comp)]                    # G(a(0), a(0)^c)
    U, s, _ = np.linalg.svd(M, full_matrices=False)
    q = U[:, -1].conj()                              # row vector, ||q|| = 1
    Gaa = g[diff_index(offs, np.array(a0))]          # G(a(0), a(0))
    qg = q @ Gaa                                     # (QG)(0, a(0))
    # assemble P: row j, column j + offset_i (periodic)
    rows, cols, vals = [], [], []
    allc = np.stack([coords[a] for a in range(dim)], axis=1)
    for i, o in enumerate(offs):
        nb = _flat(shape, [allc[:, a] + o[a] for a in range(dim)])
        rows.append(np.arange(n))
        cols.append(nb)
        vals.append(q[i] + qg[i] * (V[nb] - l))
    P = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    lu = spl.splu(P)
    return dict(shape=tuple(shape), z=z, l=l, Ghat=Ghat, q=q, qg=qg, offsets=offs, P=P,
                lu=lu, sing=s)


def apply_green(st, b):
    """G b for a row-stored block b (ncols, n)."""
    shape = st["shape"]
    lead = b.shape[:-1]
    g = b.reshape(lead + tuple(shape[::-1]))
    axes = tuple(range(len(lead), len(lead) + len(shape)))
    out = np.fft.ifftn(st["Ghat"].reshape(tuple(shape[::-1])) * np.fft.fftn(g, axes=axes), axes=axes)
    return out.reshape(lead + (-1,))


def apply_q(st, v):
    """(Q v)_j = sum_i q_i v_{j + offset_i} (periodic stencil)."""
    shape = st["shape"]
    lead = v.shape[:-1]
    g = v.reshape(lead + tuple(shape[::-1]))
    out = np.zeros_like(g)
    d = len(shape)
    for qi, o in zip(st["q"], st["offsets"]):
        # value at j + o: roll by -o along each axis (axis order in g is z, y, x)
        shift = tuple(-o[a] for a in range(d))[::-1]
        out += qi * np.roll(g, shift, axis=tuple(range(len(lead), len(lead) + d)))
    return out.reshape(lead + (-1,))


def apply(st, b):
    """u~ = P^-1 Q (G b) for a row-stored block b (ncols, n)."""
    rhs = apply_q(st, apply_green(st, b))
    if rhs.ndim == 1:
        return st["lu"].solve(rhs)
    return st["lu"].solve(np.ascontiguousarray(rhs.T)).T
