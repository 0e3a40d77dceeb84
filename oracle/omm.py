"""OMM energy, gradient, Hessian, exact quartic line search and preconditioned nonlinear
CG (oracle; test infrastructure only).

Blocks are stored as (N, n) arrays whose row j is the column x_j of the n x N matrix X,
so X^* Y = Xr.conj() @ Yr.T with Xr, Yr the row-stored blocks.

References (arXiv:1603.09724):
  eq. omm      E_omm(X) = 1/2 tr((2 I - X^*X)(X^* H X))
  Sec. 2.1     G(X) = 2 H X - X (X^* H X) - H X (X^* X)
  Sec. 2.3     Hessian H(X) Z = 2HZ - Z(X^*HX) - X(Z^*HX) - X(X^*HZ) - HZ(X^*X)
                                - HX(Z^*X) - HX(X^*Z)
  Algorithm 1  preconditioned nonlinear CG with Polak-Ribiere beta and a line search
"""
from __future__ import annotations

import numpy as np


def gram(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^* B for row-stored blocks: (N, n), (M, n) -> N x M."""
    return A.conj() @ B.T


def energy(X: np.ndarray, HX: np.ndarray) -> float:
    """E_omm = 1/2 tr((2I - S) K), S = X^*X, K = X^*HX (eq. omm).  Real for Hermitian H."""
    S = gram(X, X)
    K = gram(X, HX)
    N = S.shape[0]
    return float(0.5 * np.real(np.trace((2.0 * np.eye(N) - S) @ K)))


def gradient(X: np.ndarray, HX: np.ndarray) -> np.ndarray:
    """G(X) = 2HX - X (X^*HX) - HX (X^*X) (Sec. 2.1); returned row-stored.

    With row-stored blocks, (X M)^T = M^T X_rows, so X M becomes M.T @ Xr."""
    S = gram(X, X)
    K = gram(X, HX)
    return 2.0 * HX - K.T @ X - S.T @ HX


def hessian_apply(X, HX, Z, HZ):
    """Directional derivative of G at X along Z (Sec. 2.3, Hessian formula)."""
    return (2.0 * HZ - gram(X, HX).T @ Z - gram(Z, HX).T @ X - gram(X, HZ).T @ X
            - gram(X, X).T @ HZ - gram(Z, X).T @ HX - gram(X, Z).T @ HX)


def quartic_coefficients(X, HX, D, HD) -> np.ndarray:
    """c_0..c_4 with E_omm(X + t D) = sum_k c_k t^k.

    Expanding eq. omm with S(t) = A + tB + t^2 C and K(t) = A_H + t B_H + t^2 C_H, where
    A = X^*X, B = X^*D + D^*X, C = D^*D, A_H = X^*HX, B_H = X^*HD + D^*HX, C_H = D^*HD,
    gives E(t) = tr K(t) - 1/2 tr(S(t) K(t)), collected by powers of t."""
    A = gram(X, X)
    B = gram(X, D) + gram(D, X)
    C = gram(D, D)
    AH = gram(X, HX)
    BH = gram(X, HD) + gram(D, HX)
    CH = gram(D, HD)
    tr = lambda M: np.real(np.trace(M))
    c0 = tr(AH) - 0.5 * tr(A @ AH)
    c1 = tr(BH) - 0.5 * (tr(A @ BH) + tr(B @ AH))
    c2 = tr(CH) - 0.5 * (tr(A @ CH) + tr(B @ BH) + tr(C @ AH))
    c3 = -0.5 * (tr(B @ CH) + tr(C @ BH))
    c4 = -0.5 * tr(C @ CH)
    return np.array([c0, c1, c2, c3, c4])


def quartic_value(c, t):
    return c[0] + t * (c[1] + t * (c[2] + t * (c[3] + t * c[4])))


def line_search(c) -> float:
    """Exact minimiser of the quartic over real t.

    The stationary points are the real roots of 4c4 t^3 + 3c3 t^2 + 2c2 t + c1; with
    c4 > 0 (H negative definite) the quartic is bounded below and its minimum is at one
    of them.  Among them take the least E; on a tie the smaller |t|."""
    c = np.asarray(c, dtype=np.float64)
    if c[4] <= 0.0:
        raise ValueError("quartic not bounded below (c4 <= 0): H - sigma is not negative definite")
    r = np.roots([4.0 * c[4], 3.0 * c[3], 2.0 * c[2], c[1]])
    scale = max(1.0, np.max(np.abs(r)))
    real = [float(x.real) for x in r if abs(x.imag) <= 1e-7 * scale]
    if not real:
        real = [float(r[np.argmin(np.abs(r.imag))].real)]
    vals = [quartic_value(c, t) for t in real]
    best = min(vals)
    tol = 4.0 * np.finfo(float).eps * max(1.0, abs(best))
    cands = [t for t, v in zip(real, vals) if v <= best + tol]
    return min(cands, key=abs)


def inner(A, B) -> float:
    """Real Frobenius inner product Re tr(A^* B), used for the Polak-Ribiere beta."""
    return float(np.real(np.vdot(A, B)))


def nlcg(apply_h, precondition, X1, maxit: int, tol: float = 1e-13, min_iters: int = 1):
    """Preconditioned nonlinear CG of Algorithm 1.

    apply_h(X) -> HX;  precondition(R) -> P R (the preconditioner of Sec. 3.1).
    G_m = -P G(X_m); beta_m = Re<G_m, G_m - G_{m-1}> / <G_{m-1}, G_{m-1}> (Polak-Ribiere);
    D_m = G_m + beta_m D_{m-1} (read as the standard conjugate update); t = exact quartic
    line search; X_{m+1} = X_m + t D_m.  Stops when |E_{m+1} - E_m| <= tol |E_{m+1}| (after
    min_iters steps) or after maxit steps.

    Returns X, history (list of dicts with E, t, beta, |G|)."""
    X = np.array(X1, copy=True)
    HX = apply_h(X)
    E = energy(X, HX)
    hist = [dict(E=E, t=0.0, beta=0.0, gnorm=0.0)]
    G_prev = None
    D = None
    for it in range(maxit):
        Gr = gradient(X, HX)
        G = -precondition(Gr)
        if G_prev is None:
            beta = 0.0
            D = G
        else:
            beta = inner(G, G - G_prev) / inner(G_prev, G_prev)
            D = G + beta * D
        HD = apply_h(D)
        c = quartic_coefficients(X, HX, D, HD)
        t = line_search(c)
        X = X + t * D
        HX = HX + t * HD
        E_new = energy(X, HX)
        hist.append(dict(E=E_new, t=t, beta=beta, gnorm=float(np.linalg.norm(Gr)),
                         c=c, E_pred=quartic_value(c, t)))
        converged = abs(E_new - E) <= tol * abs(E_new)
        E = E_new
        G_prev = G
        if converged and it + 1 >= min_iters:
            break
    return X, hist
