"""Pole expansion of the Fermi projector (oracle; test infrastructure only).

Sec. 3.1, eq. FOP: Pi = (2 pi i)^-1 \\oint_Gamma (z I - H)^-1 dz with Gamma enclosing the
N lowest eigenvalues.  Eq. dFOP: a quadrature rule turns it into Pi ~ sum_j w_j (H - z_j)^-1.
The paper takes the rule of Hale-Higham-Trefethen (conformal map of an annulus, trapezoid
rule) whose error decays like exp(-c p / (log(cond) + 3)) and does not print the nodes.

This module writes that construction out from the mathematics:

  * conformal rule: the strip 0 < Im u < K' (period 4K in Re u) is mapped by the Jacobi
    function s = sn(u; k) onto the s-plane minus the slits [-1, 1] and [1/k, inf] U
    [-inf, -1/k]; a Moebius map M sends [-1, 1] to the occupied interval [a, b] and the
    outer slit to [c, +inf] (so every unoccupied eigenvalue, however large, is covered and
    the rule has no constant term).  k follows from matching cross ratios:
    ((1+k)/(1-k))^2 = (c-a)/(c-b).  The contour is the image of Im u = K'/2; the trapezoid
    rule with P points in Re u gives z_j = M(sn(u_j)) and the weights from
    dz/du = M'(s) cn(u) dn(u).  For every eigenvalue the integrand is analytic in the open
    strip, so the error decays like exp(-pi K' P / (4 K)).
  * circle rule (special case / unit test): z_j = c + R exp(i theta_j),
    theta_j = pi (2j+1)/P, which gives exactly r(lam) = 1 / (1 + ((lam - c)/R)^P).

Convention: the preconditioner is sum_j w_j (H - z_j)^-1, so the scalar filter is
r(lam) = sum_j w_j / (lam - z_j).
"""
from __future__ import annotations

import numpy as np
from scipy import special


def poles_circle(center: float, radius: float, P: int):
    """Trapezoid rule on the circle |z - center| = radius (counter-clockwise)."""
    theta = np.pi * (2 * np.arange(P) + 1) / P
    e = np.exp(1j * theta)
    z = center + radius * e
    # (2 pi i)^-1 \oint (z-H)^-1 dz, dz = i R e^{i th} d th, h = 2 pi / P
    #   = sum_j (R e_j / P) (z_j - H)^-1 = sum_j (-R e_j / P) (H - z_j)^-1
    w = -radius * e / P
    return z, w


def filter_values(z, w, lam) -> np.ndarray:
    """r(lam) = sum_j w_j / (lam - z_j) for an array of real lam."""
    lam = np.asarray(lam, dtype=np.complex128)[..., None]
    return np.sum(np.asarray(w) / (lam - np.asarray(z)), axis=-1)


def _jacobi_complex(t, y, m, mp):
    """sn, cn, dn at u = t + i y (t real array, y real scalar), modulus parameter m = k^2,
    complementary mp = 1 - m, from real-argument values by the addition theorem and the
    imaginary transformation sn(iy|m) = i sc(y|mp), cn(iy|m) = nc(y|mp), dn(iy|m) = dc(y|mp)."""
    s1, c1, d1, _ = special.ellipj(t, m)
    s2, c2, d2, _ = special.ellipj(y, mp)
    S = 1j * s2 / c2
    C = 1.0 / c2
    D = d2 / c2
    den = 1.0 - m * s1 * s1 * S * S
    sn = (s1 * C * D + S * c1 * d1) / den
    cn = (c1 * C - s1 * S * d1 * D) / den
    dn = (d1 * D - m * s1 * S * c1 * C) / den
    return sn, cn, dn


def conformal_parameters(a: float, b: float, c: float):
    """Modulus and Moebius coefficients for occupied [a, b] and unoccupied [c, inf)."""
    if not (a < b < c):
        raise ValueError("need a < b < c")
    chi = (c - a) / (c - b)
    rchi = np.sqrt(chi)
    k = (rchi - 1.0) / (rchi + 1.0)
    kp2 = 4.0 * rchi / (rchi + 1.0) ** 2            # k'^2 = 1 - k^2, without cancellation
    m = k * k
    K = special.ellipkm1(kp2)                         # K(k)  (ellipkm1(p) = K(1 - p))
    Kp = special.ellipk(kp2)                          # K'(k) = K(k')
    kappa = 1.0 / k
    alpha = 0.5 * (b * (kappa + 1.0) - a * (kappa - 1.0))
    beta = 0.5 * (b * (kappa + 1.0) + a * (kappa - 1.0))
    return dict(k=k, m=m, mp=kp2, K=K, Kp=Kp, kappa=kappa, alpha=alpha, beta=beta)


def moebius(prm, s):
    return (prm["alpha"] * s + prm["beta"]) / (s + prm["kappa"])


def poles_conformal(a: float, b: float, c: float, P: int):
    """Conformal-map trapezoid rule (see module docstring). Returns z, w (length P)."""
    prm = conformal_parameters(a, b, c)
    K, Kp, m, mp = prm["K"], prm["Kp"], prm["m"], prm["mp"]
    h = 4.0 * K / P
    t = -2.0 * K + (np.arange(P) + 0.5) * h
    sn, cn, dn = _jacobi_complex(t, 0.5 * Kp, m, mp)
    z = moebius(prm, sn)
    dMds = (prm["alpha"] * prm["kappa"] - prm["beta"]) / (sn + prm["kappa"]) ** 2
    dzdu = dMds * cn * dn
    # (2 pi i)^-1 sum_j h dz/du (z_j - H)^-1  ==  sum_j w_j (H - z_j)^-1 with
    # w_j = -h dz/du / (2 pi i); the orientation is fixed so that r = +1 on [a, b].
    w = -h * dzdu / (2j * np.pi)
    if np.real(filter_values(z, w, 0.5 * (a + b))) < 0.0:
        w = -w
    return z, w


def conformal_rate(a: float, b: float, c: float) -> float:
    """Predicted geometric decay rate per pole: exp(-pi K' / (4 K))."""
    prm = conformal_parameters(a, b, c)
    return float(np.exp(-np.pi * prm["Kp"] / (4.0 * prm["K"])))
