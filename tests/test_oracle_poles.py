"""Pins for oracle.poles (Sec. 3.1, eqs. FOP / dFOP)."""
import numpy as np
import pytest
from scipy import special

from oracle import hamiltonian as ham
from oracle import poles
from workloads import wells_2d


@pytest.mark.parametrize("P", [4, 8, 16, 30])
def test_circle_rule_closed_form(P):
    """Trapezoid rule on a circle: r(lam) = 1/(1 + ((lam - c)/R)^P) exactly (geometric
    series over the roots of w^P = -1)."""
    c, R = -3.0, 2.5
    z, w = poles.poles_circle(c, R, P)
    lam = np.linspace(-9, 4, 301)
    y = (lam - c) / R
    np.testing.assert_allclose(poles.filter_values(z, w, lam), 1.0 / (1.0 + y ** P), atol=1e-13)


def test_jacobi_complex_identities():
    """sn^2 + cn^2 = 1, dn^2 + m sn^2 = 1 and d sn/du = cn dn at complex u."""
    m = 0.81
    mp = 1 - m
    t = np.linspace(-3, 3, 13)
    y = 0.6
    sn, cn, dn = poles._jacobi_complex(t, y, m, mp)
    np.testing.assert_allclose(sn ** 2 + cn ** 2, 1.0, atol=1e-13)
    np.testing.assert_allclose(dn ** 2 + m * sn ** 2, 1.0, atol=1e-13)
    h = 1e-6
    sp, _, _ = poles._jacobi_complex(t + h, y, m, mp)
    sm, _, _ = poles._jacobi_complex(t - h, y, m, mp)
    np.testing.assert_allclose((sp - sm) / (2 * h), cn * dn, atol=1e-8)
    # sn(K + iK'/2) = 1/sqrt(k): the contour crosses the real axis in the gap
    K = special.ellipk(m)
    Kp = special.ellipk(mp)
    s, _, _ = poles._jacobi_complex(np.array([K]), 0.5 * Kp, m, mp)
    assert s[0] == pytest.approx(1 / np.sqrt(np.sqrt(m)), rel=1e-12)


def test_conformal_map_hits_interval_endpoints():
    a, b, c = -10.0, -2.0, -1.6
    prm = poles.conformal_parameters(a, b, c)
    assert poles.moebius(prm, -1.0) == pytest.approx(a, rel=1e-14)
    assert poles.moebius(prm, 1.0) == pytest.approx(b, rel=1e-14)
    assert poles.moebius(prm, 1.0 / prm["k"]) == pytest.approx(c, rel=1e-12)


@pytest.mark.parametrize("abc", [(-10.0, -2.0, -1.6), (-109.0, -103.3, -102.9), (-1.0, 3.0, 3.05)])
def test_conformal_rule_converges_at_predicted_rate(abc):
    """r -> 1 on [a, b] and -> 0 on [c, inf); the error decays like rho^P with
    rho = exp(-pi K'/(4K)) (the exp(-cP/(log cond + 3)) law of eq. dFOP)."""
    a, b, c = abc
    rho = poles.conformal_rate(a, b, c)
    lam_in = np.linspace(a, b, 3001)
    g = c - b
    lam_out = c + np.concatenate([np.linspace(0.0, 10 * g, 3001), np.geomspace(10 * g, 1e6, 3001)])
    errs = []
    Ps = [8, 16, 24]
    for P in Ps:
        z, w = poles.poles_conformal(a, b, c, P)
        ri = poles.filter_values(z, w, lam_in)
        ro = poles.filter_values(z, w, lam_out)
        assert np.max(np.abs(ri.imag)) < 1e-12 and np.max(np.abs(ro.imag)) < 1e-12
        e = max(np.max(np.abs(ri - 1)), np.max(np.abs(ro)))
        errs.append(e)
        assert e <= 8.0 * rho ** P
    # geometric decay with the predicted ratio (within a factor 3)
    ratio = errs[1] / errs[0]
    assert rho ** 8 / 3 <= ratio <= 3 * rho ** 8


def test_conformal_nodes_are_conjugate_pairs():
    z, w = poles.poles_conformal(-10.0, -2.0, -1.6, 16)
    key = lambda v: (round(v.real, 9), round(abs(v.imag), 9))
    zs = sorted(z, key=key)
    for i in range(0, 16, 2):
        assert zs[i] == pytest.approx(np.conj(zs[i + 1]), abs=1e-12)
    assert np.all(np.abs(z.imag) > 0)


def test_pole_expansion_equals_spectral_filter():
    """sum_j w_j (H - z_j)^-1 = U r(Lambda) U^* (the Fermi function computed by the
    eigendecomposition), and approaches the spectral projector as P grows."""
    shape, L = (12, 12), 10.0
    V = wells_2d(12, L, seed=5)
    sig = ham.default_shift(shape, L, V)
    H = ham.dense_h(shape, L, V, sig)
    lam, U = np.linalg.eigh(H)
    N = 5
    n = H.shape[0]
    for P in (8, 24):
        z, w = poles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
        Pm = sum(wj * np.linalg.inv(H - zj * np.eye(n)) for zj, wj in zip(z, w))
        r = poles.filter_values(z, w, lam)
        ref = (U * r) @ U.conj().T
        np.testing.assert_allclose(Pm, ref, atol=1e-11)
    Pi = U[:, :N] @ U[:, :N].conj().T
    assert np.max(np.abs(Pm - Pi)) < 1e-6


def test_conjugate_pairs_fold_for_real_blocks():
    """H - sigma is real symmetric (cosine DFT with the symmetric Nyquist multiplier), so for
    a real block R, (H - conj z)^-1 R = conj((H - z)^-1 R) and each conjugate pair of the
    pole sum contributes 2 Re(w (H - z)^-1 R): the sum over one pole per pair, doubled, has
    the same real part and the full sum is real."""
    shape, L = (10, 10), 10.0
    V = wells_2d(10, L, seed=3)
    sig = ham.default_shift(shape, L, V)
    H = ham.dense_h(shape, L, V, sig)
    assert np.max(np.abs(H.imag)) < 1e-13 * np.max(np.abs(H))   # real up to the DFT's rounding
    lam = np.linalg.eigvalsh(H)
    N, n = 6, H.shape[0]
    z, w = poles.poles_conformal(lam[0], lam[N - 1], lam[N], 16)
    R = np.random.default_rng(4).standard_normal((n, 3))
    full = sum(wj * np.linalg.solve(H - zj * np.eye(n), R) for zj, wj in zip(z, w))
    half = sum(2 * wj * np.linalg.solve(H - zj * np.eye(n), R) for zj, wj in zip(z, w) if zj.imag > 0)
    assert np.max(np.abs(full.imag)) < 1e-12 * np.max(np.abs(full))
    np.testing.assert_allclose(half.real, full.real, atol=1e-12 * np.max(np.abs(full)))
    # a planted mistake (pairs folded with conj w instead of w) fails the identity
    bad = sum(2 * np.conj(wj) * np.linalg.solve(H - zj * np.eye(n), R) for zj, wj in zip(z, w) if zj.imag > 0)
    assert np.max(np.abs(bad.real - full.real)) > 1e-6 * np.max(np.abs(full))
