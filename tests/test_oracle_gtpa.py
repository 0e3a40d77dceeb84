"""Pins for oracle.gtpa, the Fourier-diagonal comparison preconditioners of Sec. 2.2 (eqs.
Lap, TPA, gTPA): the printed TPA coefficients, the special case of eq. Lap against a
dense solve built from the explicit DFT matrix, plane waves as eigenfunctions, the two
limits that define the family (g_t = 1 - O(s^{t+1}) at 0, ~1/s at infinity), tau of
Sec. 4 against closed forms and a dense Rayleigh quotient, and OMM with TPA reaching the
exact energy in far more iterations than with the pole expansion (Tables 1-3)."""
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

from oracle import gtpa, hamiltonian as ham, omm as oomm, poles as opoles
from oracle.precond import PolePreconditioner
from workloads import gaussian_block, gaussian_block_real, wells_2d

GOLDEN = Path(__file__).parent / "golden"


def test_default_t3_is_the_printed_tpa():
    rows = [l for l in (GOLDEN / "tpa_coefficients.txt").read_text().splitlines() if l and l[0] != "#"]
    printed = [float(v) for v in rows[0].split()]
    np.testing.assert_allclose(gtpa.default_coefficients(3), printed, rtol=1e-14)
    s = np.linspace(0.0, 50.0, 11)
    p = printed[0] + printed[1] * s + printed[2] * s ** 2 + printed[3] * s ** 3
    np.testing.assert_allclose(gtpa.symbol(s, printed), p / (p + printed[4] * s ** 4), rtol=1e-14)


def test_laplacian_case_is_the_dense_shifted_inverse():
    """t = 0, c = (1, 1) is eq. Lap, the symbol (1 + |k|^2 / tau)^-1 in integer wave numbers.
    The dense kinetic matrix T (explicit DFT) has the symbol kappa |k|^2, kappa = 2 pi^2 / L^2,
    so the operator is (I + T / (kappa tau))^-1: a dense solve, no FFT."""
    shape, L, tau = (6, 8), 10.0, 3.7
    T = ham.dense_kinetic(shape, L)
    kappa = 2 * np.pi ** 2 / L ** 2
    P = np.linalg.inv(np.eye(T.shape[0]) + T / (kappa * tau))
    R = gaussian_block(48, 3, seed=1)
    np.testing.assert_allclose(gtpa.GtpaPreconditioner(shape, [1.0, 1.0], tau)(R), (P @ R.T).T, atol=1e-13)


@pytest.mark.parametrize("shape,k", [((8, 8), (3, -2)), ((8, 8), (-4, 0)), ((6, 4, 4), (1, -2, 2)),
                                     ((6, 4, 4), (-3, 0, -2))])
def test_plane_waves_are_eigenfunctions(shape, k):
    """exp(2 pi i k.x / m) is multiplied by g_t(|k|^2 / tau), the Nyquist index included."""
    grids = np.meshgrid(*[np.arange(mi) for mi in shape[::-1]], indexing="ij")[::-1]   # [0] = x
    phase = sum(2 * np.pi * k[a] * grids[a] / shape[a] for a in range(len(shape)))
    x = np.exp(1j * phase).ravel()
    c, tau = gtpa.default_coefficients(5), 2.5
    k2 = sum(ka * ka for ka in k)
    y = gtpa.GtpaPreconditioner(shape, c, tau)(x)[0]
    np.testing.assert_allclose(y, gtpa.symbol(k2 / tau, c) * x, atol=1e-13)


@pytest.mark.parametrize("t", range(0, 7))
def test_contact_order_and_tail(t):
    """The defining properties of the family (Sec. 2.2): every derivative of g_t up to
    order t vanishes at s = 0 beyond g_t(0) = 1, i.e. (1 - g_t(s)) / s^{t+1} ->
    c_{t+1} / c_0 (exact rational arithmetic), and g_t(s) ~ c_t / (c_{t+1} s) for large s
    (the inverse-Laplacian tail; 1 / (2 s) for the default coefficients)."""
    c = [Fraction(v) for v in gtpa.default_coefficients(t)]
    for e in (6, 9, 12):
        s = Fraction(1, 10 ** e)
        ratio = (1 - gtpa.symbol(s, c)) / s ** (t + 1)
        assert abs(ratio / (c[t + 1] / c[0]) - 1) < Fraction(10, 10 ** e)
    for s in (1e6, 1e9):
        assert gtpa.symbol(s, [float(v) for v in c]) * s == pytest.approx(0.5, rel=1e-5)
    s = np.linspace(0, 100, 401)
    g = gtpa.symbol(s, [float(v) for v in c])
    assert g[0] == 1.0 and np.all(np.diff(g) < 0) and np.all(g > 0)


def test_tau_closed_forms_and_dense_rayleigh_quotient():
    """V = 0 at the shell closures N = 5 (k = 0, |k| = 1) and N = 9 (adds |k|^2 = 2): the
    exact eigenvectors are plane-wave combinations within shells, so tau = |k|^2_max / 2.
    For any block, each column's (1/2) <|k|^2> equals x^* T x / (2 kappa x^* x) with the
    dense kinetic matrix T."""
    m, L = 12, 10.0
    H = ham.dense_h((m, m), L, np.zeros(m * m), 0.0)
    _, U = np.linalg.eigh(H)
    assert gtpa.kinetic_tau(U[:, :5].T, (m, m)) == pytest.approx(0.5, abs=1e-12)
    assert gtpa.kinetic_tau(U[:, :9].T, (m, m)) == pytest.approx(1.0, abs=1e-12)
    T = ham.dense_kinetic((m, m), L)
    kappa = 2 * np.pi ** 2 / L ** 2
    X = gaussian_block(m * m, 4, seed=3) * np.array([[1.0], [2.0], [0.3], [5.0]])
    rq = [np.real(x.conj() @ T @ x) / (2 * kappa * np.real(x.conj() @ x)) for x in X]
    assert gtpa.kinetic_tau(X, (m, m)) == pytest.approx(max(rq), rel=1e-12)


@pytest.mark.parametrize("scale", [0.01, 1.0])
def test_omm_with_tpa_reaches_the_energy_in_many_more_iterations(scale):
    """Sec. 4 (Tables 1-3): with TPA / gTPA (t = 5) the preconditioned OMM converges, but
    in hundreds of iterations; the pole expansion needs about ten.  scale = 0.01 is the
    kinetic-dominated V of Test 1, scale = 1 the wells at full depth."""
    m, N, L = 12, 5, 10.0
    V = scale * wells_2d(m, L, seed=2)
    sig = ham.default_shift((m, m), L, V)
    lam, U = np.linalg.eigh(ham.dense_h((m, m), L, V, sig))
    Eref = 0.5 * lam[:N].sum()
    tau = gtpa.kinetic_tau(U[:, :N].T, (m, m))
    X0 = gaussian_block_real(m * m, N, seed=7)
    H = lambda Y: ham.apply_h_fft(Y, (m, m), L, V, sig)
    iters = {}
    for t in (3, 5):
        pc = gtpa.GtpaPreconditioner((m, m), gtpa.default_coefficients(t), tau)
        _, hist = oomm.nlcg(H, pc, X0, maxit=2000, tol=1e-13)
        iters[t] = len(hist) - 1
        assert hist[-1]["E"] == pytest.approx(Eref, rel=1e-10)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], 16)
    pp = PolePreconditioner((m, m), L, V, sig, z, w, mode="exact")
    _, hist = oomm.nlcg(H, pp, pp(X0), maxit=100, tol=1e-13)
    assert hist[-1]["E"] == pytest.approx(Eref, rel=1e-10)
    assert min(iters.values()) > 8 * (len(hist) - 1), (iters, len(hist) - 1)


def test_tau_from_the_plane_wave_box_matches_the_dense_route():
    """oracle.spectrum.kinetic_tau_kspace (eigenvectors of H(k, k') in the plane-wave box,
    used for grids too large for a dense eigh) equals kinetic_tau of the dense eigenvectors
    when the box is the whole grid, and converges as the box grows for a smooth field."""
    from oracle import spectrum
    from workloads import smooth_field_2d
    m, N, L = 12, 5, 10.0
    V = wells_2d(m, L, seed=2)
    sig = ham.default_shift((m, m), L, V)
    _, U = np.linalg.eigh(ham.dense_h((m, m), L, V, sig))
    dense = gtpa.kinetic_tau(U[:, :N].T, (m, m))
    assert spectrum.kinetic_tau_kspace((m, m), L, V, sig, N, m // 2) == pytest.approx(dense, rel=1e-10)
    m, N = 32, 12
    V = smooth_field_2d(m, seed=3)
    sig = ham.default_shift((m, m), L, V)
    _, U = np.linalg.eigh(ham.dense_h((m, m), L, V, sig))
    dense = gtpa.kinetic_tau(U[:, :N].T, (m, m))
    errs = [abs(spectrum.kinetic_tau_kspace((m, m), L, V, sig, N, kc) / dense - 1) for kc in (8, 10, 12, 14)]
    assert all(a > 10 * b for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-6, errs
