"""Pins for oracle.omm: eq. omm, the gradient of Sec. 2.1, the Hessian of Sec. 2.3, the
quartic line search and Algorithm 1."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import omm
from workloads import wells_2d, gaussian_block

SHAPE, L = (12, 12), 10.0
N = 6


@pytest.fixture(scope="module")
def system():
    V = wells_2d(12, L, seed=4)
    sig = ham.default_shift(SHAPE, L, V)
    H = ham.dense_h(SHAPE, L, V, sig)
    lam, U = np.linalg.eigh(H)
    return dict(V=V, sig=sig, H=H, lam=lam, U=U)


def happ(H, X):
    return (H @ X.T).T


def test_energy_and_gradient_at_eigenvectors(system):
    """E_omm(U_N) = 1/2 sum lam_i and G(U_N) = 0 (eq. tracemin / eq. omm at X^*X = I);
    both invariant under a unitary mixing U_N Q."""
    H, lam, U = system["H"], system["lam"], system["U"]
    X = U[:, :N].T
    Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((N, N))
                        + 1j * np.random.default_rng(1).standard_normal((N, N)))
    for Xc in (X, Q.T @ X):
        HX = happ(H, Xc)
        assert omm.energy(Xc, HX) == pytest.approx(0.5 * lam[:N].sum(), rel=1e-13)
        assert np.max(np.abs(omm.gradient(Xc, HX))) < 1e-10 * abs(lam).max()


def test_omm_minimum_is_trace_minimum(system):
    """For H < 0 the minimum of E_omm is 1/2 sum of the N lowest eigenvalues: random
    points never go below it (Sec. 1, the Mauri-Galli-Car property)."""
    H, lam = system["H"], system["lam"]
    Emin = 0.5 * lam[:N].sum()
    rng = np.random.default_rng(7)
    for _ in range(20):
        X = gaussian_block(144, N, seed=int(rng.integers(1 << 30))) * rng.uniform(0.2, 3.0)
        assert omm.energy(X, happ(H, X)) >= Emin - 1e-9 * abs(Emin)


def test_gradient_by_central_differences(system):
    """dE/dt along D equals Re tr(D^* G) (G = 2 dE/dX-bar), checked by central differences."""
    H = system["H"]
    X = gaussian_block(144, N, seed=11)
    D = gaussian_block(144, N, seed=12)
    G = omm.gradient(X, happ(H, X))
    h = 1e-5
    fd = (omm.energy(X + h * D, happ(H, X + h * D)) - omm.energy(X - h * D, happ(H, X - h * D))) / (2 * h)
    assert fd == pytest.approx(np.real(np.vdot(D, G)), rel=1e-7)


def test_hessian_by_central_differences(system):
    H = system["H"]
    X = gaussian_block(144, N, seed=13)
    Z = gaussian_block(144, N, seed=14)
    h = 1e-4
    Gp = omm.gradient(X + h * Z, happ(H, X + h * Z))
    Gm = omm.gradient(X - h * Z, happ(H, X - h * Z))
    fd = (Gp - Gm) / (2 * h)
    an = omm.hessian_apply(X, happ(H, X), Z, happ(H, Z))
    np.testing.assert_allclose(fd, an, atol=1e-6 * np.max(np.abs(an)))


def test_hessian_at_minimizer_reduces_to_HZ_minus_Z_Lambda(system):
    """Sec. 2.3: at X_0 (X_0^*X_0 = I, H X_0 = X_0 Lam_0) and Z^*X_0 = 0, H(X_0) Z = HZ - Z Lam_0;
    its eigenvalues on that space are lam_j - lam_i (j > N >= i), so the condition
    number equals (lam_n - lam_1)/(lam_{N+1} - lam_N) exactly."""
    H, lam, U = system["H"], system["lam"], system["U"]
    X0 = U[:, :N].T
    Z = gaussian_block(144, N, seed=15)
    Z = Z - (Z.conj() @ X0.T).conj() @ X0                # remove the X0 components
    assert np.max(np.abs(omm.gram(Z, X0))) < 1e-13
    an = omm.hessian_apply(X0, happ(H, X0), Z, happ(H, Z))
    ref = happ(H, Z) - lam[:N, None] * Z
    np.testing.assert_allclose(an, ref, atol=1e-10 * np.max(np.abs(ref)))
    # the reduced Hessian on the orthogonal complement, built column by column
    Uc = U[:, N:]
    blocks = []
    for i in range(N):
        blocks.append(np.diag(lam[N:] - lam[i]))
    ev = np.concatenate([np.diag(b) for b in blocks])
    assert ev.max() / ev.min() == pytest.approx((lam[-1] - lam[0]) / (lam[N] - lam[N - 1]), rel=1e-12)
    assert Uc.shape[1] == 144 - N


def test_quartic_reproduces_energy(system):
    H = system["H"]
    X = gaussian_block(144, N, seed=21)
    D = gaussian_block(144, N, seed=22)
    HX, HD = happ(H, X), happ(H, D)
    c = omm.quartic_coefficients(X, HX, D, HD)
    for t in (-1.3, -0.2, 0.0, 0.37, 2.0):
        Xt = X + t * D
        assert omm.quartic_value(c, t) == pytest.approx(omm.energy(Xt, happ(H, Xt)), rel=1e-12, abs=1e-9)
    assert c[1] == pytest.approx(np.real(np.vdot(D, omm.gradient(X, HX))), rel=1e-10)
    assert c[4] > 0.0


def test_line_search_is_global_minimum_on_a_grid(system):
    H = system["H"]
    rng = np.random.default_rng(3)
    for s in range(5):
        X = gaussian_block(144, N, seed=30 + s)
        D = gaussian_block(144, N, seed=40 + s) * rng.uniform(0.1, 2.0)
        c = omm.quartic_coefficients(X, happ(H, X), D, happ(H, D))
        t = omm.line_search(c)
        grid = np.linspace(-5, 5, 200001)
        assert omm.quartic_value(c, t) <= np.min(omm.quartic_value(c, grid)) + 1e-9 * abs(c[0])
        assert abs(4 * c[4] * t ** 3 + 3 * c[3] * t ** 2 + 2 * c[2] * t + c[1]) < 1e-8 * np.max(np.abs(c))


def test_line_search_rejects_indefinite_quartic():
    with pytest.raises(ValueError):
        omm.line_search([0.0, 1.0, 1.0, 0.0, -1.0])


def test_nlcg_energy_is_monotone_and_converges(system):
    """Algorithm 1 with the exact projector (dense) as preconditioner: the energy never
    increases and reaches 1/2 sum lam_i."""
    H, lam, U = system["H"], system["lam"], system["U"]
    Pi = U[:, :N] @ U[:, :N].conj().T
    X1 = (Pi @ gaussian_block(144, N, seed=50).T).T
    X, hist = omm.nlcg(lambda Y: happ(H, Y), lambda R: (Pi @ R.T).T, X1, maxit=60, tol=1e-15)
    E = [h["E"] for h in hist]
    scale = abs(E[-1])
    assert all(E[i + 1] <= E[i] + 1e-12 * scale for i in range(len(E) - 1))
    assert E[-1] == pytest.approx(0.5 * lam[:N].sum(), rel=1e-12)
