"""Pins for oracle.precond.ProjectorPreconditioner (Sec. 3.3, Algorithm 2): the basis is
orthonormal and spans the filtered block, U U^* is an orthogonal projector, with exact
pole solves it approaches the spectral projector of the N lowest eigenvectors as the pole
rule sharpens, and the OMM preconditioned by it reaches the exact energy."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import omm as oomm, poles as opoles
from oracle.precond import PolePreconditioner, ProjectorPreconditioner
from workloads import wells_2d, gaussian_block_real


def case(m=12, N=5, L=10.0, seed=2):
    V = wells_2d(m, L, seed=seed)
    sig = ham.default_shift((m, m), L, V)
    H = ham.dense_h((m, m), L, V, sig)
    lam, Uev = np.linalg.eigh(H)
    return V, sig, H, lam, Uev


def test_basis_is_orthonormal_and_spans_the_filtered_block():
    m, N = 12, 5
    V, sig, H, lam, _ = case(m, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], 16)
    pole = PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="exact")
    B = gaussian_block_real(m * m, N, seed=3)
    pc = ProjectorPreconditioner(pole, B)
    U = pc.U
    np.testing.assert_allclose(U @ U.conj().T, np.eye(N), atol=1e-12)
    Y = pole(B)
    np.testing.assert_allclose(pc(Y), Y, atol=1e-11 * np.max(np.abs(Y)))      # U U^* Y = Y
    R = np.random.default_rng(5).standard_normal((3, m * m))
    np.testing.assert_allclose(pc(pc(R)), pc(R), atol=1e-12 * np.max(np.abs(R)))   # idempotent


def test_exact_poles_give_the_spectral_projector():
    """With exact pole solves the filtered block spans r(H) B; as P grows r -> the step and
    U U^* -> the projector onto the N lowest eigenvectors."""
    m, N = 12, 5
    V, sig, H, lam, Uev = case(m, N)
    Pi = Uev[:, :N] @ Uev[:, :N].conj().T
    B = gaussian_block_real(m * m, N, seed=4)
    errs = []
    for P in (8, 16, 24):
        z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
        pc = ProjectorPreconditioner(PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="exact"), B)
        Pu = pc.U.T @ pc.U.conj()                               # columns: U U^*
        errs.append(np.linalg.norm(Pu - Pi, 2))
    assert errs[0] > errs[1] > errs[2]
    assert errs[-1] < 1e-6
    # a planted mistake (keeping N - 1 columns) is far from the projector
    Ubad = pc.U[:-1]
    assert np.linalg.norm(Ubad.T @ Ubad.conj() - Pi, 2) > 0.5


def test_omm_with_the_projector_reaches_the_exact_energy():
    m, N = 12, 5
    V, sig, H, lam, Uev = case(m, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], 24)
    pc = ProjectorPreconditioner(PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="exact"),
                                 gaussian_block_real(m * m, N, seed=6))
    X0 = pc(gaussian_block_real(m * m, N, seed=7))
    X, hist = oomm.nlcg(lambda Y: ham.apply_h_fft(Y, (m, m), 10.0, V, sig), pc, X0, maxit=60, tol=1e-14)
    Eref = 0.5 * lam[:N].sum()
    assert hist[-1]["E"] == pytest.approx(Eref, rel=1e-10)


def test_oversampling_is_no_worse_with_noisy_pole_solves():
    """k = N extra columns and the column-pivoted choice of N of them: with GMRES pole
    solves at a loose tolerance (errors ~1e-4) the basis stays as close to the spectral
    projector as with k = 0 or closer (the chosen columns are well conditioned)."""
    m, N, L = 16, 12, 10.0
    V = wells_2d(m, L, seed=2)
    sig = ham.default_shift((m, m), L, V)
    lam, Uev = np.linalg.eigh(ham.dense_h((m, m), L, V, sig))
    Pi = Uev[:, :N] @ Uev[:, :N].conj().T
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], 16)
    pole = PolePreconditioner((m, m), L, V, sig, z, w, mode="gmres", inner="spp", rtol=1e-4)
    for seed in (3, 4, 5):
        err = {}
        for k in (0, N):
            pc = ProjectorPreconditioner(pole, gaussian_block_real(m * m, N + k, seed=seed), N=N)
            assert pc.U.shape[0] == N
            err[k] = np.linalg.norm(pc.U.T @ pc.U.conj() - Pi, 2)
        assert err[N] <= err[0] * 1.01 and err[N] < 2e-4, (seed, err)
