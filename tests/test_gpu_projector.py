"""The precomputed preconditioner U U^* (Sec. 3.3, Algorithm 2) through the C ABI: built
from the same block and the same fixed GMRES schedule as the oracle, its application
matches the oracle's; a solve preconditioned by it reaches the exact energy; dropping it
restores the pole expansion exactly."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import poles as opoles
from oracle.precond import PolePreconditioner, ProjectorPreconditioner
from workloads import wells_2d, gaussian_block, gaussian_block_real

from gpu_util import to_dev, to_host, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as m
    return m


def case(m, N, L=10.0, seed=0):
    V = wells_2d(m, L, seed=seed)
    sig = ham.default_shift((m, m), L, V)
    lam = np.linalg.eigvalsh(ham.dense_h((m, m), L, V, sig))
    return V, sig, lam


@pytest.mark.parametrize("prec,extra", [(0, 0), (1, 0), (0, 1)])
def test_projector_matches_oracle(omm, prec, extra):
    """extra = 1: k = N oversampling, 2N columns, N chosen by column pivoting on both sides."""
    m, N, P = 16, 6, 8
    V, sig, lam = case(m, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    p = omm.default_params(precision=prec, gmres_m=4, gmres_cycles=2, gmres_fixed=1)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    B = gaussian_block(m * m, N * (1 + extra), seed=31)
    R = gaussian_block(m * m, N, seed=32)
    Rd = to_dev(torch, R, dt)
    Y_pole, _ = s.pole_solve(Rd)
    s.build_projector(to_dev(torch, B, dt))
    Y_proj, _ = s.pole_solve(Rd)
    pole = PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="gmres", inner="spp", gmres_m=4, cycles=2, fixed=True)
    ref = ProjectorPreconditioner(pole, to_host(to_dev(torch, B, dt)), N=N)(to_host(Rd))
    assert rel_err(to_host(Y_proj), ref) < (1e-9 if prec == 0 else 3e-4)
    s.drop_projector()
    Y_again, _ = s.pole_solve(Rd)
    assert torch.equal(Y_again, Y_pole)
    s.close()


@pytest.mark.parametrize("prec,extra", [(0, 0), (1, 0), (1, 1)])
def test_solve_with_projector_reaches_exact_energy(omm, prec, extra):
    m, N, P = 32, 16, 16
    V, sig, lam = case(m, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    p = omm.default_params(precision=prec, maxit=40, tol=1e-13 if prec == 0 else 1e-10, real_orbitals=1)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    st_b = s.build_projector(to_dev(torch, gaussian_block_real(m * m, N * (1 + extra), seed=41), dt))
    assert st_b["gmres_relres_max"] <= 1e-5
    s.set_orbitals(to_dev(torch, gaussian_block_real(m * m, N, seed=42), dt))
    st = s.solve()
    assert st["converged"] == 1
    assert st["energy_fp64"] == pytest.approx(0.5 * lam[:N].sum(), rel=1e-8)
    s.close()
