"""Degenerate and ragged cases through the C ABI: a single state; a constant potential, for
which the sparsifying preconditioner is exact (P = Q, Sec. 3.2) and GMRES stops after one
step; a column count that leaves partial tiles in every kernel; the free particle at a
shell closure, whose energy is a closed form."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import poles as opoles
from oracle.precond import PolePreconditioner
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


def spectrum(m, V, L=10.0):
    sig = ham.default_shift((m, m), L, V)
    return sig, np.linalg.eigvalsh(ham.dense_h((m, m), L, V, sig))


@pytest.mark.parametrize("prec", [0, 1])
def test_single_state(omm, prec):
    m, N = 16, 1
    V = wells_2d(m, 10.0, seed=3)
    sig, lam = spectrum(m, V)
    gap = lam[1] - lam[0]
    z, w = opoles.poles_conformal(lam[0] - 0.01 * gap, lam[0], lam[1], 16)   # a one-point occupied interval, widened
    p = omm.default_params(precision=prec, maxit=40, tol=1e-13 if prec == 0 else 1e-10, real_orbitals=1)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    s.set_orbitals(to_dev(torch, gaussian_block_real(m * m, N, seed=9), dt))
    st = s.solve()
    assert st["energy_fp64"] == pytest.approx(0.5 * lam[0], rel=1e-10 if prec == 0 else 1e-8)
    s.close()


def test_constant_potential_makes_the_sparsifier_exact(omm):
    """V = const: P = Q and P^-1 Q G = G = (H - sigma - z)^-1 exactly, so every system
    meets the tolerance after one GMRES step and the pole sum equals the exact one."""
    m, N = 16, 5                      # the k = 0 and |k| = 1 shells
    V = np.full(m * m, -2.0)
    sig, lam = spectrum(m, V)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], 8)
    p = omm.default_params(precision=0, gmres_rtol=1e-10)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    R = gaussian_block(m * m, N, seed=10)
    Y, st = s.pole_solve(to_dev(torch, R, torch.complex128))
    assert st["gmres_iters_max"] == 1
    exact = PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="exact")(R)
    assert rel_err(to_host(Y), exact) < 1e-9
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_column_count(omm, prec):
    """N = 70 systems per pole: partial tiles in the leaf CTAs (128 columns), the product
    tiles (32 and 16 columns) and the assembly tiles (32 systems)."""
    m, N, P = 16, 70, 4
    V = wells_2d(m, 10.0, seed=4)
    sig, lam = spectrum(m, V)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    p = omm.default_params(precision=prec, gmres_m=3, gmres_cycles=1, gmres_fixed=1)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    R = gaussian_block(m * m, N, seed=11)
    Rd = to_dev(torch, R, dt)
    Y, st = s.pole_solve(Rd)
    ref = PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="gmres", inner="spp", gmres_m=3, cycles=1,
                             fixed=True)(to_host(Rd))
    assert rel_err(to_host(Y), ref) < (1e-9 if prec == 0 else 5e-4)
    s.close()


def test_free_particle_shell_closure(omm):
    """V = 0: the spectrum is (2 pi^2 / L^2)|k|^2 - sigma with the shell degeneracies of the
    square lattice; N = 5 closes the k = 0 and |k| = 1 shells, and the solve reaches the
    closed-form energy 1/2 sum."""
    m, N, L = 16, 5, 10.0
    V = np.zeros(m * m)
    sig = ham.default_shift((m, m), L, V)
    c = 2 * np.pi ** 2 / L ** 2
    shells = [0.0] + [c] * 4 + [2 * c] * 4
    lam = np.array(shells) - sig
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], 16)
    p = omm.default_params(precision=0, maxit=40, tol=1e-13, real_orbitals=1)
    s = omm.Solver(2, m, L, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    s.set_orbitals(to_dev(torch, gaussian_block_real(m * m, N, seed=12), torch.complex128))
    st = s.solve()
    assert st["energy_fp64"] == pytest.approx(0.5 * lam[:N].sum(), rel=1e-11)
    s.close()
