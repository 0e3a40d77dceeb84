"""GPU parity of the pole-expansion preconditioner (batched GMRES, Sec. 3.1 eqs. direct /
lst), of whole CG steps (Algorithm 1) and of the whole solve, against the FP64 oracle."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import metrics, omm as oomm, poles as opoles, solve as osolve
from oracle.precond import PolePreconditioner
from workloads import wells_2d, gaussian_block, WORKLOADS

from gpu_util import to_dev, to_host, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as m
    return m


def case(m=16, N=8, L=10.0, seed=0):
    V = wells_2d(m, L, seed=seed)
    sig = ham.default_shift((m, m), L, V)
    lam = np.linalg.eigvalsh(ham.dense_h((m, m), L, V, sig))
    return V, sig, lam


@pytest.mark.parametrize("inner,iname", [(0, "spp"), (1, "lap"), (2, "none")])
@pytest.mark.parametrize("prec", [0, 1])
def test_pole_solve_fixed_steps_matches_oracle(omm, inner, iname, prec):
    """Fixed GMRES schedule (every cycle m steps, no tolerance test) so that both sides do
    the same arithmetic; the result is sum_j w_j Y_j."""
    m, N, P = 16, 6, 8
    V, sig, lam = case(m, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    p = omm.default_params(precision=prec, inner=inner, gmres_m=4, gmres_cycles=2, gmres_fixed=1)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    R = gaussian_block(m * m, N, seed=11)
    Y, st = s.pole_solve(to_dev(torch, R, dt))
    pc = PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="gmres", inner=iname, gmres_m=4, cycles=2, fixed=True)
    ref = pc(R)
    err = rel_err(to_host(Y), ref)
    assert err < (1e-9 if prec == 0 else 5e-4), err
    assert st["gmres_iters_max"] == 8


def test_pole_solve_with_tolerance_converges(omm):
    """Paper schedule (rtol 1e-5, restart 15, 5 cycles): every system meets the tolerance
    and the result is close to the exactly solved filter applied to R."""
    m, N, P = 32, 16, 16
    V, sig, lam = case(m, N, seed=0)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=omm.default_params())
    s.set_poles(z, w)
    R = gaussian_block(m * m, N, seed=12)
    Y, st = s.pole_solve(to_dev(torch, R, torch.complex128))
    assert st["gmres_relres_max"] <= 1e-5
    exact = PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="exact")(R)
    assert rel_err(to_host(Y), exact) < 1e-3


@pytest.mark.parametrize("prec", [0, 1])
def test_cg_steps_match_oracle(omm, prec):
    """Two steps of Algorithm 1 (PR beta, exact quartic line search) from the same X, with
    the same fixed GMRES schedule on both sides."""
    m, N, P = 16, 6, 8
    V, sig, lam = case(m, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    p = omm.default_params(precision=prec, gmres_m=4, gmres_cycles=1, gmres_fixed=1)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    X0 = gaussian_block(m * m, N, seed=13)
    Xd = to_dev(torch, X0, dt)
    s.set_orbitals(Xd)
    st = s.iterate(2)
    Xg = to_host(s.get_orbitals())
    pc = PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="gmres", inner="spp", gmres_m=4, cycles=1, fixed=True)
    Xr, hist = oomm.nlcg(lambda Y: ham.apply_h_fft(Y, (m, m), 10.0, V, sig), pc, to_host(Xd), maxit=2, tol=0.0)
    err = rel_err(Xg, Xr)
    assert err < (1e-8 if prec == 0 else 1e-3), err
    assert st["energy"] == pytest.approx(hist[-1]["E"], rel=1e-10 if prec == 0 else 1e-5)


def reference_solution(m, N, L=10.0, seed=0):
    V, sig, lam = case(m, N, L, seed)
    _, U, _ = osolve.reference_eigs((m, m), L, V, sig, N)
    return V, sig, lam, U


@pytest.mark.parametrize("prec", [0, 1])
def test_small_solve_reaches_eigenspace(omm, prec):
    """filter + CG (+1 refilter) on the 32^2 / N = 16 well potential with 16 conformal
    poles from the exact spectrum: E_omm -> 1/2 sum lam_i, subspace -> eigh subspace."""
    m, N, P = 32, 16, 16
    V, sig, lam, U = reference_solution(m, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    p = omm.default_params(precision=prec, maxit=40, tol=1e-13 if prec == 0 else 1e-10, refilter=1)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    s.set_orbitals(to_dev(torch, gaussian_block(m * m, N, seed=1000), dt))
    st = s.solve()
    X = to_host(s.get_orbitals())
    Eref = 0.5 * lam[:N].sum()
    assert st["energy_fp64"] == pytest.approx(Eref, rel=1e-10 if prec == 0 else 1e-8)
    assert metrics.max_angle_sine(X, U) < (1e-5 if prec == 0 else 2e-5)
    assert st["resid_fp64"] < 1e-4
