"""Real orbitals with conjugate-pair folding (omm_params.real_orbitals).

H - sigma is real symmetric and the pole rules come in conjugate pairs, so for a real
block the pole sum of Sec. 3.1 equals 2 Re of the sum over one pole of each pair.  The
folded handle must give the same filtered block and the same CG iterates as the handle
that solves every pole, keep X exactly real, and reach the exact energy; a pole set
without conjugate partners is refused."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import metrics, poles as opoles, solve as osolve
from workloads import wells_2d, gaussian_block

from gpu_util import to_dev, to_host, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as m
    return m


def case(m=32, N=16, L=10.0, seed=0):
    V = wells_2d(m, L, seed=seed)
    sig = ham.default_shift((m, m), L, V)
    lam = np.linalg.eigvalsh(ham.dense_h((m, m), L, V, sig))
    return V, sig, lam


def real_block(n, N, seed):
    return np.ascontiguousarray(gaussian_block(n, N, seed=seed).real * np.sqrt(2.0))


@pytest.mark.parametrize("prec", [0, 1])
def test_folded_filter_and_steps_match_full_pole_sum(omm, prec):
    m, N, P = 16, 6, 16
    V, sig, lam = case(m, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    dt = torch.complex128 if prec == 0 else torch.complex64
    X0 = real_block(m * m, N, seed=21)
    out = {}
    for real in (0, 1):
        p = omm.default_params(precision=prec, gmres_m=4, gmres_cycles=2, gmres_fixed=1, real_orbitals=real)
        s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
        s.set_poles(z, w)
        s.set_orbitals(to_dev(torch, X0, dt))
        s.filter()
        Xf = to_host(s.get_orbitals())
        st = s.iterate(2)
        out[real] = (Xf, to_host(s.get_orbitals()), st)
        s.close()
    tol = 1e-11 if prec == 0 else 2e-5
    # the full sum of a real right-hand side is real up to rounding
    assert np.max(np.abs(out[0][0].imag)) <= tol * np.max(np.abs(out[0][0]))
    assert rel_err(out[1][0], out[0][0].real) < tol
    assert np.all(out[1][0].imag == 0) and np.all(out[1][1].imag == 0)
    assert rel_err(out[1][1], out[0][1].real) < (1e-9 if prec == 0 else 1e-3)
    assert out[1][2]["energy"] == pytest.approx(out[0][2]["energy"], rel=1e-11 if prec == 0 else 1e-5)


@pytest.mark.parametrize("prec", [0, 1])
def test_folded_solve_reaches_eigenspace(omm, prec):
    m, N, P = 32, 16, 16
    V, sig, lam = case(m, N)
    _, U, _ = osolve.reference_eigs((m, m), 10.0, V, sig, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    p = omm.default_params(precision=prec, maxit=40, tol=1e-13 if prec == 0 else 1e-10, refilter=1,
                           real_orbitals=1)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    s.set_orbitals(to_dev(torch, real_block(m * m, N, seed=1000), dt))
    st = s.solve()
    X = to_host(s.get_orbitals())
    assert np.all(X.imag == 0)
    assert st["energy_fp64"] == pytest.approx(0.5 * lam[:N].sum(), rel=1e-10 if prec == 0 else 1e-8)
    assert metrics.max_angle_sine(X, U) < (1e-5 if prec == 0 else 2e-5)


def test_unpaired_poles_are_refused(omm):
    m, N = 16, 4
    V, sig, lam = case(m, N)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], 8)
    keep = z.imag > 0                      # one pole of each pair only
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=omm.default_params(real_orbitals=1))
    with pytest.raises(omm.OmmError) as e:
        s.set_poles(z[keep], w[keep])
    assert e.value.status == omm.OMM_EINVAL
    s.set_poles(z, w)                      # the complete rule is accepted
