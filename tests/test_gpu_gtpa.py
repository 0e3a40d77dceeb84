"""The Fourier-diagonal comparison preconditioners (Sec. 2.2, eqs. Lap, TPA, gTPA) through
the C ABI against oracle.gtpa: one application on the fused (one CTA per grid function)
and the multi-pass FFT paths, FP64 and complex64, default and caller coefficients; the
first iterations of OMM with TPA against the oracle's Algorithm 1 step by step; a whole
TPA solve reaching the exact energy in many times the pole expansion's iterations
(Tables 1-3); argument checks."""
import numpy as np
import pytest

from oracle import gtpa as ogtpa, hamiltonian as ham, omm as oomm, poles as opoles
from workloads import gaussian_block, gaussian_block_real, wells_2d

from gpu_util import FP32_RTOL, FP64_RTOL, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as m
    return m


@pytest.mark.parametrize("dim,m,N,prec,t,coeffs", [
    (2, 16, 6, 0, 3, None),             # fused kernel, eq. TPA
    (2, 16, 6, 1, 5, None),             # fused kernel, complex64, gTPA t = 5
    (2, 16, 3, 0, 0, [1.0, 1.0]),       # eq. Lap from caller coefficients
    (3, 12, 4, 0, 5, None),             # fused 3D
    (2, 128, 3, 0, 3, None),            # multi-pass FFT (FP64 128^2 exceeds one CTA)
    (2, 128, 5, 1, 4, [2.0, 0.5, 1.0, 0.0, 3.0, 7.0])])   # complex64 128^2, a zero coefficient
def test_one_application(omm, dim, m, N, prec, t, coeffs):
    shape, L = (m,) * dim, 10.0
    n = m ** dim
    V = np.zeros(n)
    sig = ham.default_shift(shape, L, V)
    s = omm.Solver(dim, m, L, V, N, shift=sig, params=omm.default_params(precision=prec))
    tau = 1.7
    s.set_gtpa(t, tau, coeffs)
    dt = torch.complex128 if prec == 0 else torch.complex64
    R = to_dev(torch, gaussian_block(n, N, seed=21), dt)
    Y, st = s.pole_solve(R)
    c = coeffs if coeffs is not None else ogtpa.default_coefficients(t)
    ref = ogtpa.GtpaPreconditioner(shape, c, tau)(to_host(R))
    assert rel_err(to_host(Y), ref) < (FP64_RTOL if prec == 0 else FP32_RTOL)
    assert st["gmres_iters_max"] == 0
    s.close()


def small_case(m=16, N=5, L=10.0, scale=1.0):
    V = scale * wells_2d(m, L, seed=2)
    sig = ham.default_shift((m, m), L, V)
    lam, U = np.linalg.eigh(ham.dense_h((m, m), L, V, sig))
    tau = ogtpa.kinetic_tau(U[:, :N].T, (m, m))
    return V, sig, lam, tau


def test_iterations_follow_the_oracle(omm):
    """1, 4 and 10 steps of Algorithm 1 with TPA from the same real start: the energy
    after them matches the oracle's (FP64)."""
    m, N, L = 16, 5, 10.0
    V, sig, lam, tau = small_case(m, N, L)
    X0 = gaussian_block_real(m * m, N, seed=7)
    c = ogtpa.default_coefficients(3)
    _, hist = oomm.nlcg(lambda Y: ham.apply_h_fft(Y, (m, m), L, V, sig), ogtpa.GtpaPreconditioner((m, m), c, tau),
                        X0, maxit=10, tol=0.0)
    s = omm.Solver(2, m, L, V, N, shift=sig, params=omm.default_params(precision=0, real_orbitals=1, tol=0.0))
    s.set_gtpa(3, tau)
    s.set_orbitals(to_dev(torch, X0, torch.complex128))
    for k in (1, 4, 10):
        if k > 1:
            s.set_orbitals(to_dev(torch, X0, torch.complex128))
        st = s.iterate(k)
        assert st["energy"] == pytest.approx(hist[k]["E"], rel=1e-10), k
    s.close()


@pytest.mark.parametrize("scale", [0.01, 1.0])
def test_tpa_solve_reaches_the_energy_in_many_more_iterations(omm, scale):
    """Sec. 4: OMM with TPA converges to the exact energy, in many times the iterations
    of the pole expansion (which here runs on the same handle after omm_drop_gtpa).  The
    full-depth wells leave a gap of 0.012 in a spread of 30, so one filter with 16 poles
    leaves leakage that stalls the pole-expansion CG at E error 4.3e-9 (the oracle stops at
    the same value, exact pole solves included); one refilter round removes it.  The gTPA
    solve does not filter, so the refilter setting does not touch it."""
    m, N, L = 16, 5, 10.0
    V, sig, lam, tau = small_case(m, N, L, scale)
    Eref = 0.5 * lam[:N].sum()
    X0 = to_dev(torch, gaussian_block_real(m * m, N, seed=7), torch.complex128)
    p = omm.default_params(precision=0, maxit=3000, tol=1e-13, real_orbitals=1, refilter=1)
    s = omm.Solver(2, m, L, V, N, shift=sig, params=p)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], 16)
    s.set_poles(z, w)
    s.set_gtpa(3, tau)
    s.set_orbitals(X0)
    st_tpa = s.solve()
    assert st_tpa["converged"] == 1 and st_tpa["filters"] == 0
    assert st_tpa["energy_fp64"] == pytest.approx(Eref, rel=1e-10)
    s.drop_gtpa()
    s.set_orbitals(X0)
    st_pole = s.solve()
    assert st_pole["converged"] == 1 and st_pole["filters"] == 2
    assert st_pole["energy_fp64"] == pytest.approx(Eref, rel=1e-10)
    assert st_tpa["iters"] > 8 * st_pole["iters"], (st_tpa["iters"], st_pole["iters"])
    s.close()


def test_argument_checks(omm):
    m, N = 16, 3
    V = np.zeros(m * m)
    s = omm.Solver(2, m, 10.0, V, N, shift=ham.default_shift((m, m), 10.0, V), params=omm.default_params())
    for t, tau, c in [(-1, 1.0, None), (17, 1.0, None), (3, 0.0, None), (3, float("nan"), None),
                      (1, 1.0, [1.0, -1.0, 1.0]), (1, 1.0, [0.0, 1.0, 1.0]), (1, 1.0, [1.0, 1.0, 0.0])]:
        with pytest.raises(omm.OmmError) as e:
            s.set_gtpa(t, tau, c)
        assert e.value.status == omm.OMM_EINVAL
    s.set_gtpa(3, 1.0)
    with pytest.raises(omm.OmmError) as e:       # no poles: nothing to filter with
        s.filter()
    assert e.value.status == omm.OMM_ESTATE
    s.close()
