"""GPU checks at the edges of what the library accepts, and of the accuracy the bench line
claims:
  - the largest pole count (P = 32, the omm_set_poles limit) against the oracle;
  - a 128^2 handle with N = 1024 states (eight times the bench workload: 64 right-hand-side
    tiles per pole in the triangular solves, 16384 GMRES systems), sampled columns of the
    pole expansion against the oracle;
  - the FP64 check of a result (energy, Rayleigh-Ritz residual, residual of the orthonormal
    basis), computed on the device, against the same quantities written out in FP64 from
    the downloaded X;
  - the bench line's settings at full size (2D 128^2, N = 128, real orbitals, refilter at
    GMRES rtol 1e-6) meet both accuracy targets against the FP64 form of the same solve:
    energy within 1e-8 and the sine of the largest principal angle within 1e-6."""
import json
import os

import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import metrics, omm as oomm, poles as opoles
from oracle.precond import PolePreconditioner
from workloads import WORKLOADS, gaussian_block, wells_2d

from gpu_util import to_dev, to_host, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as m
    return m


def small_case(m=16, L=10.0, seed=0):
    V = wells_2d(m, L, seed=seed)
    sig = ham.default_shift((m, m), L, V)
    lam = np.linalg.eigvalsh(ham.dense_h((m, m), L, V, sig))
    return V, sig, lam


@pytest.mark.parametrize("prec", [0, 1])
def test_thirty_two_poles_match_oracle(omm, prec):
    """P = 32 conformal poles (the largest count a handle takes), sparsifying inner
    preconditioner, fixed GMRES schedule on both sides."""
    m, N, P = 16, 6, 32
    V, sig, lam = small_case(m)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    p = omm.default_params(precision=prec, gmres_m=4, gmres_cycles=2, gmres_fixed=1)
    s = omm.Solver(2, m, 10.0, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    R = gaussian_block(m * m, N, seed=21)
    Y, st = s.pole_solve(to_dev(torch, R, dt))
    ref = PolePreconditioner((m, m), 10.0, V, sig, z, w, mode="gmres", inner="spp", gmres_m=4, cycles=2,
                             fixed=True)(R)
    assert rel_err(to_host(Y), ref) < (1e-9 if prec == 0 else 5e-4)
    assert st["gmres_iters_max"] == 8
    s.close()


def test_thousand_states_on_128_grid_sampled_columns(omm):
    """N = 1024 at 128^2 (mixed, 16 poles, fixed 3-step GMRES): two sampled columns of the
    pole expansion against the oracle, which solves those columns alone."""
    wl = WORKLOADS["smooth2d-128"]
    sp = json.load(open(os.path.join(ROOT, "workloads", "spectra.json")))["smooth2d-128"]
    V = wl.potential_values()
    N = 1024
    z, w = omm.poles_fermi(sp["lam1"], sp["lamN"], sp["lamN1"], wl.P)
    prm = omm.default_params(precision=omm.OMM_MIXED, gmres_m=3, gmres_cycles=1, gmres_fixed=1)
    s = omm.Solver(2, wl.m, wl.L, V, N, shift=sp["sigma"], params=prm)
    s.set_poles(z, w)
    R = gaussian_block(wl.n, N, seed=31, dtype=np.complex64)
    Y, st = s.pole_solve(torch.from_numpy(R).to("cuda"))
    cols = (5, 1000)
    Yc = Y[list(cols)].cpu().numpy().astype(np.complex128)
    del Y
    s.close()
    zo, wo = opoles.poles_conformal(sp["lam1"], sp["lamN"], sp["lamN1"], wl.P)
    pc = PolePreconditioner(wl.shape, wl.L, V, sp["sigma"], zo, wo, mode="gmres", inner="spp", gmres_m=3,
                            cycles=1, fixed=True)
    for k, c in enumerate(cols):
        ref = pc(R[c:c + 1].astype(np.complex128))[0]
        assert rel_err(Yc[k], ref) < 5e-4, c


@pytest.mark.parametrize("prec", [0, 1])
def test_fp64_check_matches_its_definition(omm, prec):
    """After a solve on the 32^2 four-well potential, the device's FP64 check equals E_omm
    (eq. omm), ||HX - X S^-1 K||_F / ||X||_F and ||HQ - Q Q^*HQ||_F (Q = X R^-1, S = R^*R)
    evaluated in numpy FP64 from the same X."""
    m, N, P, L = 32, 16, 16, 10.0
    V, sig, lam = small_case(m, L)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    gap = lam[N] - lam[N - 1]
    p = omm.default_params(precision=prec, maxit=6, tol=0.0, gap=gap)
    s = omm.Solver(2, m, L, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    s.set_orbitals(to_dev(torch, gaussian_block(m * m, N, seed=41), dt))
    st = s.solve()
    X = to_host(s.get_orbitals())          # rows are the columns of X
    s.close()
    HX = ham.apply_h_fft(X, (m, m), L, V, sig)
    E = oomm.energy(X, HX)
    S = X.conj() @ X.T                      # S_ij = <x_i, x_j>
    K = X.conj() @ HX.T
    M = np.linalg.solve(S, K)               # S^-1 K
    Res = HX - M.T @ X                      # rows: HX - X S^-1 K
    resid = np.linalg.norm(Res) / np.linalg.norm(X)
    Rc = np.linalg.cholesky(S).conj().T     # S = Rc^* Rc, Rc upper
    Rinv = np.linalg.inv(Rc)
    resid_orth = np.linalg.norm(Rinv.T @ Res)
    assert st["energy_fp64"] == pytest.approx(E, rel=1e-12)
    assert st["resid_fp64"] == pytest.approx(resid, rel=1e-6)
    assert st["resid_orth"] == pytest.approx(resid_orth, rel=1e-6)
    assert st["angle_bound"] == pytest.approx(resid_orth / gap, rel=1e-6)


def test_bench_line_meets_both_accuracy_targets(omm):
    """2D 128^2, N = 128, 16 poles, real orbitals, one refilter at GMRES rtol 1e-6: the
    mixed solve and the FP64 form of the same solve agree to 1e-8 in energy and 1e-6 in
    the sine of the largest principal angle, and both reach the exact energy."""
    wl = WORKLOADS["smooth2d-128"]
    sp = json.load(open(os.path.join(ROOT, "workloads", "spectra.json")))["smooth2d-128"]
    V = wl.potential_values()
    z, w = omm.poles_fermi(sp["lam1"], sp["lamN"], sp["lamN1"], wl.P)
    out = {}
    for prec, tol, dt, npdt in ((omm.OMM_MIXED, 1e-10, torch.complex64, np.complex64),
                                (omm.OMM_FP64, 1e-13, torch.complex128, np.complex128)):
        prm = omm.default_params(precision=prec, maxit=40, tol=tol, real_orbitals=1, refilter=1,
                                 refilter_rtol=1e-6)
        s = omm.Solver(2, wl.m, wl.L, V, wl.N, shift=sp["sigma"], params=prm)
        s.set_poles(z, w)
        s.set_orbitals(torch.from_numpy(wl.initial_block(npdt, real=True)).to("cuda"))
        st = s.solve()
        out[prec] = (st, s.get_orbitals().cpu().numpy().astype(np.complex128))
        s.close()
    (sm, Xm), (sd, Xd) = out[omm.OMM_MIXED], out[omm.OMM_FP64]
    assert abs(sm["energy_fp64"] - sd["energy_fp64"]) / abs(sd["energy_fp64"]) <= 1e-8
    assert metrics.max_angle_sine(Xm, Xd) <= 1e-6
    for st in (sm, sd):
        assert st["converged"] == 1
        assert abs(st["energy_fp64"] - sp["E_ref"]) / abs(sp["E_ref"]) <= 1e-8


@pytest.mark.parametrize("prec", [0, 1])
def test_persistent_levels_match_per_height_launches(omm, prec):
    """omm_params.trsv_persistent = 1 (all supernode heights of all poles in one cooperative
    launch with grid barriers) gives the pole expansion of the launches per height, up to
    the summation order of the split-K products."""
    m, N, P, L = 32, 16, 16, 10.0
    V, sig, lam = small_case(m, L)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    dt = torch.complex128 if prec == 0 else torch.complex64
    R = to_dev(torch, gaussian_block(m * m, N, seed=51), dt)
    out = []
    for persistent in (0, 1):
        p = omm.default_params(precision=prec, gmres_m=4, gmres_cycles=2, gmres_fixed=1, trsv_persistent=persistent)
        s = omm.Solver(2, m, L, V, N, shift=sig, params=p)
        s.set_poles(z, w)
        Y, st = s.pole_solve(R)
        out.append(to_host(Y))
        s.close()
    assert rel_err(out[1], out[0]) < (1e-12 if prec == 0 else 2e-5)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("streams", [1, 0])
def test_overlapped_launches_match_ordinary(omm, prec, streams):
    """omm_params.launch_overlap = 1 (programmatic dependent launches in the triangular
    solves) changes only when each launch is scheduled, not its arithmetic: the pole
    expansion is bitwise that of ordinary launches, on one stream and on one per pole."""
    m, N, P, L = 32, 16, 16, 10.0
    V, sig, lam = small_case(m, L)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    dt = torch.complex128 if prec == 0 else torch.complex64
    R = to_dev(torch, gaussian_block(m * m, N, seed=61), dt)
    out = []
    for ov in (0, 1):
        p = omm.default_params(precision=prec, gmres_m=4, gmres_cycles=2, gmres_fixed=1, launch_overlap=ov,
                               trsv_streams=streams)
        s = omm.Solver(2, m, L, V, N, shift=sig, params=p)
        s.set_poles(z, w)
        Y, st = s.pole_solve(R)
        out.append(to_host(Y))
        s.close()
    assert np.array_equal(out[0], out[1])
