"""Full-size checks in the launch configuration bench.py times (2D 128^2, N = 128, 16
conformal poles, mixed precision): sampled columns of the pole-expansion preconditioner
against the oracle (every column is an independent set of P shifted systems, so the
oracle computes just those), and the whole solve against the exact energy stored by
workloads/make_spectra.py (1/2 sum of the lowest N eigenvalues, eq. tracemin)."""
import json
import os

import numpy as np
import pytest

from oracle import poles as opoles
from oracle.precond import PolePreconditioner
from workloads import WORKLOADS

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as omm
    wl = WORKLOADS["smooth2d-128"]
    sp = json.load(open(os.path.join(ROOT, "workloads", "spectra.json")))["smooth2d-128"]
    return omm, wl, sp, wl.potential_values()


@pytest.mark.parametrize("gm", [3, 15])
def test_full_size_pole_solve_sampled_columns(setup, gm):
    """gm = 15 runs a whole restart cycle: every basis size from 1 to 15 vectors through the
    CGS2 kernels at the full grid size."""
    omm, wl, sp, V = setup
    z, w = omm.poles_fermi(sp["lam1"], sp["lamN"], sp["lamN1"], wl.P)
    prm = omm.default_params(precision=omm.OMM_MIXED, gmres_m=gm, gmres_cycles=1, gmres_fixed=1)
    s = omm.Solver(2, wl.m, wl.L, V, wl.N, shift=sp["sigma"], params=prm)
    s.set_poles(z, w)
    R = wl.initial_block(np.complex64)
    Y, st = s.pole_solve(torch.from_numpy(R).to("cuda"))
    Y = Y.cpu().numpy().astype(np.complex128)
    zo, wo = opoles.poles_conformal(sp["lam1"], sp["lamN"], sp["lamN1"], wl.P)
    pc = PolePreconditioner(wl.shape, wl.L, V, sp["sigma"], zo, wo, mode="gmres", inner="spp", gmres_m=gm,
                            cycles=1, fixed=True)
    for c in (0, 77):
        ref = pc(R[c:c + 1].astype(np.complex128))[0]
        err = np.max(np.abs(Y[c] - ref)) / np.max(np.abs(ref))
        assert err < 5e-4, (c, err)
    s.close()


def test_full_size_solve_reaches_exact_energy(setup):
    omm, wl, sp, V = setup
    z, w = omm.poles_fermi(sp["lam1"], sp["lamN"], sp["lamN1"], wl.P)
    prm = omm.default_params(precision=omm.OMM_MIXED, maxit=40, tol=1e-10)
    s = omm.Solver(2, wl.m, wl.L, V, wl.N, shift=sp["sigma"], params=prm)
    s.set_poles(z, w)
    s.set_orbitals(torch.from_numpy(wl.initial_block(np.complex64)).to("cuda"))
    st = s.solve()
    assert st["converged"] == 1
    assert abs(st["energy_fp64"] - sp["E_ref"]) / abs(sp["E_ref"]) < 1e-8
    assert st["gmres_relres_max"] <= 1e-5
    s.close()
