"""3D solves on the simple-cubic lattice of Gaussian wells (Sec. 4, Test 3 shape): the
sparsifying inner preconditioner (3D nested dissection, up to 16^3) and the kinetic one,
against the exact spectrum of the grid H from its Bloch sectors (64 blocks)."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import poles as opoles, spectrum
from workloads import lattice_wells_3d, gaussian_block_real

from gpu_util import to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as m
    return m


@pytest.mark.parametrize("m,L,cells,N,inner,prec", [
    (12, 20.0, 2, 8, "spp", 0),        # FP64 products of 16^3 exceed shared memory; 12^3 fits
    (16, 40.0, 4, 64, "spp", 1),
    (16, 40.0, 4, 64, "kinetic", 1),
    (32, 40.0, 4, 64, "kinetic", 1)])
def test_lattice_solve_reaches_exact_energy(omm, m, L, cells, N, inner, prec):
    """N = the s band (one state per well), separated by a gap of ~5-6."""
    P = 16
    V = lattice_wells_3d(m, L, cells=cells)
    sig = ham.default_shift((m,) * 3, L, V)
    lam = spectrum.lowest_eigs_bloch((m,) * 3, L, V, sig, cells, N + 1)
    z, w = opoles.poles_conformal(lam[0], lam[N - 1], lam[N], P)
    p = omm.default_params(precision=prec, maxit=40, tol=1e-13 if prec == 0 else 1e-10, real_orbitals=1,
                           inner=omm.OMM_INNER_SPARSIFY if inner == "spp" else omm.OMM_INNER_KINETIC)
    s = omm.Solver(3, m, L, V, N, shift=sig, params=p)
    s.set_poles(z, w)
    dt = torch.complex128 if prec == 0 else torch.complex64
    s.set_orbitals(to_dev(torch, gaussian_block_real(m ** 3, N, seed=5), dt))
    st = s.solve()
    Eref = 0.5 * lam[:N].sum()
    assert st["converged"] == 1
    assert st["energy_fp64"] == pytest.approx(Eref, rel=1e-10 if prec == 0 else 1e-8)
    s.close()
