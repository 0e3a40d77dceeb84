"""The multifrontal factorisation of the sparsifying matrix P on the device
(csrc/k_factor.cu, omm_params.device_factor; Sec. 3.2, eq. P) against the host
factorisation (csrc/host_spp.cpp) of the same poles, through the preconditioner it
defines, P^-1 Q G b, and against the oracle's SuperLU solve.

Both factor in FP64; a mixed handle rounds the factor once to complex64 on either side,
so the two preconditioners agree to rounding: 1e-11 for FP64 handles, and for mixed ones
the complex64 rounding of the same factor (the solves' own FP32 arithmetic, applied to
factors that differ only by FP64 rounding, stays near 1e-6)."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import sparsify
from workloads import gaussian_block, lattice_wells_3d, wells_2d

from gpu_util import to_dev, to_host, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as m
    return m


# 3D 16^3 has fronts of 736 rows: the panels of the LU stay in global memory there
CASES = [(2, 16, 10.0), (2, 32, 10.0), (2, 128, 10.0), (3, 8, 20.0), (3, 12, 20.0), (3, 16, 40.0)]


def setup(omm, dim, m, L, prec, device_factor):
    V = wells_2d(m, L, seed=3) if dim == 2 else lattice_wells_3d(m, L, cells=2)
    shift = ham.default_shift((m,) * dim, L, V)
    p = omm.default_params(precision=prec, device_factor=device_factor)
    s = omm.Solver(dim, m, L, V, 4, shift=shift, params=p)
    z = np.array([-0.3 * shift + 0.7j, -0.05 * shift + 0.02j, -0.6 * shift + 2.0j])
    s.set_poles(z, np.ones(3))
    return s, V, shift, z


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim,m,L", CASES)
def test_device_factor_matches_host_factor(omm, prec, dim, m, L):
    if prec == 0 and m == 128:
        pytest.skip("FP64 at 128^2 is covered by the 32^2 and 3D cases (the host FP64 factor takes seconds)")
    if prec == 0 and dim == 3 and m == 16:
        pytest.skip("FP64 handles take the sparsifying solve up to 12^3")
    n = m ** dim
    dt = torch.complex128 if prec == 0 else torch.complex64
    B = to_dev(torch, gaussian_block(n, 3, seed=11), dt)
    out = {}
    for dev in (0, 1):
        s, V, shift, z = setup(omm, dim, m, L, prec, dev)
        out[dev] = [to_host(s.precond_apply(j, B)) for j in range(len(z))]
        out[dev, "info"] = [s.factor_info(j) for j in range(len(z))]
        s.close()
    for j in range(3):
        err = rel_err(out[1][j], out[0][j])
        assert err < (1e-11 if prec == 0 else 1e-5), (j, err)
        h, d = out[0, "info"][j], out[1, "info"][j]
        assert d["nperturbed"] == h["nperturbed"] == 0
        assert d["nsuper"] == h["nsuper"] and d["nnz"] == h["nnz"]
        assert d["pivot_ratio"] == pytest.approx(h["pivot_ratio"], rel=1e-9)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim,m,L", [(2, 32, 10.0), (3, 8, 20.0)])
def test_device_factor_preconditioner_matches_oracle(omm, prec, dim, m, L):
    """u~ = P^-1 Q (G b) with the device factor against the oracle's SuperLU of P."""
    n = m ** dim
    dt = torch.complex128 if prec == 0 else torch.complex64
    s, V, shift, z = setup(omm, dim, m, L, prec, 1)
    Bh = gaussian_block(n, 2, seed=13)
    for j, zj in enumerate(z):
        U = to_host(s.precond_apply(j, to_dev(torch, Bh, dt)))
        ref = sparsify.apply(sparsify.setup((m,) * dim, L, V, shift, zj), Bh)
        assert rel_err(U, ref) < (1e-9 if prec == 0 else 2e-4), j
    s.close()
