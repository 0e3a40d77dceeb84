"""GPU parity of the hot-path building blocks, called through the C ABI, against the FP64
oracle on the same seeded inputs: the pseudospectral H-apply (Sec. 4 eq. ex1mat), the
Grams (eq. omm), the gradient (Sec. 2.1), the quartic line search, and the sparsifying
preconditioner (Sec. 3.2)."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import omm as oomm
from oracle import sparsify
from workloads import wells_2d, smooth_field_2d, lattice_wells_3d, gaussian_block

from gpu_util import FP64_RTOL, FP32_RTOL, to_dev, to_host, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_09724_gb300 as m
    return m


def potential(dim, m, L, seed=0):
    if dim == 3:
        return lattice_wells_3d(m, L)
    return wells_2d(m, L, seed=seed) if m <= 64 else smooth_field_2d(m, L, seed=seed)


def make(omm, dim, m, L, N, prec, **kw):
    V = potential(dim, m, L)
    p = omm.default_params(precision=prec, **kw)
    s = omm.Solver(dim, m, L, V, N, params=p)
    return s, V


GRIDS = [(2, 8, 5.0), (2, 12, 5.0), (2, 16, 10.0), (2, 32, 10.0), (2, 48, 10.0), (2, 96, 10.0), (2, 128, 10.0),
         (3, 6, 40.0), (3, 8, 40.0), (3, 16, 40.0), (3, 32, 40.0), (3, 48, 40.0)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim,m,L", GRIDS)
def test_apply_h_matches_oracle(omm, dim, m, L, prec):
    n = m ** dim
    ncols = 3 if n > 20000 else 5
    s, V = make(omm, dim, m, L, 2, prec)
    dt = torch.complex128 if prec == 0 else torch.complex64
    X = gaussian_block(n, ncols, seed=m + dim)
    for shift in (0.0, 0.37 - 1.25j):
        Y = to_host(s.apply_h(to_dev(torch, X, dt), shift))
        ref = ham.apply_h_fft(X, (m,) * dim, L, V, s.shift + shift)
        err = rel_err(Y, ref)
        assert err < (FP64_RTOL if prec == 0 else FP32_RTOL), (dim, m, prec, err)


@pytest.mark.parametrize("prec,tensor", [(0, 0), (1, 0), (1, 1)])
@pytest.mark.parametrize("na,nb,n", [(3, 5, 256), (16, 64, 1024), (40, 33, 4096), (128, 512, 16384)])
def test_gram_matches_definition(omm, prec, tensor, na, nb, n):
    """CUDA-core Gram (FP32 products, FP64 sums) and the tcgen05 Gram (TF32 x 3 split with
    FP32 accumulation in tensor memory, FP64 split-K sum), against A^H B in FP64."""
    m = int(round(np.sqrt(n)))
    s, _ = make(omm, 2, m, 10.0, 2, prec, gram_tensor=tensor)
    dt = torch.complex128 if prec == 0 else torch.complex64
    A = gaussian_block(n, na, seed=1)
    B = gaussian_block(n, nb, seed=2)
    Ad, Bd = to_dev(torch, A, dt), to_dev(torch, B, dt)
    Cg = s.gram(Ad, Bd).cpu().numpy()
    # reference from the rounded inputs the device actually saw
    Ar, Br = to_host(Ad), to_host(Bd)
    ref = Ar.conj() @ Br.T
    err = rel_err(Cg, ref)
    assert err < (1e-13 if prec == 0 else (3e-5 if tensor else 2e-6)), err


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("m,N", [(16, 8), (32, 16), (64, 40)])
def test_gradient_matches_oracle(omm, prec, m, N):
    n = m * m
    s, V = make(omm, 2, m, 10.0, N, prec)
    dt = torch.complex128 if prec == 0 else torch.complex64
    X = gaussian_block(n, N, seed=3)
    Xd = to_dev(torch, X, dt)
    HX, G = s.gradient(Xd)
    Xr = to_host(Xd)
    HXr = ham.apply_h_fft(Xr, (m, m), 10.0, V, s.shift)
    Gr = oomm.gradient(Xr, HXr)
    assert rel_err(to_host(HX), HXr) < (FP64_RTOL if prec == 0 else FP32_RTOL)
    assert rel_err(to_host(G), Gr) < (1e-10 if prec == 0 else 2e-5)


@pytest.mark.parametrize("prec", [0, 1])
def test_quartic_and_line_search_match_oracle(omm, prec):
    m, N = 32, 16
    n = m * m
    s, V = make(omm, 2, m, 10.0, N, prec)
    dt = torch.complex128 if prec == 0 else torch.complex64
    Xd = to_dev(torch, gaussian_block(n, N, seed=4), dt)
    Dd = to_dev(torch, 0.3 * gaussian_block(n, N, seed=5), dt)
    c, t = s.quartic(Xd, Dd)
    X, D = to_host(Xd), to_host(Dd)
    H = lambda Y: ham.apply_h_fft(Y, (m, m), 10.0, V, s.shift)
    cr = oomm.quartic_coefficients(X, H(X), D, H(D))
    tr = oomm.line_search(cr)
    scale = np.max(np.abs(cr))
    tol = 1e-11 if prec == 0 else 3e-6
    assert np.max(np.abs(c - cr)) <= tol * scale, (c, cr)
    assert t == pytest.approx(tr, rel=1e-8 if prec == 0 else 1e-3)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("m,ncols", [(8, 3), (16, 4), (32, 5), (48, 3), (128, 2)])
def test_sparsifying_preconditioner_matches_oracle(omm, prec, m, ncols):
    """u~ = P^-1 Q (G b) (Sec. 3.2): device multifrontal solve vs the oracle's SuperLU."""
    L = 10.0
    n = m * m
    N = max(ncols, 2)
    s, V = make(omm, 2, m, L, N, prec)
    z = np.array([0.3 + 0.9j, -4.0 + 0.05j])
    s.set_poles(z, np.array([1.0, 1.0]))
    dt = torch.complex128 if prec == 0 else torch.complex64
    B = gaussian_block(n, ncols, seed=7)
    for j, zj in enumerate(z):
        U = to_host(s.precond_apply(j, to_dev(torch, B, dt)))
        st = sparsify.setup((m, m), L, V, s.shift, zj)
        ref = sparsify.apply(st, B)
        err = rel_err(U, ref)
        assert err < (1e-9 if prec == 0 else 2e-4), (m, prec, j, err)
        info = s.factor_info(j)
        assert info["nperturbed"] == 0
