"""Host setup of the sparsifying preconditioner (csrc/host_spp.cpp, Sec. 3.2): the nested-
dissection structure and one pole's multifrontal factor, exercised through a small C++
driver that replays the device triangular-solve algorithm on the host, against the oracle's
SuperLU solve of the same P (oracle.sparsify).  2D and 3D grids; in 2D both the dense-W and
the banded-leaf paths.  q is unique up to a unit phase, which scales P and so P^-1 b by one
global phase: the comparison removes it.  Built with AddressSanitizer where the compiler
supports it, so an out-of-bounds access in the host setup fails the test.  The elimination
tree factorised on 2 and 4 threads gives bitwise the same solve as on one."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import sparsify
from workloads import wells_2d, lattice_wells_3d

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1603_09724_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("spp") / "host_spp_driver")
    srcs = [os.path.join(HERE, "host_spp_driver.cpp"), os.path.join(CSRC, "host_spp.cpp")]
    base = [gxx, "-O1", "-g", "-std=c++17", "-I", CSRC, *srcs, "-o", out]
    for extra in (["-fsanitize=address", "-fno-omit-frame-pointer"], []):
        if subprocess.run(base + extra, capture_output=True).returncode == 0:
            return out
    pytest.fail("host_spp_driver does not compile")


def run_driver(exe, dim, m, L, V, shift, z, b, threads=1, raw=False, extra=()):
    f = lambda v: repr(float(v))
    lines = [f"{dim} {m} {f(L)} {f(shift)} {f(z.real)} {f(z.imag)}", " ".join(f(v) for v in V),
             " ".join(f"{f(v.real)} {f(v.imag)}" for v in b)]
    r = subprocess.run([exe, str(threads), *extra], input="\n".join(lines) + "\n", capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    if raw:
        return r.stdout
    out, cur = {}, None
    for ln in r.stdout.splitlines():
        if ln in ("dense", "banded"):
            cur = out.setdefault(ln, [])
        else:
            re_, im_ = ln.split()
            cur.append(complex(float(re_), float(im_)))
    return {k: np.array(v) for k, v in out.items()}


def phase_free_err(x, ref):
    c = np.vdot(x, ref) / np.vdot(x, x)          # best scalar; |c| = 1 when only the phase differs
    return float(np.linalg.norm(c * x - ref) / np.linalg.norm(ref)), abs(c)


@pytest.mark.parametrize("dim,m,L", [(2, 16, 10.0), (2, 32, 10.0), (2, 27, 10.0), (2, 48, 10.0), (3, 8, 20.0),
                                     (3, 12, 20.0)])
def test_host_factor_solves_the_oracle_P(driver, dim, m, L):
    shape = (m,) * dim
    V = wells_2d(m, L, seed=4) if dim == 2 else lattice_wells_3d(m, L, cells=2)
    shift = ham.default_shift(shape, L, V)
    z = complex(-0.35 * shift, 0.8)
    n = m ** dim
    b = np.random.default_rng(m).standard_normal(n) + 1j * np.random.default_rng(m + 1).standard_normal(n)
    ref = sparsify.setup(shape, L, V, shift, z)["lu"].solve(b)
    got = run_driver(driver, dim, m, L, V, shift, z, b)
    assert ("banded" in got) == (dim == 2)
    for mode, x in got.items():
        err, scale = phase_free_err(x, ref)
        assert err < 1e-9, (mode, err)
        assert abs(scale - 1.0) < 1e-9, (mode, scale)


@pytest.mark.parametrize("dim,m,L", [(2, 32, 10.0), (3, 8, 20.0)])
def test_threaded_tree_factorisation_is_bitwise_identical(driver, dim, m, L):
    shape = (m,) * dim
    V = wells_2d(m, L, seed=5) if dim == 2 else lattice_wells_3d(m, L, cells=2)
    shift = ham.default_shift(shape, L, V)
    z = complex(-0.3 * shift, 1.1)
    n = m ** dim
    b = np.random.default_rng(7).standard_normal(n) + 1j * np.random.default_rng(8).standard_normal(n)
    outs = [run_driver(driver, dim, m, L, V, shift, z, b, threads=t, raw=True) for t in (1, 2, 4)]
    assert outs[0] == outs[1] == outs[2]


@pytest.mark.parametrize("dim,m,L", [(2, 16, 10.0), (2, 32, 10.0), (3, 8, 20.0), (3, 12, 20.0)])
def test_device_factor_maps_reproduce_the_host_factor(driver, dim, m, L):
    """The index maps of the device factorisation (csrc/k_factor.cu) drive, replayed on the
    host in FP64 with the device's own step order (fronts assembled from the maps, the
    children's update matrices added through emap, unblocked partial LU, L_SS^-1 and U_SS^-1
    by columns, the W products, the banded leaf data), a factor equal to the host
    factorisation's to rounding: every W block and every leaf entry."""
    shape = (m,) * dim
    V = wells_2d(m, L, seed=6) if dim == 2 else lattice_wells_3d(m, L, cells=2)
    shift = ham.default_shift(shape, L, V)
    z = complex(-0.25 * shift, 0.9)
    n = m ** dim
    b = np.ones(n, dtype=complex)
    out = run_driver(driver, dim, m, L, V, shift, z, b, raw=True, extra=("maps",))
    line = [ln for ln in out.splitlines() if ln.startswith("mapsdiff")][0].split()
    assert line[1] != "unsupported"
    dfac, dleaf = float(line[1]), float(line[2])
    assert dfac < 1e-11, dfac
    assert dleaf < 1e-11, dleaf


@pytest.mark.parametrize("dim,m,L", [(2, 32, 10.0), (3, 8, 20.0), (3, 12, 20.0)])
def test_triangular_inverses_are_exactly_triangular(driver, dim, m, L):
    """The supernode products run each row block only over the k range where L_SS^-1 (the
    top block of W_f) and U_SS^-1 (the left block of W_b) can be nonzero: every entry above
    the diagonal of L_SS^-1 and below the diagonal of U_SS^-1 is exactly zero, in the host
    factor and in the device factorisation's schedule replayed on the host.  (On the device,
    fa_tinv stores zeros in the 32 x 32 tiles across the diagonal, and its diagonal-tile
    substitutions sum products with zero there; test_gpu_factor compares the resulting
    preconditioner with the host factor's.)"""
    shape = (m,) * dim
    V = wells_2d(m, L, seed=9) if dim == 2 else lattice_wells_3d(m, L, cells=2)
    shift = ham.default_shift(shape, L, V)
    z = complex(-0.4 * shift, 0.6)
    n = m ** dim
    out = run_driver(driver, dim, m, L, V, shift, z, np.ones(n, dtype=complex), raw=True, extra=("tri",))
    rows = {ln.split()[1]: (int(ln.split()[2]), int(ln.split()[3])) for ln in out.splitlines() if ln.startswith("tri")}
    assert set(rows) == {"host", "maps"}
    for who, (nonzero, entries) in rows.items():
        assert entries > 0, who
        assert nonzero == 0, (who, nonzero, entries)
