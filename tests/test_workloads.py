"""The seeded input generators follow the recipes the design states: the smooth field is
band-limited with the exp(-|k|^2/8) envelope and max|V| = 10; the wells are negative,
periodic (minimum image) Gaussians; the 3D lattice potential repeats with the cell period
(which the Bloch-sector oracle relies on) and has the cubic symmetry of its lattice; the
Gaussian blocks have the stated variances and layout; the many-Hamiltonian mixes and the
arrivals have the stated ranges; everything is reproducible from its seed."""
import numpy as np
import pytest

from workloads import (WORKLOADS, batch_mix, gaussian_block, gaussian_block_real, lattice_wells_3d,
                       poisson_arrivals, serving_mix, serving_mix_3d, serving_mix_wide, smooth_field_2d,
                       wells_2d)


def test_smooth_field_is_band_limited_with_the_stated_envelope():
    m = 128
    V = smooth_field_2d(m, seed=0)
    assert np.max(np.abs(V)) == pytest.approx(10.0, rel=1e-14)
    assert np.array_equal(V, smooth_field_2d(m, seed=0)) and not np.array_equal(V, smooth_field_2d(m, seed=1))
    c = np.fft.fft2(V.reshape(m, m)) / m ** 2
    k = np.fft.fftfreq(m, 1.0 / m)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    # the coefficients of V are (c_k + conj(c_-k)) / 2 with |c_k| ~ e^{-|k|^2/8}: beyond
    # |k|^2 = 400 the envelope is e^{-50}, far below FP64 rounding of the largest term
    tail = np.abs(c[k2 > 400]).max()
    assert tail < 1e-15 * np.abs(c).max()
    # the decay rate: log-magnitude averaged over shells falls by ~1/8 per unit |k|^2
    shells = [(8, 12), (40, 48)]
    means = [np.log(np.abs(c[(k2 >= a) & (k2 < b)])).mean() for a, b in shells]
    slope = (means[1] - means[0]) / (44 - 10)
    assert slope == pytest.approx(-1.0 / 8.0, rel=0.15)


def test_wells_are_negative_periodic_gaussians():
    m, L = 32, 10.0
    V = wells_2d(m, L, seed=0).reshape(m, m)
    assert np.all(V < 0) and -10.0 * 4 < V.min() <= -5.0 * 0.97
    # minimum image: the field is smooth across the periodic boundary (no jump between the
    # last and the first column / row larger than between interior neighbours)
    d_in = np.abs(np.diff(V, axis=1)).max()
    assert np.abs(V[:, 0] - V[:, -1]).max() <= d_in * 1.0001
    d_in = np.abs(np.diff(V, axis=0)).max()
    assert np.abs(V[0, :] - V[-1, :]).max() <= d_in * 1.0001


def test_lattice_potential_repeats_with_the_cell_and_is_cubic():
    m, cells = 48, 4
    V = lattice_wells_3d(m, 40.0, cells=cells).reshape(m, m, m)     # axes (z, y, x)
    p = m // cells
    for ax in range(3):
        np.testing.assert_allclose(np.roll(V, p, axis=ax), V, atol=1e-12)
    np.testing.assert_allclose(V.transpose(0, 2, 1), V, atol=1e-12)   # x <-> y
    np.testing.assert_allclose(V.transpose(2, 1, 0), V, atol=1e-12)   # x <-> z
    assert V.min() == pytest.approx(-8.0, rel=0.05) and np.all(V < 0)


def test_gaussian_blocks_layout_and_variance():
    n, N = 4096, 64
    Z = gaussian_block(n, N, seed=3)
    R = gaussian_block_real(n, N, seed=3)
    assert Z.shape == (N, n) and R.shape == (N, n) and Z.dtype == np.complex128
    assert np.all(R.imag == 0)
    assert np.var(Z.real) * n == pytest.approx(0.5, rel=0.05) and np.var(Z.imag) * n == pytest.approx(0.5, rel=0.05)
    assert np.var(R.real) * n == pytest.approx(1.0, rel=0.05)
    assert np.mean(np.linalg.norm(Z, axis=1)) == pytest.approx(1.0, rel=0.02)
    assert gaussian_block(n, N, seed=3, dtype=np.complex64).dtype == np.complex64
    assert np.array_equal(Z, gaussian_block(n, N, seed=3))


def test_mixes_and_arrivals_have_the_stated_ranges():
    b = batch_mix()
    assert len(b) == 64 and {h.m for h in b} <= {32, 64, 96, 128}
    assert all(16 <= h.N <= min(128, h.m * h.m // 4) and h.potential == "smooth2d" for h in b)
    s = serving_mix()
    assert len(s) == 12 and {h.m for h in s} <= {64, 72, 96, 128}
    assert all(32 <= h.N <= 128 and h.potential == "wells2d" for h in s)
    t, keys = poisson_arrivals(4000, 200.0, 12)
    assert np.all(np.diff(t) > 0) and keys.min() >= 0 and keys.max() < 12
    assert 4000 / t[-1] == pytest.approx(200.0, rel=0.05)
    w = WORKLOADS["smooth2d-128"]
    assert (w.dim, w.m, w.N, w.P, w.L, w.precision) == (2, 128, 128, 16, 10.0, "mixed")
    wide = serving_mix_wide()
    assert len(wide) == 4 and {h.m for h in wide} <= {64, 96, 128}
    assert all(129 <= h.N <= min(256, h.m * h.m // 4) and h.potential == "wells2d" and h.dim == 2 for h in wide)
    s3 = serving_mix_3d()
    assert [(h.dim, h.m, h.N, h.L, h.potential) for h in s3] == [
        (3, 32, 64, 40.0, "lattice3d"), (3, 48, 64, 40.0, "lattice3d"), (3, 48, 256, 40.0, "lattice3d")]
    assert s3[0].n == 32 ** 3 and s3[0].shape == (32, 32, 32)
    np.testing.assert_array_equal(s3[2].potential_values(), WORKLOADS["lattice3d-48"].potential_values())
