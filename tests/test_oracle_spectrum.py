"""Pins for oracle.spectrum: the truncated plane-wave spectrum and the Bloch-sector
spectrum reproduce the dense eigh of the grid H (Sec. 4, eq. ex1mat) on small grids."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import spectrum
from workloads import smooth_field_2d, lattice_wells_3d


def cell_periodic_field(m, cells, d, seed):
    """A random, asymmetric potential periodic on `cells` cells per axis (axes z, y, x)."""
    mc = m // cells
    cell = np.random.default_rng(seed).uniform(-5.0, 1.0, size=(mc,) * d)
    return np.tile(cell, (cells,) * d).ravel()


def test_kspace_full_box_is_dense_eigh():
    m, L = 12, 10.0
    V = smooth_field_2d(m, L, seed=3)
    sig = ham.default_shift((m, m), L, V)
    lam = np.linalg.eigvalsh(ham.dense_h((m, m), L, V, sig))
    got = spectrum.lowest_eigs_kspace((m, m), L, V, sig, 20, kc=m // 2)
    np.testing.assert_allclose(got, lam[:20], atol=1e-11 * np.max(np.abs(lam)))


def test_kspace_box_converges_for_a_smooth_field():
    """The smooth field's coefficients decay like exp(-|k|^2/8): the truncation error of the
    lowest eigenvalues falls geometrically with the box and vanishes at the full grid."""
    m, L = 24, 10.0
    V = smooth_field_2d(m, L, seed=1)
    sig = ham.default_shift((m, m), L, V)
    lam = np.linalg.eigvalsh(ham.dense_h((m, m), L, V, sig))[:10]
    errs = [np.max(np.abs(spectrum.lowest_eigs_kspace((m, m), L, V, sig, 10, kc=kc) - lam)) / np.max(np.abs(lam))
            for kc in (6, 8, 10, 11)]
    assert all(e1 < e0 / 3 for e0, e1 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6


def test_stored_128_spectrum_is_converged_in_the_box():
    """The stored spectrum of the 128^2 smooth-field workload (plane-wave box |k|_inf <= 24)
    agrees with a smaller box to near rounding: the truncation has converged."""
    import json, os
    from workloads import WORKLOADS
    wl = WORKLOADS["smooth2d-128"]
    stored = json.load(open(os.path.join(os.path.dirname(__file__), "..", "workloads", "spectra.json")))[wl.name]
    V = wl.potential_values()
    lam20 = spectrum.lowest_eigs_kspace(wl.shape, wl.L, V, stored["sigma"], wl.N + 1, kc=20)
    scale = abs(stored["lam1"])
    assert abs(lam20[0] - stored["lam1"]) < 1e-11 * scale
    assert abs(lam20[wl.N - 1] - stored["lamN"]) < 1e-11 * scale
    assert abs(lam20[wl.N] - stored["lamN1"]) < 1e-11 * scale
    assert abs(0.5 * lam20[:wl.N].sum() - stored["E_ref"]) < 1e-11 * abs(stored["E_ref"])


@pytest.mark.parametrize("d,m,cells", [(2, 12, 3), (2, 12, 4), (3, 8, 2)])
def test_bloch_sectors_give_the_dense_spectrum(d, m, cells):
    L = 10.0
    V = cell_periodic_field(m, cells, d, seed=m + cells)
    shape = (m,) * d
    sig = ham.default_shift(shape, L, V)
    lam = np.linalg.eigvalsh(ham.dense_h(shape, L, V, sig))
    got = spectrum.lowest_eigs_bloch(shape, L, V, sig, cells, m ** d)
    np.testing.assert_allclose(got, lam, atol=1e-11 * np.max(np.abs(lam)))


def test_bloch_needs_the_true_period():
    """A planted mistake (claiming a shorter period than V has) breaks the block structure
    and the spectrum no longer matches."""
    d, m = 2, 12
    V = cell_periodic_field(m, 2, d, seed=7)           # period m/2, not m/4
    shape = (m,) * d
    sig = ham.default_shift(shape, 10.0, V)
    lam = np.linalg.eigvalsh(ham.dense_h(shape, 10.0, V, sig))
    wrong = spectrum.lowest_eigs_bloch(shape, 10.0, V, sig, 4, m ** d)
    assert np.max(np.abs(wrong - lam)) > 1e-3


def test_lattice_workload_is_cell_periodic():
    """The 3D lattice potential repeats with the lattice constant, the premise of the
    Bloch splitting used for its stored spectrum."""
    m, cells = 24, 4
    V = lattice_wells_3d(m, 40.0, cells=cells).reshape(m, m, m)
    mc = m // cells
    for ax in range(3):
        np.testing.assert_allclose(np.roll(V, mc, axis=ax), V, atol=1e-12)


def test_stored_spectrum_of_the_served_32_lattice():
    """The stored spectral data of the served 32^3 lattice (N = 64, the s band) are those of
    the Bloch solver: lam_1, lam_N, lam_{N+1} and 1/2 sum_{i<=N} lam_i, with a clear gap."""
    import json
    import os
    from workloads import serving_mix_3d
    h = serving_mix_3d()[0]
    stored = json.load(open(os.path.join(os.path.dirname(__file__), "..", "workloads", "spectra.json")))[h.key]
    V = h.potential_values()
    lam = spectrum.lowest_eigs_bloch(h.shape, h.L, V, stored["sigma"], 4, h.N + 1)
    scale = abs(stored["lam1"])
    assert stored["N"] == h.N == 64
    assert abs(lam[0] - stored["lam1"]) < 1e-11 * scale
    assert abs(lam[h.N - 1] - stored["lamN"]) < 1e-11 * scale
    assert abs(lam[h.N] - stored["lamN1"]) < 1e-11 * scale
    assert abs(0.5 * lam[:h.N].sum() - stored["E_ref"]) < 1e-11 * abs(stored["E_ref"])
    assert stored["lamN1"] - stored["lamN"] > 1.0
