"""Writes workloads/spectra.json: the spectral data of each workload's H - sigma computed by
the oracle only (dense eigh for n <= 4096; otherwise the truncated plane-wave basis of
oracle.spectrum for the smooth 2D field and the exact Bloch sectors for the 3D lattice).

The pole rule needs the occupied interval [lam_1, lam_N] and lam_{N+1}; the paper builds
its contour from the exact spectrum (Sec. 4), so the workloads carry these stored
values.  E_ref = 1/2 sum_{i<=N} lam_i is the exact minimum of E_omm (Sec. 1).  gtpa_tau
(2D workloads) is the scale tau of the TPA-type comparison preconditioners, which Sec. 4
also takes from the exact eigenvectors.

Run: python -m workloads.make_spectra
"""
from __future__ import annotations

import json
import os

import numpy as np

from oracle import gtpa, hamiltonian as ham
from oracle import spectrum
from workloads import WORKLOADS, batch_mix, serving_mix, serving_mix_3d, serving_mix_wide

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spectra.json")


def compute(wl, kc=24):
    V = wl.potential_values()
    shape = wl.shape
    sig = ham.default_shift(shape, wl.L, V)
    if wl.n <= 4096:
        lam = np.linalg.eigvalsh(ham.dense_h(shape, wl.L, V, sig))[: wl.N + 8]
        how = "dense eigh"
    elif wl.potential == "lattice3d":
        lam = spectrum.lowest_eigs_bloch(shape, wl.L, V, sig, 4, wl.N + 8)
        how = "Bloch sectors of the 4^3 lattice (exact)"
    else:
        lam = spectrum.lowest_eigs_kspace(shape, wl.L, V, sig, wl.N + 8, kc)
        how = f"plane-wave box |k|_inf <= {kc}"
    lo, hi = ham.weyl_bounds(shape, wl.L, V, sig)
    return dict(sigma=sig, lam1=float(lam[0]), lamN=float(lam[wl.N - 1]), lamN1=float(lam[wl.N]),
                weyl_lo=lo, weyl_hi=hi, E_ref=float(0.5 * np.sum(lam[: wl.N])), method=how,
                lowest=[float(x) for x in lam])


def gtpa_tau(wl, sig, kc=24):
    """tau of the TPA-type comparison preconditioners (Sec. 4): the largest kinetic energy
    (1/2) sum_k |k|^2 |xhat_j(k)|^2 over the N exact lowest eigenvectors (dense eigh for
    n <= 4096, else the plane-wave box).  2D workloads only."""
    V = wl.potential_values()
    if wl.n <= 4096:
        _, U = np.linalg.eigh(ham.dense_h(wl.shape, wl.L, V, sig))
        return gtpa.kinetic_tau(U[:, : wl.N].T, wl.shape)
    return spectrum.kinetic_tau_kspace(wl.shape, wl.L, V, sig, wl.N, kc)


def compute_spec(h, kc=24, window=8):
    """Spectral data of one many-Hamiltonian entry (dense eigh for n <= 4096, the Bloch
    sectors for the 3D lattice, else the plane-wave box).  N is taken within +-window of the drawn value where the gap
    lam_{N+1} - lam_N is largest, so that the occupied space is well separated."""
    V = h.potential_values()
    shape = h.shape
    sig = ham.default_shift(shape, h.L, V)
    if h.potential == "lattice3d":
        window = 0                   # N is the band edge of the lattice (64: s, 256: s + p)
    cnt = h.N + window + 1
    if h.n <= 4096:
        lam = np.linalg.eigvalsh(ham.dense_h(shape, h.L, V, sig))[:cnt]
    elif h.potential == "lattice3d":
        lam = spectrum.lowest_eigs_bloch(shape, h.L, V, sig, 4, cnt)
    else:
        lam = spectrum.lowest_eigs_kspace(shape, h.L, V, sig, cnt, kc)
    cands = range(max(1, h.N - window), h.N + window + 1)
    N = max(cands, key=lambda k: lam[k] - lam[k - 1])
    return dict(sigma=sig, lam1=float(lam[0]), lamN=float(lam[N - 1]), lamN1=float(lam[N]),
                E_ref=float(0.5 * np.sum(lam[:N])), m=h.m, N=int(N), N_drawn=h.N, potential=h.potential,
                seed=h.seed, dim=h.dim)


def main(names=("wells2d-32", "smooth2d-128", "lattice3d-48")):
    data = {}
    if os.path.exists(OUT):
        data = json.load(open(OUT))
    for name in names:
        if name in data:
            continue
        data[name] = compute(WORKLOADS[name])
        print(name, data[name]["lamN1"] - data[name]["lamN"], data[name]["method"])
    for name in names:
        wl = WORKLOADS[name]
        if wl.dim == 2 and "gtpa_tau" not in data[name]:
            data[name]["gtpa_tau"] = gtpa_tau(wl, data[name]["sigma"])
            print(name, "tau", data[name]["gtpa_tau"])
    for h in batch_mix() + serving_mix() + serving_mix_wide() + serving_mix_3d():
        if h.key not in data:
            data[h.key] = compute_spec(h)
            print(h.key, h.m, h.N, data[h.key]["lamN1"] - data[h.key]["lamN"], flush=True)
    json.dump(data, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main()
