"""Write the energy-window k lists of the fcc nw=4 and diamond nw=8 workloads.

Selecting the k-points needs band energies, so this script takes them from the
CPU oracle (and nothing else).

fcc nw=4 (1000 k-points uniform in a 0.2 eV window around E_F):
* E_F = median of all band energies on a 20^3 uniform grid;
* candidates are uniform random k in [0,1)^3 (seeded); a candidate is kept
  when any band energy lies in [E_F - 0.1, E_F + 0.1] eV; the first 1000 kept
  are written.

diamond nw=8 (2000 k-points near the band edges):
* on the 20^3 grid, VBM = max of band nw/2 and CBM = min of band nw/2 + 1
  (bands counted from 1 in ascending order), E_F = (VBM + CBM) / 2;
* a candidate is kept when any band energy lies within 0.2 eV of VBM or of
  CBM; the first 2000 kept are written.

Run:  python tests/golden/make_kwindows.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def window_kpoints(model, nkeep, half_width, seed, ef=None):
    eps_grid, _ = oracle.bands(model, W.uniform_grid(20))
    EF = float(np.median(eps_grid)) if ef is None else ef
    rng = np.random.default_rng(seed)
    kept = []
    while len(kept) < nkeep:
        cand = rng.random((4 * nkeep, 3))
        eps, _ = oracle.bands(model, cand)
        ok = np.any(np.abs(eps - EF) <= half_width, axis=1)
        kept.extend(cand[ok])
    return np.array(kept[:nkeep]), EF


def edge_kpoints(model, nkeep, half_width, seed):
    eps_grid, _ = oracle.bands(model, W.uniform_grid(20))
    nw = eps_grid.shape[1]
    vbm, cbm = float(eps_grid[:, nw // 2 - 1].max()), float(eps_grid[:, nw // 2].min())
    rng = np.random.default_rng(seed)
    kept = []
    while len(kept) < nkeep:
        cand = rng.random((4 * nkeep, 3))
        eps, _ = oracle.bands(model, cand)
        ok = np.any((np.abs(eps - vbm) <= half_width) | (np.abs(eps - cbm) <= half_width), axis=1)
        kept.extend(cand[ok])
    return np.array(kept[:nkeep]), 0.5 * (vbm + cbm), vbm, cbm


def write(path, k, EF, note):
    with open(path, "w") as f:
        f.write(f"# EF={EF!r} {note}\n")
        for row in k:
            f.write(" ".join(repr(float(x)) for x in row) + "\n")


def main():
    rng = np.random.default_rng(W.models.SEED_BASE + 1)
    m = W.make_model("fcc", 4, 1, [1.0], 120, 120, rng)
    k, EF = window_kpoints(m, 1000, 0.1, W.models.SEED_BASE + 201)
    write(os.path.join(HERE, "kwindow_fcc_nw4.txt"), k, EF,
          "fcc nw=4 model (seed 160403525+1): 1000 k with a band within 0.1 eV of E_F, E_F = median of the 20^3-grid bands")
    m = W.models.diamond_nw8_model()
    k, EF, vbm, cbm = edge_kpoints(m, 2000, 0.2, W.models.SEED_BASE + 202)
    write(os.path.join(HERE, "kwindow_diamond_nw8.txt"), k, EF,
          f"diamond nw=8 model (seed 160403525+2): 2000 k with a band within 0.2 eV of VBM={vbm!r} or "
          f"CBM={cbm!r} (20^3 grid, bands 4 and 5), E_F = mid-point")


if __name__ == "__main__":
    main()
