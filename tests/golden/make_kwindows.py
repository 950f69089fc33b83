"""Write the energy-window k lists used by the fcc nw=4 workload.

The workload asks for 1000 k-points uniform in a 0.2 eV window around E_F.
Selecting them needs band energies, so this script takes them from the CPU
oracle (and nothing else):

* E_F = median of all band energies on a 20^3 uniform grid;
* candidates are uniform random k in [0,1)^3 (seeded); a candidate is kept
  when any band energy lies in [E_F - 0.1, E_F + 0.1] eV; the first 1000 kept
  are written.

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


if __name__ == "__main__":
    main()
