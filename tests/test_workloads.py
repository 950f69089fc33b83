"""The stored k lists of the energy-window workloads satisfy the rules that select them.

tests/golden/make_kwindows.py writes them from the oracle's band energies; these
checks recompute E_F (and the band edges) with the oracle and confirm every stored
k-point has a band inside its window, so a stored list cannot drift from its rule.
"""
import numpy as np

import workloads as W


def test_fcc_window_kpoints_follow_their_rule(oracle_lib):
    wl = W.make_workload("fcc_nw4", nq_sub=1)
    eps_grid, _ = oracle_lib.bands(wl.model, W.uniform_grid(20))
    EF = float(np.median(eps_grid))
    assert abs(EF - wl.EF) < 1e-12
    assert wl.k.shape == (1000, 3)
    eps, _ = oracle_lib.bands(wl.model, wl.k)
    assert np.all(np.any(np.abs(eps - EF) <= 0.1 + 1e-9, axis=1))
    assert np.all((wl.k >= 0.0) & (wl.k < 1.0))


def test_diamond_edge_kpoints_follow_their_rule(oracle_lib):
    wl = W.make_workload("diamond_nw8", nq_sub=1)
    eps_grid, _ = oracle_lib.bands(wl.model, W.uniform_grid(20))
    nw = eps_grid.shape[1]
    vbm, cbm = float(eps_grid[:, nw // 2 - 1].max()), float(eps_grid[:, nw // 2].min())
    assert abs(0.5 * (vbm + cbm) - wl.EF) < 1e-12
    assert wl.k.shape == (2000, 3)
    eps, _ = oracle_lib.bands(wl.model, wl.k)
    near = (np.abs(eps - vbm) <= 0.2 + 1e-9) | (np.abs(eps - cbm) <= 0.2 + 1e-9)
    assert np.all(np.any(near, axis=1))
