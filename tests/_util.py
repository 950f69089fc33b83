"""Helpers shared by the tests: gauge-invariant comparisons and the WS-weight builder."""
from __future__ import annotations

import itertools

import numpy as np


def group_labels(vals: np.ndarray, tol: float) -> np.ndarray:
    """Label runs of (ascending) values that lie within tol of their neighbour."""
    lab = np.zeros(len(vals), dtype=int)
    for i in range(1, len(vals)):
        lab[i] = lab[i - 1] + (0 if abs(vals[i] - vals[i - 1]) <= tol else 1)
    return lab


def degenerate_sums(g2: np.ndarray, eps_m, eps_n, omega, tol: float, tol_w: float = None) -> np.ndarray:
    """Sum |g|^2 [nu, m, n] over degenerate blocks of (nu, m, n); broadcast back to the shape.

    The per-element |g_mn,nu|^2 depends on the eigenvector gauge inside a
    degenerate subspace; the block sums do not.
    """
    tol_w = tol if tol_w is None else tol_w
    lv = group_labels(omega, tol_w)
    lm = group_labels(eps_m, tol)
    ln = group_labels(eps_n, tol)
    S = np.zeros((lv.max() + 1, lm.max() + 1, ln.max() + 1))
    V, M, N = np.meshgrid(lv, lm, ln, indexing="ij")
    np.add.at(S, (V, M, N), g2)
    return S[V, M, N]


def ws_vectors(N: int, A: np.ndarray = np.eye(3), search: int = 2):
    """Wigner-Seitz set of an N x N x N supercell with 1/degeneracy weights.

    A lattice vector R belongs to the set when it is at least as close to the
    origin as to every supercell image N*T; its weight is 1/(number of images
    at the same, minimal, distance).
    """
    out, wts = [], []
    rng = range(-N * search, N * search + 1)
    images = [np.array(t) * N for t in itertools.product(range(-search, search + 1), repeat=3)]
    for R in itertools.product(rng, repeat=3):
        R = np.array(R)
        d = [np.linalg.norm((R - T) @ A) for T in images]
        d0 = np.linalg.norm(R @ A)
        dmin = min(d)
        if d0 <= dmin + 1e-9:
            nd = sum(1 for x in d if abs(x - dmin) <= 1e-9)
            out.append(R)
            wts.append(1.0 / nd)
    return np.array(out, dtype=np.int32), np.array(wts)


def rel_err(a, b, floor=0.0):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))


def fermi_level_term_scale(oracle_lib, wm, k, q, wq, T, EF, sigma, cot, omega_min=1e-5):
    """sum over (k, q, nu, m, n) of |c_nk pi w_q |g|^2 df/dE_F (d+ - d-)|: the magnitude of the
    terms whose signed sum is dL/dE_F.  Those terms change sign with e_nk - e_mk+q, and their
    sum can be orders of magnitude below this scale; an error of relative size r per term
    then bounds the error of dL/dE_F by about r times this scale, not r times |dL/dE_F|.
    Values from the oracle's interpolation and its Gaussian difference."""
    ek, ekq, om, g = oracle_lib.interp(wm, k, q, omega_min)
    nq = len(q)
    wq = np.full(nq, 1.0 / nq) if wq is None else np.asarray(wq)
    kT = 8.617333262e-5 * T
    x = (ekq - EF) / kT                                   # [nk, nq, m]
    t = np.exp(-np.abs(x))
    dfdE = t / (1.0 + t) ** 2 / kT
    gd = np.vectorize(oracle_lib.gauss_diff)
    total = 0.0
    for iq in range(nq):
        for nu in range(om.shape[1]):
            w = om[iq, nu]
            if w < omega_min:
                continue
            xd = ek[:, None, :] - ekq[:, iq, :, None]      # [nk, m, n]
            dd = gd(xd, w, sigma)
            g2 = np.abs(g[:, iq, nu]) ** 2                  # [nk, m, n]
            total += float(np.sum(np.abs(cot[:, None, :] * np.pi * wq[iq] * g2 * dfdE[:, iq, :, None] * dd)))
    return total
