"""Per-pair kernel of the staged form for the wide shapes (nw up to 18, up to 18 modes).

Shapes beyond the register-tile per-pair kernel (nw > 8 or 3nat > 9) run, after the staged
tensor-core contraction, one warp per (k, q) pair: Householder reduction and implicit QR of
H(k+q) in FP32, the eigenvectors that some band at k can reach, and only the (m, n) terms of
Eq. (linewidthel) within the Gaussian cutoff.  These tests pin it to the FP64 oracle on
nw = 4 .. 18 and 3 .. 18 modes (odd and even nw; both compiled register widths), with every
band doubly degenerate, with most terms reachable (sigma = 0.4 eV) and almost none (6 meV),
and compare it with the every-term kernel it replaces (EPW_STAGED_PAIR=dense).

Tolerances: the split contractions give e_k+q to ~1e-5 eV and the FP32 eigensolve adds
about n eps ||H|| (~2e-5 eV for these models' 15-30 eV band spans); at sigma = 50 meV a
Gaussian moves by ~2 dx / sigma ~ 1e-3 per term and the sums over 300 q by a few 1e-4.
"""
import dataclasses
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [("fcc", 12, 1, 30), ("sc", 18, 1, 27), ("hex", 4, 4, 20), ("diamond", 9, 5, 20), ("hex", 18, 6, 20),
          ("sc", 5, 4, 27)]
TOL = {"tf32x3": 3e-4, "bf16x3": 8e-4}


def _rel(got, ref):
    floor = 1e-6 * np.abs(ref).max()
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


@pytest.fixture(scope="module")
def epw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw
    return epw


def _model(lat, nw, nat, nR, seed):
    rng = np.random.default_rng(seed)
    return W.make_model(lat, nw, nat, [1.0 + 0.1 * i for i in range(nat)], nR, nR, rng), rng


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("lat,nw,nat,nR", SHAPES)
def test_wide_staged_linewidth_matches_oracle(epw, oracle_lib, lat, nw, nat, nR, prec):
    """5 k x 300 q (three q tiles, the last ragged), T = 300 K, sigma = 50 meV."""
    wm, rng = _model(lat, nw, nat, nR, 700 + nw + nat)
    k = rng.random((5, 3))
    q = rng.random((300, 3))
    wq = np.full(300, 1.0 / 300)
    ref = oracle_lib.linewidth(wm, k, q, wq, 300.0, 0.1, 0.05)
    m = epw.Model(wm)
    got = m.linewidth(k, q, wq, T=300.0, EF=0.1, sigma=0.05, precision=epw.PRECISIONS[prec])
    m.sync()
    err = _rel(got, ref)
    print(lat, nw, 3 * nat, prec, "max rel err vs oracle", err)
    assert np.all(got >= 0)
    assert err < TOL[prec]


@pytest.mark.parametrize("sigma", [0.4, 0.006])
def test_wide_staged_cutoff_extremes(epw, oracle_lib, sigma):
    """sigma = 0.4 eV: the cutoff (max w + 9.49 sigma) reaches most (m, n); 6 meV: almost none, so
    each sum rests on a few terms near their delta peaks (there a Gaussian moves by ~2 dx / sigma
    per unit dx, hence the wider bound)."""
    wm, rng = _model("hex", 12, 4, 20, 761)
    k = rng.random((4, 3))
    q = rng.random((260, 3))
    ref = oracle_lib.linewidth(wm, k, q, None, 300.0, 0.1, sigma)
    m = epw.Model(wm)
    got = m.linewidth(k, q, T=300.0, EF=0.1, sigma=sigma, precision=epw.TF32X3)
    m.sync()
    err = _rel(got, ref)
    print("sigma", sigma, "max rel err vs oracle", err)
    assert err < (3e-4 if sigma > 0.1 else 5e-3)


def test_wide_staged_degenerate_bands(epw, oracle_lib):
    """H(R) = h(R) x I_2 and g(Re, Rp) = g_1(Re, Rp) x I_2: two identical copies, so every band
    at every k and k+q is doubly degenerate and its eigenvectors are fixed only up to rotations
    inside each pair.  The linewidths do not depend on that choice, and partners are equal."""
    base, rng = _model("sc", 9, 2, 27, 777)
    H2 = np.stack([np.kron(h, np.eye(2)) for h in base.H])
    g2 = np.kron(base.g, np.eye(2))
    wm = dataclasses.replace(base, nw=18, H=H2, g=g2)
    k = rng.random((3, 3))
    q = rng.random((200, 3))
    ref = oracle_lib.linewidth(wm, k, q, None, 300.0, 0.0, 0.05)
    m = epw.Model(wm)
    got = m.linewidth(k, q, T=300.0, EF=0.0, sigma=0.05, precision=epw.TF32X3)
    m.sync()
    err = _rel(got, ref)
    print("degenerate nw=18: max rel err vs oracle", err)
    assert np.allclose(ref[:, 0::2], ref[:, 1::2], rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(got[:, 0::2], got[:, 1::2], rtol=TOL["tf32x3"], atol=1e-6 * np.abs(got).max())
    assert err < TOL["tf32x3"]


@pytest.mark.parametrize("lat,nw,nat,nR", [("fcc", 12, 1, 30), ("hex", 18, 6, 20)])
def test_sparse_and_dense_kernels_agree(epw, lat, nw, nat, nR):
    """The same staged contraction through both per-pair kernels: the QR eigensolve and the
    cutoff against cyclic Jacobi and every term (FP32 either way)."""
    import torch
    wm, rng = _model(lat, nw, nat, nR, 790 + nw)
    k = torch.tensor(rng.random((4, 3)), device="cuda")
    q = torch.tensor(rng.random((300, 3)), device="cuda")
    m = epw.Model(wm)
    kw = dict(T=300.0, EF=0.1, sigma=0.05, precision=epw.TF32X3)
    sparse = m.linewidth(k, q, **kw).cpu().numpy()
    os.environ["EPW_STAGED_PAIR"] = "dense"
    try:
        dense = m.linewidth(k, q, **kw).cpu().numpy()
    finally:
        del os.environ["EPW_STAGED_PAIR"]
    m.sync()
    err = _rel(sparse, dense)
    print(lat, nw, 3 * nat, "sparse vs dense max rel", err)
    assert err < 2e-4
