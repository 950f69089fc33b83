"""Warp-per-pair kernel for wide shapes (nw and 3nat up to 18) against the FP64 oracle.

Shapes beyond the register-tile per-pair kernel (nw <= 8, 3nat <= 9) take one
warp per (k,q) pair with H(k+q), U and the mode vertex in shared memory.  Same
tolerances as the narrow forms: FP64 1e-6, FP32 2e-3 relative on Im Sigma; the
staged tensor-core form (q-major contraction) 1e-3 on these few-q cases (the
small-sum argument of the uneven-batch test).
"""
import numpy as np
import pytest

import workloads as W
from tests._util import degenerate_sums

pytestmark = pytest.mark.gpu

SHAPES = [("sc", 12, 4), ("fcc", 18, 6), ("hex", 9, 3), ("diamond", 5, 5)]


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


def _wide_model(lat, nw, nat, seed):
    rng = np.random.default_rng(seed)
    return W.make_model(lat, nw, nat, [1.0 + 0.1 * i for i in range(nat)], 27, 27, rng), rng


@pytest.mark.parametrize("lat,nw,nat", SHAPES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("fp32", 2e-3), ("tf32x3", 1e-3), ("bf16x3", 1e-3)])
def test_wide_linewidth_matches_oracle(epw, oracle_lib, lat, nw, nat, prec, tol):
    wm, rng = _wide_model(lat, nw, nat, 800 + nw)
    k = rng.random((3, 3))
    q = rng.random((150, 3))  # two q tiles, the second ragged
    m = epw.Model(wm)
    ref = oracle_lib.linewidth(wm, k, q, None, 300.0, 0.1, 0.08)
    got = m.linewidth(k, q, T=300.0, EF=0.1, sigma=0.08, precision=epw.PRECISIONS[prec])
    print(lat, nw, 3 * nat, prec, "max rel err", _rel(got, ref))
    assert _rel(got, ref) < tol
    m.sync()


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_wide_interp_matches_oracle(epw, oracle_lib, prec):
    wm, rng = _wide_model("fcc", 12, 5, 820)
    k = rng.random((2, 3))
    q = np.concatenate([np.zeros((1, 3)), rng.random((40, 3))])
    m = epw.Model(wm)
    ek, ekq, om, g = m.interp(k, q, precision=epw.PRECISIONS[prec])
    rk, rkq, rom, rg = oracle_lib.interp(wm, k, q)
    assert np.abs(ek - rk).max() < 1e-10
    assert np.abs(ekq - rkq).max() < (1e-10 if prec == "fp64" else 5e-5)
    assert np.all(np.diff(ekq, axis=-1) >= 0)  # ascending
    worst = 0.0
    for ik in range(len(k)):
        for iq in range(len(q)):
            a = degenerate_sums(np.abs(g[ik, iq]) ** 2, rkq[ik, iq], rk[ik], rom[iq], 1e-4)
            b = degenerate_sums(np.abs(rg[ik, iq]) ** 2, rkq[ik, iq], rk[ik], rom[iq], 1e-4)
            big = b > 1e-6 * b.max()
            if big.any():
                worst = max(worst, float(np.max(np.abs(a - b)[big] / b[big])))
    print(prec, "max |g|^2 block rel err", worst)
    assert worst < (1e-8 if prec == "fp64" else 5e-3)


def test_wide_adjoint_reports_unsupported(epw):
    wm, rng = _wide_model("sc", 12, 4, 830)
    m = epw.Model(wm)
    with pytest.raises(epw.EPWError) as e:
        m.linewidth_backward(rng.random((2, 3)), rng.random((8, 3)), np.ones((2, 12)), T=300.0, EF=0.0, sigma=0.05)
    assert e.value.status == 6
