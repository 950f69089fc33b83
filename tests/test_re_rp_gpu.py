"""Electron and phonon-displacement R sets that differ (Re != Rp) in the tensor-core forms.

g(Re, Rp) of Eq. (4) is indexed by two lattice-vector sets of their own, so the
contraction over R of Eq. (9) runs over Re (the electronic Fourier sum) and over
Rp (the phonon one) with different lengths.  The tensor-core forms lay the
contraction dimension out in two parts, [Re phases | zero pad | Rp phases], with
the Hamiltonian columns zero on the Rp part and the vertex columns zero on the Re
part (narrow fused and staged forms), or give the vertex MMAs an A operand of
their own (wide form).  Each form, and each entry point with a split form (the
linewidth, the interpolation, the adjoint, the phonon-side sums, the complex
self-energy), is checked against the FP64 oracle with Rp larger and smaller
than Re, at the tolerances of its Re = Rp tests.
"""
import numpy as np
import pytest

import workloads as W
from tests._util import degenerate_sums

pytestmark = pytest.mark.gpu


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


# (lattice, nw, nat, masses, Re shells, Rp shells, form)
CASES = [
    ("fcc", 4, 1, (1.0,), 24, 50, "fused"),
    ("sc", 2, 1, (1.0,), 40, 12, "fused"),
    ("fcc", 3, 1, (1.0,), 20, 45, "staged"),
    ("sc", 6, 2, (1.0, 1.3), 40, 20, "staged"),
    ("hex", 5, 3, (1.0, 1.1, 1.2), 20, 40, "wide"),
    ("diamond", 8, 2, (1.0, 1.2), 30, 18, "wide"),
]
TOL = {"fp64": 1e-9, "fp32": 2e-3, "tf32x3": 1e-4, "bf16x3": 6e-4}
# the wide form's few-q tolerances (FP32 eigensolve of H(k+q) per pair; a few hundred q)
TOL_WIDE = {"tf32x3": 3e-4, "bf16x3": 6e-4}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("lat,nw,nat,masses,nRe,nRp,form", CASES)
def test_linewidth_re_ne_rp(epw, oracle_lib, lat, nw, nat, masses, nRe, nRp, form, prec):
    rng = np.random.default_rng(1300 + 10 * nw + nat)
    wm = W.make_model(lat, nw, nat, list(masses), nRe, nRp, rng)
    assert len(wm.Re) != len(wm.Rp)
    k = rng.random((6, 3))
    q = rng.random((300, 3))  # ragged last q tile
    wq = rng.random(300) / 150.0
    m = epw.Model(wm)
    ref = oracle_lib.linewidth(wm, k, q, wq, 300.0, 0.1, 0.05)
    got = m.linewidth(k, q, wq, T=300.0, EF=0.1, sigma=0.05, precision=epw.PRECISIONS[prec])
    m.sync()
    err = _rel(got, ref)
    print(lat, nw, 3 * nat, len(wm.Re), len(wm.Rp), form, prec, "max rel err", err)
    tol = TOL_WIDE[prec] if (form == "wide" and prec in TOL_WIDE) else TOL[prec]
    assert np.all(got >= 0)
    assert err < tol


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("lat,nw,nat,masses,nRe,nRp,form", [c for c in CASES if c[-1] != "wide"])
def test_interp_re_ne_rp(epw, oracle_lib, lat, nw, nat, masses, nRe, nRp, form, prec):
    """eps_k+q and the vertex blocks |g|^2 (summed over degenerate subspaces) of the narrow
    fused and staged forms, whose K layout carries both R sets."""
    rng = np.random.default_rng(1350 + 10 * nw + nat)
    wm = W.make_model(lat, nw, nat, list(masses), nRe, nRp, rng)
    k = rng.random((3, 3))
    q = np.concatenate([np.zeros((1, 3)), rng.random((140, 3))])
    m = epw.Model(wm)
    ek, ekq, om, g = m.interp(k, q, precision=epw.PRECISIONS[prec])
    m.sync()
    rk, rkq, rom, rg = oracle_lib.interp(wm, k, q)
    assert np.abs(ek - rk).max() < 1e-10
    tol_e = 2e-5 if prec == "tf32x3" else 1e-4
    assert np.abs(ekq - rkq).max() < tol_e
    worst = 0.0
    for ik in range(len(k)):
        for iq in range(len(q)):
            a = degenerate_sums(np.abs(g[ik, iq]) ** 2, rkq[ik, iq], rk[ik], rom[iq], 1e-4)
            b = degenerate_sums(np.abs(rg[ik, iq]) ** 2, rkq[ik, iq], rk[ik], rom[iq], 1e-4)
            big = b > 1e-6 * b.max()
            if big.any():
                worst = max(worst, float(np.max(np.abs(a - b)[big] / b[big])))
    print(lat, nw, form, prec, "max eps err", np.abs(ekq - rkq).max(), "max |g|^2 block rel err", worst)
    assert worst < (2e-3 if prec == "tf32x3" else 1e-2)


# shapes with per-pair kernels for the adjoint and the phonon-side sums (nw <= 8, 3nat <= 9)
SMALL = [c for c in CASES if c[1] <= 8 and 3 * c[2] <= 9]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("lat,nw,nat,masses,nRe,nRp,form", SMALL)
def test_backward_re_ne_rp(epw, oracle_lib, lat, nw, nat, masses, nRe, nRp, form, prec):
    """dL/dg(Re, Rp) [nRe][nRp][3nat][nw][nw], dL/dT, dL/dE_F against the oracle gradient.  With
    Re != Rp the split forms recompute the forward through the staged contraction (both R
    sets in its K layout) for every shape."""
    rng = np.random.default_rng(1380 + 10 * nw + nat)
    wm = W.make_model(lat, nw, nat, list(masses), nRe, nRp, rng)
    k = rng.random((4, 3))
    q = rng.random((260, 3))
    cot = rng.random((4, nw))
    m = epw.Model(wm)
    dg, dT, dE = m.linewidth_backward(k, q, cot, T=300.0, EF=0.1, sigma=0.05, precision=epw.PRECISIONS[prec])
    m.sync()
    rdg, rdT, rdE = oracle_lib.linewidth_grad(wm, k, q, None, 300.0, 0.1, 0.05, cot=cot)
    assert dg.shape == rdg.shape == (len(wm.Re), len(wm.Rp), 3 * nat, nw, nw)
    eg = float(np.abs(dg - rdg).max() / np.abs(rdg).max())
    eT, eE = abs(dT - rdT) / abs(rdT), abs(dE - rdE) / abs(rdE)
    print(lat, nw, 3 * nat, form, prec, "adjoint dg", eg, "dT", eT, "dE_F", eE)
    tol = {"fp64": (1e-9, 1e-9), "fp32": (1e-3, 1e-3), "tf32x3": (2e-4, 1e-3), "bf16x3": (1e-3, 2e-3)}[prec]
    assert eg <= tol[0] and eT <= tol[0] and eE <= tol[1]


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("lat,nw,nat,masses,nRe,nRp,form", SMALL)
def test_phonon_side_re_ne_rp(epw, oracle_lib, lat, nw, nat, masses, nRe, nRp, form, prec):
    """Pi''_qnu (normwise), lambda_qnu and the nesting function (entrywise) against the oracle;
    tolerances of the Re = Rp phonon-side tests."""
    rng = np.random.default_rng(1400 + 10 * nw + nat)
    wm = W.make_model(lat, nw, nat, list(masses), nRe, nRp, rng)
    k = W.uniform_grid(5) + rng.random(3) * 0.1
    q = np.concatenate([np.zeros((1, 3)), rng.random((12, 3))])
    m = epw.Model(wm)
    got = m.phonon_selfenergy(k, q, T=300.0, EF=0.05, sigma=0.1, precision=epw.PRECISIONS[prec])
    m.sync()
    ref = oracle_lib.phonon_self(wm, k, q, None, 300.0, 0.05, 0.1)
    e_pi = float(np.abs(got[0] - ref[0]).max() / np.abs(ref[0]).max())
    e_lam, e_z = _rel(got[1], ref[1]), _rel(got[2], ref[2])
    print(lat, nw, 3 * nat, form, prec, "phonon side Pi'' / lambda / zeta", e_pi, e_lam, e_z)
    tol = {"fp64": 1e-9, "tf32x3": 1e-3, "bf16x3": 2e-3}[prec]
    assert max(e_pi, e_lam, e_z) < tol


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("lat,nw,nat,masses,nRe,nRp,form", SMALL)
def test_selfenergy_re_ne_rp(epw, oracle_lib, lat, nw, nat, masses, nRe, nRp, form, prec):
    """Complex Sigma_nk(omega) and A_nk(omega), normwise, against the oracle."""
    rng = np.random.default_rng(1420 + 10 * nw + nat)
    wm = W.make_model(lat, nw, nat, list(masses), nRe, nRp, rng, g_amp=0.03)
    k = rng.random((3, 3))
    q = rng.random((140, 3))
    omega = np.linspace(-0.6, 0.6, 25)
    m = epw.Model(wm)
    s, a = m.selfenergy(k, q, omega, T=300.0, EF=0.05, delta=0.04, precision=epw.PRECISIONS[prec])
    m.sync()
    ref_s, ref_a = oracle_lib.selfenergy(wm, k, q, omega, None, 300.0, 0.05, 0.04)
    es = float(np.abs(s - ref_s).max() / np.abs(ref_s).max())
    ea = float(np.abs(a - ref_a).max() / np.abs(ref_a).max())
    print(lat, nw, 3 * nat, form, prec, "Sigma / A normwise", es, ea)
    tol = {"fp64": 1e-9, "tf32x3": 1e-4, "bf16x3": 5e-4}[prec]
    assert max(es, ea) < tol
