"""Long-range (polar) vertex on the GPU against the FP64 oracle: every entry point adds
g^L = i C_nu(q) [U_k+q^dagger U_k] to the interpolated vertex (Eq. long-range)."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from tests._util import degenerate_sums

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 2e-3, "tf32x3": 1e-3, "bf16x3": 2e-3}


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


def _polar_model(lat, nw, nat, nR, seed, pref=0.05):
    rng = np.random.default_rng(seed)
    wm = W.make_model(lat, nw, nat, [1.0 + 0.15 * i for i in range(nat)], nR, nR, rng)
    pol = W.models.polar_terms(lat, nat, rng, prefactor=pref, gmax=2)
    if nat == 1:  # one atom: give it a charge so that the term is not zero
        pol = dataclasses.replace(pol, Zstar=np.array([[[1.3, 0.2, 0.0], [0.1, 0.9, -0.3], [0.0, 0.4, 1.1]]]))
    return dataclasses.replace(wm, polar=pol), rng


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("lat,nw,nat,nR", [("fcc", 4, 1, 40), ("diamond", 3, 2, 20), ("hex", 9, 3, 20)])
def test_polar_linewidth_matches_oracle(epw, oracle_lib, lat, nw, nat, nR, prec):
    wm, rng = _polar_model(lat, nw, nat, nR, 1000 + nw, pref=3.0)
    k = rng.random((4, 3))
    q = rng.random((200, 3))
    ref = oracle_lib.linewidth(wm, k, q, None, 300.0, 0.1, 0.06)
    short = oracle_lib.linewidth(dataclasses.replace(wm, polar=None), k, q, None, 300.0, 0.1, 0.06)
    assert np.abs(ref - short).max() > 3e-3 * np.abs(short).max()  # the term matters here
    m = epw.Model(wm)
    got = m.linewidth(k, q, T=300.0, EF=0.1, sigma=0.06, precision=epw.PRECISIONS[prec])
    err = _rel(got, ref)
    print(lat, nw, 3 * nat, prec, "polar linewidth max rel err", err)
    assert err < TOL[prec]
    m.sync()


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_polar_interp_vertex(epw, oracle_lib, prec):
    wm, rng = _polar_model("fcc", 4, 1, 40, 1010)
    k = rng.random((2, 3))
    q = np.concatenate([rng.random((20, 3)), 1e-3 * rng.random((2, 3))])  # includes small q (large g^L)
    m = epw.Model(wm)
    ek, ekq, om, g = m.interp(k, q, precision=epw.PRECISIONS[prec])
    rk, rkq, rom, rg = oracle_lib.interp(wm, k, q)
    worst = 0.0
    for ik in range(len(k)):
        for iq in range(len(q)):
            a = degenerate_sums(np.abs(g[ik, iq]) ** 2, rkq[ik, iq], rk[ik], rom[iq], 1e-4)
            b = degenerate_sums(np.abs(rg[ik, iq]) ** 2, rkq[ik, iq], rk[ik], rom[iq], 1e-4)
            big = b > 1e-6 * b.max()
            if big.any():
                worst = max(worst, float(np.max(np.abs(a - b)[big] / b[big])))
    print(prec, "polar |g|^2 block max rel err", worst)
    assert worst < (1e-9 if prec == "fp64" else 2e-3)


def test_polar_other_entry_points_fp64(epw, oracle_lib):
    wm, rng = _polar_model("diamond", 3, 2, 20, 1020)
    m = epw.Model(wm)
    k = W.uniform_grid(4) + 0.02
    q = rng.random((9, 3))
    # phonon side
    got = m.phonon_selfenergy(k, q, T=300.0, EF=0.0, sigma=0.1, precision=epw.FP64)
    ref = oracle_lib.phonon_self(wm, k, q, None, 300.0, 0.0, 0.1)
    assert np.abs(got[0] - ref[0]).max() <= 1e-9 * np.abs(ref[0]).max()
    assert _rel(got[1], ref[1]) < 1e-9 and _rel(got[2], ref[2]) < 1e-9
    # complex self-energy
    omega = np.linspace(-0.4, 0.4, 9)
    s, a = m.selfenergy(k[:3], q, omega, T=300.0, EF=0.0, delta=0.05, precision=epw.FP64)
    rs, ra = oracle_lib.selfenergy(wm, k[:3], q, omega, None, 300.0, 0.0, 0.05)
    assert np.abs(s - rs).max() <= 1e-9 * np.abs(rs).max()
    # adjoint (g^L does not depend on g(Re,Rp); it enters through |g|^2)
    cot = rng.random((3, 3))
    dg, dT, dE = m.linewidth_backward(k[:3], q, cot, T=300.0, EF=0.0, sigma=0.1, precision=epw.FP64)
    rdg, rdT, rdE = oracle_lib.linewidth_grad(wm, k[:3], q, None, 300.0, 0.0, 0.1, cot=cot)
    assert np.abs(dg - rdg).max() <= 1e-9 * np.abs(rdg).max()
    assert abs(dT - rdT) <= 1e-9 * abs(rdT) and abs(dE - rdE) <= 1e-9 * abs(rdE)


def test_polar_tensor_core_adjoint(epw, oracle_lib):
    wm, rng = _polar_model("fcc", 4, 1, 40, 1030)
    k = rng.random((5, 3))
    q = rng.random((300, 3))
    cot = rng.random((5, 4))
    m = epw.Model(wm)
    dg, dT, dE = m.linewidth_backward(k, q, cot, T=300.0, EF=0.1, sigma=0.05, precision=epw.TF32X3)
    rdg, rdT, rdE = oracle_lib.linewidth_grad(wm, k, q, None, 300.0, 0.1, 0.05, cot=cot)
    assert np.abs(dg - rdg).max() <= 2e-4 * np.abs(rdg).max()
    assert abs(dT - rdT) <= 2e-4 * abs(rdT)
    print("polar TF32x3 adjoint dE_F", abs(dE - rdE) / abs(rdE))
    assert abs(dE - rdE) <= 1e-3 * abs(rdE)
