"""Adjoint of the linewidth on the hexagonal nw=5, 9-mode model with its full R set.

L = sum_nk c_nk Im Sigma_nk (Eq. linewidthel); epw_linewidth_backward returns
dL/dg(Re, Rp) (305 x 305 x 9 x 5 x 5 complex, 335 MB), dL/dT and dL/dE_F.  The
whole vertex enters, so the model is the benchmark's at full size; k and q are
reduced (3 k of its list x 64 of its q) so that the oracle gradient takes seconds;
T = 300 K and E_F inside the sampled bands so that every derivative is far from zero.
Checks: every precision against the oracle gradient, and the FP64 GPU form
against central finite differences of the FP64 GPU linewidth at h = 1e-6 (L is
quadratic in each entry of g, so the difference quotient is exact up to rounding).
"""
import numpy as np
import pytest

import workloads as W
from tests._util import fermi_level_term_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def epw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw
    return epw


@pytest.fixture(scope="module")
def hex_problem(oracle_lib):
    """The workload's model and sigma; T = 300 K and E_F at the median band energy of the sampled
    k+q, so that df/dE_F reaches many terms (at the workload's 50 K and E_F = 0 the sampled
    states sit so far from E_F that dL/dE_F underflows to ~1e-14)."""
    wl = W.make_workload("hex_nw5")
    rng = np.random.default_rng(1500)
    k = wl.k[[0, 1234, 6001]]
    q = wl.q[np.sort(rng.choice(len(wl.q), 64, replace=False))]
    cot = rng.random((3, wl.model.nw))
    ekq, _ = oracle_lib.bands(wl.model, (k[:, None, :] + q[None, :, :]).reshape(-1, 3))
    par = dict(T=300.0, EF=float(np.median(ekq)), sigma=wl.sigma)
    ref = oracle_lib.linewidth_grad(wl.model, k, q, None, par["T"], par["EF"], par["sigma"], cot=cot)
    scale = fermi_level_term_scale(oracle_lib, wl.model, k, q, None, par["T"], par["EF"], par["sigma"], cot)
    return wl, k, q, cot, par, ref, scale


# dg: max-abs error relative to max |dg|; dT, dE: relative.  The split forms carry the
# FP32 eigensolve and contraction error of the forward (about 1e-5 eV in e_k+q).
TOL = {"fp64": (1e-9, 1e-9, 1e-9), "fp32": (1e-3, 1e-3, 1e-3), "tf32x3": (2e-4, 2e-4, 1e-3),
       "bf16x3": (5e-4, 5e-4, 2e-3)}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_hex_adjoint_matches_oracle(epw, hex_problem, prec):
    wl, k, q, cot, par, (rdg, rdT, rdE), scale = hex_problem
    m = epw.Model(wl.model)
    dg, dT, dE = m.linewidth_backward(k, q, cot, **par, precision=epw.PRECISIONS[prec])
    m.sync()
    eg = float(np.abs(dg - rdg).max() / np.abs(rdg).max())
    eT, eE = abs(dT - rdT) / abs(rdT), abs(dE - rdE) / abs(rdE)
    print("hex nw=5 adjoint", prec, "dg", eg, "dT", eT, "dE_F", eE, "(against the term magnitude",
          abs(dE - rdE) / scale, ", cancellation", scale / abs(rdE), ")")
    tg, tT, tE = TOL[prec]
    assert eg <= tg and eT <= tT and abs(dE - rdE) <= tE * max(abs(rdE), 1e-2 * scale)
    m.close()


def test_hex_adjoint_matches_finite_differences(epw, hex_problem):
    import torch
    wl, k, q, cot, par, (rdg, _, _), _ = hex_problem
    m = epw.Model(wl.model)
    kw = dict(**par, precision=epw.FP64)
    dg, dT, dE = m.linewidth_backward(k, q, cot, **kw)
    g = torch.tensor(wl.model.g, device="cuda")

    def L(gv, **over):
        m.set_vertex(gv)
        out = m.linewidth(k, q, **{**kw, **over})
        return float((out * cot).sum())

    h = 1e-6
    flat = np.abs(rdg).ravel()
    rng = np.random.default_rng(1501)
    picks = list(np.argsort(flat)[-3:]) + list(rng.choice(np.flatnonzero(flat > 1e-2 * flat.max()), 3))
    scale = np.abs(dg).max()
    for fi in picks:
        idx = np.unravel_index(int(fi), rdg.shape)
        for unit in (1.0, 1j):
            gp, gm = g.clone(), g.clone()
            gp[idx] += h * unit
            gm[idx] -= h * unit
            fd = (L(gp) - L(gm)) / (2 * h)
            an = dg[idx].real if unit == 1.0 else dg[idx].imag
            assert abs(fd - an) <= 1e-6 * scale, (idx, unit, fd, an)
    m.set_vertex(g)
    fdT = (L(g, T=par["T"] + 1e-3) - L(g, T=par["T"] - 1e-3)) / 2e-3
    fdE = (L(g, EF=par["EF"] + 1e-6) - L(g, EF=par["EF"] - 1e-6)) / 2e-6
    print("hex nw=5 FD: dT", dT, fdT, "dE_F", dE, fdE)
    assert abs(fdT - dT) <= 1e-5 * abs(dT)
    assert abs(fdE - dE) <= 1e-5 * abs(dE)
    m.close()
