"""Complex electron self-energy (Eq. elselfenergy) and spectral function (Eq. spectral_funct) on the GPU
against the FP64 oracle.

Errors are normwise per output (max |error| / max |value|): the real part of Sigma sums terms of both
signs and the spectral function is steep near its peaks.  Tolerances: FP64 1e-9; FP32 and TF32x3 1e-4;
BF16x3 5e-4 (e_k+q carries ~1e-6 / 1e-5 eV against Lorentzian widths of 30-40 meV: ~1e-5 / 1e-4 per
term; observed 5e-6 and 6e-5).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-4, "tf32x3": 1e-4, "bf16x3": 5e-4}


def _nw_err(got, ref):
    return float(np.abs(np.asarray(got) - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def epw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw
    return epw


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("lat,nw,nat,masses,nR", [("fcc", 4, 1, (1.0,), 40), ("diamond", 3, 2, (1.0, 1.2), 20),
                                                   ("hex", 5, 3, (1.0, 1.1, 1.2), 20)])
def test_selfenergy_matches_oracle(epw, oracle_lib, lat, nw, nat, masses, nR, prec):
    rng = np.random.default_rng(950 + nw)
    wm = W.make_model(lat, nw, nat, list(masses), nR, nR, rng, g_amp=0.03)
    k = rng.random((3, 3))
    q = rng.random((140, 3))  # two q blocks, the second ragged (and a ragged last warp)
    omega = np.linspace(-0.6, 0.6, 25)
    ref_s, ref_a = oracle_lib.selfenergy(wm, k, q, omega, None, 300.0, 0.05, 0.04)
    m = epw.Model(wm)
    s, a = m.selfenergy(k, q, omega, T=300.0, EF=0.05, delta=0.04, precision=epw.PRECISIONS[prec])
    es, ea = _nw_err(s, ref_s), _nw_err(a, ref_a)
    print(lat, nw, 3 * nat, prec, "Sigma / A normwise err", es, ea)
    assert max(es, ea) < TOL[prec]
    m.sync()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_many_k_in_chunks_sampled(epw, oracle_lib, prec):
    """2100 k x 20^3 q: the partial sums (and the staged contraction) run in several k chunks."""
    import torch
    rng = np.random.default_rng(960)
    wm = W.make_model("fcc", 4, 1, [1.0], 40, 40, rng, g_amp=0.03)
    k = rng.random((2100, 3))
    q = W.uniform_grid(20)
    omega = np.linspace(-0.5, 0.5, 32)
    m = epw.Model(wm)
    s, a = m.selfenergy(torch.tensor(k, device="cuda"), torch.tensor(q, device="cuda"), torch.tensor(omega, device="cuda"),
                        T=300.0, EF=0.0, delta=0.03, precision=epw.PRECISIONS[prec])
    s, a = s.cpu().numpy(), a.cpu().numpy()
    m.sync()
    idx = np.array([0, 1500, 2099])
    ref_s, ref_a = oracle_lib.selfenergy(wm, k[idx], q, omega, None, 300.0, 0.0, 0.03)
    es, ea = _nw_err(s[idx], ref_s), _nw_err(a[idx], ref_a)
    print(prec, "2100 k chunked, sampled k: Sigma / A normwise err", es, ea)
    assert max(es, ea) < TOL[prec]


def test_spectral_function_normalised_on_gpu(epw):
    """int A_nk(w) dw = 1 (a property at any size), FP64 form, weak coupling, +-40 eV grid."""
    rng = np.random.default_rng(91)
    wm = W.make_model("fcc", 2, 1, [1.0], 20, 20, rng, g_amp=0.01)
    k = rng.random((2, 3))
    q = W.uniform_grid(3) + 0.05
    omega = np.linspace(-40.0, 40.0, 160001)
    _, a = epw.Model(wm).selfenergy(k, q, omega, T=300.0, EF=0.0, delta=0.05, precision=epw.FP64)
    norm = np.trapezoid(a, omega, axis=-1)
    assert np.all(np.abs(norm - 1.0) < 1e-5), norm
