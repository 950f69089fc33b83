"""Adjoint through torch.autograd: against the oracle gradient and central finite differences (FP64)."""
import numpy as np
import pytest

import workloads as W
from tests._util import fermi_level_term_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw
    rng = np.random.default_rng(11)
    wm = W.make_model("sc", 2, 1, [1.0], None, None, rng, box=1, omega_max=0.2)
    k = rng.random((4, 3))
    q = rng.random((160, 3))
    cot = rng.random((4, 2))
    return epw, wm, k, q, cot


def test_autograd_matches_oracle_gradient(setup, oracle_lib):
    import torch
    from paper_1604_03525_gb300.autograd import linewidth
    epw, wm, k, q, cot = setup
    m = epw.Model(wm)
    g = torch.tensor(wm.g, device="cuda", requires_grad=True)
    T = torch.tensor(300.0, dtype=torch.float64, device="cuda", requires_grad=True)
    EF = torch.tensor(0.2, dtype=torch.float64, device="cuda", requires_grad=True)
    kt, qt = torch.tensor(k, device="cuda"), torch.tensor(q, device="cuda")
    out = linewidth(m, g, T, EF, kt, qt, sigma=0.2)
    L = (out * torch.tensor(cot, device="cuda")).sum()
    L.backward()
    rdg, rdT, rdE = oracle_lib.linewidth_grad(wm, k, q, None, 300.0, 0.2, 0.2, cot=cot)
    assert np.abs(g.grad.cpu().numpy() - rdg).max() <= 1e-9 * np.abs(rdg).max()
    assert abs(T.grad.item() - rdT) <= 1e-9 * abs(rdT)
    assert abs(EF.grad.item() - rdE) <= 1e-9 * abs(rdE)


def test_autograd_directional_finite_differences(setup):
    import torch
    from paper_1604_03525_gb300.autograd import linewidth
    epw, wm, k, q, cot = setup
    m = epw.Model(wm)
    kt, qt, ct = torch.tensor(k, device="cuda"), torch.tensor(q, device="cuda"), torch.tensor(cot, device="cuda")
    g0 = torch.tensor(wm.g, device="cuda")
    rng = np.random.default_rng(12)
    d = torch.tensor(rng.standard_normal(wm.g.shape) + 1j * rng.standard_normal(wm.g.shape), device="cuda")

    def L(g, T=300.0, EF=0.2):
        Tt = torch.tensor(T, dtype=torch.float64, device="cuda")
        Et = torch.tensor(EF, dtype=torch.float64, device="cuda")
        return float((linewidth(m, g, Tt, Et, kt, qt, sigma=0.2) * ct).sum())

    g = g0.clone().requires_grad_(True)
    Tt = torch.tensor(300.0, dtype=torch.float64, device="cuda", requires_grad=True)
    Et = torch.tensor(0.2, dtype=torch.float64, device="cuda", requires_grad=True)
    (linewidth(m, g, Tt, Et, kt, qt, sigma=0.2) * ct).sum().backward()
    h = 1e-6
    fd = (L(g0 + h * d) - L(g0 - h * d)) / (2 * h)
    an = float((g.grad.conj() * d).real.sum())
    assert abs(fd - an) <= 1e-6 * abs(an)
    fdT = (L(g0, T=300.0 + 1e-3) - L(g0, T=300.0 - 1e-3)) / 2e-3
    assert abs(fdT - Tt.grad.item()) <= 1e-6 * abs(fdT)
    fdE = (L(g0, EF=0.2 + 1e-6) - L(g0, EF=0.2 - 1e-6)) / 2e-6
    assert abs(fdE - Et.grad.item()) <= 1e-6 * abs(fdE)


@pytest.mark.parametrize("nw,nR", [(4, 40), (2, 30), (1, 27)])
def test_tensor_core_adjoint_matches_oracle(nw, nR, oracle_lib):
    """TF32x3 adjoint (fused recompute + tcgen05 q-contraction) against the FP64 oracle gradient."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw
    rng = np.random.default_rng(40 + nw)
    lat = "sc" if nw == 1 else "fcc"
    wm = W.make_model(lat, nw, 1, [1.0], nR, nR, rng)
    k = rng.random((5, 3))
    q = rng.random((300, 3))
    cot = rng.random((5, nw))
    m = epw.Model(wm)
    dg, dT, dE = m.linewidth_backward(k, q, cot, T=300.0, EF=0.1, sigma=0.05, precision=epw.TF32X3)
    rdg, rdT, rdE = oracle_lib.linewidth_grad(wm, k, q, None, 300.0, 0.1, 0.05, cot=cot)
    assert np.abs(dg - rdg).max() <= 2e-4 * np.abs(rdg).max()
    assert abs(dT - rdT) <= 2e-4 * abs(rdT)
    # dL/dE_F weights each pair by df/dE_F (d+ - d-); the kernels form d+ - d- as
    # -2 e^-(x^2 + w^2)/sigma^2 sinh(2xw/sigma^2), so each term keeps the forward's relative
    # error (no cancellation for soft modes).  The terms change sign with e_nk - e_mk+q and
    # their sum cancels (here by up to ~1300x against the sum of their magnitudes), so the
    # bound is on the error against that magnitude.
    scale = fermi_level_term_scale(oracle_lib, wm, k, q, None, 300.0, 0.1, 0.05, cot)
    print("fused TF32x3 adjoint nw", nw, "dT", abs(dT - rdT) / abs(rdT), "dE_F", abs(dE - rdE) / abs(rdE),
          "against the term magnitude", abs(dE - rdE) / scale, "cancellation", scale / abs(rdE))
    assert abs(dE - rdE) <= 1e-4 * scale


def test_tensor_core_adjoint_chunks_at_benchmark_q():
    """Benchmark model and 40^3 q grid, 100 k (three k chunks): TF32x3 adjoint vs the FP32 SIMT adjoint."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw
    wl = W.make_workload("fcc_nw4")
    m = epw.Model(wl.model)
    k = torch.tensor(wl.k[:100], device="cuda")
    q = torch.tensor(wl.q, device="cuda")
    wq = torch.tensor(wl.wq, device="cuda")
    cot = torch.ones((100, 4), dtype=torch.float64, device="cuda")
    a = m.linewidth_backward(k, q, cot, wq, T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=epw.TF32X3)
    b = m.linewidth_backward(k, q, cot, wq, T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=epw.FP32)
    ga, gb = a[0].cpu().numpy(), b[0].cpu().numpy()
    assert np.abs(ga - gb).max() <= 1e-3 * np.abs(gb).max()
    assert abs(a[1] - b[1]) <= 1e-3 * abs(b[1])
    print("benchmark q: TF32x3 vs FP32 adjoint dT", abs(a[1] - b[1]) / abs(b[1]), "dE_F", abs(a[2] - b[2]) / abs(b[2]))
    assert abs(a[2] - b[2]) <= 1e-3 * abs(b[2])  # see the E_F note above
