"""Phonon-side sums over k (Pi''_qnu of Eq. linewidthph on shell, lambda_qnu of Eq. lambdaEQ,
the nesting function of Eq. nestingfct, N(E_F)) on the GPU against the FP64 oracle.

Errors: Pi'' normwise (max |error| / max |Pi''|, see _normwise), lambda and nesting entrywise
relative.  Tolerances: FP64 1e-9; FP32 2e-3; the split tensor-core forms 1e-3 (tf32x3) and
2e-3 (bf16x3) on these few-k sums (each (q, nu) sum rests on few k near the delta peaks, the
argument of the uneven-batch test), 6e-4 / 2e-3 on the 300-k sums of the benchmark model.  Relative
errors use a floor of 1e-6 of the largest value of each output.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 2e-3, "tf32x3": 1e-3, "bf16x3": 2e-3}


def _rel(got, ref):
    ref = np.asarray(ref, dtype=float)
    got = np.asarray(got, dtype=float)
    floor = 1e-6 * np.abs(ref).max() + 1e-300
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def _normwise(got, ref):
    """max |got - ref| / max |ref|: Pi'' sums terms of both signs (f_nk - f_mk+q changes sign
    inside the broadened delta), so single entries can cancel far below their terms and an
    entrywise relative error measures that cancellation, not the arithmetic."""
    ref = np.asarray(ref, dtype=float)
    return float(np.abs(np.asarray(got, dtype=float) - ref).max() / (np.abs(ref).max() + 1e-300))


def _errs(got, ref):
    return [_normwise(got[0], ref[0]), _rel(got[1], ref[1]), _rel(got[2], ref[2])]


@pytest.fixture(scope="module")
def epw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw
    return epw


def test_closed_form_model_fp64(epw, oracle_lib):
    m = W.tight_binding_model(eps0=0.2, t=0.5, K=0.01, g0=0.05, mass=1.3)
    rng = np.random.default_rng(900)
    k = W.uniform_grid(6) + 0.03
    q = rng.random((7, 3))
    ref = oracle_lib.phonon_self(m, k, q, None, 300.0, 0.1, 0.08)
    got = epw.Model(m).phonon_selfenergy(k, q, T=300.0, EF=0.1, sigma=0.08, precision=epw.FP64)
    assert max(_errs(got, ref)) < 1e-9
    assert abs(got[3] - ref[3]) <= 1e-12 * ref[3]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("lat,nw,nat,masses,nR", [("fcc", 4, 1, (1.0,), 40), ("diamond", 3, 2, (1.0, 1.2), 20),
                                                   ("hex", 5, 3, (1.0, 1.1, 1.2), 20)])
def test_random_models_match_oracle(epw, oracle_lib, lat, nw, nat, masses, nR, prec):
    rng = np.random.default_rng(910 + nw)
    wm = W.make_model(lat, nw, nat, list(masses), nR, nR, rng)
    k = W.uniform_grid(5) + rng.random(3) * 0.1
    wk = rng.random(len(k))
    wk /= wk.sum()
    q = np.concatenate([np.zeros((1, 3)), rng.random((12, 3))])  # Gamma: acoustic modes left out
    ref = oracle_lib.phonon_self(wm, k, q, wk, 300.0, 0.05, 0.1)
    m = epw.Model(wm)
    got = m.phonon_selfenergy(k, q, wk, T=300.0, EF=0.05, sigma=0.1, precision=epw.PRECISIONS[prec])
    errs = _errs(got, ref)
    print(lat, nw, 3 * nat, prec, "pi normwise / lambda, zeta max rel err", errs)
    assert max(errs) < TOL[prec]
    assert abs(got[3] - ref[3]) <= 1e-12 * ref[3]  # N(E_F) stays FP64 in every form
    assert np.all(got[0][0, :3] == 0) and np.all(got[1][0, :3] == 0)
    m.sync()


# Each (q, nu) sums 300 k with sigma = 20 meV, so it rests on the few k inside the delta
# windows: the ~1e-5 eV e_k+q error of the split contraction moves each Gaussian by ~1e-3
# and these sums by a few 1e-4 (tf32x3) / ~1e-3 (bf16x3), without the averaging of the
# 64,000-q electron-side sums.
@pytest.mark.parametrize("prec,tol", [("tf32x3", 6e-4), ("bf16x3", 2e-3)])
def test_benchmark_model_full_q_grid_sampled(epw, oracle_lib, prec, tol):
    """300 k of the fcc nw=4 workload over its whole 40^3 q grid on the device (the staged contraction
    runs in 3 chunks of k), checked against the oracle on sampled q (each q's sums are independent)."""
    import torch
    wl = W.make_workload("fcc_nw4")
    m = epw.Model(wl.model)
    k = wl.k[:300]
    pi, lam, zeta, dos = m.phonon_selfenergy(torch.tensor(k, device="cuda"), torch.tensor(wl.q, device="cuda"),
                                             T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=epw.PRECISIONS[prec])
    pi, lam, zeta = pi.cpu().numpy(), lam.cpu().numpy(), zeta.cpu().numpy()
    m.sync()
    idx = np.random.default_rng(920).choice(len(wl.q), 12, replace=False)
    ref = oracle_lib.phonon_self(wl.model, k, wl.q[idx], None, wl.T, wl.EF, wl.sigma)
    errs = _errs((pi[idx], lam[idx], zeta[idx]), ref)
    print(prec, "300 k x 40^3 q, sampled q: pi normwise / lambda, zeta max rel err", errs)
    assert max(errs) < tol
    assert abs(float(dos) - ref[3]) <= 1e-12 * ref[3]


def test_edge_cases(epw, oracle_lib):
    wm = W.make_model("sc", 2, 1, [1.0], None, None, np.random.default_rng(930), box=1)
    m = epw.Model(wm)
    k = W.uniform_grid(3)
    pi, lam, zeta, dos = m.phonon_selfenergy(k, np.zeros((0, 3)), T=300.0, EF=0.0, sigma=0.1)
    assert pi.shape == (0, 3) and zeta.shape == (0,)
    ref = oracle_lib.phonon_self(wm, k, np.zeros((1, 3)) + 0.3, None, 300.0, 0.0, 0.1)
    assert abs(dos - ref[3]) <= 1e-12 * ref[3]
    pi, lam, zeta, dos = m.phonon_selfenergy(np.zeros((0, 3)), np.random.default_rng(1).random((4, 3)), T=300.0,
                                             EF=0.0, sigma=0.1)
    assert np.all(pi == 0) and np.all(lam == 0) and np.all(zeta == 0) and dos == 0
    big = epw.Model(W.make_model("sc", 12, 1, [1.0], None, None, np.random.default_rng(931), box=1))
    with pytest.raises(epw.EPWError) as e:
        big.phonon_selfenergy(k, k, T=300.0, EF=0.0, sigma=0.1)
    assert e.value.status == 6


def test_eliashberg_function_pipeline(epw, oracle_lib):
    """omega from epw_interp_g, lambda from epw_phonon_selfenergy, alpha^2 F from epw_eliashberg, against the
    oracle's chain; host and device buffers."""
    import torch
    rng = np.random.default_rng(940)
    wm = W.make_model("fcc", 2, 1, [1.0], 40, 40, rng)
    k = W.uniform_grid(5) + 0.01
    q = W.uniform_grid(6)
    wq = np.full(len(q), 1.0 / len(q))
    m = epw.Model(wm)
    _, _, om, _ = m.interp(k[:1], q, precision=epw.FP64)
    _, lam, _, _ = m.phonon_selfenergy(k, q, T=300.0, EF=0.0, sigma=0.1, precision=epw.FP64)
    grid = np.linspace(0.0, 0.15, 301)
    got = epw.eliashberg(om, lam, grid, 0.004, wq)
    rom = oracle_lib.phonons(wm, q)[0]
    rlam = oracle_lib.phonon_self(wm, k, q, None, 300.0, 0.0, 0.1)[1]
    ref = oracle_lib.eliashberg(rom, rlam, grid, 0.004, wq)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.abs(ref).max()
    dev = epw.eliashberg(torch.tensor(om, device="cuda"), torch.tensor(lam, device="cuda"),
                         torch.tensor(grid, device="cuda"), 0.004).cpu().numpy()
    assert np.max(np.abs(dev - ref)) <= 1e-9 * np.abs(ref).max()
    assert np.all(ref >= 0) and ref.max() > 0
