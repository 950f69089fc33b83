"""epw_linewidth_noalloc, the entry point for callers that cannot allocate device memory.

Some callers run where they must not call cudaMalloc (a host framework that
owns all device memory through its own pool, a loop that must never block on
the allocator).  epw_linewidth_noalloc serves them from one fixed scratch array
inside the library.  This test calls it through the C ABI twice in a row, on
different inputs, and checks each result against epw_linewidth (the same
FP64 tolerance as the other parity tests), so stale scratch contents from the
first call cannot leak into the second.  It is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-6  # FP64 path, as in test_parity_gpu.py


def _rel(got, ref):
    floor = 1e-6 * np.abs(ref).max()
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def test_noalloc_matches_linewidth_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw

    wl = W.make_workload("sc_nw1")
    m = epw.Model(wl.model)
    dev = "cuda"
    calls = [
        (wl.k, wl.q, wl.wq, 300.0, 0.0, 0.05),                # full 8^3 x 8^3
        (wl.k[::5] + 0.013, wl.q[:300], None, 77.0, 0.1, 0.03),  # different shapes and parameters
    ]
    for kk, qq, ww, T, EF, s in calls:
        kt = torch.tensor(kk, device=dev)
        qt = torch.tensor(qq, device=dev)
        wt = None if ww is None else torch.tensor(ww, device=dev)
        ref = m.linewidth(kt, qt, wt, T=T, EF=EF, sigma=s, precision=epw.FP64).cpu().numpy()
        out = torch.full((len(kk), 1), float("nan"), dtype=torch.float64, device=dev)
        got = m.linewidth_noalloc(kt, qt, wt, T=T, EF=EF, sigma=s, precision=epw.FP64, out=out)
        m.sync()
        got = got.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < TOL


def test_noalloc_rejects_oversized_and_host_inputs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw

    wl = W.make_workload("sc_nw1")
    m = epw.Model(wl.model)
    kt = torch.tensor(wl.k, device="cuda")
    big_q = torch.rand((200000, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(epw.EPWError) as e:
        m.linewidth_noalloc(kt, big_q, T=300.0, EF=0.0, sigma=0.05)
    assert e.value.status == 1 and "scratch" in str(e.value)
    with pytest.raises(epw.EPWError):
        m.linewidth_noalloc(wl.k, wl.q, T=300.0, EF=0.0, sigma=0.05, out=torch.empty((512, 1), dtype=torch.float64,
                                                                                     device="cuda"))
