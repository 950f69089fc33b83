"""Failure detection on the GPU without a fault: a bounded device wait that runs out reports
EPW_ERR_TIMEOUT through the status path, and the context keeps working afterwards."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(oracle_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw
    from paper_1604_03525_gb300 import _lib
    lib = _lib.load()
    w = ctypes.c_int(0)
    st = lib.epw_selftest_wait_timeout(2000000, ctypes.byref(w))  # ~1 ms of clock
    assert st == 5 and w.value == 1  # EPW_ERR_TIMEOUT, the wait gave up
    assert b"bounded wait" in lib.epw_last_error()
    # the context is intact: a normal tensor-core call right after matches the oracle
    wl = W.make_workload("sc_nw1")
    m = epw.Model(wl.model)
    got = m.linewidth(wl.k[:16], wl.q, wl.wq, T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=epw.TF32X3)
    ref = oracle_lib.linewidth(wl.model, wl.k[:16], wl.q, wl.wq, wl.T, wl.EF, wl.sigma)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.abs(ref).max()
    m.sync()
