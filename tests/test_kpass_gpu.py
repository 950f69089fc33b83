"""Linewidth in k passes: large k lists run in equal passes under a byte budget.

Im Sigma_nk of Eq. (linewidthel) is independent for every k, and each k's sum over q
is formed in the same order whatever other k share its pass, so a call run in
passes (EPW_K_SIDE_BYTES forced down to one k per pass, or to a few passes) must
give the one-pass result bit for bit, in every form: the fused narrow kernel, the
wide-shape kernel, the staged form and the SIMT forms, host and device buffers,
single calls and batches.
"""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def epw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03525_gb300 as epw
    return epw


class _Budget:
    def __init__(self, nbytes):
        self.nbytes = nbytes

    def __enter__(self):
        os.environ["EPW_K_SIDE_BYTES"] = str(self.nbytes)

    def __exit__(self, *a):
        del os.environ["EPW_K_SIDE_BYTES"]


SHAPES = [("fcc", 4, 1, (1.0,), 30, "fused"), ("diamond", 8, 2, (1.0, 1.2), 20, "wide"),
          ("sc", 6, 2, (1.0, 1.3), 27, "staged")]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "fp32", "fp64"])
@pytest.mark.parametrize("lat,nw,nat,masses,nR,form", SHAPES)
def test_passes_equal_one_pass(epw, lat, nw, nat, masses, nR, form, prec):
    """Budgets of 1 byte (one k per pass), 1 MiB and 16 MiB (a few passes of unequal counts,
    depending on the form's bytes per k) against the one-pass call."""
    import torch
    rng = np.random.default_rng(1600 + nw)
    wm = W.make_model(lat, nw, nat, list(masses), nR, nR, rng)
    k = rng.random((37, 3))
    q = rng.random((300, 3))
    m = epw.Model(wm)
    kw = dict(T=300.0, EF=0.1, sigma=0.05, precision=epw.PRECISIONS[prec])
    one = m.linewidth(k, q, **kw)
    kd, qd = torch.tensor(k, device="cuda"), torch.tensor(q, device="cuda")
    for budget in (1, 1 << 20, 1 << 24):
        with _Budget(budget):
            host = m.linewidth(k, q, **kw)
            dev = m.linewidth(kd, qd, **kw).cpu().numpy()
        m.sync()
        assert np.array_equal(one, host), (form, prec, budget)
        assert np.array_equal(one, dev), (form, prec, budget)
    m.close()


def test_batch_jobs_in_passes_equal_single_calls(epw):
    import torch
    rng = np.random.default_rng(1650)
    models = [epw.Model(W.make_model("fcc", 4, 1, [1.0], 30, 30, rng)),
              epw.Model(W.make_model("diamond", 8, 2, [1.0, 1.2], 20, 20, rng)),
              epw.Model(W.make_model("sc", 6, 2, [1.0, 1.3], 27, 27, rng))]
    jobs = []
    for i, m in enumerate(models):
        k = torch.tensor(rng.random((29 + 5 * i, 3)), device="cuda")
        q = torch.tensor(rng.random((200 + 50 * i, 3)), device="cuda")
        jobs.append(dict(model=m, k=k, q=q, wq=None, T=300.0, EF=0.1, sigma=0.05, precision=epw.BF16X3))
    ref = [m.linewidth(j["k"], j["q"], T=300.0, EF=0.1, sigma=0.05, precision=epw.BF16X3).cpu().numpy()
           for m, j in zip(models, jobs)]
    with _Budget(1):
        b = epw.Batch(jobs)
        outs = [o.cpu().numpy() for o in b.run()]
    torch.cuda.synchronize()
    for r, o in zip(ref, outs):
        assert np.array_equal(r, o)
    b.close()
    for m in models:
        m.sync()
