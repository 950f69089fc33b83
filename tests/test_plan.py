"""Workspace planning by shape alone (epw_plan_linewidth): CPU only, no model, no device.

The library lays out one device workspace per call and, when the buffers that grow with the
k list would pass EPW_K_SIDE_BYTES, runs the k list in equal passes over the whole q list.  The
pass is the longest whose plan exceeds the plan of one k by at most that budget; a staged
contraction chunk (capped by its own budget) counts once.  These tests pin those rules through
the planning entry point, which runs the same planners as the library's calls.
"""
import math
import os

import pytest

import paper_1604_03525_gb300 as epw

GiB = 1 << 30


class _Env:
    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        for k, v in self.kv.items():
            os.environ[k] = str(v)

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


def _plan(shape, nk, nq, prec=epw.BF16X3):
    nw, nat, nRe, nRp, same = shape
    return epw.plan_linewidth(nw, nat, nRe, nRp, nRe, nk, nq, prec, same_ep=same, same_eph=same)


DIAMOND_NW8 = (8, 2, 249, 249, True)     # the diamond nw=8 workload's model (wide fused form)
FCC_NW4 = (4, 1, 135, 135, True)         # the fcc nw=4 workload's model (narrow fused form)
FCC_NW12 = (12, 6, 135, 135, True)       # an uneven-batch system (staged form)
HEX_NW18 = (18, 6, 155, 233, False)      # an uneven-batch system, Re != Rp (staged form)


def test_benchmark_workloads_run_in_one_pass():
    ws, kpp = _plan(DIAMOND_NW8, 2000, 316000)
    assert kpp == 2000
    # at least the A operand of the wide form: 316,000 q x 512 K x (hi + lo) bf16
    assert ws > 316000 * 512 * 2 * 2
    ws2, kpp2 = _plan(FCC_NW4, 1000, 64000)
    assert kpp2 == 1000 and 0 < ws2 < ws


@pytest.mark.parametrize("shape,nk,nq", [(FCC_NW12, 1562, 46656), (HEX_NW18, 2187, 54872), (DIAMOND_NW8, 2000, 316000)])
def test_pass_is_the_longest_within_the_budget(shape, nk, nq):
    """kpp k fit the budget over the plan of one k; passes are equal (kpp = ceil(nk / npass)),
    and the shortest pass that would save one pass does not fit."""
    ws1, _ = _plan(shape, 1, nq)
    ws, kpp = _plan(shape, nk, nq)
    budget = 8 * GiB
    assert 1 <= kpp <= nk
    wsk, kppk = _plan(shape, kpp, nq)
    assert kppk == kpp and wsk - ws1 <= budget
    npass = math.ceil(nk / kpp)
    assert kpp == math.ceil(nk / npass)
    if npass > 1:
        fewer = math.ceil(nk / (npass - 1))
        assert _plan(shape, fewer, nq)[1] < fewer
        with _Env(EPW_K_SIDE_BYTES=0):  # its plan in one pass
            wsf, kppf = _plan(shape, fewer, nq)
        assert kppf == fewer and wsf - ws1 > budget


def test_staged_chunk_counts_once():
    """The staged contraction chunk of a wide shape grows with k up to its cap: measured as growth
    per k it would split this job into passes of a few k.  Its plan per k beyond the chunk is the
    k-side vertex alone, so the job takes at most two passes."""
    ws1, _ = _plan(FCC_NW12, 1, 46656)
    ws2, _ = _plan(FCC_NW12, 2, 46656)
    assert ws2 - ws1 > 512 << 20          # the chunk grows by ~1 GB per k at first
    _, kpp = _plan(FCC_NW12, 1562, 46656)
    assert math.ceil(1562 / kpp) <= 2


def test_budget_from_the_environment():
    with _Env(EPW_K_SIDE_BYTES=1):
        assert _plan(DIAMOND_NW8, 37, 300)[1] == 1
    with _Env(EPW_K_SIDE_BYTES=0):  # 0: no passes
        assert _plan(HEX_NW18, 2187, 54872)[1] == 2187
    with _Env(EPW_K_SIDE_BYTES=16 << 20):
        _, kpp = _plan(FCC_NW4, 1000, 64000)
        npass = math.ceil(1000 / kpp)
        assert npass > 1 and kpp == math.ceil(1000 / npass)


def test_workspace_grows_with_the_lists():
    prev = 0
    for nk in (1, 8, 64, 512):
        ws, kpp = _plan(FCC_NW4, nk, 64000)
        assert kpp == nk and ws >= prev
        prev = ws
    assert _plan(FCC_NW4, 64, 128000)[0] > _plan(FCC_NW4, 64, 64000)[0]


@pytest.mark.parametrize("prec", [epw.FP64, epw.FP32, epw.TF32X3, epw.BF16X3])
def test_every_precision_and_shape_plans(prec):
    for shape in (DIAMOND_NW8, FCC_NW4, FCC_NW12, HEX_NW18, (1, 1, 27, 27, True), (5, 3, 305, 305, True)):
        ws, kpp = _plan(shape, 50, 4096, prec)
        assert ws > 0 and 1 <= kpp <= 50


@pytest.mark.parametrize("args", [
    dict(nw=19, nat=1), dict(nw=0, nat=1), dict(nw=4, nat=7), dict(nw=4, nat=0),
    dict(nw=4, nat=1, nk=0), dict(nw=4, nat=1, nq=0), dict(nw=4, nat=1, nRe=0),
    dict(nw=4, nat=1, precision=9), dict(nw=4, nat=1, nRp=28, same_ep=True)])
def test_invalid_arguments(args):
    a = dict(nw=4, nat=1, nRe=27, nRp=27, nRph=27, nk=10, nq=100, precision=epw.BF16X3)
    a.update(args)
    with pytest.raises(epw.EPWError) as e:
        epw.plan_linewidth(**a)
    assert e.value.status == 1
