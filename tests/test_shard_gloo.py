"""k- and q-sharding of one linewidth problem, and of its adjoint, over two ranks (gloo, CPU processes).

The per-rank evaluation here is the CPU oracle, so the test covers the host
logic (slicing, weights, gather, rank-ordered compensated sums) without a GPU.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    import workloads as W
    from paper_1604_03525_gb300.shard import linewidth_sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(5)
    m = W.make_model("fcc", 2, 1, [1.0], 20, 20, rng)
    k = rng.random((7, 3))
    q = rng.random((23, 3))

    def compute(kk, qq, ww):
        return oracle.linewidth(m, kk, qq, ww, 300.0, 0.1, 0.1)

    res = linewidth_sharded(compute, k, q, None, mode=mode)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), res)
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["k", "q"])
def test_sharded_equals_unsharded(tmp_path, mode, oracle_lib):
    import workloads as W
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), mode, str(tmp_path)), nprocs=world, join=True)
    rng = np.random.default_rng(5)
    m = W.make_model("fcc", 2, 1, [1.0], 20, 20, rng)
    k = rng.random((7, 3))
    q = rng.random((23, 3))
    ref = oracle_lib.linewidth(m, k, q, None, 300.0, 0.1, 0.1)
    for r in range(world):
        got = np.load(tmp_path / f"r{r}.npy")
        assert got.shape == ref.shape
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)


def test_shard_bounds_cover_exactly():
    from paper_1604_03525_gb300.shard import shard_bounds
    for n in (0, 1, 5, 64, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1


def _bwd_worker(rank, world, port, mode, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    import workloads as W
    from paper_1604_03525_gb300.shard import linewidth_backward_sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, k, q, cot = _bwd_problem()

    def compute_bwd(kk, qq, cc, ww):
        return oracle.linewidth_grad(m, kk, qq, ww, 300.0, 0.1, 0.1, cot=cc)

    # a chunk smaller than the vertex so that the rank-ordered sum runs in several rounds
    import paper_1604_03525_gb300.shard as sh
    sh._CHUNK = 1000
    dg, dT, dE = linewidth_backward_sharded(compute_bwd, k, q, cot, None, mode=mode)
    np.save(os.path.join(out_dir, f"g{rank}.npy"), dg)
    np.save(os.path.join(out_dir, f"s{rank}.npy"), np.array([dT, dE]))
    dist.destroy_process_group()


def _bwd_problem():
    import workloads as W
    rng = np.random.default_rng(6)
    m = W.make_model("fcc", 2, 1, [1.0], 20, 24, rng)
    k = rng.random((5, 3))
    q = rng.random((19, 3))
    cot = rng.random((5, 2))
    return m, k, q, cot


@pytest.mark.parametrize("mode", ["k", "q"])
def test_sharded_adjoint_equals_unsharded(tmp_path, mode, oracle_lib):
    """dL/dg, dL/dT, dL/dE_F of the two shards, added in rank order, equal the unsharded adjoint."""
    world = 2
    mp.spawn(_bwd_worker, args=(world, _free_port(), mode, str(tmp_path)), nprocs=world, join=True)
    m, k, q, cot = _bwd_problem()
    rdg, rdT, rdE = oracle_lib.linewidth_grad(m, k, q, None, 300.0, 0.1, 0.1, cot=cot)
    g0 = np.load(tmp_path / "g0.npy")
    for r in range(world):
        dg = np.load(tmp_path / f"g{r}.npy")
        dT, dE = np.load(tmp_path / f"s{r}.npy")
        assert dg.shape == rdg.shape and dg.dtype == np.complex128
        assert np.array_equal(dg, g0)  # every rank holds the same sum
        assert np.abs(dg - rdg).max() <= 1e-12 * np.abs(rdg).max()
        assert abs(dT - rdT) <= 1e-12 * abs(rdT) and abs(dE - rdE) <= 1e-12 * abs(rdE)


def test_compensated_sum_in_rank_order():
    """The rank-ordered sum keeps the bits a plain FP64 sum drops: 1e16 + 1 - 1e16 = 1."""
    import torch
    from paper_1604_03525_gb300.shard import compensated_sum
    parts = [np.array([1e16, 0.1, 3.0]), np.array([1.0, 0.2, -3.0]), np.array([-1e16, 0.3, 1e-300])]
    got = compensated_sum(parts)
    assert got[0] == 1.0 and (1e16 + 1.0) - 1e16 != 1.0
    assert got[1] == 0.6000000000000001 or abs(got[1] - 0.6) <= 1e-16
    assert got[2] == 1e-300
    tgot = compensated_sum([torch.tensor(p) for p in parts])
    assert torch.equal(tgot, torch.tensor(got))
