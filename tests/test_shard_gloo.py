"""k- and q-sharding of one linewidth problem over two ranks (gloo, CPU processes).

The per-rank evaluation here is the CPU oracle, so the test covers the host
logic (slicing, weights, gather, rank-ordered sum) without a GPU.
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
