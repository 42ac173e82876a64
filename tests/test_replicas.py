"""Multi-process host logic of the replica bench (two gloo ranks on CPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 17.25][rank]
    pairs = [1000, 3000][rank]
    q.put((rank, bench.reduce_across_ranks(ms, pairs, dist)))
    # replicas use different seeds: the workload generator gives distinct inputs per rank
    from paper_2603_24688_gb300 import workloads as W
    w = W.box_workload(n_dm=64, n_gas=64, seed=W.SEED_BASE + 1 + rank)
    q.put((rank, float(w["dm"]["pos"][0, 0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(4)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    red = [v for r, v in out if isinstance(v, tuple)]
    assert red == [(17.25, 4000.0), (17.25, 4000.0)]
    firsts = sorted(v for r, v in out if not isinstance(v, tuple))
    assert firsts[0] != firsts[1]


def test_single_process_is_identity():
    import bench
    assert bench.reduce_across_ranks(3.0, 7, None) == (3.0, 7.0)
