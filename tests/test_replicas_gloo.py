"""Replica host path (several processes, one realisation each) with two gloo ranks on CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1803_02132_gb300 import replicas

    # rank r is slower on the first timing and faster on the second
    t = replicas.max_over_ranks([10.0 + rank, 5.0 - rank], dist)
    out = {"B": np.full((2, 3, 3), float(rank)), "nmodes": np.arange(3, dtype=np.float64) + rank}
    got = replicas.gather_outputs(out, dist)
    dist.barrier()
    q.put((rank, t, None if got is None else [{k: v.tolist() for k, v in g.items()} for g in got]))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, t, got = q.get(timeout=120)
        res[r] = (t, got)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r][0] == [11.0, 5.0]  # the slowest rank's time on every rank
    assert res[1][1] is None
    got = res[0][1]
    assert [g["B"][0][0][0] for g in got] == [0.0, 1.0]  # rank order
    assert got[1]["nmodes"] == [1.0, 2.0, 3.0]


def test_single_process_passthrough():
    from paper_1803_02132_gb300 import replicas

    assert replicas.max_over_ranks([3, 4]) == [3.0, 4.0]
    assert replicas.gather_outputs({"B": [1.0]})[0]["B"] == [1.0]
    assert replicas.weak_scaling_rate(100, 500.0, 4) == pytest.approx(800.0)

