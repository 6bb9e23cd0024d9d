"""The multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1)
agree on the slowest rank's time and on the whole-job rate, and draw disjoint
walker shards (weak scaling, no data-path collective)."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)   # rank 1 is the slow one
    rate = bench.whole_job_rate(world, 64, 3, ms / 1e3)
    out.put((rank, ms, rate, bench.walker_first(rank, 64)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_time_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert all(abs(r[2] - 2 * 64 * 3 / 0.015) < 1e-6 for r in res)
    assert [r[3] for r in res] == [0, 64]


def test_walker_shards_are_distinct():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2202_00832_b300 import synth
    mol = synth.CHAIN_60.molecule()
    a = synth.CHAIN_60.walkers(mol, W=2, first=bench.walker_first(0, 2), processes=1)
    b = synth.CHAIN_60.walkers(mol, W=2, first=bench.walker_first(1, 2), processes=1)
    assert not np.allclose(a, b)
