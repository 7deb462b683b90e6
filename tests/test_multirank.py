"""The multi-rank path of bench.py on CPU with the gloo backend, world size 2:
max-over-ranks timing, independent shards per rank and whole-job aggregation
(no collective touches the data path)."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import grid_inputs as gi
    sec = 1.0 + 0.5 * rank                     # rank 1 is the slow one
    m = bench.max_over_ranks(sec, dist, device="cpu")
    q, _, _ = gi.states(7, 16, bench.rank_seed(rank))
    out[rank] = (m, bench.aggregate_value(world, 1000, 10, m), float(q[0, 0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_sharding():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.5                 # both ranks report the max
    assert np.isclose(res[0][1], 2 * 1000 * 10 / 1.5)   # all ranks' work over the slowest time
    assert res[0][2] != res[1][2]                        # independent shards
