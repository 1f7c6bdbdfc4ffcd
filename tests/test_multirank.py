"""Multi-rank paths on CPU ranks (gloo, world_size 2): the batched workload
is sharded over ranks by instance (no exchange on the data path) and the
whole-job rate uses the slowest rank's time."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from paper_1909_07439_gb300 import inputs  # noqa: E402


def test_shard_instances_is_a_balanced_partition():
    sides = inputs.batch_sizes(512, seed=4)
    sizes = sides ** 3
    for ws in (1, 2, 3, 8):
        parts = bench.shard_instances(sizes, ws)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(512))
        loads = [int(sizes[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= int(sizes.max())


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sides = inputs.batch_sizes(40, seed=9, nmin=64, nmax=4096)
    mine = bench.shard_instances(sides ** 3, ws)[rank]
    w, off = inputs.sedov_batch(40, seed=9, only=mine, nmin=64, nmax=4096)
    local_ms = 10.0 * (rank + 1)

    def _max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    value, ms = bench.aggregate(local_ms, 1000, ws, _max)
    n = torch.tensor([w.n], dtype=torch.int64)
    dist.all_reduce(n)
    out[rank] = (value, ms, int(n.item()), sorted(mine))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ws = 2
    port = 29500 + os.getpid() % 1000
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    sides = inputs.batch_sizes(40, seed=9, nmin=64, nmax=4096)
    total = int((sides ** 3).sum())
    for r in range(ws):
        value, ms, n_all, mine = out[r]
        assert ms == 20.0                       # the slowest rank's time
        assert value == 1000 * ws / 0.020       # units of all ranks over that time
        assert n_all == total                   # every instance on exactly one rank
    assert sorted(out[0][3] + out[1][3]) == list(range(40))
