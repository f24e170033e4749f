"""Multi-rank host logic on CPU ranks (gloo, world size 2): the whole-job
rate (units of all ranks over the slowest rank's time) and the partition of
a batch's instances over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2510_22221_b300.distributed import job_rate, shard_instances


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r did (r+1) * 1e9 units in (1 + r) * 0.5 s
    rate, t = job_rate((rank + 1) * 1e9, (1 + rank) * 0.5)
    out[rank] = (rate, t)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_sums_units_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        res = dict(out)
    for r in range(2):
        assert res[r][1] == pytest.approx(1.0)
        assert res[r][0] == pytest.approx(3e9)


def test_job_rate_single_process():
    assert job_rate(2e9, 0.5) == (4e9, 0.5)


def test_shard_instances_balanced_and_complete():
    rng = np.random.default_rng(0)
    cells = rng.integers(48, 97, size=64) ** 3
    for world in (1, 2, 3, 8):
        sh = shard_instances(cells, world)
        flat = sorted(q for s in sh for q in s)
        assert flat == list(range(64))
        loads = [int(sum(cells[q] for q in s)) for s in sh]
        assert max(loads) - min(loads) <= int(cells.max())
        assert sh == shard_instances(cells, world)       # deterministic
