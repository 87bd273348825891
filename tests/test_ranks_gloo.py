"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every
rank gets its own batch seed, the timed region's time is the maximum over
ranks, and the whole-job rate counts every rank's units."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_06902_gb300 import ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, l = ranks.rank_info()
    ranks.barrier(w)
    t = ranks.max_over_ranks(1.5 + r, w)
    out[r] = (w, r, l, t, ranks.batch_seed(2, r), ranks.aggregate_rate(10, w, t))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][3] == out[1][3] == 2.5                 # max over ranks
    assert out[0][4] != out[1][4]                        # distinct batches
    assert out[0][5] == pytest.approx(2 * 10 / 2.5)      # whole-job rate
    assert (out[0][0], out[1][1]) == (2, 1)


def test_single_rank_defaults():
    assert ranks.max_over_ranks(3.0, 1) == 3.0
    assert ranks.aggregate_rate(5, 1, 0.5) == 10.0
