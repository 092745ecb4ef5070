"""Host logic of the multi-GPU replica mode, on CPU with world_size-2 gloo process groups."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_00316_gb300 import replicas as REP


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    info = REP.RankInfo.from_env()
    elapsed = 1.0 + 0.5 * info.rank                     # rank 1 is the slow one
    slowest = REP.max_over_ranks(elapsed)
    units = REP.sum_over_ranks(5)                        # 5 updates per rank
    mine = REP.assign_slices(32, info.rank, info.world)
    dist.barrier()
    q.put((info.rank, info.world, slowest, units, REP.aggregate_throughput(units, slowest), mine,
           REP.replica_seed(info.rank)))
    dist.destroy_process_group()


def test_replica_mode_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == pytest.approx(1.5) for r in res)          # max over ranks
    assert all(r[3] == 10 for r in res)
    assert all(r[4] == pytest.approx(10 / 1.5) for r in res)     # weak scaling aggregate
    slices = sorted(res[0][5] + res[1][5])
    assert slices == list(range(32)) and not set(res[0][5]) & set(res[1][5])
    assert res[0][6] != res[1][6]                                 # independent replicas


def test_single_process_defaults():
    assert REP.max_over_ranks(3.0) == 3.0
    assert REP.assign_slices(5, 0, 1) == [0, 1, 2, 3, 4]
