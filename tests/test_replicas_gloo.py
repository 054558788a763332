"""The multi-GPU form is replicas only (independent images, keys replicated, no collective on
the data path).  Its host logic -- a barrier, then the slowest rank's time, then the
whole-job rate -- is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = [10.0 + rank, 20.0 - rank]          # rank 1 slower on the first, faster on the second
    got = bench.max_over_ranks(ms, "cpu")
    out[rank] = got + [bench.whole_job_rate(160 * 24, world, got[0])]
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time():
    ctx = mp.get_context("spawn")
    world = 2
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][:2] == res[1][:2] == [11.0, 20.0]
    assert res[0][2] == pytest.approx(2 * 160 * 24 / 0.011)
