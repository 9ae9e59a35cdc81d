"""The multi-rank bench path on CPU: world size 2 over gloo.  Each rank runs an
independent halo (replicas, weak scaling); the only collective is the MAX of
the per-rank timed region used for the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, _ = bench.dist_env()
    assert (ws, r) == (world, rank)
    local_ms = 100.0 + 50.0 * rank              # rank 1 is the slow one
    m = bench.max_over_ranks(local_ms, "cpu")
    out[rank] = (m, bench.job_throughput(1 << 20, world, 10, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_whole_job_throughput():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    assert res[0][1] == pytest.approx(2 * (1 << 20) * 10 / 0.150)
