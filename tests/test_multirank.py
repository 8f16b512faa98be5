"""Multi-rank host logic of the bench on CPU (gloo, world size 2): replicas
report the slowest rank's time and the whole job's rate.  The exchange of a
row-sharded Lloyd iteration is tested in test_sharded.py."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 * (rank + 1), world)        # rank 1 is the slower one
    rate = bench.whole_job_rate(1.0e9, world, ms / 1e3)
    out.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_report_slowest_rank_and_whole_job_rate():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    assert all(abs(r[2] - 2 * 1.0e9 / 0.020) < 1e-3 for r in res)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
