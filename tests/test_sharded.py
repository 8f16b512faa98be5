"""The data-parallel exchange (paper_2407_12208_gb300/dp.py) on CPU ranks:
two gloo processes holding half the rows each give the centres, labels and
empty-cluster re-seeding of one process holding all rows, bit for bit.  The
per-shard computations run in a stand-in for the library with its
documented arithmetic (exact 64-bit fixed-point sums at the agreed scale,
binary64 division, fp32 centres; assignments by the CPU oracle), so the test
checks the protocol: the scale agreement, the exact integer reductions, the
candidate merge for empty clusters and the row broadcast."""
import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class ModelBackend:
    """CPU stand-in for the Context calls the exchange makes."""

    def __init__(self):
        self.sse = 0.0

    def absmax(self, X):
        m = np.float32(np.abs(X.numpy()).max())
        return int(np.array([m], np.float32).view(np.uint32)[0])

    def assign(self, X, C, p, want_flagged=False):
        import torch
        import oracle
        lab, d1, _ = oracle.assign(X.numpy(), C.numpy())
        self.sse = float(np.sum(d1))
        return torch.from_numpy(lab), torch.from_numpy(d1), None

    def stats(self):
        return {"sse": self.sse}

    @staticmethod
    def _shift(absmax_bits, n_total):
        amax = float(np.array([absmax_bits], np.uint32).view(np.float32)[0])
        E = math.frexp(amax)[1] - 1 if amax > 0 else -126
        return 60 - math.ceil(math.log2(n_total)) - E

    def update_partial(self, X, labels, k, absmax_bits, n_total, p=None):
        import torch
        S = self._shift(absmax_bits, n_total)
        q = np.rint(X.numpy().astype(np.float64) * 2.0 ** S).astype(np.int64)
        sums = np.zeros((k, X.shape[1]), np.int64)
        np.add.at(sums, labels.numpy(), q)
        counts = np.bincount(labels.numpy(), minlength=k).astype(np.int64)
        return torch.from_numpy(sums), torch.from_numpy(counts)

    def update_finalize(self, sums, counts, C_old, absmax_bits, n_total):
        import torch
        S = self._shift(absmax_bits, n_total)
        s, c = sums.numpy(), counts.numpy()
        Cn = C_old.numpy().copy()
        nz = c > 0
        Cn[nz] = ((s[nz].astype(np.float64) * 2.0 ** -S) / c[nz, None]).astype(np.float32)
        shift = float(np.max(np.linalg.norm(Cn.astype(np.float64) - C_old.numpy(), axis=1)))
        return torch.from_numpy(Cn), shift

    def farthest_rows(self, md, e, k=None):
        import torch
        v = md.numpy()
        order = np.lexsort((np.arange(v.size), -v))[:e]
        return torch.from_numpy(order.astype(np.int64)), torch.from_numpy(v[order])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2407_12208_gb300 import workloads
    from paper_2407_12208_gb300._binding import Params
    from paper_2407_12208_gb300.dp import ShardedLloyd
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X, C0 = workloads.gaussian_mixture(2001, 8, 6, seed=91)
    C0[2] += 1e3   # a centre far from every point: an empty cluster to re-seed
    bounds = np.linspace(0, len(X), world + 1).astype(int)
    Xs = torch.from_numpy(np.ascontiguousarray(X[bounds[rank]:bounds[rank + 1]]))
    p = Params()
    p.empty = 1
    lloyd = ShardedLloyd(ModelBackend(), Xs, 6, p)
    C = torch.from_numpy(C0)
    traj = []
    for _ in range(4):
        C, lab, md, sse, shift = lloyd.step(C)
        traj.append((C.numpy().copy(), lab.numpy().copy(), sse))
    out.put((rank, world, lloyd.n_total, lloyd.row0, traj))
    dist.barrier()
    dist.destroy_process_group()


def _run(world):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_two_shards_equal_one_process():
    one = _run(1)[0]
    two = _run(2)
    assert two[0][2] == two[1][2] == one[2] == 2001
    assert (two[0][3], two[1][3]) == (0, 1000)
    for it in range(4):
        C1, lab1, sse1 = one[4][it]
        for r in range(2):
            Cr, labr, sser = two[r][4][it]
            assert np.array_equal(Cr.view(np.uint32), C1.view(np.uint32)), it
            assert sser == pytest.approx(sse1, rel=1e-12)
        assert np.array_equal(np.concatenate([two[0][4][it][1], two[1][4][it][1]]), lab1)
    # the far centre's cluster was empty in the first iteration and re-seeded
    # with a data row (the one of largest min_dist)
    sys.path.insert(0, ROOT)
    from paper_2407_12208_gb300 import workloads
    X, _ = workloads.gaussian_mixture(2001, 8, 6, seed=91)
    assert np.any(np.all(X == one[4][0][0][2], axis=1))
