"""Row-sharded (data-parallel) Lloyd iterations over torch.distributed ranks.

The rows of X are split over the ranks (one GPU each), the centres are
replicated.  An iteration of Alg. 3 needs one exchange: the per-cluster sums
and counts of Eq. (center).  The library forms them as exact 64-bit
fixed-point integers (km_update_partial), so their all-reduction is exact in
any order and every rank finalises the same centres, bit for bit equal to one
process holding all rows.  Before the first iteration the ranks agree on the
fixed-point scale: the largest |x| over all shards (an integer maximum of its
binary32 bits) and the total row count.  Empty clusters under
KM_EMPTY_FARTHEST: every rank proposes its rows of largest min_dist
(km_farthest_rows), the candidates are gathered and merged (largest min_dist
first, ties to the lowest global row index) and the winners' rows are
broadcast from the ranks that hold them.

`backend` is a libmpkm Context (every computation runs in its kernels); the
exchange itself is torch.distributed collectives (NCCL between GPUs).
"""
from __future__ import annotations

from ._binding import EMPTY_FARTHEST, Params


class ShardedLloyd:
    def __init__(self, backend, X, k: int, p: Params, group=None):
        import torch
        import torch.distributed as dist
        self.b, self.X, self.k, self.p, self.group = backend, X, int(k), p, group
        dev = X.device
        self.n_local = int(X.shape[0])
        self.d = int(X.shape[1])
        world = dist.get_world_size(group)
        ns = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
        dist.all_gather(ns, torch.tensor([self.n_local], dtype=torch.int64, device=dev), group=group)
        ns = [int(t.item()) for t in ns]
        rank = dist.get_rank(group)
        self.row0 = sum(ns[:rank])          # this shard's first global row
        self.n_total = sum(ns)
        a = torch.tensor([backend.absmax(X)], dtype=torch.int64, device=dev)
        dist.all_reduce(a, op=dist.ReduceOp.MAX, group=group)
        self.absmax_bits = int(a.item())

    def step(self, C):
        """One iteration from the replicated centres C (k x d): returns (the
        new centres, this shard's labels and min_dist, the SSE of all rows,
        the shift)."""
        import torch
        import torch.distributed as dist
        labels, md, _ = self.b.assign(self.X, C, self.p, want_flagged=False)
        sse = torch.tensor([self.b.stats()["sse"]], dtype=torch.float64, device=C.device)
        sums, counts = self.b.update_partial(self.X, labels, self.k, self.absmax_bits, self.n_total, self.p)
        dist.all_reduce(sums, group=self.group)     # integers: exact in any order
        dist.all_reduce(counts, group=self.group)
        dist.all_reduce(sse, group=self.group)
        C_new, shift = self.b.update_finalize(sums, counts, C, self.absmax_bits, self.n_total)
        empty = torch.nonzero(counts == 0).flatten().tolist()
        if empty and self.p.empty == EMPTY_FARTHEST:
            empty = sorted(empty)
            C_new = self._reseed(C_new, md, empty)
            # the re-seeded centres moved too (the kernel's shift kept them)
            moved = torch.linalg.vector_norm(C_new[empty].double() - C[empty].double(), dim=1)
            shift = max(shift, float(moved.max()))
        return C_new, labels, md, float(sse.item()), shift

    def _reseed(self, C_new, md, empty):
        import torch
        import torch.distributed as dist
        e = min(len(empty), self.n_local)
        rows, vals = self.b.farthest_rows(md, e, k=self.k)
        world = dist.get_world_size(self.group)
        E = len(empty)
        # every rank's candidates (padded to E): min_dist and global row index
        cv = torch.full((E,), -1.0, dtype=torch.float64, device=C_new.device)
        ci = torch.full((E,), -1, dtype=torch.int64, device=C_new.device)
        cv[:e] = vals
        ci[:e] = rows + self.row0
        allv = [torch.empty_like(cv) for _ in range(world)]
        alli = [torch.empty_like(ci) for _ in range(world)]
        dist.all_gather(allv, cv, group=self.group)
        dist.all_gather(alli, ci, group=self.group)
        cand = [(float(v), int(i)) for vv, ii in zip(allv, alli) for v, i in zip(vv.tolist(), ii.tolist()) if i >= 0]
        cand.sort(key=lambda t: (-t[0], t[1]))
        win = [i for _, i in cand[:E]]
        # the winners' rows, from the ranks that hold them
        picked = torch.zeros((E, self.d), dtype=torch.float32, device=C_new.device)
        for r, gi in enumerate(win):
            if self.row0 <= gi < self.row0 + self.n_local:
                picked[r] = self.X[gi - self.row0]
        dist.all_reduce(picked, group=self.group)   # one holder per row; the others add zeros
        C_new = C_new.clone()
        for r, j in enumerate(empty[:len(win)]):
            C_new[j] = picked[r]
        return C_new
