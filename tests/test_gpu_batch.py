"""GPU tests of km_lloyd_run_batch: many small Lloyd jobs in one launch give,
job by job, exactly km_lloyd_run's centres, labels, SSE trajectory and
iteration count (and so the oracle's labels, as km_lloyd_run does)."""
import numpy as np
import pytest

import oracle
from paper_2407_12208_gb300 import workloads
from gpu_util import MARGIN

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300 import build
    build.build()
    c = pkg.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _jobs(seed, count):
    r = np.random.default_rng(seed)
    jobs = []
    for q in range(count):
        d = int(r.integers(1, 9))
        k = int(r.integers(1, 65))
        n = int(r.integers(k, 16385)) if q % 3 else int(r.integers(k, k + 50))
        kind = q % 4
        if kind == 0:
            X, C0 = workloads.blobs(n, d, k, seed=seed * 100 + q)
        elif kind == 1:
            X, C0 = workloads.uniform_pairs(n, d, k, seed=seed * 100 + q)
        elif kind == 2:  # coarse grid values: many equal distances (ties)
            X = r.integers(0, 4, size=(n, d)).astype(np.float32)
            C0 = X[workloads.init_indices(n, k, seed * 100 + q)].copy()
        else:  # some initial centres far away: empty clusters from the first iteration
            X, C0 = workloads.blobs(n, d, k, seed=seed * 100 + q)
            C0[::3] += 1e3
        jobs.append((X, C0))
    return jobs


@pytest.mark.parametrize("empty,tau", [("farthest", 0.0), ("keep", 0.0), ("farthest", 1e-3)])
def test_batch_equals_single_runs(ctx, empty, tau):
    import paper_2407_12208_gb300 as pkg
    p = pkg.params("fp32", max_iter=12, empty=empty, tau=tau)
    jobs = _jobs(5 if tau == 0.0 else 6, 45)
    dev = [(_dev(X), _dev(C0)) for X, C0 in jobs]
    got = ctx.lloyd_run_batch(dev, p)
    torch.cuda.synchronize()
    for q, ((Xd, C0d), (C, lab, sse, it)) in enumerate(zip(dev, got)):
        C1, lab1, sse1, eta1, it1 = ctx.lloyd_run(Xd, C0d, p)
        torch.cuda.synchronize()
        assert it == it1, q
        assert np.array_equal(C.cpu().numpy().view(np.uint32), C1.cpu().numpy().view(np.uint32)), q
        assert np.array_equal(lab.cpu().numpy(), lab1.cpu().numpy()), q
        assert np.array_equal(sse.view(np.uint64), np.asarray(sse1).view(np.uint64)), q


def test_batch_matches_the_oracle(ctx):
    import paper_2407_12208_gb300 as pkg
    X, C0 = workloads.blobs(3000, 5, 12, seed=77)
    p = pkg.params("fp32", max_iter=8, empty="farthest")
    (C, lab, sse, it), = ctx.lloyd_run_batch([(_dev(X), _dev(C0))], p)
    oC, olab, osse, oit = oracle.lloyd(X, C0, 8, 0.0, 1)
    assert it == oit
    np.testing.assert_allclose(sse, osse, rtol=1e-12)
    o2, d1, d2 = oracle.assign(X, C.cpu().numpy())
    margin = (d2 - d1) / np.maximum(d2, 1e-300)
    sel = margin > MARGIN
    assert np.array_equal(lab.cpu().numpy()[sel], o2[sel])


def test_batch_rejects_what_it_does_not_take(ctx):
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300._binding import KmError
    X, C0 = workloads.blobs(500, 9, 4, seed=1)
    with pytest.raises(KmError, match="EUNSUPPORTED"):
        ctx.lloyd_run_batch([(_dev(X), _dev(C0))], pkg.params("fp32"))
    X, C0 = workloads.blobs(500, 4, 4, seed=1)
    with pytest.raises(KmError, match="EUNSUPPORTED"):
        ctx.lloyd_run_batch([(_dev(X), _dev(C0))], pkg.params("bf16"))
    X, C0 = workloads.blobs(20000, 4, 4, seed=1)
    with pytest.raises(KmError, match="EUNSUPPORTED"):
        ctx.lloyd_run_batch([(_dev(X), _dev(C0))], pkg.params("fp32"))
