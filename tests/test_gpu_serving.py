"""GPU tests of the serving engine (km_submit / km_poll / km_release /
km_cancel): jobs of uneven n, d, k submitted together overlap on the device,
and each result equals the same job run alone through the synchronous calls,
bit for bit; admission refuses a job that can never fit the arena."""
import time

import numpy as np
import pytest

from paper_2407_12208_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sctx():
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300 import build
    build.build()
    c = pkg.Context(0, arena_bytes=1 << 30)
    yield c
    c.close()


def _wait(ctx, jid, timeout=120.0):
    t0 = time.time()
    while True:
        r = ctx.poll(jid)
        if r is not None:
            return r
        assert time.time() - t0 < timeout, "job %d did not finish" % jid
        time.sleep(0.002)


def _jobs():
    """A mix: Lloyd runs and single assignments, 16-bit, E4M3 and direct paths."""
    specs = [(0, "bf16", 20000, 128, 64), (1, "bf16", 30001, 32, 200), (0, "fp16", 9000, 64, 37),
             (0, "e4m3", 12000, 64, 16), (1, "fp32", 8000, 8, 10), (0, "fp64", 3000, 2, 5),
             (0, "bf16", 5000, 256, 128), (1, "fp16", 40000, 128, 1024)]
    out = []
    for i, (kind, low, n, d, k) in enumerate(specs):
        X, C = workloads.gaussian_mixture(n, d, k, seed=100 + i)
        out.append(dict(kind=kind, low=low, X=X, C=C))
    return out


def test_serving_mix_equals_alone(sctx):
    import paper_2407_12208_gb300 as pkg
    jobs = _jobs()
    ids = []
    for jb in jobs:
        p = pkg.params(jb["low"], max_iter=6)
        ids.append(sctx.submit(jb["X"], jb["C"], p, kind=jb["kind"]))
    results = [_wait(sctx, j) for j in ids]
    for jb, jid, r in zip(jobs, ids, results):
        assert r["status"] == pkg._binding.KM_OK
        n, d = jb["X"].shape
        k = jb["C"].shape[0]
        lab_s = pkg.device_array(r["labels"], (n,), "<i4").cpu().numpy()
        C_s = pkg.device_array(r["C"], (k, d), "<f4").cpu().numpy()
        p = pkg.params(jb["low"], max_iter=6)
        Xd = torch.from_numpy(jb["X"]).cuda()
        Cd = torch.from_numpy(jb["C"]).cuda()
        if jb["kind"] == 0:
            C_a, lab_a, _, _, _ = sctx.lloyd_run(Xd, Cd, p)
            torch.cuda.synchronize()
            assert np.array_equal(C_s.view(np.uint32), C_a.cpu().numpy().view(np.uint32))
        else:
            lab_a, _, _ = sctx.assign(Xd, Cd, p)
            torch.cuda.synchronize()
            assert np.array_equal(C_s.view(np.uint32), jb["C"].view(np.uint32))  # centres returned as given
        assert np.array_equal(lab_s, lab_a.cpu().numpy())
        assert r["latency_ms"] >= r["queue_ms"] >= 0.0
        sctx.release(jid)


def test_serving_refuses_a_job_that_never_fits(sctx):
    import paper_2407_12208_gb300 as pkg
    X = np.zeros((20_000_000, 16), dtype=np.float32)  # 1.3 GB of points alone: more than the 1 GB arena
    C = np.zeros((4, 16), dtype=np.float32)
    with pytest.raises(pkg.KmError) as ei:
        sctx.submit(X, C, pkg.params("bf16"), kind=1)
    assert ei.value.status == pkg._binding.KM_ENOMEM


def test_serving_cancel_and_release(sctx):
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.gaussian_mixture(50000, 64, 64, seed=7)
    jid = sctx.submit(X, C, pkg.params("bf16", max_iter=200, tau=0.0), kind=0)
    sctx.cancel(jid)
    r = _wait(sctx, jid)
    assert r["status"] in (pkg._binding.KM_ECANCELLED, pkg._binding.KM_OK)
    sctx.release(jid)
    # the arena is free again: a job of half its size is admitted and finishes
    X2, C2 = workloads.gaussian_mixture(200000, 128, 32, seed=8)
    j2 = sctx.submit(X2, C2, pkg.params("bf16", max_iter=2), kind=0)
    r2 = _wait(sctx, j2)
    assert r2["status"] == pkg._binding.KM_OK
    sctx.release(j2)


def test_serving_resident_data_equals_alone(sctx):
    """Jobs whose points and centres are resident on the device
    (KM_JOB_DEVICE_DATA, read in place) give the results of the same jobs
    run alone, bit for bit, while they run side by side."""
    import paper_2407_12208_gb300 as pkg
    jobs = _jobs()
    dev = [(torch.from_numpy(jb["X"]).cuda(), torch.from_numpy(jb["C"]).cuda()) for jb in jobs]
    ids = [sctx.submit(Xd, Cd, pkg.params(jb["low"], max_iter=6), kind=jb["kind"]) for jb, (Xd, Cd) in zip(jobs, dev)]
    results = [_wait(sctx, j) for j in ids]
    for jb, (Xd, Cd), jid, r in zip(jobs, dev, ids, results):
        assert r["status"] == pkg._binding.KM_OK, r["message"]
        n, d = jb["X"].shape
        k = jb["C"].shape[0]
        lab_s = pkg.device_array(r["labels"], (n,), "<i4").cpu().numpy()
        C_s = pkg.device_array(r["C"], (k, d), "<f4").cpu().numpy()
        p = pkg.params(jb["low"], max_iter=6)
        if jb["kind"] == 0:
            C_a, lab_a, _, _, _ = sctx.lloyd_run(Xd, Cd, p)
        else:
            lab_a, _, _ = sctx.assign(Xd, Cd, p)
            C_a = Cd
        torch.cuda.synchronize()
        assert np.array_equal(C_s.view(np.uint32), C_a.cpu().numpy().view(np.uint32))
        assert np.array_equal(lab_s, lab_a.cpu().numpy())
        sctx.release(jid)


def test_serving_groups_small_jobs(sctx):
    """120 small FP32 Lloyd jobs (d <= 8, k <= 64, n <= 16384: grouped launches
    of up to 32 jobs) submitted among larger ones: each small job's centres,
    labels, SSE and iteration count equal km_lloyd_run on it alone."""
    import paper_2407_12208_gb300 as pkg
    r = np.random.default_rng(9)
    big = workloads.gaussian_mixture(60000, 64, 128, seed=9)
    small, others = [], []
    for q in range(120):
        d, k = int(r.integers(1, 9)), int(r.integers(1, 65))
        n = int(r.integers(k, 16385))
        X, C = workloads.blobs(n, d, k, seed=500 + q)
        p = pkg.params("fp32", max_iter=10, empty="farthest")
        small.append((sctx.submit(X, C, p, kind=0), X, C, p))
        if q % 40 == 0:
            others.append(sctx.submit(big[0], big[1], pkg.params("bf16", max_iter=4), kind=0))
    for jid in others:
        assert _wait(sctx, jid)["status"] == pkg._binding.KM_OK
    for q, (jid, X, C, p) in enumerate(small):
        out = _wait(sctx, jid)
        assert out["status"] == pkg._binding.KM_OK, q
        n, d = X.shape
        k = C.shape[0]
        C_a, lab_a, sse_a, _, it_a = sctx.lloyd_run(torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), p)
        torch.cuda.synchronize()
        C_s = pkg.device_array(out["C"], (k, d), "<f4").cpu().numpy()
        lab_s = pkg.device_array(out["labels"], (n,), "<i4").cpu().numpy()
        assert np.array_equal(C_s.view(np.uint32), C_a.cpu().numpy().view(np.uint32)), q
        assert np.array_equal(lab_s, lab_a.cpu().numpy()), q
        assert out["iters"] == it_a and out["sse"] == sse_a[-1], q
    for jid in others + [s_[0] for s_ in small]:
        sctx.release(jid)


def test_serving_hundred_mixed_jobs_equal_alone(sctx):
    """100 jobs drawn like the served stream (n log-uniform [1e3, 3e4], d in
    {2, 8, 32, 128, 256}, k log-uniform [4, 256]; BF16, FP16 and E4M3 on the
    tensor cores, FP32 and FP64 direct for d <= 8; one in four a single
    assignment) submitted at once: every result equals the same job run alone
    through km_lloyd_run / km_assign, bit for bit."""
    import paper_2407_12208_gb300 as pkg
    specs = workloads.serving_jobs(100, seed=77, n_lo=1e3, n_hi=3e4, k_hi=256)
    jobs = []
    for i, s in enumerate(specs):
        n, d, k = s["n"], s["d"], s["k"]
        low = ("fp32", "fp64")[i % 2] if d <= 8 else ("bf16", "fp16", "e4m3")[i % 3]
        kind = 1 if i % 4 == 3 else 0
        X, C = workloads.gaussian_mixture(n, d, k, seed=700 + i)
        p = pkg.params(low, max_iter=5)
        jobs.append((sctx.submit(X, C, p, kind=kind), X, C, p, kind))
    for i, (jid, X, C, p, kind) in enumerate(jobs):
        out = _wait(sctx, jid)
        assert out["status"] == pkg._binding.KM_OK, (i, out["message"])
        n, d = X.shape
        k = C.shape[0]
        lab_s = pkg.device_array(out["labels"], (n,), "<i4").cpu().numpy()
        C_s = pkg.device_array(out["C"], (k, d), "<f4").cpu().numpy()
        Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
        if kind == 0:
            C_a, lab_a, _, _, _ = sctx.lloyd_run(Xd, Cd, p)
            torch.cuda.synchronize()
            assert np.array_equal(C_s.view(np.uint32), C_a.cpu().numpy().view(np.uint32)), i
        else:
            lab_a, _, _ = sctx.assign(Xd, Cd, p)
            torch.cuda.synchronize()
        assert np.array_equal(lab_s, lab_a.cpu().numpy()), i
        sctx.release(jid)
