"""GPU parity: the CUDA path through the C-ABI against the CPU oracle, on the
same seeded inputs, at sizes that span several tiles and a ragged tail."""
import numpy as np
import pytest

import oracle
from paper_2407_12208_gb300 import workloads
from gpu_util import MARGIN, RTOL_FP64, RTOL_MD, RTOL_MIXED, check_assign

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


def _run_assign(ctx, X, C, low, test="tc", rho=5.0, c_A=2.0):
    import paper_2407_12208_gb300 as pkg
    p = pkg.params(low, test, rho=rho, paper_factor=c_A)
    lab, md, nf = ctx.assign(_dev(X), _dev(C), p)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), md.cpu().numpy(), nf, ctx.stats()


# ------------------------------------------------------------- direct paths
def test_fp64_direct_blobs(ctx):
    X, C = workloads.blobs(4099, 16, 8, seed=1)
    lab, md, nf, st = _run_assign(ctx, X, C, "fp64")
    olab, od1, _ = oracle.assign(X, C)
    assert np.array_equal(lab, olab)
    np.testing.assert_allclose(md, od1, rtol=RTOL_FP64)
    assert nf == 0
    check_assign(lab, md, X, C, oracle, RTOL_FP64)


@pytest.mark.parametrize("n,d,k", [(5000, 5, 16), (1000, 16, 8), (777, 33, 40), (300, 2, 300),
                                   (3001, 128, 300), (2000, 64, 1000), (129, 96, 65)])
def test_fp32_direct_certified(ctx, n, d, k):
    if d == 5:
        X, C = workloads.voronoi_image(50, 100, 16, k, seed=2)
    else:
        X, C = workloads.blobs(n, d, k, seed=3)
    lab, md, nf, st = _run_assign(ctx, X, C, "fp32")
    check_assign(lab, md, X, C, oracle, RTOL_MD)


# ------------------------------------------------------- tensor-core paths
CASES = [
    ("uniform", 3001, 128, 300),
    ("uniform", 2000, 128, 1024),
    ("mixture", 2500, 64, 256),
    ("cancellation", 1500, 128, 64),
    ("uniform", 700, 37, 130),
    ("mixture", 129, 256, 100),
]


def _data(kind, n, d, k, seed):
    if kind == "uniform":
        return workloads.uniform_pairs(n, d, k, seed)
    if kind == "mixture":
        return workloads.gaussian_mixture(n, d, k, seed)
    return workloads.cancellation(n, d, k, seed)


@pytest.mark.parametrize("low", ["bf16", "fp16", "e4m3"])
@pytest.mark.parametrize("kind,n,d,k", CASES)
def test_tc_assign_parity(ctx, low, kind, n, d, k):
    X, C = _data(kind, n, d, k, seed=n + d + k)
    lab, md, nf, st = _run_assign(ctx, X, C, low)
    check_assign(lab, md, X, C, oracle, RTOL_MD)
    fmt = {"fp16": 0, "bf16": 1, "e4m3": 2}[low]
    sure, maybe = oracle.predict_tc_flags(X, C, fmt, 5.0, per_row_scale=(fmt == 2))
    lo, hi = int(sure.sum()), int((sure | maybe).sum())
    assert lo <= nf <= hi, (nf, lo, hi)
    assert st["pairs"] == n * k


@pytest.mark.parametrize("low", ["bf16", "fp16"])
def test_tc_paper_test_flags_everything_at_r128_bf16(ctx, low):
    X, C = workloads.uniform_pairs(600, 128, 50, seed=4)
    lab, md, nf, st = _run_assign(ctx, X, C, low, test="paper", c_A=1.0)
    check_assign(lab, md, X, C, oracle, RTOL_MD)
    fmt = {"fp16": 0, "bf16": 1}[low]
    sure, maybe = oracle.predict_tc_flags(X, C, fmt, 5.0, test="paper", c_A=1.0)
    assert int(sure.sum()) <= nf <= int((sure | maybe).sum())
    if low == "bf16":
        assert nf == 600 * 50  # Alg. 2 at r >= 72 with BF16: 100% fallback (Table 6.1)


def test_tc_test_off_still_certified(ctx):
    X, C = workloads.gaussian_mixture(2000, 64, 64, seed=5)
    lab, md, nf, st = _run_assign(ctx, X, C, "bf16", test="off")
    check_assign(lab, md, X, C, oracle, RTOL_MD)
    assert nf == 0


@pytest.mark.parametrize("low", ["bf16", "fp16"])
def test_tc_edges(ctx, low):
    # k = 1; k = n; duplicate centres (ties -> lowest index); n < one tile
    X, C = workloads.uniform_pairs(50, 96, 1, seed=6)
    lab, md, *_ = _run_assign(ctx, X, C, low)
    assert np.all(lab == 0)
    check_assign(lab, md, X, C, oracle, RTOL_MD)
    X = workloads.uniform_pairs(200, 64, 200, seed=7)[0]
    lab, md, *_ = _run_assign(ctx, X, X.copy(), low)
    assert np.array_equal(lab, np.arange(200))
    assert np.all(md == 0.0)
    X, C = workloads.uniform_pairs(400, 64, 40, seed=8)
    C[25] = C[3]
    lab, md, *_ = _run_assign(ctx, X, C, low)
    check_assign(lab, md, X, C, oracle, RTOL_MD)
    assert not np.any(lab == 25)


def test_tc_rejects_bad_arguments(ctx):
    import paper_2407_12208_gb300 as pkg
    X = _dev(np.zeros((10, 8), np.float32))
    with pytest.raises(pkg.KmError) as e:
        ctx.assign(X, _dev(np.zeros((11, 8), np.float32)), pkg.params("bf16"))  # k > n
    assert e.value.status == 1
    with pytest.raises(pkg.KmError) as e:
        ctx.assign(X, X[:2], pkg.params("e4m3"))  # E4M3 needs d >= 16
    assert e.value.status == 7
    with pytest.raises(pkg.KmError) as e:
        ctx.assign(X, X[:2], pkg.params("bf16", "paper", rho=2.0))  # rho~ > 2 required
    assert e.value.status == 1


# ------------------------------------------------------------ distance matrix
@pytest.mark.parametrize("low", ["fp16", "bf16", "e4m3"])
@pytest.mark.parametrize("scenario", ["far", "near"])
def test_distances_alg2(ctx, low, scenario):
    import paper_2407_12208_gb300 as pkg
    if scenario == "far":
        X, C = workloads.near_far(600, 128, 0.0, seed=9)
    else:
        X, C = workloads.near_far(600, 128, 0.5, seed=9)
    C = C[:500]
    p = pkg.params(low, "tc")
    D, bits, nf = ctx.distances(_dev(X), _dev(C), p)
    D = D.cpu().numpy().astype(np.float64)
    bits = bits.cpu().numpy().view(np.uint32)
    n, k = D.shape
    flags = ((bits[(np.arange(n * k) >> 5)] >> (np.arange(n * k) & 31)) & 1).reshape(n, k).astype(bool)
    assert flags.sum() == nf
    Dex = oracle.dist_direct(X, C)
    fmt = {"fp16": 0, "bf16": 1, "e4m3": 2}[low]
    prs = fmt == 2  # E4M3: power-of-two scales per row of X and per centre
    B = oracle.tc_bound_matrix(X, C, fmt, per_row_scale=prs)
    # unflagged: within the bound (Theorem 4.2 + conversion error); relative error <= 1/(rho-1)
    un = ~flags
    assert np.all(np.abs(D[un] - Dex[un]) <= B[un] + 1e-6 * Dex[un])
    assert np.all(np.abs(D[un] - Dex[un]) <= Dex[un] / 4.0)
    # flagged: binary64 direct value stored in fp32
    np.testing.assert_allclose(D[flags], Dex[flags], rtol=2 ** -23, atol=1e-38)
    sure, maybe = oracle.predict_tc_flags(X, C, fmt, 5.0, per_row_scale=prs)
    assert np.all(flags[sure & ~maybe]) and not np.any(flags[~sure & ~maybe])
    assert np.all(D >= 0.0)  # no pair is left with its flag mark


# ---------------------------------------------------------------- centre update
@pytest.mark.parametrize("policy", ["keep", "farthest"])
def test_update_centroids(ctx, policy):
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.gaussian_mixture(5003, 24, 37, seed=10)
    olab, od1, _ = oracle.assign(X, C)
    olab = olab.copy()
    olab[olab == 5] = 6  # make clusters 5 empty
    olab[olab == 30] = 0
    p = pkg.params("fp64", empty=policy)
    Cn, cnt, shift = ctx.update_centroids(_dev(X), _dev(olab), _dev(C), p, min_dist=_dev(od1))
    oC, ocnt, oshift = oracle.update(X, olab, C, 1 if policy == "farthest" else 0, od1)
    assert np.array_equal(cnt.cpu().numpy(), ocnt)
    Cn = Cn.cpu().numpy()
    # exact sums: at most a one-ulp difference from binary64 recursive summation
    np.testing.assert_allclose(Cn, oC, rtol=2 ** -22, atol=1e-30)
    assert shift == pytest.approx(oshift, rel=1e-6)


@pytest.mark.parametrize("n,d,k", [(20011, 5, 16), (3001, 7, 9), (10000, 64, 256), (5000, 2, 1),
                                   (4099, 32, 50), (3000, 48, 7), (2500, 12, 300)])
def test_update_shapes(ctx, n, d, k):
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.gaussian_mixture(n, d, k, seed=n + d)
    lab, od1, _ = oracle.assign(X, C)
    p = pkg.params("fp64", empty="farthest")
    Cn, cnt, shift = ctx.update_centroids(_dev(X), _dev(lab), _dev(C), p, min_dist=_dev(od1))
    oC, ocnt, oshift = oracle.update(X, lab, C, 1, od1)
    assert np.array_equal(cnt.cpu().numpy(), ocnt)
    np.testing.assert_allclose(Cn.cpu().numpy(), oC, rtol=2 ** -22, atol=1e-30)


def test_update_large_kd_sliced(ctx):
    # k*d too large for one block's shared memory: dimension-sliced accumulation
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.uniform_pairs(30001, 128, 1024, seed=21)
    lab = np.random.default_rng(3).integers(0, 1024, size=len(X)).astype(np.int32)
    lab[lab == 7] = 8  # an empty cluster
    p = pkg.params("bf16", empty="keep")
    Cn, cnt, shift = ctx.update_centroids(_dev(X), _dev(lab), _dev(C), p)
    oC, ocnt, oshift = oracle.update(X, lab, C, 0)
    assert np.array_equal(cnt.cpu().numpy(), ocnt)
    np.testing.assert_allclose(Cn.cpu().numpy(), oC, rtol=2 ** -22, atol=1e-30)
    assert shift == pytest.approx(oshift, rel=1e-6)


def test_update_is_bitwise_reproducible(ctx):
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.gaussian_mixture(20000, 64, 64, seed=11)
    lab = _dev(oracle.assign(X, C)[0])
    p = pkg.params("fp64")
    a = ctx.update_centroids(_dev(X), lab, _dev(C), p)[0].cpu().numpy()
    b = ctx.update_centroids(_dev(X), lab, _dev(C), p)[0].cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


# --------------------------------------------------------------------- Lloyd
def test_lloyd_fp64_config_plain():
    import paper_2407_12208_gb300 as pkg
    c = pkg.Context(0)
    X, C0 = workloads.blobs(10000, 16, 8, seed=12)
    p = pkg.params("fp64", max_iter=20)
    C, lab, sse, eta, it = c.lloyd_run(_dev(X), _dev(C0), p)
    oC, olab, osse, oit = oracle.lloyd(X, C0, 20)
    assert it == oit == 20
    np.testing.assert_allclose(sse, osse, rtol=RTOL_FP64)
    assert np.array_equal(lab.cpu().numpy(), olab)
    np.testing.assert_allclose(C.cpu().numpy(), oC, rtol=2 ** -22)


@pytest.mark.parametrize("low", ["fp16", "e4m3", "bf16"])
def test_lloyd_mixed_trajectory(low):
    import paper_2407_12208_gb300 as pkg
    c = pkg.Context(0)
    X, C0 = workloads.gaussian_mixture(20000, 64, 32, seed=13)
    p = pkg.params(low, max_iter=8)
    C, lab, sse, eta, it = c.lloyd_run(_dev(X), _dev(C0), p)
    oC, olab, osse, oit = oracle.lloyd(X, C0, 8)
    np.testing.assert_allclose(sse, osse, rtol=RTOL_MIXED)
    assert np.array_equal(lab.cpu().numpy(), olab)
    assert np.all(eta >= 0) and np.all(eta <= 1)


def test_tau_stop():
    import paper_2407_12208_gb300 as pkg
    c = pkg.Context(0)
    X, C0 = workloads.blobs(3000, 4, 3, seed=14)
    p = pkg.params("fp16", max_iter=100, tau=1e-8)
    C, lab, sse, eta, it = c.lloyd_run(_dev(X), _dev(C0), p)
    oC, olab, osse, oit = oracle.lloyd(X, C0, 100, tau=1e-8)
    assert it == oit < 100
    np.testing.assert_allclose(sse, osse, rtol=RTOL_MIXED)


# ------------------------------------------------- full size, sampled outputs
def test_full_size_bf16_sampled():
    """n=1e6, d=128, k=1024 (the headline shape) in the bench's launch
    configuration; labels and distances checked on 2000 sampled rows."""
    import paper_2407_12208_gb300 as pkg
    c = pkg.Context(0)
    X, C = workloads.uniform_pairs(1_000_000, 128, 1024, seed=15)
    lab, md, nf = c.assign(_dev(X), _dev(C), pkg.params("bf16"))
    lab = lab.cpu().numpy()
    md = md.cpu().numpy()
    rows = np.random.default_rng(0).choice(len(X), 2000, replace=False)
    check_assign(lab[rows], md[rows], X[rows], C, oracle, RTOL_MD)
    st = c.stats()
    assert st["pairs"] == 1_000_000 * 1024


@pytest.mark.parametrize("wl,n,d,k,low", [
    ("uniform_pairs", 1_000_000, 128, 1024, "bf16"),     # the benchmark's default workload
    ("cancellation", 1_000_000, 128, 1024, "bf16"),      # every pair flagged, every list overflows
    ("gaussian_mixture", 4_000_000, 64, 256, "bf16"),     # the mixed Lloyd iteration shape
    ("voronoi", 4096 * 4096, 5, 16, "fp32"),              # the image shape, fp32 direct
])
def test_full_size_lloyd_step_sampled(wl, n, d, k, low):
    """One km_lloyd_step at the full benchmark sizes (the bench's launch
    configuration): labels and min_dist on 2000 sampled rows against the
    oracle; the new centres against the oracle's update from the GPU's own
    labels (exact fixed-point sums: within one ulp of binary64 summation)."""
    import paper_2407_12208_gb300 as pkg
    c = pkg.Context(0)
    if wl == "voronoi":
        X, C = workloads.voronoi_image(4096, 4096, 16, k, seed=7)
    else:
        X, C = getattr(workloads, wl)(n, d, k, seed=15)
    assert X.shape == (n, d)
    p = pkg.params(low)
    lab, md, Cn, cnt, _ = c.lloyd_step(_dev(X), _dev(C), p)
    torch.cuda.synchronize()
    lab, md, Cn, cnt = lab.cpu().numpy(), md.cpu().numpy(), Cn.cpu().numpy(), cnt.cpu().numpy()
    assert lab.min() >= 0 and lab.max() < k
    rows = np.random.default_rng(1).choice(n, 2000, replace=False)
    check_assign(lab[rows], md[rows], X[rows], C, oracle, RTOL_MD)
    oC, ocnt, _ = oracle.update(X, lab, C, 1, md)
    assert np.array_equal(cnt, ocnt)
    np.testing.assert_allclose(Cn, oC, rtol=2 ** -22, atol=1e-30)
    assert c.stats()["pairs"] == n * k


# ------------------------------------------------ one fused Lloyd iteration
@pytest.mark.parametrize("low,empty,shape", [("bf16", "farthest", (20000, 128, 300)), ("fp16", "keep", (7001, 64, 96)),
                                             ("e4m3", "farthest", (5000, 64, 40)), ("fp32", "farthest", (3000, 16, 24)),
                                             ("fp64", "keep", (2000, 8, 9))])
def test_lloyd_step_equals_assign_then_update(ctx, low, empty, shape):
    import paper_2407_12208_gb300 as pkg
    n, d, k = shape
    X, C = workloads.gaussian_mixture(n, d, k, seed=61)
    C[-1] = C[-1] + 1e3  # a centre far from every point: an empty cluster
    Xd, Cd = _dev(X), _dev(C)
    p = pkg.params(low, empty=empty)
    lab1, md1, _ = ctx.assign(Xd, Cd, p)
    Cn1, cnt1, sh1 = ctx.update_centroids(Xd, lab1, Cd, p, min_dist=md1)
    torch.cuda.synchronize()
    ref = [t.cpu().numpy() for t in (lab1, md1, Cn1, cnt1)]
    lab2, md2, Cn2, cnt2, sh2 = ctx.lloyd_step(Xd, Cd, p)
    torch.cuda.synchronize()
    got = [t.cpu().numpy() for t in (lab2, md2, Cn2, cnt2)]
    assert np.array_equal(got[0], ref[0])
    assert np.array_equal(got[1].view(np.uint64), ref[1].view(np.uint64))
    assert np.array_equal(got[2].view(np.uint32), ref[2].view(np.uint32))
    assert np.array_equal(got[3], ref[3])
    assert sh2 == sh1
    assert ref[3][-1] == 0 or empty == "farthest"


@pytest.mark.parametrize("low,empty,shape", [("bf16", "farthest", (20000, 128, 300)), ("fp16", "keep", (7001, 64, 96)),
                                             ("e4m3", "farthest", (5000, 64, 40)), ("fp32", "farthest", (3000, 16, 24)),
                                             ("fp64", "keep", (2000, 8, 9)), ("bf16", "farthest", (300, 32, 7)),
                                             ("bf16", "keep", (1000, 16, 600))])
def test_lloyd_step_host_equals_device(ctx, low, empty, shape):
    """km_lloyd_step_host (host buffers, rows in chunks overlapping copies and
    kernels) gives km_lloyd_step's results bit for bit, pinned or pageable."""
    import paper_2407_12208_gb300 as pkg
    n, d, k = shape
    X, C = workloads.gaussian_mixture(n, d, k, seed=62)
    p = pkg.params(low, empty=empty)
    lab1, md1, Cn1, cnt1, sh1 = ctx.lloyd_step(_dev(X), _dev(C), p)
    torch.cuda.synchronize()
    ref = [t.cpu().numpy() for t in (lab1, md1, Cn1, cnt1)]
    Xh, Ch = torch.from_numpy(X).pin_memory(), torch.from_numpy(C).pin_memory()
    md = torch.full((n,), -1.0, dtype=torch.float64).pin_memory()
    cnt = torch.full((k,), -1, dtype=torch.int64).pin_memory()
    lab2, md2, Cn2, cnt2, sh2 = ctx.lloyd_step_host(Xh, Ch, p, min_dist=md, counts=cnt)
    assert np.array_equal(lab2.numpy(), ref[0])
    assert np.array_equal(md2.numpy().view(np.uint64), ref[1].view(np.uint64))
    assert np.array_equal(Cn2.numpy().view(np.uint32), ref[2].view(np.uint32))
    assert np.array_equal(cnt2.numpy(), ref[3])
    assert sh2 == sh1
    assert ctx.stats()["pairs"] == n * k
    lab3, _, Cn3, _, _ = ctx.lloyd_step_host(torch.from_numpy(X), torch.from_numpy(C), p)  # pageable
    assert np.array_equal(lab3.numpy(), ref[0])
    assert np.array_equal(Cn3.numpy().view(np.uint32), ref[2].view(np.uint32))


@pytest.mark.parametrize("low,shape", [("bf16", (20000, 32, 50)), ("fp32", (30000, 5, 16)), ("fp16", (12000, 128, 64))])
@pytest.mark.parametrize("where", ["later", "first"])
def test_lloyd_step_host_chunk_scales(ctx, low, shape, where):
    """km_lloyd_step_host with the largest |x| (and with it the fixed-point
    scale of the centre sums) in the last chunk, or only in the first: both
    ways it equals km_lloyd_step bit for bit."""
    import paper_2407_12208_gb300 as pkg
    n, d, k = shape
    X, C = workloads.gaussian_mixture(n, d, k, seed=63)
    if where == "later":
        X[n - n // 10:] *= 8.0  # the last chunk holds the largest |x|
    else:
        X[: n // 20] *= 8.0     # only the first chunk does
    p = pkg.params(low, empty="keep")
    lab1, md1, Cn1, cnt1, sh1 = ctx.lloyd_step(_dev(X), _dev(C), p)
    torch.cuda.synchronize()
    Xh, Ch = torch.from_numpy(X).pin_memory(), torch.from_numpy(C).pin_memory()
    md = torch.full((n,), -1.0, dtype=torch.float64).pin_memory()
    cnt = torch.full((k,), -1, dtype=torch.int64).pin_memory()
    lab2, md2, Cn2, cnt2, sh2 = ctx.lloyd_step_host(Xh, Ch, p, min_dist=md, counts=cnt)
    assert np.array_equal(lab2.numpy(), lab1.cpu().numpy())
    assert np.array_equal(md2.numpy().view(np.uint64), md1.cpu().numpy().view(np.uint64))
    assert np.array_equal(Cn2.numpy().view(np.uint32), Cn1.cpu().numpy().view(np.uint32))
    assert np.array_equal(cnt2.numpy(), cnt1.cpu().numpy())
    assert sh2 == sh1


def test_lloyd_step_host_rejects_bad_arguments(ctx):
    import paper_2407_12208_gb300 as pkg
    p = pkg.params("bf16")
    X, C = torch.zeros((100, 16)), torch.zeros((4, 16))
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.KmError) as ei:
        ctx.lloyd_step_host(X, C, p, ws=small)
    assert ei.value.status == pkg._binding.KM_ENOMEM
    with pytest.raises(pkg.KmError) as ei:
        ctx.lloyd_step_host(torch.zeros((3, 16)), C, p)  # k > n
    assert ei.value.status == pkg._binding.KM_EINVAL
    with pytest.raises(pkg.KmError) as ei:
        ctx.lloyd_step_host(torch.zeros((100, 8)), torch.zeros((4, 8)), pkg.params("e4m3"))  # E4M3 needs d >= 16
    assert ei.value.status == pkg._binding.KM_EUNSUPPORTED


def test_tc_large_k_full_row_path(ctx):
    """k = 57344: the full-row kernel's per-centre values no longer fit in
    shared memory and are recomputed in its binary64 pass.  In the
    cancellation regime every pair fails the reliability test, so every row
    goes through that kernel; a duplicated centre makes ties that only the
    binary64 pass decides (lowest index)."""
    import paper_2407_12208_gb300 as pkg
    n, d, k = 60000, 16, 57344
    X, C = workloads.cancellation(n, d, k, seed=71)
    C[1] = C[0]
    lab, md, nf, st = _run_assign(ctx, X, C, "bf16")
    assert st["overflow_rows"] + st["ambiguous_rows"] > 0
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([rng.choice(n, 48, replace=False), np.nonzero((X == C[0]).all(1))[0]]))
    olab, od1, od2 = oracle.assign(X[rows], C)
    margin = np.where(np.isfinite(od2), (od2 - od1) / np.maximum(od2, 1e-300), np.inf)
    sel = margin > MARGIN
    assert np.array_equal(lab[rows][sel], olab[sel])
    ties = ~sel
    if ties.any():  # exact ties: lowest index, as the oracle
        assert np.array_equal(lab[rows][ties], olab[ties])
    np.testing.assert_allclose(md[rows], oracle.dist_labelled(X[rows], C, lab[rows]), rtol=RTOL_MD, atol=1e-30)


def test_update_small_d_long_label_runs(ctx):
    """The small-d centre sums: labels in long runs (as an image's pixels) and
    enough rows that every warp folds its shared accumulators several times."""
    import paper_2407_12208_gb300 as pkg
    n, d, k = 12_000_000, 1, 3
    rng = np.random.default_rng(9)
    X = (rng.standard_normal((n, d)) * 10.0).astype(np.float32)
    lab = ((np.arange(n) // 1000) % k).astype(np.int32)
    lab[::7777] = 1  # a few short runs inside the long ones
    C = np.zeros((k, d), dtype=np.float32)
    p = pkg.params("fp64", empty="keep")
    Cn, cnt, _ = ctx.update_centroids(_dev(X), _dev(lab), _dev(C), p, min_dist=None)
    oC, ocnt, _ = oracle.update(X, lab, C, 0, np.zeros(n))
    assert np.array_equal(cnt.cpu().numpy(), ocnt)
    np.testing.assert_allclose(Cn.cpu().numpy(), oC, rtol=2 ** -22, atol=1e-30)


@pytest.mark.parametrize("d", [1, 3, 5, 8])
@pytest.mark.parametrize("pattern", ["runs", "random", "mixed"])
def test_small_d_sums_label_patterns(ctx, d, pattern):
    """The small-d centre sums (one warp scan over runs of equal labels) for
    labels in long runs, in no order, and both mixed, at ragged row counts:
    counts exact and centres within the Lemma 4.4 bound of the oracle's."""
    import paper_2407_12208_gb300 as pkg
    k = 16 if d <= 5 else 40
    r = np.random.default_rng(100 + d)
    for n in (777, 262_417, 1_500_001):
        X = (r.standard_normal((n, d)) * 3.0 + 1.0).astype(np.float32)
        if pattern == "runs":
            lab = ((np.arange(n) // 613) % k).astype(np.int32)
        elif pattern == "random":
            lab = r.integers(0, k, size=n).astype(np.int32)
        else:
            lab = ((np.arange(n) // 4001) % k).astype(np.int32)
            noisy = r.random(n) < 0.02
            lab[noisy] = r.integers(0, k, size=int(noisy.sum())).astype(np.int32)
        C = r.standard_normal((k, d)).astype(np.float32)
        p = pkg.params("fp64", empty="keep")
        Cn, cnt, _ = ctx.update_centroids(_dev(X), _dev(lab), _dev(C), p, min_dist=None)
        torch.cuda.synchronize()
        oC, ocnt, _ = oracle.update(X, lab, C, 0, np.zeros(n))
        assert np.array_equal(cnt.cpu().numpy(), ocnt)
        np.testing.assert_allclose(Cn.cpu().numpy(), oC, rtol=2 ** -22, atol=1e-30)


def test_small_d_image_step_equals_assign_then_update(ctx):
    """A Voronoi image's pixels (d = 5, labels in long runs): km_lloyd_step,
    whose small-d centre sums carry each row's distance in the same pass over
    X, equals km_assign followed by km_update_centroids bit for bit."""
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.voronoi_image(640, 480, 12, 12, seed=66)
    Xd, Cd = _dev(X), _dev(C)
    p = pkg.params("fp32", empty="keep")
    lab1, md1, _ = ctx.assign(Xd, Cd, p)
    Cn1, cnt1, _ = ctx.update_centroids(Xd, lab1, Cd, p, min_dist=md1)
    lab2, md2, Cn2, cnt2, _ = ctx.lloyd_step(Xd, Cd, p)
    torch.cuda.synchronize()
    assert np.array_equal(lab2.cpu().numpy(), lab1.cpu().numpy())
    assert np.array_equal(md2.cpu().numpy().view(np.uint64), md1.cpu().numpy().view(np.uint64))
    assert np.array_equal(Cn2.cpu().numpy().view(np.uint32), Cn1.cpu().numpy().view(np.uint32))
    assert np.array_equal(cnt2.cpu().numpy(), cnt1.cpu().numpy())
    olab, od, _ = oracle.assign(X, C)
    assert np.array_equal(lab2.cpu().numpy(), olab)
    np.testing.assert_allclose(md2.cpu().numpy(), od, rtol=1e-12)


# ------------------------------------------------------ quantisation (step a1)
def _e4m3_edge_rows(d):
    rows = []
    for j in range(-24, 25, 4):
        edge = np.float32(448.0 * 2.0 ** j)
        for m in (edge, np.nextafter(edge, np.float32(np.inf)), np.nextafter(edge, np.float32(0))):
            r = np.linspace(-0.9, 0.9, d).astype(np.float32) * m
            r[j % d] = -m
            rows.append(r)
    rows.append(np.zeros(d, np.float32))
    rows.append(np.full(d, 1e-40, np.float32))       # binary32 subnormal maximum: the clamped scale
    rows.append(np.full(d, 3e-37, np.float32))
    return np.stack(rows)


@pytest.mark.parametrize("low", ["fp16", "bf16", "e4m3"])
@pytest.mark.parametrize("d", [37, 128])
def test_quantize_bitexact(ctx, low, d):
    """km_quantize (Alg. 2's first line) against the oracle's quantisation:
    the low-format values and the E4M3 row scales bit for bit, ||x||^2 to
    the binary32 rounding, the norms as upper bounds within (1 + 2^-11)."""
    fmt = {"fp16": 0, "bf16": 1, "e4m3": 2}[low]
    r = np.random.default_rng(d)
    X = (r.normal(size=(700, d)) * 10.0 ** r.uniform(-3, 3, size=(700, 1))).astype(np.float32)
    if fmt == 2:
        X = np.concatenate([X, _e4m3_edge_rows(d)])
    Xq, stats, scale = ctx.quantize(_dev(X), low)
    torch.cuda.synchronize()
    n = X.shape[0]
    tdt = {0: torch.float16, 1: torch.bfloat16, 2: torch.float8_e4m3fn}[fmt]
    vals = Xq.view(tdt).float().cpu().numpy().astype(np.float64)
    sc = scale.cpu().numpy().astype(np.float64)
    st = stats.cpu().numpy().astype(np.float64)
    oq, op, onx, onq, onr, osc = oracle.row_quant_stats(X, fmt, per_row_scale=(fmt == 2))
    np.testing.assert_array_equal(sc, osc)
    np.testing.assert_array_equal(vals[:, :d] * sc[:, None], oq.astype(np.float64))
    assert np.all(vals[:, d:] == 0.0)
    # ||x||^2: the binary64 value rounded to binary32 (ties below 2^-44 aside)
    np.testing.assert_allclose(st[:, 0], op, rtol=2.0 ** -23, atol=0)
    # rows whose squares approach binary32's underflow: infinite bound terms
    # (every pair of such a row goes to the direct formula)
    tiny = (np.abs(X).max(axis=1) > 0) & (onx ** 2 < 2.0 ** -100)
    assert np.all(np.isinf(st[tiny, 2])) and np.all(np.isinf(st[tiny, 3]))
    ok = ~tiny
    for col, ref in ((1, onx), (2, onq), (3, onr)):
        assert np.all(st[ok, col] >= ref[ok] * (1 - 2.0 ** -40)), col
        assert np.all(st[ok, col] <= ref[ok] * (1 + 2.0 ** -11) + 1e-37), col


# ------------------------------------------- empty clusters on the mixed path
@pytest.mark.parametrize("low", ["bf16", "fp16", "e4m3"])
def test_lloyd_mixed_empty_cluster_farthest(low):
    """A centre far from every point empties its cluster in the first
    iteration: KM_EMPTY_FARTHEST re-seeds it with the point of largest
    min_dist (binary64-accurate on the mixed path, as the oracle's).  Labels,
    centres and the SSE trajectory follow oracle.lloyd."""
    import paper_2407_12208_gb300 as pkg
    c = pkg.Context(0)
    X, C0 = workloads.gaussian_mixture(20000, 64, 32, seed=63)
    C0[5] = C0[5] + 1e3
    C0[17] = C0[17] - 1e3
    p = pkg.params(low, max_iter=6, empty="farthest")
    C, lab, sse, eta, it = c.lloyd_run(_dev(X), _dev(C0), p)
    oC, olab, osse, oit = oracle.lloyd(X, C0, 6, empty_policy=1)
    assert np.array_equal(lab.cpu().numpy(), olab)
    np.testing.assert_allclose(C.cpu().numpy(), oC, rtol=2 ** -22, atol=1e-30)
    np.testing.assert_allclose(sse, osse, rtol=RTOL_MIXED)
    # the first SSE (before any update) is the sum of binary64-accurate distances
    np.testing.assert_allclose(sse[0], osse[0], rtol=1e-12)


def test_workspace_is_linear_in_n(ctx):
    """The workspace of every synchronous call is O(n): below 1 GB at the
    1e6 x 128, k = 1024 benchmark shape, in every low format."""
    import paper_2407_12208_gb300 as pkg
    for low in ("bf16", "fp16", "e4m3", "fp32", "fp64"):
        b = ctx.workspace_size(1_000_000, 128, 1024, pkg.params(low))
        assert b < 1_000_000_000, (low, b)


def test_distances_queue_overflow_scans(ctx):
    """More flagged pairs than the bounded queue holds (every pair of the
    cancellation data): the binary64 patch finds them by their marks."""
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.cancellation(300, 32, 300, seed=64)
    D, bits, nf = ctx.distances(_dev(X), _dev(C), pkg.params("bf16", "tc"))
    D = D.cpu().numpy().astype(np.float64)
    assert nf == 300 * 300
    np.testing.assert_allclose(D, oracle.dist_direct(X, C), rtol=2 ** -23, atol=1e-38)


def test_empty_farthest_many_clusters_at_scale(ctx):
    """64 empty clusters at n = 4e6: the rows of largest min_dist (ties to
    the lowest index: min_dist on a coarse grid makes many ties) in one
    cooperative radix selection, as the oracle's ordered walk picks them, in
    well under a millisecond more than keeping the old centres."""
    import paper_2407_12208_gb300 as pkg
    n, d, k = 4_000_000, 8, 256
    r = np.random.default_rng(65)
    X = r.normal(size=(n, d)).astype(np.float32)
    lab = r.integers(0, k, size=n).astype(np.int32)
    lab[lab % 4 == 1] -= 1  # clusters 1, 5, 9, ...: 64 empty
    md = np.round(r.random(n) * 1e5) / 1e5
    C = r.normal(size=(k, d)).astype(np.float32)
    Xd, labd, Cd, mdd = _dev(X), _dev(lab), _dev(C), _dev(md)
    pf, pk = pkg.params("fp64", empty="farthest"), pkg.params("fp64", empty="keep")
    for p in (pf, pk):
        ctx.update_centroids(Xd, labd, Cd, p, min_dist=mdd, want_shift=False)
    torch.cuda.synchronize()

    def timed(p):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            ctx.update_centroids(Xd, labd, Cd, p, min_dist=mdd, want_shift=False)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 5

    extra_ms = timed(pf) - timed(pk)
    Cn, cnt, _ = ctx.update_centroids(Xd, labd, Cd, pf, min_dist=mdd)
    oC, ocnt, _ = oracle.update(X, lab, C, 1, md)
    assert np.array_equal(cnt.cpu().numpy(), ocnt)
    empty = np.nonzero(ocnt == 0)[0]
    assert empty.size == 64
    Cn = Cn.cpu().numpy()
    np.testing.assert_array_equal(Cn[empty], oC[empty])  # the same rows, in the same order
    np.testing.assert_allclose(Cn, oC, rtol=2 ** -22, atol=1e-30)
    assert extra_ms < 1.0, extra_ms


# --------------------------------------- config-3 trajectories at full size
@pytest.mark.parametrize("low", ["fp16", "e4m3"])
def test_mixture_lloyd_full_size_teacher_forced(low):
    """The mixed-precision Lloyd iteration at its full size (Gaussian mixture
    n = 4e6, d = 64, k = 256) for 50 iterations, teacher-forced: every GPU
    iteration starts from the oracle's centres; labels and min_dist on 2000
    sampled rows against the oracle's assignment, counts and centres against
    the oracle's update (Eq. (center)) of the GPU's labels, every iteration."""
    import paper_2407_12208_gb300 as pkg
    c = pkg.Context(0)
    n, d, k = 4_000_000, 64, 256
    X, C0 = workloads.gaussian_mixture(n, d, k, seed=15)
    Xd = _dev(X)
    p = pkg.params(low, empty="farthest")
    rows = np.sort(np.random.default_rng(17).choice(n, 2000, replace=False))
    C = C0.copy()
    sse = []
    for it in range(50):
        lab, md, Cn, cnt, _ = c.lloyd_step(Xd, _dev(C), p)
        torch.cuda.synchronize()
        lab, md, Cn, cnt = lab.cpu().numpy(), md.cpu().numpy(), Cn.cpu().numpy(), cnt.cpu().numpy()
        check_assign(lab[rows], md[rows], X[rows], C, oracle, RTOL_MD)
        oC, ocnt, _ = oracle.update(X, lab, C, 1, md)
        assert np.array_equal(cnt, ocnt), it
        np.testing.assert_allclose(Cn, oC, rtol=2 ** -22, atol=1e-30)
        sse.append(float(md.sum()))
        C = oC
    # SSE never increases along the (teacher-forced) iteration, Lemma 2.1
    assert all(b <= a * (1 + 1e-9) for a, b in zip(sse, sse[1:]))


# ------------------------------------------------- choosing the low format
def test_choose_low_predicts_list_overflow(ctx):
    """km_choose_low: on uniform data E4M3's error bound exceeds the spread of
    the distances (every row's candidates overflow its list) and BF16 is
    chosen; on points tight around well-separated centres E4M3 keeps one
    candidate per row and is chosen.  The predicted overflow share is what an
    E4M3 assignment of the same data then measures, within 0.1."""
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.uniform_pairs(20000, 128, 256, seed=66)
    # points tightly around 64 centres N(0, 25) apart, and those centres
    r = np.random.default_rng(67)
    C2 = r.normal(0.0, 5.0, size=(64, 128)).astype(np.float32)
    X2 = (C2[r.integers(0, 64, size=20000)] + r.normal(0.0, 0.01, size=(20000, 128))).astype(np.float32)
    for Xh, Ch, expect in ((X, C, "bf16"), (X2, C2, "e4m3")):
        Xd, Cd = _dev(Xh), _dev(Ch)
        low, st = ctx.choose_low(Xd, Cd, max_overflow_share=0.01)
        assert low == expect, (low, st)
        ctx.assign(Xd, Cd, pkg.params("e4m3"))
        measured = ctx.stats()["overflow_rows"] / Xh.shape[0]
        assert abs(measured - st["e4m3"][1]) <= 0.1, (measured, st)
        assert st["bf16"][1] <= 0.01 and st["bf16"][0] >= 1.0
    with pytest.raises(pkg.KmError) as ei:
        ctx.choose_low(_dev(X), _dev(C), max_overflow_share=2.0)
    assert ei.value.status == pkg._binding.KM_EINVAL


# ------------------------------- the precision matrix of Tables 6.1 / 6.2
def _flags_of(bits, n, k):
    bits = bits.cpu().numpy().view(np.uint32)
    idx = np.arange(n * k)
    return ((bits[idx >> 5] >> (idx & 31)) & 1).reshape(n, k).astype(bool)


@pytest.mark.parametrize("fb", ["fp64", "fp32"])
@pytest.mark.parametrize("c_A", [1.0, 2.0])
def test_distances_fp32_alg2_bitexact(ctx, fb, c_A):
    """Alg. 2 with binary32 as the low precision (FP32 -> FP64 and FP32 ->
    FP32 of Table 6.1): every pair's flag and value equal the oracle's
    emulation of Alg. 2 bit for bit (values stored in binary32)."""
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.near_far(120, 64, 0.5, seed=68)
    C = C[:90]
    p = pkg.params("fp32x", "paper", rho=5.0, paper_factor=c_A, fallback=fb)
    D, bits, nf = ctx.distances(_dev(X), _dev(C), p)
    D = D.cpu().numpy()
    flags = _flags_of(bits, 120, 90)
    fbf = 4 if fb == "fp64" else 3
    ref_d = np.empty((120, 90), np.float32)
    ref_f = np.empty((120, 90), bool)
    for i in range(120):
        for j in range(90):
            f, d, _, _ = oracle.mp_dist_fb(X[i], C[j], 5.0, 3, fbf, c_A)
            ref_d[i, j], ref_f[i, j] = np.float32(d), f
    assert np.array_equal(flags, ref_f) and nf == int(ref_f.sum())
    assert 0 < nf < 120 * 90
    np.testing.assert_array_equal(D.view(np.uint32), ref_d.view(np.uint32))


@pytest.mark.parametrize("low,fb", [("fp16", "low"), ("bf16", "low"), ("fp16", "fp32"), ("bf16", "fp32")])
def test_distances_fallback_precisions(ctx, low, fb):
    """Eq. (fallback-rule) in the chosen precision: the flagged pairs hold
    the direct formula evaluated with every operation rounded to the low
    format (the same-precision fallback) or to binary32, as the oracle
    emulates it, bit for bit; the unflagged ones are within the bound."""
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.near_far(300, 128, 0.5, seed=69)
    C = C[:200]
    p = pkg.params(low, "tc", fallback=fb)
    D, bits, nf = ctx.distances(_dev(X), _dev(C), p)
    D = D.cpu().numpy()
    flags = _flags_of(bits, 300, 200)
    assert flags.sum() == nf > 0
    fmt = {"fp16": 0, "bf16": 1}[low]
    fbf = fmt if fb == "low" else 3
    ii, jj = np.nonzero(flags)
    ref = np.array([oracle.dist_direct_fmt(X[i], C[j], fbf) for i, j in zip(ii, jj)], dtype=np.float32)
    np.testing.assert_array_equal(D[ii, jj].view(np.uint32), ref.view(np.uint32))
    Dex = oracle.dist_direct(X, C)
    B = oracle.tc_bound_matrix(X, C, fmt)
    un = ~flags
    assert np.all(np.abs(D[un] - Dex[un]) <= B[un] + 1e-6 * Dex[un])


@pytest.mark.parametrize("low", ["fp64", "fp32"])
def test_distances_direct_modes(ctx, low):
    """The direct formula for every pair (the FP64 direct row of Table 6.1,
    and binary32): the oracle's values bit for bit, nothing flagged."""
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.blobs(150, 40, 70, seed=70)
    D, bits, nf = ctx.distances(_dev(X), _dev(C), pkg.params(low))
    D = D.cpu().numpy()
    if low == "fp64":
        ref = oracle.dist_direct(X, C).astype(np.float32)
    else:
        ref = np.array([[oracle.dist_direct_fmt(x, c, 3) for c in C] for x in X], dtype=np.float32)
    np.testing.assert_array_equal(D.view(np.uint32), ref.view(np.uint32))
    assert nf == 0


def test_precision_modes_rejected_where_undefined(ctx):
    import paper_2407_12208_gb300 as pkg
    X = _dev(np.random.default_rng(0).random((64, 32), dtype=np.float32))
    for p in (pkg.params("fp32x"), pkg.params("bf16", fallback="fp32")):
        with pytest.raises(pkg.KmError) as ei:
            ctx.assign(X, X[:4], p)  # the assignment certifies in fp32 and binary64 itself
        assert ei.value.status == pkg._binding.KM_EUNSUPPORTED
    with pytest.raises(pkg.KmError) as ei:
        ctx.distances(X, X[:4], pkg.params("e4m3", fallback="low"))
    assert ei.value.status == pkg._binding.KM_EUNSUPPORTED


# ------------------------------------------- replayed (graph-recorded) iterations
@pytest.mark.parametrize("low,shape", [("bf16", (30000, 128, 200)), ("fp16", (20000, 64, 64)),
                                       ("fp32", (50000, 5, 16)), ("fp64", (5000, 16, 8))])
def test_lloyd_graph_replay_equals_direct_launches(low, shape):
    """km_lloyd_run replays its iterations as two recorded CUDA graphs; with
    phase timing on it launches them kernel by kernel.  Both give the same
    centres, labels, SSE and flag trajectories bit for bit, and the library
    counts the same kernels plus the one that appends each replayed
    iteration's SSE and flag count."""
    import paper_2407_12208_gb300 as pkg
    n, d, k = shape
    X, C0 = workloads.gaussian_mixture(n, d, k, seed=90)
    C0[-1] += 1e3  # an empty cluster in the first iteration
    p = pkg.params(low, max_iter=7, empty="farthest")
    out = []
    for prof in (False, True):
        c = pkg.Context(0)
        c.set_profiling(prof)
        l0 = c.launch_count()
        C, lab, sse, eta, it = c.lloyd_run(_dev(X), _dev(C0), p)
        torch.cuda.synchronize()
        out.append((C.cpu().numpy(), lab.cpu().numpy(), sse.copy(), eta.copy(), it, c.launch_count() - l0))
        c.close()
    (Cg, lg, sg, eg, ig, ng), (Cd, ld, sd, ed, idd, nd) = out
    assert ig == idd == 7 and ng == nd + 7
    assert np.array_equal(Cg.view(np.uint32), Cd.view(np.uint32))
    assert np.array_equal(lg, ld)
    assert np.array_equal(sg.view(np.uint64), sd.view(np.uint64)) and np.array_equal(eg, ed)


# ------------------------------------------- row-sharded updates on one GPU
def test_sharded_update_equals_whole(ctx):
    """Two row shards' fixed-point partial sums, added as integers and
    finalised, give km_update_centroids' centres of all rows bit for bit
    (the exchange of a data-parallel iteration); km_farthest_rows orders the
    rows by min_dist, ties to the lowest index."""
    import paper_2407_12208_gb300 as pkg
    n, d, k = 30001, 32, 40
    X, C = workloads.gaussian_mixture(n, d, k, seed=92)
    lab = oracle.assign(X, C)[0]
    lab[lab == 7] = 8  # an empty cluster
    Xd, Cd, labd = _dev(X), _dev(C), _dev(lab)
    bits = ctx.absmax(Xd)
    assert bits == int(np.array([np.abs(X).max()], np.float32).view(np.uint32)[0])
    cut = 12345
    s1, c1 = ctx.update_partial(Xd[:cut], labd[:cut], k, bits, n)
    s2, c2 = ctx.update_partial(Xd[cut:], labd[cut:], k, bits, n)
    Cn, sh = ctx.update_finalize(s1 + s2, c1 + c2, Cd, bits, n)
    Cr, cnt_r, sh_r = ctx.update_centroids(Xd, labd, Cd, pkg.params("bf16", empty="keep"))
    torch.cuda.synchronize()
    assert np.array_equal(Cn.cpu().numpy().view(np.uint32), Cr.cpu().numpy().view(np.uint32))
    assert np.array_equal((c1 + c2).cpu().numpy(), cnt_r.cpu().numpy())
    assert sh == sh_r
    md = np.round(np.random.default_rng(3).random(n) * 1e3) / 1e3  # many ties
    rows, vals = ctx.farthest_rows(_dev(md), 50, k=k)
    ref = np.lexsort((np.arange(n), -md))[:50]
    assert np.array_equal(rows.cpu().numpy(), ref) and np.array_equal(vals.cpu().numpy(), md[ref])


def test_data_parallel_iteration_on_the_gpu(ctx):
    """ShardedLloyd (the row-sharded iteration with its exact integer
    exchange) driving the library on this GPU through a one-rank NCCL group:
    centres, labels, min_dist and SSE equal km_lloyd_step's, iteration after
    iteration, empty clusters re-seeded the same way."""
    import socket
    import torch.distributed as dist
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300.dp import ShardedLloyd
    X, C = workloads.gaussian_mixture(20000, 32, 48, seed=93)
    C[::7] += 500.0  # far centres: empty clusters in the first iteration
    Xd, Cd = _dev(X), _dev(C)
    p = pkg.params("bf16", empty="farthest")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, world_size=1, rank=0)
    try:
        sl = ShardedLloyd(ctx, Xd, C.shape[0], p)
        Cs, Cr = Cd.clone(), Cd.clone()
        for it in range(4):
            Cs, lab_s, md_s, sse_s, sh_s = sl.step(Cs)
            lab_r, md_r, Cr2, cnt_r, sh_r = ctx.lloyd_step(Xd, Cr, p)
            sse_r = ctx.stats()["sse"]
            torch.cuda.synchronize()
            assert np.array_equal(lab_s.cpu().numpy(), lab_r.cpu().numpy()), it
            assert np.array_equal(md_s.cpu().numpy().view(np.uint64), md_r.cpu().numpy().view(np.uint64)), it
            assert np.array_equal(Cs.cpu().numpy().view(np.uint32), Cr2.cpu().numpy().view(np.uint32)), it
            assert sse_s == sse_r, it
            assert sh_s == pytest.approx(sh_r, rel=1e-12), it
            Cr = Cr2
    finally:
        dist.destroy_process_group()
