"""GPU tests of the screening kernel's epilogue variants and of km_autotune.

The three variants (64-column steps staging all quads or half of them, and
32-column steps) must give the same labels, distances and flag counts, each
equal to the oracle's; the autotuner must time them and keep the fastest."""
import numpy as np
import pytest

import oracle
from paper_2407_12208_gb300 import workloads
from gpu_util import check_assign

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VARIANTS = ("full", "half", "c32")


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


def _data(kind, n, d, k, seed):
    if kind == "uniform":
        return workloads.uniform_pairs(n, d, k, seed)
    if kind == "mixture":
        return workloads.gaussian_mixture(n, d, k, seed)
    return workloads.cancellation(n, d, k, seed)


def _assign_with(ctx, X, C, low, variant):
    import paper_2407_12208_gb300 as pkg
    n, d = X.shape
    ctx.set_screen_variant(n, d, C.shape[0], low, variant)
    try:
        lab, md, nf = ctx.assign(_dev(X), _dev(C), pkg.params(low))
        torch.cuda.synchronize()
    finally:
        ctx.set_screen_variant(n, d, C.shape[0], low, "auto")
    return lab.cpu().numpy(), md.cpu().numpy(), nf


CASES = [
    ("uniform", 3001, 128, 300, "bf16"),
    ("uniform", 2000, 128, 1024, "fp16"),
    ("mixture", 2500, 64, 256, "fp16"),
    ("cancellation", 1500, 128, 64, "bf16"),
    ("mixture", 1200, 200, 130, "e4m3"),
    ("uniform", 700, 37, 130, "bf16"),
    ("mixture", 300, 16, 5, "e4m3"),
]


@pytest.mark.parametrize("kind,n,d,k,low", CASES)
def test_screen_variants_agree_with_oracle(ctx, kind, n, d, k, low):
    X, C = _data(kind, n, d, k, seed=n + 3 * d + k)
    out = {}
    for v in VARIANTS:
        lab, md, nf = _assign_with(ctx, X, C, low, v)
        check_assign(lab, md, X, C, oracle)
        out[v] = (lab, md, nf)
    for v in VARIANTS[1:]:
        assert np.array_equal(out[v][0], out["full"][0]), v
        assert np.array_equal(out[v][1].view(np.uint64), out["full"][1].view(np.uint64)), v
        assert out[v][2] == out["full"][2], v


def test_screen_variants_identical_at_scale(ctx):
    """200,000 x 128 rows, k = 1024 (the 1e6-row benchmark's row blocks and
    tiles): the variants agree bit for bit; sampled rows match the oracle."""
    X, C = workloads.uniform_pairs(200_000, 128, 1024, seed=91)
    out = {v: _assign_with(ctx, X, C, "bf16", v) for v in VARIANTS}
    for v in VARIANTS[1:]:
        assert np.array_equal(out[v][0], out["full"][0]), v
        assert np.array_equal(out[v][1].view(np.uint64), out["full"][1].view(np.uint64)), v
    rows = np.random.default_rng(5).choice(X.shape[0], 400, replace=False)
    lab, md, _ = out["full"]
    check_assign(lab[rows], md[rows], X[rows], C, oracle)


def test_autotune_times_the_variants_and_keeps_the_fastest(ctx):
    import paper_2407_12208_gb300 as pkg
    X, C = workloads.uniform_pairs(100_000, 128, 1024, seed=17)
    Xd, Cd = _dev(X), _dev(C)
    p = pkg.params("bf16")
    v, ms = ctx.autotune(Xd, Cd, p)
    assert v in VARIANTS
    assert all(m > 0 for m in ms), ms
    assert ms[VARIANTS.index(v)] == min(ms)
    # the kept variant gives the results of every other
    lab, md, nf = ctx.assign(Xd, Cd, p)
    ref = _assign_with(ctx, X, C, "bf16", "c32")
    assert np.array_equal(lab.cpu().numpy(), ref[0])
    assert np.array_equal(md.cpu().numpy().view(np.uint64), ref[1].view(np.uint64))
    ctx.set_screen_variant(100_000, 128, 1024, "bf16", "auto")
    # K wider than two atoms: one variant, nothing timed; direct formats: none
    X2, C2 = workloads.uniform_pairs(3000, 256, 100, seed=18)
    v2, ms2 = ctx.autotune(_dev(X2), _dev(C2), p)
    assert v2 == "reg" and ms2 == [-1.0, -1.0, -1.0]
    v3, _ = ctx.autotune(_dev(X2), _dev(C2), pkg.params("fp32"))
    assert v3 == "none"


def test_set_screen_variant_rejects_what_does_not_exist(ctx):
    from paper_2407_12208_gb300._binding import KmError
    with pytest.raises(KmError, match="EUNSUPPORTED"):
        ctx.set_screen_variant(1000, 256, 100, "bf16", "full")
    with pytest.raises(KmError, match="EUNSUPPORTED"):
        ctx.set_screen_variant(1000, 64, 100, "fp32", "full")
    ctx.set_screen_variant(1000, 256, 100, "bf16", "auto")  # nothing to clear: fine
