"""Seeded random shapes through the assignment and the Lloyd step: n from 1,
k from 1 up to n, d from 1 to 300 (odd widths, tails past every tile), every
format, three data families.  Labels, min_dist, counts and centres against
the oracle on every case."""
import numpy as np
import pytest

import oracle
from paper_2407_12208_gb300 import workloads
from gpu_util import RTOL_MD, check_assign

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


def _case(i):
    r = np.random.default_rng(1000 + i)
    n = int(r.choice([1, 2, 7, 129, 1000, 2500, 4097]))
    k = int(r.integers(1, min(n, 1100) + 1))
    d = int(r.choice([1, 3, 5, 8, 13, 16, 31, 64, 100, 128, 130, 256, 300]))
    lows = ["fp16", "bf16", "fp32", "fp64"] + (["e4m3"] if d >= 16 else [])
    low = str(r.choice(lows))
    if d > 256 and low in ("fp16", "bf16"):
        low = "fp32"  # wider rows than the 16-bit tiles take
    fam = int(r.integers(0, 3))
    seed = 2000 + i
    if fam == 0:
        X, C = workloads.uniform_pairs(n, d, k, seed)
    elif fam == 1:
        X, C = workloads.gaussian_mixture(n, d, k, seed)
    else:
        X, C = workloads.blobs(n, d, k, seed)
    return low, X, C


@pytest.mark.parametrize("i", range(36))
def test_random_shapes_against_the_oracle(ctx, i):
    import paper_2407_12208_gb300 as pkg
    low, X, C = _case(i)
    p = pkg.params(low)
    Xd, Cd = _dev(X), _dev(C)
    lab, md, _ = ctx.assign(Xd, Cd, p)
    torch.cuda.synchronize()
    lab, md = lab.cpu().numpy(), md.cpu().numpy()
    check_assign(lab, md, X, C, oracle, RTOL_MD)
    lab2, md2, Cn, cnt, _ = ctx.lloyd_step(Xd, Cd, p)
    torch.cuda.synchronize()
    assert np.array_equal(lab2.cpu().numpy(), lab)
    assert np.array_equal(md2.cpu().numpy().view(np.uint64), md.view(np.uint64))
    oC, ocnt, _ = oracle.update(X, lab, C, 1, md)
    assert np.array_equal(cnt.cpu().numpy(), ocnt)
    np.testing.assert_allclose(Cn.cpu().numpy(), oC, rtol=2 ** -22, atol=1e-30)
