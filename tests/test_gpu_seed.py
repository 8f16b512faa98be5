"""GPU parity of km_seed_pp (D^2-sampling seeding) with the oracle.

The draws are inputs, so both sides see the same ones.  The oracle follows
the GPU's picks step by step and reports, per step, its own pick and how far
the draw lies from the nearest boundary between two rows; wherever that
margin exceeds the rounding of the two implementations' sums (1e-9 of T),
the picks must be equal -- elsewhere either row is a correct pick."""
import numpy as np
import pytest

import oracle
from paper_2407_12208_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MARGIN_TOL = 1e-9


@pytest.fixture(scope="module")
def ctx():
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300 import build
    build.build()
    c = pkg.Context(0)
    yield c
    c.close()


def _check(ctx, X, u):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    C, idx = ctx.seed_pp(Xd, u)
    torch.cuda.synchronize()
    oidx, margin = oracle.kmeanspp(X, u, follow=idx)
    unique = margin > MARGIN_TOL
    bad = np.nonzero(unique & (oidx != idx))[0]
    assert bad.size == 0, "picks differ at steps %s (gpu %s oracle %s)" % (bad[:5], idx[bad[:5]], oidx[bad[:5]])
    assert np.array_equal(C.cpu().numpy(), X[idx])
    return idx, unique


@pytest.mark.parametrize("d", [2, 5, 16, 37, 128, 300])
def test_seed_matches_oracle(ctx, d):
    X, _ = workloads.blobs(2000, d, 20, seed=100 + d)
    u = workloads.seed_uniforms(50, seed=200 + d)
    idx, unique = _check(ctx, X, u)
    assert unique.mean() > 0.9
    assert len(set(idx.tolist())) == 50  # distinct points: a picked row has D^2 = 0


def test_seed_at_scale(ctx):
    X, _ = workloads.uniform_pairs(100_000, 128, 1, seed=301)
    u = workloads.seed_uniforms(128, seed=302)
    _check(ctx, X, u)


def test_seed_every_row_and_coincident_points(ctx):
    X = np.random.default_rng(7).normal(size=(20, 3)).astype(np.float32)
    u = workloads.seed_uniforms(20, seed=8)
    idx, _ = _check(ctx, X, u)
    assert sorted(idx.tolist()) == list(range(20))  # k = n: every row once
    Z = np.zeros((64, 8), dtype=np.float32)           # every point on the first pick: the uniform rule
    u = np.array([0.0, 0.5, 0.25, 0.999])
    idx, _ = _check(ctx, Z, u)
    assert idx.tolist() == [0, 32, 16, 63]


def test_seed_rejects_draws_outside_the_unit_interval(ctx):
    from paper_2407_12208_gb300._binding import KmError
    X = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(KmError, match="EINVAL"):
        ctx.seed_pp(X, [0.1, 1.0])
    with pytest.raises(KmError, match="EINVAL"):
        ctx.seed_pp(X, [0.1] * 11)  # k > n
