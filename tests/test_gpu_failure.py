"""GPU test of the failure path: a device-side wait that nothing satisfies
runs out of its bounded budget, the call reports KM_ETIMEOUT with a message,
and the context and device keep working.  No fault, trap or hang: the wait is
the library's own bounded one (about a second)."""
import numpy as np
import pytest

from paper_2407_12208_gb300 import workloads
from gpu_util import RTOL_MIXED, check_assign

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_wait_runs_out_and_context_stays_usable():
    import oracle
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300 import build
    build.build()
    ctx = pkg.Context(0)
    try:
        rc = ctx.selftest_timeout()
        assert rc == pkg._binding.KM_ETIMEOUT
        assert "wait" in ctx.lib.km_last_error(ctx.h).decode()
        # the same context still computes correct assignments afterwards
        X, C = workloads.blobs(3000, 64, 20, seed=81)
        lab, md, _ = ctx.assign(torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), pkg.params("bf16"))
        torch.cuda.synchronize()
        check_assign(lab.cpu().numpy(), md.cpu().numpy(), X, C, oracle, RTOL_MIXED)
        assert ctx.stats()["pairs"] == 3000 * 20
    finally:
        ctx.close()
