"""GPU tests of km_assign_static, the fp32 direct assignment whose scratch is
a static device array of the library (no workspace, no allocation).  It must
give the same labels and min_dist as km_assign on the FP32 direct path, bit
for bit, on consecutive calls (the second call sees the scratch the first one
left), and reject sizes above its static limit before any launch.  The file
sorts last so that it also runs after every other GPU test in one process."""
import gc

import numpy as np
import pytest

from paper_2407_12208_gb300 import workloads

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


def _reference(ctx, X, C):
    """The existing entry point, km_assign with low = FP32 direct."""
    import paper_2407_12208_gb300 as pkg
    lab, md, _ = ctx.assign(X, C, pkg.params("fp32"))
    torch.cuda.synchronize()
    return lab.cpu().numpy(), md.cpu().numpy(), ctx.stats()


def _outputs(n):
    return (torch.full((n,), -7, dtype=torch.int32, device="cuda"),
            torch.full((n,), -1.0, dtype=torch.float64, device="cuda"))


def test_static_matches_assign_on_two_calls_in_a_row(ctx):
    # first call: centres 90..99 repeat centres 0..9, so the rows nearest to
    # them tie exactly and go through the list of open rows; second call:
    # fewer rows, so a stale count or list from the first call would reach
    # rows past n or change min_dist
    X1, C1 = workloads.blobs(20000, 64, 100, seed=41)
    C1[90:] = C1[:10]
    X2, C2 = workloads.cancellation(5003, 32, 40, seed=42)
    X1, C1, X2, C2 = _dev(X1), _dev(C1), _dev(X2), _dev(C2)
    lab1, md1 = _outputs(X1.shape[0])
    lab2, md2 = _outputs(X2.shape[0])
    ctx.assign_static(X1, C1, lab1, md1)
    ctx.assign_static(X2, C2, lab2, md2)
    torch.cuda.synchronize()
    got1 = (lab1.cpu().numpy(), md1.cpu().numpy())
    got2 = (lab2.cpu().numpy(), md2.cpu().numpy())
    ref1 = _reference(ctx, X1, C1)
    assert ref1[2]["ambiguous_rows"] > 0  # the list of open rows was exercised
    ref2 = _reference(ctx, X2, C2)
    for got, ref in ((got1, ref1), (got2, ref2)):
        assert np.array_equal(got[0], ref[0])
        assert np.array_equal(got[1].view(np.uint64), ref[1].view(np.uint64))
    # and once more in the other order, on a side stream
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.assign_static(X2, C2, lab2, md2, stream=s)
        ctx.assign_static(X1, C1, lab1, md1, stream=s)
    s.synchronize()
    assert np.array_equal(lab1.cpu().numpy(), ref1[0])
    assert np.array_equal(md1.cpu().numpy().view(np.uint64), ref1[1].view(np.uint64))
    assert np.array_equal(lab2.cpu().numpy(), ref2[0])
    assert np.array_equal(md2.cpu().numpy().view(np.uint64), ref2[1].view(np.uint64))


def test_static_rejects_more_rows_than_its_scratch(ctx):
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300._binding import STATIC_MAX_ROWS
    n = STATIC_MAX_ROWS + 1
    X = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    C = torch.zeros((2, 4), dtype=torch.float32, device="cuda")
    lab, md = _outputs(n)
    with pytest.raises(pkg.KmError) as ei:
        ctx.assign_static(X, C, lab, md)
    assert ei.value.status == 2 and "static scratch" in str(ei.value)
    torch.cuda.synchronize()
    assert int((lab != -7).sum()) == 0  # nothing was launched
    # the largest accepted size still runs and matches km_assign
    Xm, Cm = workloads.blobs(STATIC_MAX_ROWS, 8, 16, seed=43)
    Xm, Cm = _dev(Xm), _dev(Cm)
    lab, md = _outputs(STATIC_MAX_ROWS)
    ctx.assign_static(Xm, Cm, lab, md)
    torch.cuda.synchronize()
    ref = _reference(ctx, Xm, Cm)
    assert np.array_equal(lab.cpu().numpy(), ref[0])
    assert np.array_equal(md.cpu().numpy().view(np.uint64), ref[1].view(np.uint64))


def test_static_requires_both_outputs(ctx):
    import ctypes
    import paper_2407_12208_gb300 as pkg
    X = torch.zeros((8, 4), dtype=torch.float32, device="cuda")
    C = torch.zeros((2, 4), dtype=torch.float32, device="cuda")
    lab = torch.empty(8, dtype=torch.int32, device="cuda")
    rc = ctx.lib.km_assign_static(ctx.h, ctypes.c_void_p(X.data_ptr()), 8, ctypes.c_void_p(C.data_ptr()), 2, 4,
                                  ctypes.c_void_p(lab.data_ptr()), None, None)
    assert rc == pkg._binding.KM_EINVAL


def test_static_allocates_no_device_memory(ctx):
    """After the first call (which resolves the scratch address), further
    calls leave the device's free memory and torch's allocator untouched."""
    X, C = workloads.blobs(30000, 32, 50, seed=44)
    X, C = _dev(X), _dev(C)
    lab, md = _outputs(X.shape[0])
    ctx.assign_static(X, C, lab, md)
    torch.cuda.synchronize()
    # tensors of earlier tests still waiting for the cycle collector must not
    # be freed inside the measured window
    gc.collect()
    gc.disable()
    try:
        free0, _ = torch.cuda.mem_get_info()
        used0 = torch.cuda.memory_allocated()
        for _ in range(3):
            ctx.assign_static(X, C, lab, md)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        used1 = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    assert free1 == free0
    assert used1 == used0
