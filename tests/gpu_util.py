"""Helpers shared by the GPU parity tests (comparison logic only)."""
import numpy as np

MARGIN = 1e-6      # labels must match where the oracle's (d2 - d1) / d2 exceeds this
RTOL_MIXED = 1e-5  # distances / SSE of the mixed path
RTOL_FP64 = 1e-12  # binary64 steps


def check_assign(lab, md, X, C, oracle, rtol):
    """Labels equal the oracle's wherever its relative best/second-best margin
    exceeds MARGIN; elsewhere the GPU label must still be a minimiser within
    tolerance.  min_dist within rtol of the oracle's best distance."""
    olab, od1, od2 = oracle.assign(X, C)
    with np.errstate(invalid="ignore", divide="ignore"):  # k = 1: od2 is inf (the other branch)
        margin = np.where(np.isfinite(od2), (od2 - od1) / np.maximum(od2, 1e-300), np.inf)
    sel = margin > MARGIN
    bad = np.nonzero(sel & (lab != olab))[0]
    assert bad.size == 0, "label mismatch at rows %s (gpu %s oracle %s)" % (bad[:5], lab[bad[:5]], olab[bad[:5]])
    # rows inside the margin: the chosen centre is (nearly) optimal
    if (~sel).any():
        rows = np.nonzero(~sel)[0][:200]
        D = oracle.dist_direct(X[rows], C)
        chosen = D[np.arange(rows.size), lab[rows]]
        assert np.all(chosen <= D.min(axis=1) * (1 + 2 * MARGIN) + 1e-300)
    err = np.abs(md - od1) / np.maximum(np.abs(od1), 1e-300)
    ok = (err <= rtol) | (np.abs(md - od1) <= 1e-30)
    assert ok.all(), "min_dist rel. err %.3e at row %d" % (err.max(), int(np.argmax(err)))
    return olab, od1, od2
