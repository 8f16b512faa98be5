"""Helpers shared by the GPU parity tests (comparison logic only)."""
import numpy as np

MARGIN = 1e-6      # labels must match where the oracle's (d2 - d1) / d2 exceeds this
RTOL_MIXED = 1e-5  # SSE trajectories of the mixed path (centres may differ by an ulp)
RTOL_FP64 = 1e-12  # binary64 steps
RTOL_MD = 1e-12    # min_dist: the chosen centre's direct distance, binary64-accurate on every path


def check_assign(lab, md, X, C, oracle, rtol=RTOL_MD):
    """Labels equal the oracle's wherever its relative best/second-best margin
    exceeds MARGIN; elsewhere the GPU label must still be a minimiser within
    that margin.  min_dist within rtol of the oracle's binary64 distance to
    the centre the GPU chose (Eq. (dist-direct) for that pair)."""
    olab, od1, od2 = oracle.assign(X, C)
    with np.errstate(invalid="ignore", divide="ignore"):  # k = 1: od2 is inf (the other branch)
        margin = np.where(np.isfinite(od2), (od2 - od1) / np.maximum(od2, 1e-300), np.inf)
    sel = margin > MARGIN
    bad = np.nonzero(sel & (lab != olab))[0]
    assert bad.size == 0, "label mismatch at rows %s (gpu %s oracle %s)" % (bad[:5], lab[bad[:5]], olab[bad[:5]])
    chosen = oracle.dist_labelled(X, C, lab)
    # rows inside the margin: the chosen centre is (nearly) optimal
    assert np.all(chosen <= od1 * (1 + 2 * MARGIN) + 1e-300)
    err = np.abs(md - chosen) / np.maximum(np.abs(chosen), 1e-300)
    ok = (err <= rtol) | (np.abs(md - chosen) <= 1e-30)
    assert ok.all(), "min_dist rel. err %.3e at row %d" % (err.max(), int(np.argmax(err)))
    return olab, od1, od2
