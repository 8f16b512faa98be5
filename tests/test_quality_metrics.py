"""CPU tests of the clustering-quality measures bench.py reports (Section 6.2:
ARI, AMI, and Table 6.7's matched-label Diff).  Pinned by hand-worked cases,
by their invariances, and against scikit-learn's implementations where that
library is installed."""
import itertools
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_ari_hand_worked():
    # a = {0,0,0,1,1,1}, b = {0,0,1,1,2,2}: contingency [[2,1,0],[0,1,2]]
    # sum_ij C(nij,2) = 1 + 1 = 2; sum_i C(3,2) = 6; sum_j C(2,2) = 3; C(6,2) = 15
    # expected = 6 * 3 / 15 = 1.2; max = (6 + 3) / 2 = 4.5 -> ARI = 0.8 / 3.3
    a = [0, 0, 0, 1, 1, 1]
    b = [0, 0, 1, 1, 2, 2]
    assert bench.adjusted_rand_index(a, b) == pytest.approx(0.8 / 3.3, rel=1e-12)


def test_ami_brute_force_expected_mutual_information():
    """AMI with the expected mutual information summed by brute force over
    every labelling with the same cluster sizes (n = 6)."""
    a = np.array([0, 0, 0, 1, 1, 2])
    b = np.array([0, 1, 1, 1, 2, 2])
    n = len(a)

    def mi(x, y):
        m = bench.contingency(x, y)
        ax, by = m.sum(1), m.sum(0)
        return sum(m[i, j] / n * math.log(n * m[i, j] / (ax[i] * by[j]))
                   for i in range(m.shape[0]) for j in range(m.shape[1]) if m[i, j])

    perms = set(itertools.permutations(b.tolist()))
    emi = sum(mi(a, np.array(p)) for p in perms) / len(perms)
    ha = -sum(c / n * math.log(c / n) for c in np.bincount(a))
    hb = -sum(c / n * math.log(c / n) for c in np.bincount(b))
    want = (mi(a, b) - emi) / (0.5 * (ha + hb) - emi)
    assert bench.adjusted_mutual_info(a, b) == pytest.approx(want, rel=1e-10)


def test_measures_are_label_permutation_invariant():
    r = np.random.default_rng(3)
    a = r.integers(0, 7, 500)
    b = np.where(r.random(500) < 0.8, a, r.integers(0, 7, 500))
    perm = r.permutation(7)
    assert bench.adjusted_rand_index(a, perm[b]) == pytest.approx(bench.adjusted_rand_index(a, b), rel=1e-12)
    assert bench.adjusted_mutual_info(a, perm[b]) == pytest.approx(bench.adjusted_mutual_info(a, b), rel=1e-12)
    assert bench.adjusted_rand_index(a, a) == 1.0
    assert bench.adjusted_mutual_info(a, perm[a]) == pytest.approx(1.0, abs=1e-12)
    assert bench.matched_label_diff(a, perm[a]) == 0.0


def test_matched_diff_hand_worked():
    ref = [0, 0, 1, 1, 2, 2]
    lab = [5, 5, 7, 9, 9, 9]  # best matching 0->5, 1->7, 2->9: 5 of 6 agree
    assert bench.matched_label_diff(ref, lab) == pytest.approx(1.0 / 6.0, rel=1e-12)


@pytest.mark.parametrize("ka,kb,n", [(5, 5, 300), (20, 12, 2000), (100, 100, 5000)])
def test_measures_match_scikit_learn(ka, kb, n):
    metrics = pytest.importorskip("sklearn.metrics")
    r = np.random.default_rng(ka * 7 + kb)
    a = r.integers(0, ka, n)
    b = np.where(r.random(n) < 0.6, a % kb, r.integers(0, kb, n))
    assert bench.adjusted_rand_index(a, b) == pytest.approx(metrics.adjusted_rand_score(a, b), rel=1e-9, abs=1e-12)
    assert bench.adjusted_mutual_info(a, b) == pytest.approx(metrics.adjusted_mutual_info_score(a, b), rel=1e-7,
                                                             abs=1e-10)
