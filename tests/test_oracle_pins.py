"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: exact
rational arithmetic on tiny inputs, closed forms, the paper's printed values
(tests/golden/), the error bounds it proves, invariants, or a library
conversion routine.  A plausible mistake in the oracle (dropped term, wrong
sign or index, transposed operand, wrong tie-break, wrong rounding) fails at
least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2407_12208_gb300 import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")
pytestmark = pytest.mark.filterwarnings("ignore")


def _exact_dist(x, y):
    return sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, y))


# --- Table 1.1 -------------------------------------------------------------
def test_unit_roundoffs_match_table_1_1():
    g = json.load(open(os.path.join(GOLD, "table_1_1.json")))["formats"]
    for name, fmt in (("fp16", 0), ("bf16", 1), ("fp32", 3), ("fp64", 4)):
        u = oracle.unit_roundoff(fmt)
        assert abs(u - g[name]["u"]) / g[name]["u"] < 5e-3, name
        assert u == 2.0 ** -g[name]["t"]
    for name, fmt in (("fp16", 0), ("bf16", 1)):
        xmax = g[name]["xmax"]
        got = oracle.round_to_format(1e300 if fmt == 1 else 6.55e4, fmt)
        if fmt == 0:
            assert abs(got - xmax) / xmax < 5e-3
        xmin = 2.0 ** g[name]["emin"]
        assert abs(xmin - g[name]["xmin"]) / g[name]["xmin"] < 5e-3
        assert oracle.round_to_format(xmin, fmt) == xmin


@pytest.mark.parametrize("fmt,tdtype", [(0, "float16"), (1, "bfloat16"), (2, "float8_e4m3fn")])
def test_quantize_matches_torch_conversion(fmt, tdtype):
    torch = pytest.importorskip("torch")
    if not hasattr(torch, tdtype):
        pytest.skip("torch lacks " + tdtype)
    r = np.random.default_rng(5)
    lim = {0: 6e4, 1: 1e30, 2: 440.0}[fmt]
    xs = [r.uniform(-1, 1, 4000) * 10.0 ** r.uniform(-12, np.log10(lim), 4000)]
    # ties, subnormals, exact values
    if fmt == 0:
        xs.append(np.array([2.0 ** -24, 1.5 * 2.0 ** -24, 2.5 * 2.0 ** -24, 2.0 ** -25, 1 + 2.0 ** -11,
                            1 + 3 * 2.0 ** -11, 65504.0, 65519.0, -3e-8]))
    if fmt == 1:
        xs.append(np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 2.0 ** -133, 3 * 2.0 ** -134,
                            1e-39, -1.5e-40]))
    if fmt == 2:
        xs.append(np.array([2.0 ** -9, 1.5 * 2.0 ** -9, 2.5 * 2.0 ** -9, 2.0 ** -10, 448.0, 1.0625,
                            1.1875, -0.013]))
    x = np.concatenate(xs).astype(np.float32)
    ref = torch.from_numpy(x).to(getattr(torch, tdtype)).to(torch.float32).numpy()
    got = oracle.quantize(x, fmt)
    np.testing.assert_array_equal(got, ref)


def _e4m3_scales(rows):
    d = max(len(r) for r in rows)
    X = np.zeros((len(rows), d), np.float32)
    for i, r in enumerate(rows):
        X[i, :len(r)] = r
    Xq, _, _, _, _, sc = oracle.row_quant_stats(X, 2, per_row_scale=True)
    return X, Xq, sc


def test_e4m3_row_scale_rule():
    # The per-row E4M3 scale (reading R12): the smallest power of two s with
    # max|x| / s <= 448 -- the row maximum lands in (224, 448] and never
    # saturates -- kept a normal binary32 number (s >= 2^-126); s = 1 for an
    # all-zero row.  Checked from its definition on edge rows: maxima exactly
    # 448 2^j and one binary32 ulp either side, negative maxima, rows whose
    # maximum is a binary32 subnormal, and the all-zero row.
    rows, expect = [], []
    for j in range(-30, 31, 3):
        edge = np.float32(448.0 * 2.0 ** j)
        up = np.nextafter(edge, np.float32(np.inf))
        dn = np.nextafter(edge, np.float32(0))
        rows += [[edge, edge * np.float32(0.25)], [-up, edge * np.float32(0.5)], [dn, -dn]]
        expect += [2.0 ** j, 2.0 ** (j + 1), 2.0 ** j]
    X, Xq, sc = _e4m3_scales(rows)
    np.testing.assert_array_equal(sc, np.array(expect))
    r = np.random.default_rng(12)
    rand = [list((r.normal(size=16) * 10.0 ** r.uniform(-35, 35)).astype(np.float32)) for _ in range(200)]
    tiny = [[1e-40, 2e-41], [np.float32(2.0 ** -149)], [np.float32(3e-38), -1e-39], [np.float32(448 * 2.0 ** -126)],
            [np.float32(448 * 2.0 ** -127)]]
    X, Xq, sc = _e4m3_scales(rand + tiny + [[0.0, 0.0]])
    amax = np.abs(X).max(axis=1).astype(np.float64)
    for i in range(len(X)):
        if amax[i] == 0.0:
            assert sc[i] == 1.0
            continue
        m, e = math.frexp(sc[i])
        assert m == 0.5, sc[i]                        # a power of two
        assert amax[i] / sc[i] <= 448.0               # never saturates
        if sc[i] > 2.0 ** -126:
            assert amax[i] / sc[i] > 224.0            # the smallest such power
            # the row maximum is represented to E4M3's unit roundoff (no saturation)
            k = int(np.argmax(np.abs(X[i])))
            assert abs(Xq[i, k] - X[i, k]) <= 2.0 ** -4 * abs(X[i, k])
        else:
            assert sc[i] == 2.0 ** -126 and amax[i] <= 448.0 * 2.0 ** -126
    assert list(sc[-6:-1]) == [2.0 ** -126] * 4 + [2.0 ** -126]


def test_binary32_rounding_matches_numpy():
    # fmt 3 of round_to_format is binary32: numpy's float64 -> float32 cast
    # (IEEE round to nearest even) on normals, ties, subnormals and overflow
    r = np.random.default_rng(13)
    v = r.uniform(-1, 1, 20000) * 10.0 ** r.uniform(-46, 39, 20000)
    ties = (np.arange(1, 200, dtype=np.float64) + 0.5) * 2.0 ** -23
    v = np.concatenate([v, ties, ties * 2.0 ** -130, [3.5e38, 3.41e38, -1e39, 1e-46]])
    with np.errstate(over="ignore"):
        ref = v.astype(np.float32).astype(np.float64)
    got = np.array([oracle.round_to_format(float(a), 3) for a in v])
    np.testing.assert_array_equal(got, ref)
    assert oracle.unit_roundoff(3) == 2.0 ** -24


@pytest.mark.parametrize("fmt", [0, 1, 3])
def test_dist_direct_fmt_matches_library_arithmetic(fmt):
    # the direct formula with every operation rounded to the format, against
    # the same sequence of operations done in the library's own arithmetic of
    # that format (numpy float32 / float16, torch bfloat16); the inputs keep
    # every exact intermediate within 24 bits, so the library's float32
    # evaluation followed by one rounding is the format's own rounding
    r = np.random.default_rng(14 + fmt)
    for _ in range(200):
        x = r.uniform(-4, 4, 8)
        y = x + r.choice([-1, 1], 8) * r.uniform(0.5, 2, 8)
        x32, y32 = x.astype(np.float32), y.astype(np.float32)
        got = oracle.dist_direct_fmt(x32, y32, fmt)
        if fmt == 3:
            s = np.float32(0)
            for a, b in zip(x32, y32):
                t = np.float32(a - b)
                s = np.float32(s + np.float32(t * t))
            ref = float(s)
        elif fmt == 0:
            xh, yh = x32.astype(np.float16), y32.astype(np.float16)
            s = np.float16(0)
            for a, b in zip(xh, yh):
                t = np.float16(a - b)
                s = np.float16(s + np.float16(t * t))
            ref = float(s)
        else:
            torch = pytest.importorskip("torch")
            xb = torch.from_numpy(x32).to(torch.bfloat16)
            yb = torch.from_numpy(y32).to(torch.bfloat16)
            s = torch.zeros((), dtype=torch.bfloat16)
            for a, b in zip(xb, yb):
                t = a - b
                s = s + t * t
            ref = float(s)
        assert got == ref, (fmt, got, ref)
    # the binary64 case is Eq. (dist-direct) itself
    x = r.normal(size=16).astype(np.float32)
    y = r.normal(size=16).astype(np.float32)
    assert oracle.dist_direct_fmt(x, y, 4) == oracle.dist_direct(x[None], y[None])[0, 0]


def test_alg2_fallback_precisions():
    # Eq. (fallback-rule): a flagged pair is recomputed by the direct formula
    # in the fallback's precision (binary64, binary32, or the low format
    # itself); an unflagged pair keeps Alg. 2's d^ whatever the fallback
    u = 2.0 ** -24
    x = np.zeros(8, np.float32); x[0] = 1.0
    y = x.copy(); y[1] = np.float32(10 * u)
    for fmt in (0, 1):
        for fb in (4, 3, fmt):
            flag, d, _, _ = oracle.mp_dist_fb(x, y, 5.0, fmt, fb)
            assert flag and d == oracle.dist_direct_fmt(x, y, fb)
        assert oracle.mp_dist_fb(x, y, 5.0, fmt, 4)[1] == (10 * u) ** 2   # exact in binary64
        # in the low format itself: the square (10u)^2 underflows binary16;
        # bfloat16 has binary32's exponent range and holds it exactly
        assert oracle.mp_dist_fb(x, y, 5.0, fmt, fmt)[1] == (0.0 if fmt == 0 else (10 * u) ** 2)
        far = np.full(8, 3.0, np.float32)
        fl, d, dh, _ = oracle.mp_dist_fb(x, far, 5.0, fmt, 3)
        assert not fl and d == dh
    # Alg. 2 in binary32 (the FP32 -> FP64 mode): the same worked example is
    # flagged at u = 2^-24 too, and x = y always
    flag, d, dh, E = oracle.mp_dist_fb(x, y, 5.0, 3, 4)
    assert flag and d == (10 * u) ** 2 and E > 0
    assert oracle.mp_dist_fb(x, x, 5.0, 3, 4)[0]


def test_e4m3_saturates():
    assert oracle.round_to_format(1e6, 2) == 448.0
    assert oracle.round_to_format(-465.0, 2) == -448.0
    assert oracle.round_to_format(70000.0, 0) == math.inf


# --- Eq. (dist-direct), Theorem 4.1 -----------------------------------------
def test_dist_direct_exact_on_tiny_inputs_and_theorem_4_1():
    r = np.random.default_rng(1)
    for d in (1, 3, 7, 16):
        X = (r.normal(size=(5, d)) * 10.0 ** r.uniform(-3, 3, size=(5, 1))).astype(np.float32)
        C = (X[:3] + r.normal(size=(3, d)) * 1e-3).astype(np.float32)
        D = oracle.dist_direct(X, C)
        g = oracle.gamma(d + 2, 2.0 ** -53)
        for i in range(5):
            for j in range(3):
                ex = _exact_dist(X[i], C[j])
                assert abs(Fraction(D[i, j]) - ex) <= Fraction(g) * ex
        # transposition / index check: D[i, j] belongs to (X_i, C_j)
        assert D[1, 2] == pytest.approx(float(_exact_dist(X[1], C[2])), rel=1e-14)


def test_dist_labelled_exact_on_tiny_inputs():
    # the distance to a given centre per point: exact rational arithmetic
    # within Theorem 4.1's bound, and the right (point, centre) pair
    r = np.random.default_rng(11)
    for d in (1, 4, 9, 33):
        X = (r.normal(size=(7, d)) * 10.0 ** r.uniform(-2, 2, size=(7, 1))).astype(np.float32)
        C = (r.normal(size=(4, d))).astype(np.float32)
        lab = r.integers(0, 4, size=7).astype(np.int32)
        got = oracle.dist_labelled(X, C, lab)
        g = oracle.gamma(d + 2, 2.0 ** -53)
        for i in range(7):
            ex = _exact_dist(X[i], C[lab[i]])
            assert abs(Fraction(got[i]) - ex) <= Fraction(g) * ex
            other = _exact_dist(X[i], C[(lab[i] + 1) % 4])
            assert other == ex or abs(Fraction(got[i]) - other) > Fraction(g) * other


def test_dist_direct_zero_and_symmetry():
    r = np.random.default_rng(2)
    X = r.normal(size=(6, 5)).astype(np.float32)
    D = oracle.dist_direct(X, X)
    assert np.all(np.diag(D) == 0.0)
    np.testing.assert_array_equal(D, D.T)


# --- Alg. 1 assignment ------------------------------------------------------
def test_assign_brute_force_and_ties():
    r = np.random.default_rng(3)
    X = r.integers(-3, 4, size=(40, 3)).astype(np.float32)
    C = r.integers(-3, 4, size=(6, 3)).astype(np.float32)
    C[4] = C[1]  # duplicate centre: ties must go to the lower index
    lab, d1, d2 = oracle.assign(X, C)
    for i in range(40):
        ds = [_exact_dist(X[i], C[j]) for j in range(6)]
        m = min(ds)
        assert lab[i] == ds.index(m)
        assert Fraction(d1[i]) == m
        rest = sorted(ds)
        assert Fraction(d2[i]) == rest[1]
    assert not np.any(lab == 4)


def test_assign_k1_second_is_inf():
    X = np.ones((3, 2), np.float32)
    lab, d1, d2 = oracle.assign(X, X[:1])
    assert np.all(lab == 0) and np.all(np.isinf(d2))


# --- Eq. (center), Lemma 4.4, Lemma 2.1 ------------------------------------
def test_update_is_mean_within_lemma_4_4():
    r = np.random.default_rng(4)
    n, d, k = 300, 4, 5
    X = (r.normal(size=(n, d)) * 3 + 100).astype(np.float32)
    lab = r.integers(0, k, size=n).astype(np.int32)
    C0 = np.zeros((k, d), np.float32)
    C, cnt, shift = oracle.update(X, lab, C0, empty_policy=0)
    for j in range(k):
        mem = X[lab == j]
        assert cnt[j] == len(mem)
        for l in range(d):
            mu = sum(Fraction(float(v)) for v in mem[:, l]) / len(mem)
            abar = sum(abs(Fraction(float(v))) for v in mem[:, l]) / len(mem)
            tol = Fraction(oracle.gamma(len(mem), 2.0 ** -53)) * abar + Fraction(2.0 ** -24) * abs(mu)
            assert abs(Fraction(float(C[j, l])) - mu) <= tol
    ex_shift = max(math.sqrt(float(sum(Fraction(float(v)) ** 2 for v in C[j]))) for j in range(k))
    assert shift == pytest.approx(ex_shift, rel=1e-12)


def test_lemma_2_1_identity():
    # phi(p, S) = phi(mu, S) + |S| dist(p, mu)^2 with mu the exact mean
    r = np.random.default_rng(6)
    S = r.integers(-20, 20, size=(8, 3)).astype(np.float32)
    p = np.array([[1.5, -2.0, 7.25]], np.float32)
    lab = np.zeros(8, np.int32)
    C, _, _ = oracle.update(S, lab, np.zeros((1, 3), np.float32))
    mu = [sum(Fraction(float(v)) for v in S[:, l]) / 8 for l in range(3)]
    # the fp32 mean equals the exact mean when it is representable (here: multiples of 1/8)
    assert [Fraction(float(v)) for v in C[0]] == mu
    phi_p = Fraction(float(oracle.dist_direct(S, p).sum()))
    phi_mu = Fraction(float(oracle.dist_direct(S, C).sum()))
    dpm = Fraction(float(oracle.dist_direct(p, C)[0, 0]))
    assert phi_p == phi_mu + 8 * dpm


def test_empty_cluster_policies():
    X = np.array([[0.0], [1.0], [5.0], [9.0]], np.float32)
    lab = np.array([0, 0, 0, 0], np.int32)
    C0 = np.array([[1.0], [50.0], [60.0]], np.float32)
    md = np.array([1.0, 0.0, 16.0, 64.0])
    C, cnt, _ = oracle.update(X, lab, C0, empty_policy=0)
    assert C[1, 0] == 50.0 and C[2, 0] == 60.0 and cnt.tolist() == [4, 0, 0]
    C, cnt, _ = oracle.update(X, lab, C0, empty_policy=1, min_dist=md)
    assert C[0, 0] == 3.75 and C[1, 0] == 9.0 and C[2, 0] == 5.0


# --- Alg. 1 driver ----------------------------------------------------------
def test_lloyd_closed_form_1d():
    g = json.load(open(os.path.join(GOLD, "lloyd_1d_closed_form.json")))
    X = np.array(g["X"], np.float32)
    C0 = np.array(g["C_init"], np.float32)
    C, lab, sse, it = oracle.lloyd(X, C0, g["max_iter"])
    assert it == g["max_iter"]
    np.testing.assert_allclose(sse, g["sse_per_iter"], rtol=1e-15)
    assert lab.tolist() == g["final_labels"]
    np.testing.assert_array_equal(C, np.array(g["final_centres"], np.float32))
    # tau stop: the shift is 0 after the third update, so tau = 1e-8 stops there
    C, lab, sse, it = oracle.lloyd(X, C0, 50, tau=1e-8)
    assert it == 3


def test_lloyd_invariants_on_blobs():
    X, C0 = workloads.blobs(2000, 6, 7, seed=11)
    C, lab, sse, it = oracle.lloyd(X, C0, 15)
    # SSE never increases (Lemma 2.1 + argmin, Section 3)
    assert np.all(np.diff(sse) <= 1e-9 * sse[:-1])
    # every label is an argmin with the lowest-index tie-break
    D = oracle.dist_direct(X, C)
    assert np.all(D[np.arange(len(X)), lab] <= D.min(axis=1))
    # one more Lloyd step from C reproduces update(assign(C))
    lab1, md1, _ = oracle.assign(X, C)
    C1, _, _ = oracle.update(X, lab1, C, empty_policy=1, min_dist=md1)
    C2, _, _, _ = oracle.lloyd(X, C, 1)
    np.testing.assert_array_equal(C1, C2)


# --- Alg. 2 -----------------------------------------------------------------
def test_alg2_closed_form_thresholds():
    g = json.load(open(os.path.join(GOLD, "alg2_closed_forms.json")))["bf16_rho5"]
    for cA, key in ((1.0, "c_A_1_first_r_all_flagged"), (2.0, "c_A_2_first_r_all_flagged")):
        rstar = g[key]
        for r in range(8, 140):
            x = np.zeros(r, np.float32); x[0] = 1.0
            flag, d, dh, E = oracle.mp_dist_paper(x, -x, 5.0, 1, c_A=cA)
            assert flag == (r >= rstar), (cA, r)
            assert dh == 4.0
            assert d == 4.0  # flagged pairs fall back to the exact direct value
        # beyond the threshold every pair is flagged
        rng = np.random.default_rng(7)
        for r in (rstar, 128):
            for _ in range(50):
                x = rng.normal(size=r).astype(np.float32)
                y = rng.normal(size=r).astype(np.float32) * rng.uniform(0.1, 10)
                assert oracle.mp_dist_paper(x, y, 5.0, 1, c_A=cA)[0]


def test_alg2_same_point_always_flagged():
    rng = np.random.default_rng(8)
    for fmt in (0, 1):
        x = rng.normal(size=16).astype(np.float32)
        flag, d, _, _ = oracle.mp_dist_paper(x, x, 5.0, fmt)
        assert flag and d == 0.0


def test_alg2_undefined_gamma():
    x = np.ones(300, np.float32)
    assert oracle.mp_dist_paper(x, x, 5.0, 1)[0] is None  # bf16: (r+2) u >= 1


@pytest.mark.parametrize("fmt", [0, 1])
def test_worked_cancellation_example(fmt):
    # Section 4.3: x unit, y = x + delta, ||delta|| = 10 u (u = fp32 unit roundoff)
    u = 2.0 ** -24
    rng = np.random.default_rng(9)
    for r in (4, 16):
        x = rng.normal(size=r); x /= np.linalg.norm(x); x = x.astype(np.float32)
        delta = np.zeros(r); delta[1] = 10 * u
        y = (x.astype(np.float64) + delta).astype(np.float32)
        flag, d, _, _ = oracle.mp_dist_paper(x, y, 5.0, fmt, c_A=2.0)
        assert flag
        ex = _exact_dist(x, y)
        assert abs(Fraction(d) - ex) <= Fraction(oracle.gamma(r + 2, 2.0 ** -53)) * ex
        # quantisation destroys the true difference (Eq. (quantis-necess-cond) fails)
        xq, yq = oracle.quantize(x, fmt), oracle.quantize(y, fmt)
        assert abs(float(_exact_dist(xq, yq)) - float(ex)) >= 0.5 * float(ex)
    x = np.zeros(8, np.float32); x[0] = 1.0
    y = x.copy(); y[1] = np.float32(10 * u)
    flag, d, _, _ = oracle.mp_dist_paper(x, y, 5.0, fmt)
    assert flag and d == (10 * u) ** 2


def test_alg2_unflagged_relative_error_bound():
    # Eq. (quantis-rel-bound-expand): unflagged => rel. err <= 2/(rho~ - 2)
    rng = np.random.default_rng(10)
    rho = 5.0
    seen = 0
    for r in (4, 8, 16):
        for _ in range(300):
            x = rng.normal(size=r).astype(np.float32)
            y = (x * rng.uniform(-1, 1) + rng.normal(size=r) * 10.0 ** rng.uniform(-3, 0)).astype(np.float32)
            flag, d, dh, E = oracle.mp_dist_paper(x, y, rho, 0, c_A=2.0)
            ex = float(_exact_dist(x, y))
            if not flag:
                seen += 1
                assert abs(d - ex) / ex <= 2.0 / (rho - 2.0)
                assert d == dh
            else:
                assert abs(d - ex) <= oracle.gamma(r + 2, 2.0 ** -53) * ex
    assert seen > 100


# --- tensor-core instantiation of the test ----------------------------------
def _tc_model_dhat(xq, cq, p, q, truncate=False):
    """d^ under a model of the hardware: exact products, fp32 accumulation in
    order (round-to-nearest, or toward zero), e = fl32(q - 2 g), d^ = fl32(p + e)."""
    acc = np.float32(0.0)
    for a, b in zip(xq.astype(np.float64), cq.astype(np.float64)):
        s = float(acc) + a * b
        if truncate:
            f = np.float32(s)
            if abs(float(f)) > abs(s):
                f = np.nextafter(f, np.float32(0.0))
            acc = f
        else:
            acc = np.float32(s)
    e = np.float32(float(np.float32(q)) - 2.0 * float(acc))
    return float(np.float32(float(np.float32(p)) + float(e)))


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_tc_bound_holds_under_hardware_models(fmt):
    rng = np.random.default_rng(12)
    d = 64 if fmt == 2 else 128
    cases = []
    X = rng.random((20, d)).astype(np.float32)
    cases.append((X, X[::-1].copy()))
    Xc, Cc = workloads.cancellation(20, d, 10, seed=3)
    cases.append((Xc, Cc))
    Xg, Cg = workloads.gaussian_mixture(20, d, 10, seed=4)
    cases.append((Xg, Cg))
    for X, C in cases:
        Xq, p, nx, nxq, nrx, _ = oracle.row_quant_stats(X, fmt, per_row_scale=(fmt == 2))
        Cq, q, nc, ncq, nrc, _ = oracle.row_quant_stats(C, fmt, per_row_scale=(fmt == 2))
        B = oracle.tc_bound_matrix(X, C, fmt, per_row_scale=(fmt == 2))
        for i in range(len(X)):
            for j in range(len(C)):
                ex = float(_exact_dist(X[i], C[j]))
                for trunc in (False, True):
                    dh = _tc_model_dhat(Xq[i], Cq[j], p[i], q[j], truncate=trunc)
                    assert abs(dh - ex) <= B[i, j], (i, j, dh, ex, B[i, j])
                # the C entry point evaluates the same formula
                bc = oracle.tc_bound(nrx[i], nc[j], nxq[i], nrc[j], ncq[j], p[i], q[j], d, fmt)
                assert bc == pytest.approx(B[i, j], rel=1e-14)


def test_tc_bound_scale_and_unflagged_rel_error():
    # B is of the order of the quantisation error (not vacuous), and unflagged
    # pairs have relative error <= 1/(rho - 1) (Eq. (expanded-rel-bound))
    rng = np.random.default_rng(13)
    X = rng.random((30, 128)).astype(np.float32)
    C = rng.random((30, 128)).astype(np.float32)
    B = oracle.tc_bound_matrix(X, C, 1)
    nx = np.linalg.norm(X.astype(np.float64), axis=1)
    nc = np.linalg.norm(C.astype(np.float64), axis=1)
    assert np.all(B <= 4.5 * 2.0 ** -8 * np.outer(nx, nc))
    assert np.all(B >= 0.5 * 2.0 ** -8 * np.outer(nx, nc) / np.sqrt(3) * 0.5)
    Xq, p, *_ = oracle.row_quant_stats(X, 1)
    Cq, q, *_ = oracle.row_quant_stats(C, 1)
    D = oracle.dist_direct(X, C)
    rho = 5.0
    for i in range(30):
        for j in range(30):
            dh = _tc_model_dhat(Xq[i], Cq[j], p[i], q[j])
            if dh > rho * B[i, j]:
                assert abs(dh - D[i, j]) / D[i, j] <= 1.0 / (rho - 1.0)


def test_predict_flags_consistent():
    X, C = workloads.cancellation(50, 128, 20, seed=5)
    sure, maybe = oracle.predict_tc_flags(X, C, 1, 5.0)
    assert sure.all()  # cancellation data: every pair flagged for certain
    X, C = workloads.uniform_pairs(200, 128, 32, seed=6)
    sure, maybe = oracle.predict_tc_flags(X, C, 1, 5.0)
    # far data: only the 32 rows that are centres (d = 0) are flagged
    D = oracle.dist_direct(X, C)
    assert (sure == (D == 0)).all()
    sure, maybe = oracle.predict_tc_flags(X, C, 1, 5.0, test="paper", c_A=1.0)
    assert sure.all()  # Alg. 2 with bf16 at r = 128: 100% fallback (Table 6.1)


# ---- D^2-sampling seeding (k-means++) --------------------------------------
def test_kmeanspp_hand_worked_1d():
    """X = {0, 1, 3} on a line: u_0 = 0.1 picks row 0; D^2 = (0, 1, 9), T = 10,
    so u_1 = 0.05 (target 0.5) picks row 1 and u_1 = 0.2 (target 2) row 2."""
    X = np.array([[0.0], [1.0], [3.0]], dtype=np.float32)
    idx, mg = oracle.kmeanspp(X, [0.1, 0.05])
    assert idx.tolist() == [0, 1]
    assert mg[1] == pytest.approx(0.05, rel=1e-15)  # |P_0 - 0.5| / 10 with P_0 = 0
    idx, _ = oracle.kmeanspp(X, [0.1, 0.2])
    assert idx.tolist() == [0, 2]
    # after rows 0 and 2: D^2 = (0, 1, 0), so any third draw picks row 1
    idx, _ = oracle.kmeanspp(X, [0.1, 0.2, 0.999])
    assert idx.tolist() == [0, 2, 1]


def test_kmeanspp_first_pick_and_coincident_points():
    X = np.zeros((8, 3), dtype=np.float32)
    idx, mg = oracle.kmeanspp(X, [0.0, 0.5, 0.999999])
    # every point on the first centre: T = 0, the uniform rule
    assert idx.tolist() == [0, 4, 7]
    assert np.isinf(mg).all()


def test_kmeanspp_draws_follow_the_d2_distribution():
    """Second pick over a fine grid of draws: the share of draws that pick row
    i equals D^2_i / T (the D^2 distribution), exactly up to the grid."""
    r = np.random.default_rng(4)
    X = r.normal(size=(7, 2)).astype(np.float32)
    D2 = oracle.dist_direct(X, X[[2]])[:, 0]   # the first pick below is row 2 (u_0 = 0.3)
    grid = (np.arange(20000) + 0.5) / 20000
    picks = np.array([oracle.kmeanspp(X, [0.3, g])[0][1] for g in grid])
    share = np.bincount(picks, minlength=7) / len(grid)
    np.testing.assert_allclose(share, D2 / D2.sum(), atol=1.5 / len(grid))
    assert share[2] == 0.0


def test_kmeanspp_picks_distinct_points_and_follows():
    r = np.random.default_rng(5)
    X = r.normal(size=(300, 4)).astype(np.float32)
    u = r.random(40)
    idx, mg = oracle.kmeanspp(X, u)
    assert len(set(idx.tolist())) == 40       # a chosen point has D^2 = 0
    idx2, mg2 = oracle.kmeanspp(X, u, follow=idx)
    assert np.array_equal(idx2, idx) and np.array_equal(mg2, mg)
