"""Pins for the CPU oracle: each checks it against something other than itself
(closed forms, textbook special cases, library routines, invariants, brute force).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.ndimage
import scipy.stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
QS = [0.3, 0.5, 0.8, 1.0, 1.5, 2.5]


def _rand_hist(rng, L, zero_frac=0.3, hi=1000):
    h = rng.integers(0, hi, L).astype(np.int64)
    h[rng.random(L) < zero_frac] = 0
    if h.sum() == 0:
        h[0] = 1
    return h


def _safe_eval(expr):
    return float(eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt, "log": math.log}))


# ------------------------------------------------------------ histograms

def test_hist1d_matches_bincount():
    rng = np.random.default_rng(1)
    v = rng.integers(-32768, 32768, 50_001).astype(np.int16)
    v[:100] = -1024
    v[100:200] = 3071
    v[200:300] = 3072
    v[300:400] = -1025
    ref = np.bincount(np.clip(v.astype(np.int64) + 1024, 0, 4095), minlength=4096)
    assert np.array_equal(oracle.hist1d(v), ref)


@pytest.mark.parametrize("shape", [(1, 7, 9), (5, 6, 11), (3, 1, 4), (1, 1, 1)])
def test_hist2d_matches_scipy_box_sum(shape):
    rng = np.random.default_rng(sum(shape))
    v = rng.integers(-1500, 3500, shape).astype(np.int16)
    h, f, m = oracle.hist2d(v, return_levels=True)
    grey = (np.clip(v.astype(np.int64) + 1024, 0, 4095) >> 4)
    if shape[0] == 1:
        s = scipy.ndimage.correlate(grey[0], np.ones((3, 3), np.int64), mode="nearest")[None]
        mean = s // 9
    else:
        s = scipy.ndimage.correlate(grey, np.ones((3, 3, 3), np.int64), mode="nearest")
        mean = s // 27
    assert np.array_equal(f, grey)
    assert np.array_equal(m, mean)
    ref = np.bincount((grey * 256 + mean).ravel(), minlength=65536).reshape(256, 256)
    assert np.array_equal(h, ref)


def test_hist2d_rejects_levels_that_do_not_fill_the_grey_range():
    # grey = b >> shift must index L >> shift levels, so L is a multiple of 2^shift
    v = np.zeros((1, 4, 4), np.int16)
    with pytest.raises(RuntimeError):
        oracle.hist2d(v, -1024, 4001, 4)
    assert oracle.hist2d(v, -1024, 4000, 4).shape == (250, 250)


# ------------------------------------------------------------ objective pins

@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "hand_examples.json")))["cases"],
                         ids=lambda c: c["name"])
@pytest.mark.parametrize("mode", ["definition", "prefix"])
def test_hand_worked_examples(case, mode):
    h = np.array(case["h"], np.int64)
    t, best, gap, phi, valid = oracle.search1d(h, case["q"], mode)
    want = [_safe_eval(e) for e in case["phi"]]
    assert valid.all()
    np.testing.assert_allclose(phi, want, rtol=1e-13, atol=1e-14)
    assert t == case["t"]
    if "gap" in case:
        assert gap == pytest.approx(_safe_eval(case["gap"]), rel=1e-12)


@pytest.mark.parametrize("mode", ["definition", "prefix"])
def test_q2_is_gini_simpson(mode):
    """At q = 2 the Tsallis entropy is the Gini-Simpson index 1 - sum r^2, and
    H1 + H2 - H1 H2 = 1 - (sum r1^2)(sum r2^2)."""
    rng = np.random.default_rng(7)
    h = _rand_hist(rng, 40)
    phi, valid = oracle.objective1d(h, 2.0, mode)
    for t in range(39):
        a, b = h[: t + 1].astype(float), h[t + 1:].astype(float)
        if a.sum() == 0 or b.sum() == 0:
            assert not valid[t]
            continue
        ga = np.sum((a / a.sum()) ** 2)
        gb = np.sum((b / b.sum()) ** 2)
        assert phi[t] == pytest.approx(1 - ga * gb, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("q", [0.3, 0.5, 0.8, 1.5, 2.5])
@pytest.mark.parametrize("mode", ["definition", "prefix"])
def test_pseudo_additivity_is_joint_entropy(q, mode):
    """H1 + H2 + (1-q) H1 H2 is the Tsallis entropy of the product of the two
    class distributions (pseudo-additivity), computed here from the joint."""
    rng = np.random.default_rng(int(q * 10))
    h = _rand_hist(rng, 24)
    phi, valid = oracle.objective1d(h, q, mode)
    for t in range(23):
        if not valid[t]:
            continue
        a, b = h[: t + 1].astype(float), h[t + 1:].astype(float)
        joint = np.outer(a / a.sum(), b / b.sum()).ravel()
        joint = joint[joint > 0]
        s_joint = (1.0 - np.sum(joint ** q)) / (q - 1.0)
        assert phi[t] == pytest.approx(s_joint, rel=1e-11, abs=1e-12)


@pytest.mark.parametrize("mode", ["definition", "prefix"])
def test_q1_is_kapur_shannon(mode):
    """alpha = 1: the Shannon (Kapur) sum H(class 1) + H(class 2), via scipy."""
    rng = np.random.default_rng(11)
    h = _rand_hist(rng, 50)
    phi, valid = oracle.objective1d(h, 1.0, mode)
    for t in range(49):
        if not valid[t]:
            continue
        ref = scipy.stats.entropy(h[: t + 1]) + scipy.stats.entropy(h[t + 1:])
        assert phi[t] == pytest.approx(ref, rel=1e-12, abs=1e-13)


def test_q_to_1_limit_is_continuous():
    rng = np.random.default_rng(12)
    h = _rand_hist(rng, 64)
    p1, v = oracle.objective1d(h, 1.0)
    for eps in (1e-5, -1e-5):
        pq, vq = oracle.objective1d(h, 1.0 + eps)
        assert np.array_equal(v, vq)
        np.testing.assert_allclose(pq[v], p1[v], rtol=1e-4, atol=1e-4)
    # and the argmax partition agrees near the limit
    assert oracle.search1d(h, 1.0 + 1e-7)[0] == oracle.search1d(h, 1.0)[0]


@pytest.mark.parametrize("q", [0.3, 0.5, 0.8, 1.5, 2.5])
@pytest.mark.parametrize("w,gap_bins,L", [(16, 10, 64), (5, 1, 16), (32, 200, 4096)])
def test_two_uniform_modes_split_at_gap(q, w, gap_bins, L):
    """Two disjoint modes of w equal bins: every split of the 2w bins into m and
    2w - m gives ab = (m(2w - m))^(1-q), extremal at m = w, so the maximiser is
    the gap and phi* = (1 - w^(2(1-q))) / (q - 1)."""
    h = np.zeros(L, np.int64)
    start = 3
    h[start:start + w] = 7
    h[start + w + gap_bins:start + 2 * w + gap_bins] = 7
    for mode in ("prefix", "definition") if L <= 64 else ("prefix",):
        t, best, gap, phi, valid = oracle.search1d(h, q, mode)
        assert t == start + w - 1
        assert best == pytest.approx((1 - w ** (2 * (1 - q))) / (q - 1), rel=1e-12)
        assert gap > 0


@pytest.mark.parametrize("q", QS)
def test_count_scaling_invariance(q):
    rng = np.random.default_rng(13)
    h = _rand_hist(rng, 128)
    a, va = oracle.objective1d(h, q)
    b, vb = oracle.objective1d(h * 37, q)
    assert np.array_equal(va, vb)
    np.testing.assert_allclose(a[va], b[vb], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("q", QS)
def test_mirror_symmetry(q):
    """Reversing the levels swaps the classes: phi'(L-2-t) = phi(t)."""
    rng = np.random.default_rng(14)
    h = _rand_hist(rng, 100)
    a, va = oracle.objective1d(h, q)
    b, vb = oracle.objective1d(h[::-1].copy(), q)
    assert np.array_equal(va, vb[::-1])
    np.testing.assert_allclose(a[va], b[::-1][va], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("L", [2, 3, 17, 64])
def test_prefix_mode_equals_definition_mode(q, L):
    """Brute force (no prefix sums, O(L^2)) pins the O(L) prefix formulas."""
    rng = np.random.default_rng(L * 100 + int(q * 10))
    for trial in range(5):
        h = _rand_hist(rng, L, zero_frac=0.4)
        a, va = oracle.objective1d(h, q, "definition")
        b, vb = oracle.objective1d(h, q, "prefix")
        assert np.array_equal(va, vb)
        np.testing.assert_allclose(a[va], b[vb], rtol=1e-11, atol=1e-12)


def test_empty_classes_are_invalid_and_no_valid_threshold():
    h = np.zeros(16, np.int64)
    h[5] = 10
    t, best, gap, phi, valid = oracle.search1d(h, 0.8)
    assert not valid.any() and t == -1
    h[9] = 1
    t, best, gap, phi, valid = oracle.search1d(h, 0.8)
    assert valid.sum() == 4 and t == 5 and best == 0.0


def test_argmax_plateau_and_gap_brute_force():
    rng = np.random.default_rng(15)
    for trial in range(20):
        h = _rand_hist(rng, 30, zero_frac=0.5)
        t, best, gap, phi, valid = oracle.search1d(h, 0.8)
        vals = np.where(valid, phi, -np.inf)
        assert t == int(np.argmax(vals))          # numpy argmax is the first maximiser
        cum = np.cumsum(h)[:-1]
        others = vals[cum != cum[t]]
        second = others.max() if others.size and np.isfinite(others).any() else -np.inf
        want = (best - second) / max(abs(best), 1.0) if np.isfinite(second) else math.inf
        assert gap == pytest.approx(want, rel=1e-12)


# ------------------------------------------------------------ 2-D pins

@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("L", [2, 5, 12])
def test_2d_prefix_equals_definition(q, L):
    rng = np.random.default_rng(L + int(10 * q))
    h = rng.integers(0, 50, (L, L)).astype(np.int64)
    h[rng.random((L, L)) < 0.4] = 0
    h[0, 0] += 1
    h[-1, -1] += 1
    a, va = oracle.objective2d(h, q, "definition")
    b, vb = oracle.objective2d(h, q, "prefix")
    assert np.array_equal(va, vb)
    np.testing.assert_allclose(a[va], b[vb], rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("q", QS)
def test_2d_diagonal_reduces_to_1d(q):
    """A histogram on the diagonal gives phi_2D(t, t) = phi_1D(t) on its diagonal."""
    rng = np.random.default_rng(16)
    d = _rand_hist(rng, 20, zero_frac=0.2)
    h2 = np.diag(d)
    p2, v2 = oracle.objective2d(h2, q, "prefix")
    p1, v1 = oracle.objective1d(d, q, "prefix")
    diag = np.diagonal(p2)
    assert np.array_equal(np.diagonal(v2), v1)
    np.testing.assert_allclose(diag[v1], p1[v1], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("q", [0.5, 0.8, 1.5])
def test_2d_pseudo_additivity_joint(q):
    rng = np.random.default_rng(17)
    L = 9
    h = rng.integers(0, 20, (L, L)).astype(np.int64)
    h[0, 0] += 1
    h[-1, -1] += 1
    phi, valid = oracle.objective2d(h, q, "definition")
    for t in range(L - 1):
        for s in range(L - 1):
            if not valid[t, s]:
                continue
            a = h[: t + 1, : s + 1].astype(float).ravel()
            b = h[t + 1:, s + 1:].astype(float).ravel()
            joint = np.outer(a / a.sum(), b / b.sum()).ravel()
            joint = joint[joint > 0]
            assert phi[t, s] == pytest.approx((1 - np.sum(joint ** q)) / (q - 1), rel=1e-11, abs=1e-12)


def test_2d_argmax_and_gap_brute_force():
    rng = np.random.default_rng(18)
    L = 10
    h = rng.integers(0, 9, (L, L)).astype(np.int64)
    h[rng.random((L, L)) < 0.5] = 0
    h[0, 0] += 3
    h[-1, -1] += 3
    t, s, best, gap, phi, valid = oracle.search2d(h, 0.8)
    vals = np.where(valid, phi, -np.inf)
    flat = int(np.argmax(vals))
    assert (t, s) == divmod(flat, L - 1)
    ca = np.array([[h[: i + 1, : j + 1].sum() for j in range(L - 1)] for i in range(L - 1)])
    cb = np.array([[h[i + 1:, j + 1:].sum() for j in range(L - 1)] for i in range(L - 1)])
    same = (ca == ca[t, s]) & (cb == cb[t, s])
    second = vals[~same].max()
    assert gap == pytest.approx((best - second) / max(abs(best), 1.0), rel=1e-12)


# ------------------------------------------------------------ binarise / step

@pytest.mark.parametrize("polarity", [0, 1])
def test_binarize_algorithm1(polarity):
    rng = np.random.default_rng(19)
    v = rng.integers(-2000, 4000, 10_000).astype(np.int16)
    for t in (0, 17, 1000, 4094):
        b = np.clip(v.astype(np.int64) + 1024, 0, 4095)
        want = (b >= t + 1) if polarity else (b <= t)
        assert np.array_equal(oracle.binarize(v, t, polarity=polarity), want.astype(np.uint8))
    # 2-D grey levels (shift 4) and the no-threshold case
    g = np.clip(v.astype(np.int64) + 1024, 0, 4095) >> 4
    assert np.array_equal(oracle.binarize(v, 100, shift=4, polarity=polarity),
                          ((g >= 101) if polarity else (g <= 100)).astype(np.uint8))
    assert not oracle.binarize(v, -1, polarity=polarity).any()


def test_segment1d_threads_match_single_calls():
    rng = np.random.default_rng(20)
    vol = (rng.normal(-500, 400, (6, 32, 32))).astype(np.int16)
    t, phi, gap, mask = oracle.segment1d(vol, 32 * 32, 0.8, nthreads=3)
    for z in range(6):
        h = oracle.hist1d(vol[z])
        tz, bz, gz, _, _ = oracle.search1d(h, 0.8)
        assert t[z] == tz and phi[z] == bz and gap[z] == gz
        assert np.array_equal(mask.reshape(6, 32, 32)[z], oracle.binarize(vol[z], tz))
