"""Pins for the oracle's pre-processing (section II-B) and morphology
(section II-C): hand-worked levels, the digital disk's size from Gauss's
circle problem, scipy's flat grey erosion and dilation (a library routine
for the same min/max filters), and the algebra of openings and closings."""
import json
import os

import numpy as np
import pytest
import scipy.ndimage

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "preprocess_examples.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_rescale_hand_examples():
    g = _golden()["rescale"]
    v = np.array([c["v"] for c in g["cases"]], np.int16)
    out = oracle.rescale8(v, g["background"], g["hu_min"], g["hu_max"])
    assert out.tolist() == [c["g"] for c in g["cases"]]


@pytest.mark.parametrize("lo,hi,bg", [(-2000, 2500, -2000), (-1024, 3071, -1500), (-100, 155, -2000),
                                      (-5, 2, -32768)])
def test_rescale_is_nearest_level_and_monotone(lo, hi, bg):
    """Every int16 value: within half a level of the exact linear map,
    non-decreasing in v, every level 0..255 reached (when the range has at
    least 256 values), and 0 at or below the background."""
    v = np.arange(-32768, 32768, dtype=np.int64)
    g = oracle.rescale8(v.astype(np.int16), bg, lo, hi).astype(np.int64)
    x = (np.clip(v, lo, hi) - lo) * 255.0 / (hi - lo)
    keep = v > bg
    assert np.all(np.abs(g[keep] - x[keep]) <= 0.5 + 1e-12)
    assert np.all(g[~keep] == 0)
    assert np.all(np.diff(g[keep]) >= 0)
    if hi - lo >= 255 and bg < lo:
        assert set(np.unique(g[keep])) == set(range(256))


def test_disk_size_is_the_gauss_circle_count():
    d = _golden()["disk_points"]
    for r, n in zip(d["r"], d["n"]):
        a = np.zeros((1, 2 * r + 5, 2 * r + 7), np.uint8)
        a[0, r + 2, r + 3] = 200
        dil = oracle.morph2d(a, r, "dilate")
        assert int((dil > 0).sum()) == n, r
        # erosion of a single dark pixel marks the same disk
        b = np.full_like(a, 90)
        b[0, r + 2, r + 3] = 7
        assert int((oracle.morph2d(b, r, "erode") == 7).sum()) == n, r


def _disk(r):
    y, x = np.mgrid[-r:r + 1, -r:r + 1]
    return (x * x + y * y) <= r * r


@pytest.mark.parametrize("shape", [(2, 37, 23), (1, 5, 64), (1, 1, 1), (1, 40, 3)])
@pytest.mark.parametrize("r", [0, 1, 3, 6])
def test_erode_dilate_match_scipy(shape, r):
    """Flat erosion/dilation with the offsets outside the image left out
    equal scipy's grey filters padded with the neutral value (255 for the
    minimum, 0 for the maximum), slice by slice."""
    rng = np.random.default_rng(r * 100 + shape[1])
    a = rng.integers(0, 256, shape).astype(np.uint8)
    fp = _disk(r)
    er = np.stack([scipy.ndimage.grey_erosion(s, footprint=fp, mode="constant", cval=255) for s in a])
    di = np.stack([scipy.ndimage.grey_dilation(s, footprint=fp, mode="constant", cval=0) for s in a])
    assert np.array_equal(oracle.morph2d(a, r, "erode"), er)
    assert np.array_equal(oracle.morph2d(a, r, "dilate"), di)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_opening_closing_algebra(r):
    rng = np.random.default_rng(7 + r)
    # blocky image so that openings do more than flatten noise
    a = np.kron(rng.integers(0, 256, (2, 9, 7)), np.ones((1, 4, 5))).astype(np.uint8)
    a = a + rng.integers(0, 3, a.shape).astype(np.uint8)
    er, di = oracle.morph2d(a, r, "erode"), oracle.morph2d(a, r, "dilate")
    op, cl = oracle.morph2d(a, r, "open"), oracle.morph2d(a, r, "close")
    # duality under complement
    assert np.array_equal(er, 255 - oracle.morph2d(255 - a, r, "dilate"))
    assert np.array_equal(cl, 255 - oracle.morph2d(255 - a, r, "open"))
    # ordering and idempotence
    assert np.all(er <= op) and np.all(op <= a) and np.all(a <= cl) and np.all(cl <= di)
    assert np.array_equal(oracle.morph2d(op, r, "open"), op)
    assert np.array_equal(oracle.morph2d(cl, r, "close"), cl)
    # the two subtractions
    assert np.array_equal(oracle.morph2d(a, r, "chest_mask"), a - op)
    assert np.array_equal(oracle.morph2d(a, r, "black_tophat"), cl - a)
    assert np.array_equal(oracle.morph2d(a, r, "copy"), a)


def test_chest_mask_keeps_small_bright_spots_only():
    """A 3x3 bright spot (200 on 50) is thinner than the radius-2 disk, so
    the opening removes it and the subtraction leaves exactly 150 there; a
    flat image gives 0 everywhere."""
    a = np.full((1, 20, 20), 50, np.uint8)
    a[0, 8:11, 8:11] = 200
    cm = oracle.morph2d(a, 2, "chest_mask")
    exp = np.zeros_like(a)
    exp[0, 8:11, 8:11] = 150
    assert np.array_equal(cm, exp)
    assert not oracle.morph2d(np.full((1, 9, 9), 77, np.uint8), 3, "chest_mask").any()


def test_slices_are_independent_images():
    rng = np.random.default_rng(3)
    a = rng.integers(0, 256, (3, 17, 19)).astype(np.uint8)
    whole = oracle.morph2d(a, 3, "open")
    for z in range(3):
        assert np.array_equal(whole[z], oracle.morph2d(a[z:z + 1], 3, "open")[0])


def test_preprocess_histograms_count_every_voxel():
    rng = np.random.default_rng(4)
    v = rng.integers(-2500, 3000, (4, 21, 33)).astype(np.int16)
    o, h = oracle.preprocess(v, r=2)
    assert h.shape == (4, 256) and np.all(h.sum(axis=1) == 21 * 33)
    assert o.dtype == np.int16 and o.min() >= 0 and o.max() <= 255
    _, hv = oracle.preprocess(v, r=2, per_slice=False)
    assert np.array_equal(hv[0], h.sum(axis=0))


def _divider(D):
    """The level map's division by 2D as the kernel does it: a 32-bit
    multiply-high and a shift, m = floor(2^(32+s) / d) + 1 with
    s = max(ceil(log2 d) - 2, 0), d = 2D."""
    d = 2 * D
    l = int(np.ceil(np.log2(d))) if d > 1 else 0
    while (1 << l) < d:
        l += 1
    s = max(l - 2, 0)
    return ((1 << (32 + s)) // d) + 1, s


def test_level_map_divider_is_exact_for_every_range():
    """For range widths D = hu_max - hu_min from 1 to 65535 (a sample plus
    both ends and every power of two), the multiplier fits 32 bits and
    umulhi(n, m) >> s equals n // (2D) for every n = 2 c 255 + D the map
    forms (c = 0..D): the division the pre-processing kernel avoids."""
    rng = np.random.default_rng(11)
    Ds = sorted(set([1, 2, 3, 4500, 4096, 65535] + [1 << k for k in range(16)] + [(1 << k) + 1 for k in range(16)] +
                    list(rng.integers(1, 65536, 120))))
    for D in Ds:
        m, s = _divider(int(D))
        assert m < (1 << 32), D
        c = np.arange(D + 1, dtype=np.uint64)
        n = np.uint64(2 * 255) * c + np.uint64(D)
        got = ((n * np.uint64(m)) >> np.uint64(32)) >> np.uint64(s)
        assert np.array_equal(got, n // np.uint64(2 * D)), D
