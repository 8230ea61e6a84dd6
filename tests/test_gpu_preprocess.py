"""GPU parity of the pre-processing and chest-mask morphology
(tsallis_preprocess) against the oracle: levels, morphology results and
256-level histograms bit-exact, on ragged and tile-crossing shapes, every
radius class and every op, at the full 512 x 512 x 400 size on sampled
slices, and the paper's whole segmentation step (8-bit levels, chest mask,
Tsallis threshold per slice, Algorithm 1) against the oracle's."""
import numpy as np
import pytest
import torch

import oracle
import phantom
import paper_2012_10684_gb300 as tg
from test_gpu_1d import check_thresholds, f32

pytestmark = pytest.mark.gpu

OPS = ["none", "erode", "dilate", "open", "close", "chest_mask", "black_tophat"]
ORACLE_OP = {"none": "copy"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _ct(rng, shape):
    """CT-like values with background, out-of-range and exact-tie entries."""
    v = rng.integers(-2600, 3200, shape).astype(np.int16)
    f = v.reshape(-1)
    k = f.size
    f[: k // 6] = -2000
    f[k // 6: k // 5] = 250            # 127.5: the rounding tie
    f[k // 5: k // 4] = -1024
    rng.shuffle(f)
    # a few blocky structures so that openings and closings do something
    z, y, x = shape
    for _ in range(4):
        y0, x0 = rng.integers(0, max(1, y - 8)), rng.integers(0, max(1, x - 8))
        v[:, y0:y0 + rng.integers(1, 12), x0:x0 + rng.integers(1, 12)] = rng.integers(-1100, 1500)
    return v


def _oracle(v, r, op, per_slice=True):
    return oracle.preprocess(v, r=r, op=ORACLE_OP.get(op, op), per_slice=per_slice)


def _gpu(v, r, op, per_slice=True, **kw):
    pp = tg.preprocess_params(op=op, radius=r, per_slice=per_slice, **kw)
    return tg.tsallis_preprocess(torch.from_numpy(v).cuda(), pp)


@pytest.mark.parametrize("shape", [(3, 77, 203), (2, 33, 129), (1, 1, 1), (1, 40, 3), (2, 64, 256)])
@pytest.mark.parametrize("r", [0, 1, 2, 5, 10])
def test_chest_mask_bit_exact(shape, r):
    rng = np.random.default_rng(r * 1000 + shape[1] + shape[2])
    v = _ct(rng, shape)
    o, h = _gpu(v, r, "chest_mask")
    oo, ho = _oracle(v, r, "chest_mask")
    assert np.array_equal(o.cpu().numpy(), oo)
    assert np.array_equal(h.cpu().numpy(), ho)


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("r", [3, 15])
def test_every_op_bit_exact(op, r):
    rng = np.random.default_rng(len(op) * 31 + r)
    v = _ct(rng, (2, 45, 150))
    for per_slice in (True, False):
        o, h = _gpu(v, r, op, per_slice=per_slice)
        oo, ho = _oracle(v, r, op, per_slice=per_slice)
        assert np.array_equal(o.cpu().numpy(), oo), (op, r)
        assert np.array_equal(h.cpu().numpy(), ho), (op, r)


@pytest.mark.parametrize("r", [4, 6, 7, 8, 9, 11, 12, 13, 14])
def test_other_radii_bit_exact(r):
    rng = np.random.default_rng(500 + r)
    v = _ct(rng, (1, 70, 140))
    for op in ("open", "close"):
        o, _ = _gpu(v, r, op)
        oo, _ = _oracle(v, r, op)
        assert np.array_equal(o.cpu().numpy(), oo), (op, r)


def test_level_map_settings():
    """Other background and range settings: every int16 value once."""
    v = np.arange(-32768, 32768, dtype=np.int16).reshape(1, 256, 256)
    for bg, lo, hi in ((-2000, -2000, 2500), (-1500, -1024, 3071), (-32768, -5, 2), (100, -200, 65335 - 200)):
        pp = tg.preprocess_params(op="none", background=bg, hu_min=lo, hu_max=hi)
        o, h = tg.tsallis_preprocess(torch.from_numpy(v).cuda(), pp)
        g = oracle.rescale8(v, bg, lo, hi)
        assert np.array_equal(o.cpu().numpy(), g.astype(np.int16)), (bg, lo, hi)
        assert np.array_equal(h.cpu().numpy()[0], np.bincount(g.reshape(-1), minlength=256))


def test_outputs_are_optional_and_agree():
    rng = np.random.default_rng(9)
    v = torch.from_numpy(_ct(rng, (3, 50, 60))).cuda()
    pp = tg.preprocess_params(radius=4)
    o, h = tg.tsallis_preprocess(v, pp)
    o2, none = tg.tsallis_preprocess(v, pp, want_hist=False)
    none2, h2 = tg.tsallis_preprocess(v, pp, want_out=False)
    assert none is None and none2 is None
    assert torch.equal(o, o2) and torch.equal(h, h2)


def test_argument_errors():
    v = torch.zeros((2, 16, 16), dtype=torch.int16, device="cuda")
    bad = [dict(radius=16), dict(radius=-1), dict(op=7), dict(hu_min=5, hu_max=5), dict(hu_min=-40000 + 1,
                                                                                         hu_max=30000)]
    for kw in bad:
        with pytest.raises(tg.TsallisError):
            tg.tsallis_preprocess(v, tg.preprocess_params(**kw))
    with pytest.raises(tg.TsallisError):
        tg.tsallis_preprocess(v, want_out=False, want_hist=False)
    with pytest.raises(tg.TsallisError):
        tg.tsallis_preprocess(v, out=v)            # in-place is refused
    e = torch.zeros((0, 16, 16), dtype=torch.int16, device="cuda")
    o, h = tg.tsallis_preprocess(e)
    assert o.numel() == 0 and h.shape == (0, 256)


def test_full_size_chest_phantom_sampled_slices():
    """512 x 512 x 400 chest phantom, radius 10, as the benchmark runs it:
    the sampled slices equal the oracle's slice by slice, every slice's
    histogram counts its 262,144 pixels, and the volume histogram is the sum
    of the slice histograms."""
    spec = phantom.chest_volume(2012106842, 512, 512, 400)
    v = phantom.generate_cuda(spec)
    o, h = tg.tsallis_preprocess(v, tg.preprocess_params())
    _, hv = tg.tsallis_preprocess(v, tg.preprocess_params(per_slice=False), want_out=False)
    assert torch.all(h.sum(dim=1) == 512 * 512)
    assert torch.equal(hv[0].long(), h.long().sum(dim=0))
    vh = v.cpu().numpy()
    for z in (0, 137, 399):
        oo, ho = _oracle(vh[z:z + 1], 10, "chest_mask")
        assert np.array_equal(o[z:z + 1].cpu().numpy(), oo), z
        assert np.array_equal(h[z].cpu().numpy(), ho[0]), z


@pytest.mark.parametrize("q", [0.5, 0.8, 1.5])
def test_paper_segmentation_step(q):
    """Pre-processing, chest mask (disk of radius 10), per-slice Tsallis
    threshold on the 256 levels and Algorithm 1, all on the GPU, against the
    oracle's same chain."""
    spec = phantom.chest_volume(2012106842, 256, 256, 12)
    v = phantom.generate_cuda(spec)
    o, h = tg.tsallis_preprocess(v, tg.preprocess_params())
    p = tg.tsallis_params(q=q, lo=0, nbins=256, mode="slice")
    t, phi, st = tg.tsallis_search(h, p)
    m = tg.tsallis_binarize(o, t, p)
    oo, _ = _oracle(v.cpu().numpy(), 10, "chest_mask")
    to, phio, gapo, mo = oracle.segment1d(oo, 256 * 256, f32(q), lo=0, L=256)
    check_thresholds(t.cpu().numpy(), phi.cpu().numpy(), st.cpu().numpy(), to, phio, gapo, ("paper", q))
    same = gapo >= 1e-9
    mg = m.cpu().numpy().reshape(12, -1)
    assert np.array_equal(mg[same], mo.reshape(12, -1)[same])
    # the fused tsallis_segment on the chest-masked levels agrees as well
    m2, t2, _, _ = tg.tsallis_segment(o, p)
    assert torch.equal(t2, t) and torch.equal(m2, m)
