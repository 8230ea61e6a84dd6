"""GPU parity of the pipelined per-slice kernel against the CPU oracle,
through the C ABI.

The kernel counts chunks of the slices in order, searches each slice when
its last chunk is counted, and binarises each chunk after its slice's
search. The result must be the exhaustive method's, under the rules of the
1-D tests:
  * masks bit-exact (Algorithm 1 at the returned t);
  * t equal to the oracle's unless the oracle's top-two gap between distinct
    partitions is below 1e-9 relative;
  * |phi_gpu - phi_oracle| <= 1e-5 * max(|phi_oracle|, 1).
Each chunk is also binarised in its counting pass at a predicted threshold
and its voxels near the prediction listed; after the search a chunk is
left as it is, patched from its lists, or binarised again. The cases drive
each of those (exact predictions, windows of 1 to 127 levels, lists that
overflow, no predictions at all) and cover chunkings (one chunk a slice, a
ragged last chunk, eight chunks), thousands of small slices, clamped
tails, degenerate slices, a threshold that never arrives, and graph replay.
"""
import numpy as np
import pytest
import torch

import oracle
import phantom
import paper_2012_10684_gb300 as tg
from test_gpu_1d import check_thresholds, f32, _cuda, _chest400

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


@pytest.fixture(autouse=True)
def _pipeline_kernel():
    tg.set_slice_kernel("pipeline")
    yield
    tg.set_prediction(16, 8)
    tg.withhold_predictions(False)
    tg.set_slice_kernel("auto")


def _check(v, q=0.8, polarity="low", lo=-1024, nbins=4096):
    pol = 0 if polarity == "low" else 1
    p = tg.tsallis_params(q=q, polarity=polarity, lo=lo, nbins=nbins)
    mask, t, phi, st = tg.tsallis_segment(_cuda(v), p)
    torch.cuda.synchronize()
    g = v.shape[1] * v.shape[2]
    t_o, phi_o, gap_o, mask_o = oracle.segment1d(v, g, f32(q), lo=lo, L=nbins, polarity=pol, nthreads=16)
    t_g, st_g = t.cpu().numpy(), st.cpu().numpy()
    check_thresholds(t_g, phi.cpu().numpy(), st_g, t_o, phi_o, gap_o, (q, polarity))
    m = mask.cpu().numpy().reshape(len(t_o), -1)
    vg = v.reshape(len(t_o), -1)
    for z in range(len(t_o)):
        want = mask_o.reshape(len(t_o), -1)[z] if t_g[z] == t_o[z] else \
            oracle.binarize(vg[z], int(t_g[z]), lo=lo, L=nbins, polarity=pol)
        assert np.array_equal(m[z], want), z
    return t_g, st_g


@pytest.mark.parametrize("q", [0.5, 0.8, 1.0, 1.5])
@pytest.mark.parametrize("polarity", ["low", "high"])
def test_chest_volume_every_q(q, polarity):
    v = phantom.generate_host(phantom.chest_volume(2012106853, nz=48))
    _check(v, q, polarity)


@pytest.mark.parametrize("shape", [(9, 40, 100), (17, 8, 8), (3, 1, 8), (2, 300, 304), (1, 512, 512),
                                   (2, 1000, 1000), (1, 2048, 2048), (3, 7, 9)])
def test_ragged_shapes_and_chunkings(shape):
    """Slices of one chunk, of a full chunk plus a ragged one, of eight
    chunks (1 and 4 million voxels), a single slice, and a slice size that is
    not a multiple of 8 (served by the tile kernel)."""
    rng = np.random.default_rng(sum(shape))
    v = rng.normal(-400, 500, shape).astype(np.int16)
    _check(v, 0.8, "high")


def test_many_small_slices():
    """3000 slices of 256 voxels: one chunk each, thousands of searches and
    claims, rings that fill."""
    rng = np.random.default_rng(12)
    v = rng.normal(-500, 300, (3000, 16, 16)).astype(np.int16)
    _check(v, 0.8)


def test_level_ranges_and_clamped_tails():
    rng = np.random.default_rng(5)
    v = rng.normal(-850, 300, (10, 64, 64)).astype(np.int16)
    v.reshape(10, -1)[:, ::7] = -32768     # far below the range: level 0
    v.reshape(10, -1)[:, 3::11] = 32767    # far above: the top level
    for lo, L in ((-1024, 4096), (-1000, 100), (-900, 2), (-1100, 300), (-2000, 4096)):
        _check(v, 0.8, "low", lo, L)


def test_degenerate_slices():
    """Constant slices (no valid threshold: all-zero mask), a slice whose
    voxels are all at level 0, two-level slices, and slices without any
    voxel at level 0."""
    v = np.zeros((8, 32, 32), np.int16)
    v[0] = -1024
    v[1] = 500
    v[2, :, :16] = -1024
    v[2, :, 16:] = 200
    v[3] = -30000
    v[4] = np.arange(32 * 32).reshape(32, 32) - 600
    rng = np.random.default_rng(2)
    v[5:] = rng.integers(-1000, 3000, (3, 32, 32))
    t, st = _check(v)
    assert t[0] == -1 and t[1] == -1 and t[3] == -1


def test_skipped_arrival_reports_timeout_and_next_call_is_exact():
    """One chunk never arrives on its slice's counter: that slice is never
    searched, the bounded wait for its threshold (20 ms) runs out, every
    slice of that call reports TIMEOUT, and the next call is exact
    everywhere (the scratch state is restored)."""
    v = phantom.generate_host(phantom.chest_volume(2012106854, nz=12))
    tg.set_wait_timeout(20_000_000)
    try:
        p = tg.tsallis_params(q=0.8, flags=tg.TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL)
        mask, t, phi, st = tg.tsallis_segment(_cuda(v), p)
        torch.cuda.synchronize()
        st = st.cpu().numpy()
        assert np.all((st & 0xff) == tg.TSALLIS_ERR_TIMEOUT) and bool((t == -1).all())
    finally:
        tg.set_wait_timeout(1_000_000_000)
    _check(v)


def test_repeated_calls_and_graph_replay():
    v = phantom.generate_host(phantom.chest_volume(2012106855, nz=32))
    dv = _cuda(v)
    p = tg.tsallis_params(q=0.8)
    ref = [x.clone() for x in tg.tsallis_segment(dv, p)]
    for _ in range(3):
        for a, b in zip(tg.tsallis_segment(dv, p), ref):
            assert torch.equal(a, b)
    outs = [torch.empty_like(x) for x in ref]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        tg.tsallis_segment(dv, p, *outs)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            tg.tsallis_segment(dv, p, *outs)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        outs[0].zero_()
        outs[1].fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)


def test_kernels_agree_on_the_chest_volume():
    """Pipelined and tile kernels: same masks and thresholds on the full
    512x512x400 volume, values within the objective tolerance."""
    dv = _cuda(_chest400())
    p = tg.tsallis_params(q=0.8)
    ref = [x.clone() for x in tg.tsallis_segment(dv, p)]
    tg.set_slice_kernel("tiles")
    out = tg.tsallis_segment(dv, p)
    assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])
    d = (out[2] - ref[2]).abs()
    assert bool((d <= 1e-5 * ref[2].abs().clamp(min=1.0)).all()), d.max().item()


@pytest.mark.parametrize("q", [0.5, 0.8, 1.5])
def test_full_size_chest_volume(q):
    """The 512x512x400 chest volume in the launch shape the benchmark times."""
    _check(_chest400(), q)


@pytest.mark.parametrize("polarity", ["low", "high"])
@pytest.mark.parametrize("window", [1, 2, 8, 127])
def test_windows_and_polarity(window, polarity):
    """A one-level window sends most chunks to a second pass; wide windows
    list many voxels; both give the exhaustive result."""
    tg.set_prediction(16, window)
    v = phantom.generate_host(phantom.chest_volume(2012106857, nz=24))
    _check(v, 0.8, polarity)


def test_list_overflow_falls_back():
    """Noise concentrated around the threshold (every voxel within the
    127-level window) overflows the warps' lists (each keeps up to 1/16 of
    the voxels it counts): those chunks are binarised again, with the same
    result."""
    tg.set_prediction(16, 127)
    rng = np.random.default_rng(9)
    v = rng.normal(-400, 40, (16, 512, 512)).astype(np.int16)
    _check(v)


def test_without_predictions_every_chunk_is_binarised_again():
    tg.withhold_predictions(True)
    v = phantom.generate_host(phantom.chest_volume(2012106858, nz=10))
    _check(v)
