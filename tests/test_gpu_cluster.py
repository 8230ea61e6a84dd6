"""GPU parity of the two per-slice 1-D kernels against the CPU oracle.

tsallis_segment serves per-slice 1-D work with either the cluster kernel
(each slice held in the shared memory of an 8-CTA cluster between histogram
and binarisation) or the persistent tile kernel. Both are checked here
against the oracle under the rules of test_gpu_1d (histograms and masks
bit-exact, t equal unless the oracle's top-two gap is below 1e-9, phi within
1e-5 relative), and against each other.
"""
import contextlib

import numpy as np
import pytest
import torch

import oracle
import phantom
import paper_2012_10684_gb300 as tg
from test_gpu_1d import _check_step, _cuda, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


@contextlib.contextmanager
def kernel(kind):
    tg.set_slice_kernel(kind)
    try:
        yield
    finally:
        tg.set_slice_kernel("auto")


def cluster_eligible(shape):
    s = shape[1] * shape[2]
    return s % 8 == 0 and s <= 8 * 32768


@pytest.mark.parametrize("kind", ["cluster", "tiles"])
@pytest.mark.parametrize("q", [0.5, 0.8, 1.0, 1.5, 3.0])
def test_single_slice_phantom(kind, q):
    v = phantom.generate_host(phantom.slice_phantom(2012106841))
    with kernel(kind):
        _check_step(v, "slice", q)


@contextlib.contextmanager
def speculation(on):
    tg.set_speculation(on)
    try:
        yield
    finally:
        tg.set_speculation(False)


@pytest.mark.parametrize("kind,spec", [("cluster", True), ("tiles", True), ("tiles", False)])
@pytest.mark.parametrize("q", [0.5, 0.8, 1.5])
def test_chest_volume_full_size(kind, spec, q):
    """All 400 slices of the 512x512x400 chest phantom (more slices than
    resident clusters, so clusters take several slices each); the tile
    kernel with and without first-pass binarisation."""
    v = phantom.generate_host(phantom.chest_volume(2012106842, nz=400))
    with kernel(kind), speculation(spec):
        _, st = _check_step(v, "slice", q)
    first = (st & tg.TSALLIS_STATUS_FIRST_PASS_EXACT) != 0
    if kind == "cluster" or not spec:
        assert not first.any()
    else:
        # slices that start after the first search has finished get a
        # prediction; on this phantom it is exact, or exact after the
        # listed voxels are rewritten, for most of them
        assert first.sum() > 50, first.sum()


def test_first_pass_prediction_that_fails_falls_back_exactly():
    """Slices whose thresholds differ, with every level between them
    occupied: a prediction from another slice is wrong, the slice is
    binarised again, and the masks are still exact."""
    rng = np.random.default_rng(77)
    nz = 120
    v = np.empty((nz, 128, 128), np.int16)
    for z in range(nz):
        shift = 150 * (z % 3)
        v[z] = np.clip(rng.normal(-700 + shift, 120, (128, 128)), -1024, 3071).astype(np.int16)
        v[z, :40] = np.clip(rng.normal(60 + shift, 40, (40, 128)), -1024, 3071).astype(np.int16)
    with kernel("tiles"), speculation(True):
        tg.set_launch_shape(4096, 0)
        try:
            _, st = _check_step(v, "slice", 0.8)
        finally:
            tg.set_launch_shape()
    first = (st & tg.TSALLIS_STATUS_FIRST_PASS_EXACT) != 0
    assert first.sum() < nz


# slice shapes the cluster kernel takes: parts shorter than a chunk, parts
# that are empty (slices smaller than eight parts), and a full 512x512 slice
@pytest.mark.parametrize("shape", [(3, 1, 8), (2, 8, 9), (4, 40, 64), (5, 128, 136), (9, 256, 130), (2, 512, 512),
                                   (37, 64, 64)])
@pytest.mark.parametrize("polarity", ["low", "high"])
def test_cluster_ragged_shapes(shape, polarity):
    assert cluster_eligible(shape)
    rng = np.random.default_rng(shape[1] * shape[2] + shape[0])
    v = rng.normal(-400, 500, shape).astype(np.int16)
    with kernel("cluster"):
        _check_step(v, "slice", 0.8, polarity=polarity)


@pytest.mark.parametrize("lo,L", [(-1024, 4096), (-2000, 4096), (0, 256), (-100, 2), (32000, 4096)])
def test_cluster_level_ranges_and_adversarial_values(lo, L):
    rng = np.random.default_rng(L * 7 + (lo & 0xffff))
    v = rng.integers(-32768, 32768, (6, 64, 128)).astype(np.int16)
    flat = v.reshape(-1)
    flat[: flat.size // 4] = lo          # a hot level
    flat[flat.size // 4: flat.size // 3] = -32768
    flat[flat.size // 3: flat.size // 3 + 5] = 32767
    rng.shuffle(flat)
    p = tg.tsallis_params(q=0.8, lo=lo, nbins=L, mode="slice")
    with kernel("cluster"):
        mask, t, phi, st = tg.tsallis_segment(_cuda(v), p)
    torch.cuda.synchronize()
    t_o, phi_o, gap_o, mask_o = oracle.segment1d(v, 64 * 128, f32(0.8), lo=lo, L=L)
    t_g = t.cpu().numpy()
    for g in range(6):
        if t_o[g] < 0:
            assert t_g[g] == -1
            continue
        if gap_o[g] >= 1e-9:
            assert t_g[g] == t_o[g], (g, t_g[g], t_o[g])
        assert abs(phi.cpu().numpy()[g] - phi_o[g]) <= 1e-5 * max(abs(phi_o[g]), 1.0)
    m = mask.cpu().numpy().reshape(6, -1)
    vg = v.reshape(6, -1)
    for g in range(6):
        assert np.array_equal(m[g], oracle.binarize(vg[g], int(t_g[g]), lo=lo, L=L))


def test_cluster_degenerate_slices():
    """A constant slice and a slice with one other voxel: no valid threshold
    and exactly one, respectively; an all-zero mask for the first."""
    v = np.full((3, 64, 64), 40, dtype=np.int16)
    v[1, 5, 7] = -900
    v[2, ::2] = -1024
    with kernel("cluster"):
        mask, t, phi, st = tg.tsallis_segment(_cuda(v), tg.tsallis_params(q=0.8))
    torch.cuda.synchronize()
    t, st, mask = t.cpu().numpy(), st.cpu().numpy(), mask.cpu().numpy()
    assert t[0] == -1 and (st[0] & 0xff) == tg.TSALLIS_ERR_NO_VALID_THRESHOLD
    assert not mask[0].any()
    assert t[1] == 124 and (st[1] & 0xff) == 0                   # level of -900 is 124
    assert mask[1].sum() == 1 and mask[1, 5, 7] == 1
    assert t[2] == 0 and np.array_equal(mask[2], (v[2] <= -1024).astype(np.uint8))


def test_cluster_matches_tiles_kernel_bit_for_bit_on_masks():
    v = _cuda(phantom.generate_host(phantom.chest_volume(31, nz=90)))
    p = tg.tsallis_params(q=0.8)
    with kernel("cluster"):
        a = [x.cpu().numpy() for x in tg.tsallis_segment(v, p)]
    with kernel("tiles"):
        b = [x.cpu().numpy() for x in tg.tsallis_segment(v, p)]
    # thresholds may differ only where the oracle's gap is tiny; then both
    # masks follow Algorithm 1 at their own t (checked in the parity tests)
    same = a[1] == b[1]
    assert same.mean() > 0.95
    assert np.array_equal(a[0][same], b[0][same])
    assert np.all(np.abs(a[2] - b[2]) <= 1e-5 * np.maximum(np.abs(b[2]), 1.0))


def test_cluster_repeated_calls_and_graph_replay():
    v = _cuda(phantom.generate_host(phantom.chest_volume(7, nz=80)))
    p = tg.tsallis_params(q=1.5)
    with kernel("cluster"):
        ref = [x.clone() for x in tg.tsallis_segment(v, p)]
        for _ in range(3):
            for a, b in zip(tg.tsallis_segment(v, p), ref):
                assert torch.equal(a, b)
        outs = [torch.empty_like(x) for x in ref]
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            tg.tsallis_segment(v, p, *outs)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                tg.tsallis_segment(v, p, *outs)
        torch.cuda.current_stream().wait_stream(s)
        for _ in range(3):
            for o in outs:
                o.fill_(0)
            g.replay()
            torch.cuda.synchronize()
            for a, b in zip(outs, ref):
                assert torch.equal(a, b)


def test_cluster_chunk_wait_timeout_reports_status_and_recovers():
    """Test hook: the first chunk of slice 0 is never copied, so that
    slice's bounded wait runs out; the slice reports TIMEOUT with an
    all-zero mask, the other slices are unaffected, and the next call is
    exact again."""
    v = phantom.generate_host(phantom.chest_volume(9, nz=12))
    dv = _cuda(v)
    tg.set_wait_timeout(20_000_000)   # 20 ms
    try:
        with kernel("cluster"):
            p = tg.tsallis_params(q=0.8, flags=tg.TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL)
            mask, t, phi, st = tg.tsallis_segment(dv, p)
            torch.cuda.synchronize()
            st = st.cpu().numpy()
            assert (st[0] & 0xff) == tg.TSALLIS_ERR_TIMEOUT and t[0].item() == -1
            assert not mask[0].any().item()
            assert np.all((st[1:] & 0xff) == 0)
    finally:
        tg.set_wait_timeout(1_000_000_000)
    with kernel("cluster"):
        _check_step(v, "slice", 0.8)


@pytest.mark.parametrize("kind", ["cluster", "tiles"])
@pytest.mark.parametrize("q", [0.7, 1.0, 2.0])
def test_exact_ties_between_mirror_partitions_are_reranked(kind, q):
    """Three equal, disjoint blocks of levels: splitting after the first or
    after the second gives mirror-image partitions with equal objective
    values, so the maximum is a tie that the FP64 re-rank decides. The oracle
    reports a zero gap; the threshold must be one of the two."""
    v = np.empty((4, 48, 64), np.int16)   # 3072 voxels: three blocks of 1024
    flat = v.reshape(4, -1)
    for z in range(4):
        flat[z] = np.repeat(np.array([-1000 + z, -500 + z, z], np.int16), 1024)
    t_o, phi_o, gap_o, _ = oracle.segment1d(v, 48 * 64, f32(q), want_mask=False)
    assert np.all(gap_o == 0)
    with kernel(kind):
        mask, t, phi, st = tg.tsallis_segment(_cuda(v), tg.tsallis_params(q=q))
    torch.cuda.synchronize()
    t, st = t.cpu().numpy(), st.cpu().numpy()
    for z in range(4):
        lv = np.unique(np.clip(flat[z].astype(np.int32) + 1024, 0, 4095))
        assert t[z] in (lv[0], lv[1]), (z, t[z], lv)
        assert abs(phi.cpu().numpy()[z] - phi_o[z]) <= 1e-5 * max(abs(phi_o[z]), 1.0)
        assert (st[z] & 0xff) == 0
        assert np.array_equal(mask[z].cpu().numpy().reshape(-1), oracle.binarize(flat[z], int(t[z])))
