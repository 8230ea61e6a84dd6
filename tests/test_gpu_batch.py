"""GPU parity of the batched path (tsallis_segment_batch): many volumes of
uneven depth in one persistent launch, one threshold per volume or per slice,
checked against the CPU oracle volume by volume under the rules of
test_gpu_1d (histograms and masks bit-exact, t equal unless the oracle's
top-two gap is below 1e-9, phi within 1e-5 relative)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import phantom
import paper_2012_10684_gb300 as tg
from test_gpu_1d import check_thresholds, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _oracle_batch(vols_np, mode, q, polarity=0):
    """Per-volume oracle results, concatenated in batch order."""
    ts, phis, gaps, masks = [], [], [], []
    for v in vols_np:
        gv = v.shape[1] * v.shape[2] if mode == "slice" else v.size
        t, phi, gap, m = oracle.segment1d(v, gv, f32(q), polarity=polarity)
        ts.append(t); phis.append(phi); gaps.append(gap); masks.append(m.reshape(v.shape))
    return np.concatenate(ts), np.concatenate(phis), np.concatenate(gaps), masks


def _check_batch(vols_np, mode, q, polarity="low"):
    pol = 0 if polarity == "low" else 1
    vols = [torch.from_numpy(v).cuda() for v in vols_np]
    p = tg.tsallis_params(q=q, mode=mode, polarity=polarity)
    masks, t, phi, st = tg.tsallis_segment_batch(vols, p)
    torch.cuda.synchronize()
    t_o, phi_o, gap_o, masks_o = _oracle_batch(vols_np, mode, q, pol)
    t_g = t.cpu().numpy()
    check_thresholds(t_g, phi.cpu().numpy(), st.cpu().numpy(), t_o, phi_o, gap_o, ("batch", mode, q))
    h = 0
    for v, m, mo in zip(vols_np, masks, masks_o):
        m = m.cpu().numpy()
        ng = v.shape[0] if mode == "slice" else 1
        mg, mog, vg = m.reshape(ng, -1), mo.reshape(ng, -1), v.reshape(ng, -1)
        for g in range(ng):
            if t_g[h + g] == t_o[h + g]:
                assert np.array_equal(mg[g], mog[g]), (h, g)
            else:
                assert np.array_equal(mg[g], oracle.binarize(vg[g], int(t_g[h + g]), polarity=pol)), (h, g)
        h += ng
    return t_g, st.cpu().numpy()


def _uneven(seed, n, nx, ny, dmin, dmax):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nz = int(rng.integers(dmin, dmax + 1))
        spec = phantom.chest_volume(seed * 100 + i, nx, ny, nz, generations=int(rng.integers(4, 9)),
                                    noise_sd=int(rng.integers(5, 31)), vol_id=i)
        out.append(phantom.generate_host(spec))
    return out


@pytest.mark.parametrize("mode", ["volume", "slice"])
@pytest.mark.parametrize("q", [0.5, 0.8, 1.0, 1.5])
def test_batch_uneven_phantoms(mode, q):
    _check_batch(_uneven(3, 7, 128, 96, 1, 23), mode, q)


@pytest.mark.parametrize("mode", ["volume", "slice"])
def test_batch_ragged_shapes_and_polarity(mode):
    rng = np.random.default_rng(5)
    shapes = [(1, 1, 1), (3, 7, 5), (2, 33, 45), (5, 64, 64), (1, 300, 301), (4, 17, 9)]
    vols = [rng.normal(-400, 500, s).astype(np.int16) for s in shapes]
    _check_batch(vols, mode, 0.8, polarity="high")


def test_batch_equals_one_call_per_volume():
    vols_np = _uneven(11, 5, 256, 256, 10, 40)
    vols = [torch.from_numpy(v).cuda() for v in vols_np]
    for mode in ("volume", "slice"):
        p = tg.tsallis_params(q=0.8, mode=mode)
        masks, t, phi, st = tg.tsallis_segment_batch(vols, p)
        h = 0
        for v, m in zip(vols, masks):
            m1, t1, phi1, st1 = tg.tsallis_segment(v, p)
            n = t1.numel()
            assert torch.equal(m, m1)
            assert torch.equal(t[h:h + n], t1)
            assert torch.equal(phi[h:h + n], phi1)
            assert torch.equal(st[h:h + n] & 0xff, st1 & 0xff)
            h += n


def test_batch_graph_capture_and_replay():
    vols = [torch.from_numpy(v).cuda() for v in _uneven(13, 6, 192, 160, 5, 30)]
    p = tg.tsallis_params(q=0.8, mode="volume")
    ref = tg.tsallis_segment_batch(vols, p)
    ref = ([m.clone() for m in ref[0]],) + tuple(x.clone() for x in ref[1:])
    masks = [torch.empty_like(m) for m in ref[0]]
    outs = tuple(torch.empty_like(x) for x in ref[1:])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        tg.tsallis_segment_batch(vols, p, masks, outs)   # sizes the scratch before capture
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            tg.tsallis_segment_batch(vols, p, masks, outs)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        for m in masks:
            m.fill_(3)
        outs[0].fill_(-9)
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(masks, ref[0]):
            assert torch.equal(a, b)
        assert torch.equal(outs[0], ref[1]) and torch.equal(outs[1], ref[2])


def test_batch_autotune_picks_a_valid_shape_and_keeps_results():
    vols_np = _uneven(17, 4, 256, 256, 8, 24)
    vols = [torch.from_numpy(v).cuda() for v in vols_np]
    p = tg.tsallis_params(q=0.8, mode="volume")
    ref = [x.clone() for x in tg.tsallis_segment_batch(vols, p)[1:3]]
    try:
        tile, bps, ms = tg.tsallis_autotune_batch(vols, p)
        assert tile in (16384, 32768, 65536, 131072, 262144) and bps >= 1 and ms > 0
        out = tg.tsallis_segment_batch(vols, p)
        assert torch.equal(out[1], ref[0]) and torch.equal(out[2], ref[1])
    finally:
        tg.set_launch_shape()
    _check_batch(vols_np, "volume", 0.8)


def test_batch_autotune_cache(tmp_path):
    """The first call times the shapes and stores the winner; the second
    finds it for the same GPU, parameters and shapes and applies it without
    timing; other shapes miss."""
    vols_np = _uneven(19, 3, 256, 256, 8, 20)
    vols = [torch.from_numpy(v).cuda() for v in vols_np]
    p = tg.tsallis_params(q=0.8, mode="volume")
    cache = str(tmp_path / "tune.json")
    try:
        first = tg.tsallis_autotune_batch(vols, p, cache=cache)
        entries = tg.autotune_cache_load(cache)
        assert len(entries) == 1 and list(entries.values())[0]["tile_vox"] == first[0]
        tg.set_launch_shape()
        import time
        t0 = time.time()
        second = tg.tsallis_autotune_batch(vols, p, cache=cache)
        assert second == first and time.time() - t0 < 0.5
        tg.tsallis_autotune_batch(vols[:2], p, cache=cache)
        assert len(tg.autotune_cache_load(cache)) == 2
    finally:
        tg.set_launch_shape()


def test_batch_argument_errors():
    L = tg.lib()
    ctx = tg.context()
    p = tg.tsallis_params()
    v = torch.zeros((2, 16, 16), dtype=torch.int16, device="cuda")
    m = torch.zeros((2, 16, 16), dtype=torch.uint8, device="cuda")
    t = torch.empty(4, dtype=torch.int32, device="cuda")
    phi = torch.empty(4, device="cuda")
    st = torch.empty(4, dtype=torch.int32, device="cuda")

    def call(vols):
        arr = (tg.Volume * len(vols))(*vols)
        return L.tsallis_segment_batch(ctx, arr, len(vols), ctypes.byref(p), t.data_ptr(), phi.data_ptr(),
                                       st.data_ptr(), None)

    assert call([tg.Volume(v.data_ptr() + 2, m.data_ptr(), 16, 16, 1)]) == tg.TSALLIS_ERR_ALIGNMENT
    assert call([tg.Volume(v.data_ptr(), m.data_ptr(), 16, 16, 0)]) == tg.TSALLIS_ERR_INVALID_ARG
    assert call([tg.Volume(None, m.data_ptr(), 16, 16, 2)]) == tg.TSALLIS_ERR_INVALID_ARG
    assert L.tsallis_segment_batch(ctx, None, 0, ctypes.byref(p), t.data_ptr(), phi.data_ptr(), st.data_ptr(),
                                   None) == tg.TSALLIS_OK
    torch.cuda.synchronize()


def test_batch_of_64_uneven_chest_volumes_full_size():
    """The 64-volume workload: 512x512xD chest phantoms, D uniform in
    [120, 600], sensor noise sd in [5, 30] HU, 4-8 airway generations,
    q = 0.8, one threshold per volume, in one launch. Every volume's
    threshold and value are checked against the oracle, and its mask on
    three sampled slices."""
    specs = phantom.batch_specs(2012106844, nvol=64)
    vols = [phantom.generate_cuda(s) for s in specs]
    p = tg.tsallis_params(q=0.8, mode="volume")
    masks, t, phi, st = tg.tsallis_segment_batch(vols, p)
    torch.cuda.synchronize()
    t_g, phi_g, st_g = t.cpu().numpy(), phi.cpu().numpy(), st.cpu().numpy()
    rng = np.random.default_rng(0)
    for i, (spec, v, m) in enumerate(zip(specs, vols, masks)):
        vh = v.cpu().numpy()
        h = oracle.hist1d(vh)
        assert np.array_equal(h, tg.tsallis_histogram(v, p).cpu().numpy().reshape(-1)), i
        t_o, phi_o, gap_o, _, _ = oracle.search1d(h, f32(0.8))
        check_thresholds(t_g[i:i + 1], phi_g[i:i + 1], st_g[i:i + 1], [t_o], [phi_o], [gap_o], ("vol", i))
        for z in rng.integers(0, spec.nz, 3):
            assert np.array_equal(m[z].cpu().numpy(), oracle.binarize(vh[z], int(t_g[i]))), (i, z)
        del vh


@pytest.mark.parametrize("predictor", ["subsample", "proposer"])
def test_batch_predicted_first_pass_equals_exhaustive(predictor):
    """Whole-volume batch binarised in the histogram pass with a threshold
    predicted from the middle sixteenth of each volume: thresholds, values
    and masks equal those of the exhaustive path, and the volumes whose
    prediction was close finish without a second read."""
    import os
    from oracle import mlp
    weights = os.path.join(os.path.dirname(tg.__file__), "proposer_weights.bin")
    if predictor == "proposer":
        if os.path.exists(weights):
            tg.proposer_load(weights)
        else:
            tg.proposer_set(np.zeros(mlp.NPARAM, np.float32))
    flag = tg.TSALLIS_FLAG_PREDICT_PROPOSER if predictor == "proposer" else tg.TSALLIS_FLAG_PREDICT_SUBSAMPLE
    vols_np = _uneven(19, 6, 256, 256, 24, 80)
    vols = [torch.from_numpy(v).cuda() for v in vols_np]
    m0, t0, phi0, st0 = tg.tsallis_segment_batch(vols, tg.tsallis_params(q=0.8, mode="volume"))
    for rep in range(2):
        mk, tk, phik, stk = tg.tsallis_segment_batch(vols, tg.tsallis_params(q=0.8, mode="volume", flags=flag))
        torch.cuda.synchronize()
        assert torch.equal(t0, tk) and torch.equal(phi0, phik)
        assert torch.equal(st0 & 0xff, stk & 0xff)
        for a, b in zip(m0, mk):
            assert torch.equal(a, b)
    first = ((stk.cpu().numpy() & tg.TSALLIS_STATUS_FIRST_PASS_EXACT) != 0)
    print(predictor, "volumes finished in the first pass:", int(first.sum()), "of", len(first))
    _check_batch(vols_np, "volume", 0.8)


def test_batch_misleading_prediction_falls_back_exactly():
    """Volumes whose middle slab differs from the rest (shifted values), so
    the prediction from it is far from the exact threshold: the volumes are
    binarised again and the results still equal the exhaustive path's."""
    rng = np.random.default_rng(23)
    vols_np = []
    for i in range(4):
        v = np.clip(rng.normal(-600, 200, (32, 96, 128)), -1024, 3071).astype(np.int16)
        v[:, :30] = np.clip(rng.normal(100, 50, (32, 30, 128)), -1024, 3071).astype(np.int16)
        v[15:17] = np.clip(v[15:17].astype(np.int32) + 700, -1024, 3071).astype(np.int16)   # the sampled slab
        vols_np.append(v)
    vols = [torch.from_numpy(v).cuda() for v in vols_np]
    m0, t0, phi0, _ = tg.tsallis_segment_batch(vols, tg.tsallis_params(q=0.8, mode="volume"))
    p = tg.tsallis_params(q=0.8, mode="volume", flags=tg.TSALLIS_FLAG_PREDICT_SUBSAMPLE)
    mk, tk, phik, stk = tg.tsallis_segment_batch(vols, p)
    torch.cuda.synchronize()
    assert torch.equal(t0, tk) and torch.equal(phi0, phik)
    for a, b in zip(m0, mk):
        assert torch.equal(a, b)
    assert not ((stk.cpu().numpy() & tg.TSALLIS_STATUS_FIRST_PASS_EXACT) != 0).all()


def test_batch_prediction_argument_rules():
    vols = [torch.zeros((2, 16, 16), dtype=torch.int16, device="cuda")]
    for p in (tg.tsallis_params(mode="slice", flags=tg.TSALLIS_FLAG_PREDICT_SUBSAMPLE),
              tg.tsallis_params(mode="volume", topk=64, flags=tg.TSALLIS_FLAG_PREDICT_SUBSAMPLE)):
        with pytest.raises(tg.TsallisError):
            tg.tsallis_segment_batch(vols, p)
