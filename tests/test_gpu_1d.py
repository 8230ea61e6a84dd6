"""GPU parity of the 1-D path against the CPU oracle, through the C ABI.

Rules (written here so a reader sees them):
  * histograms and masks: bit-exact;
  * threshold t: equal to the oracle's unless the oracle's relative gap
    between its best and second-best distinct partitions is below 1e-9;
    when t differs the mask must equal Algorithm 1 at the GPU's t;
  * objective values: |phi_gpu - phi_oracle| <= 1e-5 * max(|phi_oracle|, 1).
"""
import numpy as np
import pytest
import torch

import oracle
import phantom
import paper_2012_10684_gb300 as tg

pytestmark = pytest.mark.gpu

GAP = 1e-9
PHI_RTOL = 1e-5


def f32(q):
    """The Tsallis index as the C ABI receives it (a float). The oracle is
    given this value so both sides evaluate the same objective."""
    return float(np.float32(q))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_thresholds(t_g, phi_g, st_g, t_o, phi_o, gap_o, ctx=""):
    t_g, phi_g, st_g = np.asarray(t_g), np.asarray(phi_g), np.asarray(st_g)
    for i in range(len(t_o)):
        if t_o[i] < 0:
            assert t_g[i] == -1 and (st_g[i] & 0xff) == tg.TSALLIS_ERR_NO_VALID_THRESHOLD, (ctx, i)
            continue
        assert (st_g[i] & 0xff) == 0, (ctx, i, st_g[i])
        if gap_o[i] >= GAP:
            assert t_g[i] == t_o[i], (ctx, i, t_g[i], t_o[i], gap_o[i])
        assert abs(phi_g[i] - phi_o[i]) <= PHI_RTOL * max(abs(phi_o[i]), 1.0), (ctx, i, phi_g[i], phi_o[i])


# ------------------------------------------------------------ histogram

def _adversarial_volume(rng, shape):
    v = rng.integers(-32768, 32768, shape).astype(np.int16)
    flat = v.reshape(-1)
    k = flat.size
    flat[: k // 5] = -1024                     # the hot clamp level
    flat[k // 5: k // 4] = -32768
    flat[k // 4: k // 3] = 3071
    flat[k // 3: k // 3 + 7] = 32767
    rng.shuffle(flat)
    return v


@pytest.mark.parametrize("shape", [(1, 512, 512), (7, 33, 45), (3, 1, 1), (2, 300, 301), (1, 1, 9)])
@pytest.mark.parametrize("mode", ["slice", "volume"])
def test_histogram_bit_exact(shape, mode):
    rng = np.random.default_rng(sum(shape))
    v = _adversarial_volume(rng, shape)
    p = tg.tsallis_params(mode=mode)
    h = tg.tsallis_histogram(_cuda(v), p).cpu().numpy()
    groups = v.reshape(shape[0], -1) if mode == "slice" else v.reshape(1, -1)
    for g in range(groups.shape[0]):
        assert np.array_equal(h[g], oracle.hist1d(groups[g])), g


def test_histogram_phantom_and_level_range():
    v = phantom.generate_host(phantom.chest_volume(2012106842, nz=24))
    for lo, L in ((-1024, 4096), (-1000, 100), (-900, 2)):
        p = tg.tsallis_params(lo=lo, nbins=L)
        h = tg.tsallis_histogram(_cuda(v), p).cpu().numpy()
        for z in range(v.shape[0]):
            assert np.array_equal(h[z], oracle.hist1d(v[z], lo, L)), (lo, L, z)


def test_histogram_misaligned_volume_is_rejected():
    v = torch.zeros((4, 5, 3), dtype=torch.int16, device="cuda")   # 30-byte slices
    with pytest.raises(tg.TsallisError) as e:
        tg.tsallis_histogram(v[1:])
    assert e.value.code == tg.TSALLIS_ERR_ALIGNMENT


# ------------------------------------------------------------ search

def _rand_hist(rng, L, zero_frac, hi):
    h = rng.integers(0, hi, L).astype(np.int64)
    h[rng.random(L) < zero_frac] = 0
    return h


@pytest.mark.parametrize("q", [0.3, 0.5, 0.8, 1.0, 1.5, 2.5])
@pytest.mark.parametrize("L", [2, 3, 100, 511, 4096])
def test_search_random_histograms(q, L):
    rng = np.random.default_rng(L * 10 + int(q * 10))
    H = np.stack([_rand_hist(rng, L, zf, hi) for zf, hi in
                  ((0.0, 1000), (0.5, 100), (0.9, 10 ** 6), (0.3, 3), (0.0, 2 ** 20))])
    p = tg.tsallis_params(q=q, nbins=L)
    t, phi, st, curve = tg.tsallis_search(_cuda(H.astype(np.int32)), p, curve=True)
    t, phi, st, curve = t.cpu().numpy(), phi.cpu().numpy(), st.cpu().numpy(), curve.cpu().numpy()
    res = [oracle.search1d(h, f32(q)) for h in H]
    check_thresholds(t, phi, st, [r[0] for r in res], [r[1] for r in res], [r[2] for r in res], (q, L))
    for i, (to, bo, go, po, vo) in enumerate(res):
        assert np.array_equal(~np.isnan(curve[i]), vo), i
        d = np.abs(curve[i][vo] - po[vo])
        assert np.all(d <= PHI_RTOL * np.maximum(np.abs(po[vo]), 1.0)), (i, d.max())


@pytest.mark.parametrize("q", [0.5, 0.8, 1.5])
def test_search_two_uniform_modes_closed_form(q):
    L, w = 4096, 40
    h = np.zeros(L, np.int64)
    h[100:100 + w] = 500
    h[1000:1000 + w] = 500
    t, phi, st = tg.tsallis_search(_cuda(h[None].astype(np.int32)), tg.tsallis_params(q=q))
    assert int(t.item()) == 100 + w - 1
    want = (1 - w ** (2 * (1 - f32(q)))) / (f32(q) - 1)
    assert abs(phi.item() - want) <= PHI_RTOL * max(abs(want), 1)


def test_search_degenerate_histograms():
    L = 64
    H = np.zeros((4, L), np.int32)
    H[1, 10] = 5            # one level only
    H[2, 0] = 1
    H[2, L - 1] = 1         # the two end levels
    H[3, 5] = 3
    H[3, 6] = 9             # two adjacent levels
    t, phi, st = tg.tsallis_search(_cuda(H), tg.tsallis_params(nbins=L))
    t, st = t.cpu().numpy(), st.cpu().numpy()
    assert t[0] == -1 and (st[0] & 0xff) == tg.TSALLIS_ERR_NO_VALID_THRESHOLD
    assert t[1] == -1 and (st[1] & 0xff) == tg.TSALLIS_ERR_NO_VALID_THRESHOLD
    assert t[2] == 0 and (st[2] & 0xff) == 0
    assert t[3] == 5 and (st[3] & 0xff) == 0
    # two one-level classes: phi = 0 exactly; FP32 is held to the objective tolerance
    assert np.all(np.abs(phi.cpu().numpy()) <= PHI_RTOL)


def test_search_phantom_slices_near_ties_rerank():
    """Phantom slice histograms at q = 1.5 have many top-two gaps below 1e-6;
    the FP64 re-rank must still land on the oracle's partition."""
    v = phantom.generate_host(phantom.chest_volume(2012106842, nz=96))
    H = np.stack([oracle.hist1d(v[z]) for z in range(v.shape[0])])
    for q in (0.5, 0.8, 1.5):
        t, phi, st = tg.tsallis_search(_cuda(H.astype(np.int32)), tg.tsallis_params(q=q))
        res = [oracle.search1d(h, f32(q)) for h in H]
        check_thresholds(t.cpu().numpy(), phi.cpu().numpy(), st.cpu().numpy(), [r[0] for r in res],
                         [r[1] for r in res], [r[2] for r in res], q)
        if q == 1.5:
            assert (st.cpu().numpy() & tg.TSALLIS_STATUS_RERANKED).any()


# ------------------------------------------------------------ binarise

@pytest.mark.parametrize("polarity", ["low", "high"])
@pytest.mark.parametrize("shape", [(3, 64, 64), (5, 37, 29), (1, 1, 3)])
def test_binarize_bit_exact(polarity, shape):
    rng = np.random.default_rng(3)
    v = _adversarial_volume(rng, shape)
    pol = 0 if polarity == "low" else 1
    ts = np.array([-1, 0, 4094, 4095, 77, 2000, 10 ** 6][: shape[0]] + [5] * max(0, shape[0] - 7), np.int32)
    p = tg.tsallis_params(polarity=polarity)
    m = tg.tsallis_binarize(_cuda(v), _cuda(ts[: shape[0]]), p).cpu().numpy()
    for z in range(shape[0]):
        t = int(ts[z])
        if t >= 4095:   # every level is <= t
            want = np.full(v[z].shape, 1 - pol, np.uint8)
        else:
            want = oracle.binarize(v[z], t, polarity=pol)
        assert np.array_equal(m[z], want), (z, t)


# ------------------------------------------------------------ fused step

def _oracle_step(v, mode, q, polarity=0):
    g = v.shape[1] * v.shape[2] if mode == "slice" else v.size
    return oracle.segment1d(v, g, f32(q), polarity=polarity, nthreads=16)


def _check_step(v, mode, q, polarity="low"):
    pol = 0 if polarity == "low" else 1
    p = tg.tsallis_params(q=q, mode=mode, polarity=polarity)
    mask, t, phi, st = tg.tsallis_segment(_cuda(v), p)
    torch.cuda.synchronize()
    t_o, phi_o, gap_o, mask_o = _oracle_step(v, mode, q, pol)
    t_g = t.cpu().numpy()
    check_thresholds(t_g, phi.cpu().numpy(), st.cpu().numpy(), t_o, phi_o, gap_o, (mode, q))
    m = mask.cpu().numpy().reshape(len(t_o), -1)
    mo = mask_o.reshape(len(t_o), -1)
    vg = v.reshape(len(t_o), -1)
    for g in range(len(t_o)):
        if t_g[g] == t_o[g]:
            assert np.array_equal(m[g], mo[g]), g
        else:
            assert np.array_equal(m[g], oracle.binarize(vg[g], int(t_g[g]), polarity=pol)), g
    return t_g, st.cpu().numpy()


def test_segment_single_slice_phantom():
    v = phantom.generate_host(phantom.slice_phantom(2012106841))
    for q in (0.5, 0.8, 1.0, 1.5):
        _check_step(v, "slice", q)


@pytest.mark.parametrize("q", [0.5, 0.8, 1.5])
@pytest.mark.parametrize("mode", ["slice", "volume"])
def test_segment_chest_volume_full_size(q, mode):
    """The 512x512x400 chest volume, in the launch shape the benchmark times."""
    v = _chest400()
    _check_step(v, mode, q)


_CHEST = {}


def _chest400():
    if "v" not in _CHEST:
        _CHEST["v"] = phantom.generate_host(phantom.chest_volume(2012106842, nz=400))
    return _CHEST["v"]


@pytest.mark.parametrize("shape", [(5, 37, 29), (3, 300, 301), (2, 1, 1), (1, 7, 3), (9, 256, 130)])
@pytest.mark.parametrize("mode", ["slice", "volume"])
def test_segment_ragged_shapes(shape, mode):
    rng = np.random.default_rng(shape[1] * shape[2])
    v = (rng.normal(-400, 500, shape)).astype(np.int16)
    _check_step(v, mode, 0.8, polarity="high")


def _same(outs, ref):
    """Equal masks, thresholds, values and statuses. The first-pass bit of a
    status depends on which searches finished first, so it is not compared."""
    for i, (a, b) in enumerate(zip(outs, ref)):
        if i == 3:
            a, b = a & ~tg.TSALLIS_STATUS_FIRST_PASS_EXACT, b & ~tg.TSALLIS_STATUS_FIRST_PASS_EXACT
        assert torch.equal(a, b), i


def test_segment_repeated_calls_and_graph_replay():
    v = phantom.generate_host(phantom.chest_volume(7, nz=40))
    dv = _cuda(v)
    p = tg.tsallis_params(q=0.8)
    ref = [x.clone() for x in tg.tsallis_segment(dv, p)]
    for _ in range(3):
        _same(tg.tsallis_segment(dv, p), ref)
    mask = torch.empty_like(ref[0])
    t = torch.empty_like(ref[1])
    phi = torch.empty_like(ref[2])
    st = torch.empty_like(ref[3])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        tg.tsallis_segment(dv, p, mask, t, phi, st)   # scratch allocated before capture
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            tg.tsallis_segment(dv, p, mask, t, phi, st)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        mask.zero_()
        t.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        _same((mask, t, phi, st), ref)


def test_wait_timeout_reports_status_and_context_recovers():
    v = phantom.generate_host(phantom.chest_volume(9, nz=6))
    dv = _cuda(v)
    tg.set_wait_timeout(50_000_000)   # 50 ms
    try:
        p = tg.tsallis_params(q=0.8, flags=tg.TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL)
        mask, t, phi, st = tg.tsallis_segment(dv, p)
        torch.cuda.synchronize()
        st = st.cpu().numpy()
        assert (st[0] & 0xff) == tg.TSALLIS_ERR_TIMEOUT
        assert np.all((st[1:] & 0xff) == 0)
    finally:
        tg.set_wait_timeout(1_000_000_000)
    _check_step(v, "slice", 0.8)


def test_phantom_gpu_generator_matches_host():
    for spec in (phantom.slice_phantom(5), phantom.chest_volume(11, nz=37, generations=5),
                 phantom.chest_volume(12, 100, 60, 9)):
        a = phantom.generate_host(spec)
        b = phantom.generate_cuda(spec).cpu().numpy()
        assert np.array_equal(a, b)


def test_double_float_pow_and_log2_accuracy():
    """The search's double-float (h/N)^q and log2 h against numpy float64."""
    rng = np.random.default_rng(21)
    for N in (262_144, 104_857_600, 2 ** 31 - 1):
        hs = np.concatenate([np.arange(1, 2000), rng.integers(1, N + 1, 20_000),
                             [N, N - 1, 2 ** 16, 2 ** 16 - 1, 2 ** 16 + 1, 2 ** 24 - 1, 2 ** 24, 2 ** 24 + 1]])
        hs = hs[(hs >= 1) & (hs <= N)].astype(np.int64)
        dh = _cuda(hs.astype(np.uint32).view(np.int32))
        for q in (0.3, 0.5, 0.8, 1.5, 2.5, 4.0):
            pw, lg = tg.tsallis_probe_dfmath(dh, N, q)
            pw, lg = pw.cpu().numpy(), lg.cpu().numpy()
            want = (hs.astype(np.float64) / N) ** f32(q)
            rel = np.abs(pw - want) / want
            assert rel.max() < 1e-12, (N, q, rel.max(), hs[np.argmax(rel)])
        wl = np.log2(hs.astype(np.float64))
        assert np.max(np.abs(lg - wl) / np.maximum(wl, 1.0)) < 1e-13


# ------------------------------------------------------------ host buffers

@pytest.mark.parametrize("pinned", [True, False])
def test_segment_host_full_size_equals_device(pinned):
    """The 512x512x400 chest volume through the host-buffer entry point (7
    pipelined chunks of 64 slices): masks, thresholds, values and statuses
    equal the device path's."""
    v = phantom.generate_cuda(phantom.chest_volume(2012106842, 512, 512, 400))
    p = tg.tsallis_params(q=0.8, mode="slice")
    m0, t0, phi0, st0 = tg.tsallis_segment(v, p)
    hv = v.cpu()
    if pinned:
        hv = hv.pin_memory()
    m, t, phi, st = tg.tsallis_segment_host(hv, p)
    assert torch.equal(m, m0.cpu()) and torch.equal(t, t0.cpu())
    assert torch.equal(phi, phi0.cpu()) and torch.equal(st, st0.cpu())


@pytest.mark.parametrize("shape,mode,two_d", [((3, 37, 53), "slice", False), ((2, 300, 301), "volume", False),
                                              ((70, 512, 520), "slice", False), ((4, 64, 64), "slice", True),
                                              ((5, 48, 40), "volume", True)])
def test_segment_host_shapes_and_forms(shape, mode, two_d):
    rng = np.random.default_rng(sum(shape))
    hv = torch.from_numpy(rng.integers(-1500, 3200, shape).astype(np.int16))
    p = tg.tsallis_params(q=0.8, mode=mode, two_d=two_d)
    m0, t0, phi0, st0 = tg.tsallis_segment(hv.cuda(), p)
    m, t, phi, st = tg.tsallis_segment_host(hv, p)
    assert torch.equal(m, m0.cpu()) and torch.equal(t, t0.cpu())
    assert torch.equal(phi, phi0.cpu()) and torch.equal(st, st0.cpu())
