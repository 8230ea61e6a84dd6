"""GPU parity of the 2-D path (grey level x 3x3(x3) floor-mean level,
section II-C) against the CPU oracle, through the C ABI.

Rules (written here so a reader sees them):
  * 2-D histograms and masks: bit-exact;
  * the pair (t, s): equal to the oracle's unless the oracle's relative gap
    between its best and second-best distinct partitions (distinct quadrant
    count pairs) is below 1e-9; when t differs the mask must equal
    Algorithm 1 at the GPU's t;
  * objective values (maximum and the whole phi(t, s) surface):
    |phi_gpu - phi_oracle| <= 1e-5 * max(|phi_oracle|, 1).
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
    """The Tsallis index as the C ABI receives it (a float)."""
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


def _oracle_hists(v, mode, lo=-1024, L=4096, shift=4):
    """Per slice (3x3 window) or whole volume (3x3x3 when nz > 1)."""
    if mode == "slice":
        return np.stack([oracle.hist2d(v[z:z + 1], lo, L, shift) for z in range(v.shape[0])])
    return oracle.hist2d(v, lo, L, shift)[None]


# ------------------------------------------------------------ histogram

def _mixed_volume(rng, shape):
    """Random values (most neighbourhoods far off the diagonal band) mixed
    with flat runs (on the band) and the int16 extremes."""
    v = rng.integers(-1500, 3500, shape).astype(np.int16)
    flat = v.reshape(-1)
    k = flat.size
    flat[: k // 3] = -1024
    flat[k // 3: k // 3 + k // 20] = -32768
    flat[k // 2: k // 2 + k // 20] = 32767
    blocks = v.reshape(shape)
    blocks[:, : shape[1] // 2, : shape[2] // 2] = 40      # a flat quadrant
    return v


@pytest.mark.parametrize("shape", [(1, 37, 53), (5, 64, 128), (3, 130, 522), (7, 20, 8), (2, 1, 1), (4, 3, 5),
                                   (1, 512, 512), (2, 65, 516)])
@pytest.mark.parametrize("mode", ["slice", "volume"])
def test_hist2d_bit_exact(shape, mode):
    rng = np.random.default_rng(sum(shape) + (mode == "volume"))
    v = _mixed_volume(rng, shape)
    p = tg.tsallis_params(mode=mode, two_d=True)
    h = tg.tsallis_histogram(_cuda(v), p).cpu().numpy()
    ref = _oracle_hists(v, mode)
    assert h.shape == ref.shape
    assert np.array_equal(h, ref)


@pytest.mark.parametrize("mode", ["slice", "volume"])
def test_hist2d_rejects_a_volume_off_its_16_byte_boundary(mode):
    """The 2-D histogram, like every entry point, takes only 16-byte aligned
    volumes (its staged and 8-byte load paths rely on it); rows of a length
    that is not a multiple of 4 voxels take the per-element path instead,
    which the ragged shapes above cover."""
    flat = torch.zeros(3 * 40 * 132 + 8, dtype=torch.int16, device="cuda")
    dv = flat[1:1 + 3 * 40 * 132].view(3, 40, 132)
    with pytest.raises(tg.TsallisError) as e:
        tg.tsallis_histogram(dv, tg.tsallis_params(mode=mode, two_d=True))
    assert e.value.code == tg.TSALLIS_ERR_ALIGNMENT


@pytest.mark.parametrize("lo,L,shift", [(-1000, 1024, 2), (-1024, 512, 4), (32000, 4096, 4), (-32768, 4096, 8),
                                        (0, 2, 0), (-1024, 4096, 5)])
def test_hist2d_level_ranges(lo, L, shift):
    rng = np.random.default_rng(L + shift)
    v = _mixed_volume(rng, (3, 40, 44))
    for mode in ("slice", "volume"):
        p = tg.tsallis_params(mode=mode, two_d=True, lo=lo, nbins=L, shift=shift)
        h = tg.tsallis_histogram(_cuda(v), p).cpu().numpy()
        assert np.array_equal(h, _oracle_hists(v, mode, lo, L, shift)), mode


def test_hist2d_phantom_volume():
    v = phantom.generate_host(phantom.chest_volume(2012106850, nx=256, ny=192, nz=24))
    for mode in ("slice", "volume"):
        p = tg.tsallis_params(mode=mode, two_d=True)
        h = tg.tsallis_histogram(_cuda(v), p).cpu().numpy()
        assert np.array_equal(h, _oracle_hists(v, mode)), mode


def test_two_d_params_rejected_when_grey_levels_do_not_fill_L2():
    v = torch.zeros((2, 8, 8), dtype=torch.int16, device="cuda")
    with pytest.raises(RuntimeError):
        tg.tsallis_histogram(v, tg.tsallis_params(two_d=True, nbins=4001, shift=4))
    with pytest.raises(RuntimeError):
        tg.tsallis_histogram(v, tg.tsallis_params(two_d=True, nbins=4096, shift=3))   # 512 grey levels


# ------------------------------------------------------------ search

def _rand_hist2d(rng, L, kind):
    if kind == "dense":
        return rng.integers(0, 1000, (L, L)).astype(np.int32)
    if kind == "sparse":
        h = rng.integers(0, 5000, (L, L)).astype(np.int32)
        h[rng.random((L, L)) < 0.9] = 0
        return h
    # near the diagonal, like an image's grey x mean histogram
    h = np.zeros((L, L), np.int32)
    for _ in range(3):
        c = rng.integers(0, L)
        w = max(1, L // 10)
        n = rng.integers(10_000, 2_000_000)
        f = np.clip(rng.normal(c, w, n).astype(int), 0, L - 1)
        g = np.clip(f + rng.normal(0, 1.5, n).astype(int), 0, L - 1)
        np.add.at(h, (f, g), 1)
    return h


def _check_pairs(t_g, phi_g, st_g, hs, q, ctx=""):
    for i, h in enumerate(hs):
        t, s, best, gap, phi, valid = oracle.search2d(h, f32(q))
        if t < 0:
            assert tuple(t_g[i]) == (-1, -1) and (st_g[i] & 0xff) == tg.TSALLIS_ERR_NO_VALID_THRESHOLD, (ctx, i)
            continue
        assert (st_g[i] & 0xff) == 0, (ctx, i, st_g[i])
        if gap >= GAP:
            assert tuple(t_g[i]) == (t, s), (ctx, i, tuple(t_g[i]), (t, s), gap)
        assert abs(phi_g[i] - best) <= PHI_RTOL * max(abs(best), 1.0), (ctx, i, phi_g[i], best)


@pytest.mark.parametrize("q", [0.5, 0.8, 1.0, 1.5, 2.5])
@pytest.mark.parametrize("L", [2, 3, 16, 33, 256])
@pytest.mark.parametrize("kind", ["dense", "sparse", "diagonal"])
def test_search2d_random_histograms(q, L, kind):
    rng = np.random.default_rng(L * 31 + int(q * 10) + len(kind))
    hs = np.stack([_rand_hist2d(rng, L, kind) for _ in range(3)])
    # the C ABI expresses L2 as nbins >> shift
    p = tg.tsallis_params(q=q, two_d=True, nbins=L, shift=0)
    t, phi, st, curve = tg.tsallis_search(_cuda(hs), p, curve=True)
    t, phi, st, curve = (x.cpu().numpy() for x in (t, phi, st, curve))
    _check_pairs(t, phi, st, hs, q, (q, L, kind))
    for i, h in enumerate(hs):
        ref, valid = oracle.objective2d(h, f32(q))
        assert np.array_equal(~np.isnan(curve[i]), valid), i
        d = np.abs(curve[i][valid] - ref[valid])
        assert np.all(d <= PHI_RTOL * np.maximum(np.abs(ref[valid]), 1.0)), (i, d.max())


def test_search2d_degenerate_and_many_histograms():
    L = 8
    hs = np.zeros((70, L, L), np.int32)        # more than one launch chunk
    hs[0, 3, 3] = 100                          # one bin: no pair splits it
    hs[1] = 0                                  # empty
    hs[2, 0, 0] = 5; hs[2, 7, 7] = 5           # two bins on opposite corners
    hs[3, 0, 7] = 9; hs[3, 7, 0] = 9           # mass only in the ignored quadrants
    rng = np.random.default_rng(7)
    for k in range(4, 70):
        hs[k] = _rand_hist2d(rng, L, "sparse" if k % 2 else "dense")
    p = tg.tsallis_params(q=0.8, two_d=True, nbins=L, shift=0)
    t, phi, st = tg.tsallis_search(_cuda(hs), p)
    _check_pairs(t.cpu().numpy(), phi.cpu().numpy(), st.cpu().numpy(), hs, 0.8, "degenerate")


def test_search2d_phantom_histograms():
    v = phantom.generate_host(phantom.chest_volume(2012106851, nz=6))
    hs = _oracle_hists(v, "slice").astype(np.int32)
    for q in (0.5, 0.8, 1.5):
        p = tg.tsallis_params(q=q, two_d=True)
        t, phi, st = tg.tsallis_search(_cuda(hs), p)
        _check_pairs(t.cpu().numpy(), phi.cpu().numpy(), st.cpu().numpy(), hs, q, q)


# ------------------------------------------------------------ binarise and the whole step

@pytest.mark.parametrize("polarity", ["low", "high"])
def test_binarize2d_uses_t_on_grey_levels(polarity):
    rng = np.random.default_rng(11)
    v = _mixed_volume(rng, (4, 33, 70))
    pairs = np.array([[3, 200], [120, 5], [-1, -1], [254, 254]], np.int32)
    p = tg.tsallis_params(mode="slice", two_d=True, polarity=polarity)
    m = tg.tsallis_binarize(_cuda(v), _cuda(pairs), p).cpu().numpy()
    pol = 1 if polarity == "high" else 0
    for z in range(4):
        assert np.array_equal(m[z], oracle.binarize(v[z], int(pairs[z, 0]), shift=4, polarity=pol)), z


def _check_segment2d(v, mode, q, polarity="low"):
    p = tg.tsallis_params(q=q, mode=mode, two_d=True, polarity=polarity)
    mask, t, phi, st = (x.cpu().numpy() for x in tg.tsallis_segment(_cuda(v), p))
    hs = _oracle_hists(v, mode)
    _check_pairs(t, phi, st, hs, q, (mode, q))
    pol = 1 if polarity == "high" else 0
    groups = [v[z] for z in range(v.shape[0])] if mode == "slice" else [v]
    masks = [mask[z] for z in range(v.shape[0])] if mode == "slice" else [mask]
    for i, (g, m) in enumerate(zip(groups, masks)):
        assert np.array_equal(m, oracle.binarize(g, int(t[i, 0]), shift=4, polarity=pol)), i


@pytest.mark.parametrize("mode", ["slice", "volume"])
@pytest.mark.parametrize("q", [0.8, 1.0])
def test_segment2d_phantom(mode, q):
    v = phantom.generate_host(phantom.chest_volume(2012106852, nz=12))
    _check_segment2d(v, mode, q)


@pytest.mark.parametrize("shape", [(5, 37, 29), (3, 130, 522), (1, 7, 3), (2, 1, 1)])
def test_segment2d_ragged_shapes(shape):
    rng = np.random.default_rng(sum(shape))
    v = _mixed_volume(rng, shape)
    for mode in ("slice", "volume"):
        _check_segment2d(v, mode, 0.8, polarity="high")


def test_segment2d_chest_full_size():
    """The 2-D workload itself: 512 x 512 x 256, whole volume, 3x3x3 mean, q = 0.8."""
    v = phantom.generate_host(phantom.chest_volume(2012106842, nz=256))
    _check_segment2d(v, "volume", 0.8)


# ------------------------------------------------------------ brute-force search (one thread per pair)

def _check_pairs_brute(t_g, phi_g, st_g, hs, q, ctx=""):
    """The brute-force search is held to the same rule as the default one:
    the oracle's (t, s) wherever its gap to the next partition is 1e-9 or
    more, phi within PHI_RTOL."""
    _check_pairs(t_g, phi_g, st_g, hs, q, ctx)


@pytest.mark.parametrize("q", [0.5, 0.8, 1.0, 1.5, 2.5])
@pytest.mark.parametrize("L", [2, 3, 16, 33, 256])
@pytest.mark.parametrize("kind", ["dense", "sparse", "diagonal"])
def test_brute_force_search_matches_oracle(q, L, kind):
    rng = np.random.default_rng(L * 37 + int(q * 10) + len(kind))
    hs = np.stack([_rand_hist2d(rng, L, kind) for _ in range(2)])
    p = tg.tsallis_params(q=q, two_d=True, nbins=L, shift=0, flags=tg.TSALLIS_FLAG_BRUTE_FORCE_2D)
    t, phi, st, curve = (x.cpu().numpy() for x in tg.tsallis_search(_cuda(hs), p, curve=True))
    _check_pairs_brute(t, phi, st, hs, q, (q, L, kind))
    for i, h in enumerate(hs):
        ref, valid = oracle.objective2d(h, f32(q))
        assert np.array_equal(~np.isnan(curve[i]), valid), i
        d = np.abs(curve[i][valid] - ref[valid])
        assert np.all(d <= PHI_RTOL * np.maximum(np.abs(ref[valid]), 1.0)), (i, d.max())


def test_brute_force_degenerate_many_and_plateaus():
    """More histograms than one launch chunk, empty and one-bin histograms,
    and empty rows/columns (plateaus: the smallest (t, s) of a partition)."""
    L = 12
    hs = np.zeros((67, L, L), np.int32)
    hs[0, 3, 3] = 100
    hs[2, 0, 0] = 5; hs[2, 11, 11] = 5
    hs[3, 0, 11] = 9; hs[3, 11, 0] = 9
    rng = np.random.default_rng(17)
    for k in range(4, 67):
        h = _rand_hist2d(rng, L, "dense")
        h[rng.integers(0, L, 3), :] = 0              # empty grey rows
        h[:, rng.integers(0, L, 3)] = 0              # empty mean columns
        hs[k] = h
    for q in (0.8, 1.0, 2.0):
        p = tg.tsallis_params(q=q, two_d=True, nbins=L, shift=0, flags=tg.TSALLIS_FLAG_BRUTE_FORCE_2D)
        t, phi, st = (x.cpu().numpy() for x in tg.tsallis_search(_cuda(hs), p))
        _check_pairs_brute(t, phi, st, hs, q, ("plateau", q))


def test_brute_force_agrees_with_summed_area_search_on_phantoms():
    v = phantom.generate_host(phantom.chest_volume(2012106852, nz=4))
    hs = _cuda(_oracle_hists(v, "slice").astype(np.int32))
    for q in (0.5, 0.8, 1.5):
        p0 = tg.tsallis_params(q=q, two_d=True)
        pb = tg.tsallis_params(q=q, two_d=True, flags=tg.TSALLIS_FLAG_BRUTE_FORCE_2D)
        t0, phi0, _ = tg.tsallis_search(hs, p0)
        tb, phib, stb = tg.tsallis_search(hs, pb)
        _check_pairs_brute(tb.cpu().numpy(), phib.cpu().numpy(), stb.cpu().numpy(), hs.cpu().numpy(), q, q)
        assert torch.allclose(phib, phi0, rtol=1e-5, atol=1e-5)
        # the whole 2-D step with the brute-force search: its thresholds,
        # and each slice's mask against Algorithm 1 at them
        vol = _cuda(v)
        mb, tb2, _, _ = tg.tsallis_segment(vol, pb)
        assert torch.equal(tb2, tb)
        mb = mb.cpu().numpy()
        for z in range(v.shape[0]):
            assert np.array_equal(mb[z], oracle.binarize(v[z], int(tb2[z, 0]), shift=4)), (q, z)


def test_brute_force_flag_needs_two_d():
    h = torch.zeros((1, 4096), dtype=torch.int32, device="cuda")
    with pytest.raises(tg.TsallisError):
        tg.tsallis_search(h, tg.tsallis_params(flags=tg.TSALLIS_FLAG_BRUTE_FORCE_2D))
