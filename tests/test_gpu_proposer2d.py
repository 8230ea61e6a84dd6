"""GPU tests of the 2-D search's proposer (slot 1) and its certified window
search: 2-D features against the oracle; the window search (params.topk > 0
with two_d) gives the exhaustive 2-D search's pair and value on every
histogram whatever the proposer says (random and all-zero weights), for
several q; with the trained weights, how often the candidate cells already
hold the maximiser and how many other cells are searched."""
import os

import numpy as np
import pytest
import torch

import phantom
import paper_2012_10684_gb300 as tg
from oracle import mlp
from test_gpu_2d import _rand_hist2d

pytestmark = pytest.mark.gpu

WEIGHTS2D = os.path.join(os.path.dirname(tg.__file__), "proposer2d_weights.bin")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield
    tg.proposer_select(0)


def _params(seed):
    rng = np.random.default_rng(seed)
    out = []
    for name, s in mlp.SHAPES:
        fan_in = s[-1] if len(s) == 2 else 256
        out.append(rng.normal(0, 1.0 / np.sqrt(fan_in), int(np.prod(s))))
    return np.concatenate(out).astype(np.float32)


def _hists(seed):
    v = phantom.generate_cuda(phantom.chest_volume(seed, nz=6))
    hs = tg.tsallis_histogram(v, tg.tsallis_params(mode="slice", two_d=True))
    hv = tg.tsallis_histogram(v, tg.tsallis_params(mode="volume", two_d=True))
    rng = np.random.default_rng(seed)
    extra = np.stack([_rand_hist2d(rng, 256, k) for k in ("diagonal", "sparse", "diagonal")]).astype(np.int32)
    special = np.zeros((4, 256, 256), np.int32)
    special[0, 40, 40] = 7                      # one cell: no pair
    special[1, 3, 3], special[1, 250, 250] = 5, 9
    special[2, 10:20, 10:20] = 1                # one block
    return torch.cat([hs, hv, torch.from_numpy(extra).cuda(), torch.from_numpy(special).cuda()])


def test_features2d_match_oracle():
    tg.proposer_select(1)
    h = _hists(11)
    x = tg.proposer_features(h).cpu().numpy()
    want = mlp.features2d(h.cpu().numpy())
    assert np.allclose(x, want, rtol=2e-6, atol=2e-7)
    # histograms 4 bytes past a 16-byte boundary take the 4-byte-load variant
    flat = torch.empty(h.numel() + 1, dtype=torch.int32, device=h.device)
    flat[1:] = h.reshape(-1)
    hu = flat[1:].view(h.shape)
    assert hu.data_ptr() % 16 == 4
    assert np.array_equal(tg.proposer_features(hu).cpu().numpy(), x)
    tg.proposer_select(0)


@pytest.mark.parametrize("q", [0.5, 0.8, 1.0, 1.5, 3.0])
@pytest.mark.parametrize("weights", ["random", "zero"])
def test_window2d_gives_the_exhaustive_result(q, weights):
    tg.proposer_select(1)
    tg.proposer_set(_params(21) if weights == "random" else np.zeros(mlp.NPARAM, np.float32))
    tg.proposer_select(0)
    h = _hists(12)
    t0, phi0, st0 = tg.tsallis_search(h, tg.tsallis_params(q=q, two_d=True))
    tk, phik, stk = tg.tsallis_search(h, tg.tsallis_params(q=q, two_d=True, topk=16))
    assert torch.equal(tk, t0), (q, weights)
    assert torch.equal(phik, phi0), (q, weights)
    assert torch.equal(stk & 0xff, st0 & 0xff)


def test_segment2d_with_window_equals_exhaustive():
    tg.proposer_select(1)
    tg.proposer_set(_params(22))
    tg.proposer_select(0)
    v = phantom.generate_cuda(phantom.chest_volume(13, 256, 256, 5))
    for mode in ("slice", "volume"):
        m0, t0, _, _ = tg.tsallis_segment(v, tg.tsallis_params(mode=mode, two_d=True))
        mk, tk, _, _ = tg.tsallis_segment(v, tg.tsallis_params(mode=mode, two_d=True, topk=8))
        assert torch.equal(t0, tk) and torch.equal(m0, mk)


def test_window2d_argument_rules():
    h = torch.zeros((1, 256, 256), dtype=torch.int32, device="cuda")
    tg.proposer_select(1)
    tg.proposer_set(_params(23))
    tg.proposer_select(0)
    with pytest.raises(tg.TsallisError):            # 128 grey levels
        tg.tsallis_search(torch.zeros((1, 128, 128), dtype=torch.int32, device="cuda"),
                          tg.tsallis_params(two_d=True, shift=5, topk=4))
    with pytest.raises(tg.TsallisError):            # with the brute-force search
        tg.tsallis_search(h, tg.tsallis_params(two_d=True, topk=4, flags=tg.TSALLIS_FLAG_BRUTE_FORCE_2D))
    with pytest.raises(tg.TsallisError):            # with a curve
        tg.tsallis_search(h, tg.tsallis_params(two_d=True, topk=4), curve=True)
    with pytest.raises(tg.TsallisError):
        tg.proposer_select(2)


@pytest.mark.skipif(not os.path.exists(WEIGHTS2D), reason="no trained 2-D weights in the package")
def test_trained_2d_proposer_narrows_the_search():
    """Held-out chest phantoms (seeds not used in training), per-slice 2-D
    histograms: the trained proposer's 16 cells hold the maximiser for most
    slices and fewer other cells need a search than with an uninformed
    proposer (all-zero weights: cells 0..15); both give the exhaustive pair."""
    v = phantom.generate_cuda(phantom.chest_volume(9090, nz=32, generations=6, noise_sd=12))
    h = tg.tsallis_histogram(v, tg.tsallis_params(mode="slice", two_d=True))
    t0, _, _ = tg.tsallis_search(h, tg.tsallis_params(two_d=True))
    res = {}
    for name in ("trained", "uninformed"):
        tg.proposer_select(1)
        if name == "trained":
            tg.proposer_load(WEIGHTS2D)
        else:
            tg.proposer_set(np.zeros(mlp.NPARAM, np.float32))
        tg.proposer_select(0)
        tk, _, stk = tg.tsallis_search(h, tg.tsallis_params(two_d=True, topk=16))
        assert torch.equal(tk, t0)
        stk = stk.cpu().numpy()
        res[name] = (float(((stk & tg.TSALLIS_STATUS_WINDOW_HIT) != 0).mean()),
                     float(((stk >> tg.TSALLIS_STATUS_FALLBACK_SHIFT) & 0xff).mean()))
    print("2-D window hit rate, mean cells searched beyond the candidates:", res)
    assert res["trained"][0] >= 0.5, res
    assert res["trained"][1] < res["uninformed"][1], res
