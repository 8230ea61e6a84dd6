"""GPU tests of the learned threshold proposer and of the window search.

Against the FP64 oracle (oracle/mlp.py, with the same bfloat16-rounded
matrices the GPU multiplies with): features, logits, gradients, one Adam
step. The window search (params.topk > 0) must give the exhaustive search's
threshold on every histogram, whatever the proposer says (random weights
included): 0 misses after fallback. With the trained weights, a test shows
what the proposer gains: how often its window already holds the maximiser
and how many 64-level blocks still need an exhaustive search, against the
same search with an uninformed proposer."""
import os

import numpy as np
import pytest
import torch

import oracle
import phantom
import paper_2012_10684_gb300 as tg
from oracle import mlp
from paper_2012_10684_gb300 import proposer as P
from test_gpu_1d import check_thresholds, f32

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(tg.__file__), "proposer_weights.bin")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for name, s in mlp.SHAPES:
        fan_in = s[-1] if len(s) == 2 else 256
        out.append(rng.normal(0, scale / np.sqrt(fan_in), int(np.prod(s))))
    return np.concatenate(out).astype(np.float32)


def _as_used(params):
    """The parameters as the GPU uses them: matrices rounded to bfloat16,
    biases as stored (float32), in FP64."""
    d = mlp.unpack(np.asarray(params, np.float64))
    return mlp.pack({k: (mlp.bf16_round(v) if k.startswith("W") else v) for k, v in d.items()})


def _histograms(seed, n):
    rng = np.random.default_rng(seed)
    h = np.zeros((n, 4096), np.int32)
    for i in range(n):
        k = rng.integers(2, 600)
        lv = rng.choice(4096, k, replace=False)
        h[i, lv] = rng.integers(1, 5000, k)
    return h


def test_features_match_oracle():
    v = phantom.generate_host(phantom.chest_volume(41, nz=20))
    hp = tg.tsallis_histogram(torch.from_numpy(v).cuda(), tg.tsallis_params(mode="slice"))
    h = torch.cat([hp, torch.from_numpy(_histograms(1, 30)).cuda(), torch.zeros((1, 4096), dtype=torch.int32,
                                                                                device="cuda")])
    x = tg.proposer_features(h).cpu().numpy()
    xo = mlp.features(h.cpu().numpy())
    assert np.allclose(x, xo, rtol=2e-6, atol=2e-7)


def test_forward_matches_oracle():
    params = _params(2)
    tg.proposer_set(params)
    x = np.random.default_rng(3).random((37, 256)).astype(np.float32)
    z = tg.proposer_forward(torch.from_numpy(x).cuda()).cpu().numpy()
    zo, _ = mlp.forward(_as_used(params), x)
    assert np.max(np.abs(z - zo)) <= 1e-4 * (1 + np.max(np.abs(zo)))


@pytest.mark.parametrize("B", [1, 16, 17, 64, 65, 300])
def test_forward_both_paths_match_oracle(B):
    """Up to 64 rows the fused tensor-core inference kernel, above them the
    tiled tensor-core GEMMs: both within the forward tolerance of the FP64
    oracle (bfloat16 weights as used)."""
    params = _params(21)
    tg.proposer_set(params)
    x = np.random.default_rng(B).random((B, 256)).astype(np.float32)
    z = tg.proposer_forward(torch.from_numpy(x).cuda()).cpu().numpy()
    zo, _ = mlp.forward(_as_used(params), x)
    assert np.max(np.abs(z - zo)) <= 1e-4 * (1 + np.max(np.abs(zo))), B


def test_gradients_match_oracle():
    params = _params(4)
    tg.proposer_set(params)
    rng = np.random.default_rng(5)
    B = 6
    x = rng.random((B, 256)).astype(np.float32)
    h = _histograms(6, B)
    t = np.array([int(np.flatnonzero(h[i])[len(np.flatnonzero(h[i])) // 2]) for i in range(B)])
    y = mlp.targets(h, t).astype(np.float32)
    loss, g = tg.proposer_train_step(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), update=False,
                                     want_grad=True)
    lo, go = mlp.grads(_as_used(params), x, y)
    assert float(loss[0]) == pytest.approx(lo, rel=1e-5)
    g = g.cpu().numpy()
    o = 0
    for name, s in mlp.SHAPES:
        n = int(np.prod(s))
        a, b = g[o:o + n], go[o:o + n]
        assert np.max(np.abs(a - b)) <= 2e-3 * np.max(np.abs(b)) + 1e-8, name
        o += n


def test_adam_step_matches_oracle():
    params = _params(7)
    tg.proposer_set(params)
    rng = np.random.default_rng(8)
    x = torch.from_numpy(rng.random((4, 256)).astype(np.float32)).cuda()
    y = torch.zeros((4, 4096), device="cuda")
    y[:, 1000] = 1
    _, g = tg.proposer_train_step(x, y, lr=1e-3, update=True, want_grad=True)
    p1 = tg.proposer_get()
    po, _, _ = mlp.adam_step(params.astype(np.float64), g.cpu().numpy().astype(np.float64),
                             np.zeros(mlp.NPARAM), np.zeros(mlp.NPARAM), 1, 1e-3)
    assert np.allclose(p1, po, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("k", [1, 2, 16, 64, 65, 256])
def test_topk_matches_a_sort(k):
    """Both top-k kernels (warp rounds for k <= 64, bitonic sort above)
    against a stable numpy sort: descending value, equal values by smaller
    index; rows with many exact ties and with negative values included."""
    rng = np.random.default_rng(k)
    z = rng.normal(0, 1, (6, 4096)).astype(np.float32)
    z[1] = np.round(z[1] * 2) / 2 + np.float32(0.0)   # many exact ties (no negative zeros)
    z[2] = -np.abs(z[2])                              # all negative
    z[3] = 0.0                                        # all equal
    z[4, ::7] = 5.0                                   # a tied top group
    got = tg.probe_topk(torch.from_numpy(z).cuda(), k).cpu().numpy()
    for r in range(z.shape[0]):
        order = np.lexsort((np.arange(4096), -z[r].astype(np.float64)))
        assert np.array_equal(got[r], order[:k]), (k, r)


def test_save_load_round_trip(tmp_path):
    params = _params(9)
    tg.proposer_set(params)
    f = str(tmp_path / "w.bin")
    tg.proposer_save(f)
    tg.proposer_set(np.zeros_like(params))
    tg.proposer_load(f)
    assert np.array_equal(tg.proposer_get(), params)


def test_checkpoint_resume_is_bit_exact(tmp_path):
    """An interrupted run (stopped after 7 of 20 steps, checkpoint every 7)
    resumed from its checkpoint ends with the same parameters, bit for bit,
    as the uninterrupted run; a damaged checkpoint is refused and leaves the
    context as it was. (The loss is summed over rows with atomics, so only
    its value, not its last bits, is compared.)"""
    rng = np.random.default_rng(14)
    h = torch.from_numpy(_histograms(15, 64)).cuda()
    t = torch.tensor([int(np.flatnonzero(r)[len(np.flatnonzero(r)) // 3]) for r in h.cpu().numpy()],
                     dtype=torch.int32, device="cuda")
    x, y = tg.proposer_features(h), P.soft_targets(h, t)
    kw = dict(steps=20, batch=16, lr=2e-3, seed=int(rng.integers(1 << 30)))
    full = P.train(x, y, **kw)
    p_full = tg.proposer_get()
    ck = str(tmp_path / "c.ckpt")
    part = P.train(x, y, checkpoint=ck, checkpoint_every=7, stop_after=8, **kw)
    assert np.isnan(part[8:]).all() and np.allclose(part[:8], full[:8], rtol=1e-5)
    tg.proposer_set(_params(16))                     # another run's weights in between
    rest = P.train(x, y, resume=ck, **kw)
    assert np.isnan(rest[:7]).all() and np.allclose(rest[7:], full[7:], rtol=1e-5)
    assert np.array_equal(tg.proposer_get(), p_full)
    raw = bytearray(open(ck, "rb").read())
    raw[100] ^= 1
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(RuntimeError):
        tg.proposer_checkpoint_load(bad)
    assert np.array_equal(tg.proposer_get(), p_full)


def test_training_reduces_the_loss():
    v = torch.from_numpy(phantom.generate_host(phantom.chest_volume(43, nz=64))).cuda()
    p = tg.tsallis_params(q=0.8, mode="slice")
    h = tg.tsallis_histogram(v, p)
    t, _, _ = tg.tsallis_search(h, p)
    x, y = tg.proposer_features(h), P.soft_targets(h, t)
    losses = P.train(x, y, steps=300, batch=32, lr=2e-3, seed=1)
    assert losses[-20:].mean() < 0.5 * losses[:5].mean(), (losses[:5], losses[-20:])


def _window_vs_exhaustive(h, q, k=64):
    p0 = tg.tsallis_params(q=q)
    pk = tg.tsallis_params(q=q, topk=k)
    t0, phi0, st0 = tg.tsallis_search(h, p0)
    tk, phik, stk = tg.tsallis_search(h, pk)
    return (t0.cpu().numpy(), phi0.cpu().numpy(), st0.cpu().numpy(), tk.cpu().numpy(), phik.cpu().numpy(),
            stk.cpu().numpy())


@pytest.mark.parametrize("q", [0.5, 0.8, 1.0, 1.5, 3.0])
@pytest.mark.parametrize("weights", ["random", "zero"])
def test_window_search_gives_the_exhaustive_result(q, weights):
    tg.proposer_set(_params(10) if weights == "random" else np.zeros(mlp.NPARAM, np.float32))
    v = phantom.generate_host(phantom.chest_volume(45, nz=48))
    hv = tg.tsallis_histogram(torch.from_numpy(v).cuda(), tg.tsallis_params(mode="slice"))
    h = torch.cat([hv, torch.from_numpy(_histograms(11, 40)).cuda()])
    special = np.zeros((4, 4096), np.int32)
    special[0, 7] = 10                          # one level: no threshold
    special[1, [0, 4095]] = [3, 4]              # two levels far apart
    special[2, 100:164] = 5                     # one full block
    special[3, ::2] = 1                         # every other level
    h = torch.cat([h, torch.from_numpy(special).cuda()])
    t0, phi0, st0, tk, phik, stk = _window_vs_exhaustive(h, q)
    hh = h.cpu().numpy()
    t_o, phi_o, gap_o = [], [], []
    for i in range(hh.shape[0]):
        a, b, c, _, _ = oracle.search1d(hh[i], f32(q))
        t_o.append(a); phi_o.append(b); gap_o.append(c)
    check_thresholds(tk, phik, stk & 0xff, t_o, phi_o, gap_o, ("window", q, weights))
    same = np.array(gap_o) >= 1e-9
    assert np.array_equal(tk[same], t0[same])


def test_batch_with_window_equals_exhaustive_masks():
    tg.proposer_set(_params(12))
    rng = np.random.default_rng(13)
    vols = [torch.from_numpy(phantom.generate_host(phantom.chest_volume(50 + i, 160, 128, int(rng.integers(3, 20)),
                                                                        vol_id=i))).cuda() for i in range(5)]
    for mode in ("volume", "slice"):
        m0, t0, _, _ = tg.tsallis_segment_batch(vols, tg.tsallis_params(q=0.8, mode=mode))
        mk, tk, _, stk = tg.tsallis_segment_batch(vols, tg.tsallis_params(q=0.8, mode=mode, topk=64))
        assert torch.equal(t0, tk)
        for a, b in zip(m0, mk):
            assert torch.equal(a, b)


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained weights in the package")
def test_trained_proposer_narrows_the_search():
    """Held-out 512x512 chest phantoms of the batch distribution (seeds not
    used in training): with the trained weights the top-64 window holds the
    exact threshold for most volumes and few blocks need an exhaustive
    search; with an uninformed proposer (all weights zero: the window is
    levels 0..63) the window never holds it and many blocks are searched.
    Both give the exhaustive result."""
    specs = phantom.batch_specs(777, nvol=24, dmin=120, dmax=600)
    p = tg.tsallis_params(q=0.8, mode="volume")
    h = torch.cat([tg.tsallis_histogram(phantom.generate_cuda(s), p) for s in specs])
    res = {}
    for name in ("trained", "uninformed"):
        if name == "trained":
            tg.proposer_load(WEIGHTS)
        else:
            tg.proposer_set(np.zeros(mlp.NPARAM, np.float32))
        t0, _, _, tk, _, stk = _window_vs_exhaustive(h, 0.8)
        assert np.array_equal(t0, tk)
        res[name] = (float(((stk & tg.TSALLIS_STATUS_WINDOW_HIT) != 0).mean()),
                     float(((stk >> tg.TSALLIS_STATUS_FALLBACK_SHIFT) & 0xff).mean()))
    print("window hit rate, mean blocks searched:", res)
    assert res["trained"][0] >= 0.75, res
    assert res["uninformed"][0] == 0.0
    assert res["trained"][1] < res["uninformed"][1], res


def test_training_labels_are_the_oracles():
    """The proposer's training data: 64 generated volumes (64 x 64 x D, D in
    [8, 40], the training generator's noise and airway ranges), labelled on
    the GPU by make_dataset. Each whole-volume histogram must equal the
    oracle's histogram of the same volume generated on the host, and each
    label the oracle's threshold of that histogram (oracle.search1d), except
    where the oracle's top-two gap between partitions is below 1e-9."""
    from paper_2012_10684_gb300 import proposer
    seed, n, dmin, dmax, nx = 7, 64, 8, 40, 64
    hist, _, t, st = proposer.make_dataset(n, seed, dmin, dmax, nx=nx, ny=nx)
    hist, t, st = hist.cpu().numpy(), t.cpu().numpy(), st.cpu().numpy()
    rng = np.random.default_rng(seed)
    checked = 0
    for i in range(n):
        # the generator's draws, in make_dataset's order
        nz = int(rng.integers(dmin, dmax + 1))
        spec = phantom.chest_volume(seed * 100000 + i, nx, nx, nz, generations=int(rng.integers(4, 9)),
                                    noise_sd=int(rng.integers(5, 31)), vol_id=i)
        h_o = oracle.hist1d(phantom.generate_host(spec))
        assert np.array_equal(hist[i], h_o), i
        t_o, best, gap, _, _ = oracle.search1d(h_o, float(np.float32(0.8)))
        if t_o < 0:
            assert t[i] == -1, i
            continue
        assert (st[i] & 0xff) == 0, i
        if gap >= 1e-9:
            assert t[i] == t_o, (i, t[i], t_o, gap)
            checked += 1
    assert checked >= 60
