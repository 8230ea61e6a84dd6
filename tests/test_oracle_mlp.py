"""Pins of the FP64 proposer oracle (oracle/mlp.py) against values fixed
independently of it: the normal distribution function, closed forms of the
cross-entropy and of Adam's first step, central finite differences of the
loss, hand-built feature and target examples, and torch's bfloat16 rounding.
CPU only."""
import numpy as np
import pytest
import torch

from oracle import mlp


def test_gelu_is_z_times_normal_cdf():
    # Phi(1) = 0.841344746068542948585232545632 (normal table)
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)
    assert mlp.gelu(np.array([-1.0]))[0] == pytest.approx(-0.15865525393145705, rel=1e-14)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([40.0]))[0] == 40.0
    z = np.linspace(-6, 6, 101)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def test_features_hand_example():
    h = np.zeros((2, 4096))
    h[0, 0:16] = 1                      # group 0 holds all 16 counts
    h[1, 4080:4096] = 2                 # last group holds 32
    h[1, 17] = 32                       # group 1 holds 32
    x = mlp.features(h)
    assert x.shape == (2, 256)
    assert x[0, 0] == pytest.approx(1.0) and np.all(x[0, 1:] == 0)
    assert x[1, 1] == pytest.approx(np.log(33) / np.log(65))
    assert x[1, 255] == pytest.approx(np.log(33) / np.log(65))
    assert np.count_nonzero(x[1]) == 2


def test_cross_entropy_closed_forms():
    rng = np.random.default_rng(0)
    y = rng.random((3, 4096))
    y /= y.sum(axis=1, keepdims=True)
    assert mlp.loss(np.zeros((3, 4096)), y) == pytest.approx(np.log(4096), rel=1e-14)
    z = rng.normal(size=(1, 4096))
    onehot = np.zeros((1, 4096))
    onehot[0, 77] = 1
    lse = np.log(np.exp(z[0]).sum())
    assert mlp.loss(z, onehot) == pytest.approx(lse - z[0, 77], rel=1e-13)


def _small_params(rng, scale=0.3):
    return rng.normal(0, scale, mlp.NPARAM) * np.concatenate(
        [np.full(int(np.prod(s)), 1.0 / np.sqrt(s[-1] if len(s) == 2 else 1.0)) for _, s in mlp.SHAPES])


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    params = _small_params(rng)
    x = rng.random((3, 256))
    y = np.zeros((3, 4096))
    y[0, 100:104] = 0.25
    y[1, 2000] = 1.0
    y[2, 4094] = 1.0
    _, g = mlp.grads(params, x, y)
    # coordinates from every parameter block
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    idx = np.concatenate([rng.integers(offs[i], offs[i + 1], 40) for i in range(len(mlp.SHAPES))])
    idx = np.concatenate([idx, [offs[4] + 2000 * 256 + 3, offs[5] + 2000, offs[5] + 100]])
    eps = 1e-4          # truncation error O(eps^2) stays below the rounding error of smaller steps
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (mlp.loss(mlp.forward(pp, x)[0], y) - mlp.loss(mlp.forward(pm, x)[0], y)) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=2e-10), i   # abs: loss rounding / 2 eps


def test_targets_cover_the_equivalent_thresholds():
    h = np.zeros((3, 4096), np.int64)
    h[0, [3, 10, 15, 300]] = 5           # t* = 10: levels 11..14 are empty
    h[1, [0, 4095]] = 1                  # t* = 0: levels 1..4094 are empty
    h[2, 7] = 9                          # no valid threshold
    y = mlp.targets(h, [10, 0, -1])
    assert np.allclose(y[0, 10:15], 0.2) and y[0].sum() == pytest.approx(1.0) and y[0, 15] == 0
    assert np.allclose(y[1, 0:4095], 1 / 4095) and y[1, 4095] == 0
    assert not y[2].any()


def test_adam_first_step_is_signed_learning_rate():
    rng = np.random.default_rng(2)
    p = rng.normal(size=1000)
    g = rng.normal(size=1000)
    p1, m, v = mlp.adam_step(p, g, np.zeros(1000), np.zeros(1000), 1, 0.01)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0]]).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(a), ref)


def test_pack_unpack_round_trip():
    rng = np.random.default_rng(4)
    flat = rng.normal(size=mlp.NPARAM)
    assert np.array_equal(mlp.pack(mlp.unpack(flat)), flat)
    assert mlp.NPARAM == 256 * 256 + 256 + 256 * 256 + 256 + 4096 * 256 + 4096


def test_features2d_hand_examples():
    """Block sums worked by hand: one cell (37, 200) lies in grey block 2 and
    mean block 12 (feature 44); two cells of block 0 add up; cells in the
    first and last blocks give log(2)/log(5) and log(4)/log(5)."""
    h = np.zeros((3, 256, 256), np.int64)
    h[0, 37, 200] = 9
    h[1, 0, 0], h[1, 15, 15] = 3, 4
    h[2, 0, 0], h[2, 255, 255] = 1, 3
    x = mlp.features2d(h)
    e0 = np.zeros(256); e0[44] = 1.0
    assert np.allclose(x[0], e0)
    e1 = np.zeros(256); e1[0] = 1.0
    assert np.allclose(x[1], e1)
    e2 = np.zeros(256); e2[0] = np.log(2) / np.log(5); e2[255] = np.log(4) / np.log(5)
    assert np.allclose(x[2], e2)
    assert not mlp.features2d(np.zeros((1, 256, 256))).any()
    assert mlp.cell2d(37, 200) == 64 * 9 + 50 and mlp.cell2d(254, 254) == 4095
