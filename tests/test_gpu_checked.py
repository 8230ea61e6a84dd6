"""The checked build (-DTSALLIS_CHECKED: the kernels test their computed
indices against buffer extents, skip and record a failing access) run over
small, odd and tile-crossing cases of every path, compared with the oracle:
no check may fail and every result must match. It stands in for a memory
sanitizer on GPUs where none may run. The checked library is built, then a
child process loads it (TSALLIS_CHECKED=1) and runs the cases."""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import oracle, phantom
import paper_2012_10684_gb300 as tg
from oracle import mlp
assert tg.library_path().endswith("_build_checked/libtsallis.so")
torch.cuda.set_device(0)
def no_fail(what):
    site = tg.check_status()
    assert site == 0, (what, site)
rng = np.random.default_rng(5)
# 1-D: per slice (tile kernel, table search), whole volume, odd shapes, batch
for shape in [(3, 37, 53), (2, 300, 301), (1, 512, 512), (5, 1, 9)]:
    v = rng.integers(-1500, 3200, shape).astype(np.int16)
    for mode in ("slice", "volume"):
        m, t, phi, st = tg.tsallis_segment(torch.from_numpy(v).cuda(), tg.tsallis_params(q=0.8, mode=mode))
        gv = shape[1] * shape[2] if mode == "slice" else v.size
        to, _, gap, mo = oracle.segment1d(v, gv, float(np.float32(0.8)))
        same = gap >= 1e-9
        assert np.array_equal(t.cpu().numpy()[same], to[same]), (shape, mode)
        no_fail(("segment", shape, mode))
vols = [torch.from_numpy(rng.integers(-1500, 3200, (int(rng.integers(1, 9)), 64, 72)).astype(np.int16)).cuda()
        for _ in range(5)]
masks, t, phi, st = tg.tsallis_segment_batch(vols, tg.tsallis_params(mode="volume"))
for v, m, tt in zip(vols, masks, t.cpu().numpy()):
    assert np.array_equal(m.cpu().numpy(), oracle.binarize(v.cpu().numpy(), int(tt)))
no_fail("batch")
# pre-processing: every radius class and op on odd shapes
for shape, r, op in [((2, 45, 150), 3, "chest_mask"), ((1, 77, 203), 10, "open"), ((3, 33, 129), 15, "close"),
                     ((1, 1, 1), 2, "erode"), ((2, 40, 3), 1, "dilate"), ((1, 64, 256), 0, "none")]:
    v = rng.integers(-2600, 3200, shape).astype(np.int16)
    o, h = tg.tsallis_preprocess(torch.from_numpy(v).cuda(), tg.preprocess_params(op=op, radius=r))
    oo, ho = oracle.preprocess(v, r=r, op={"none": "copy"}.get(op, op))
    assert np.array_equal(o.cpu().numpy(), oo) and np.array_equal(h.cpu().numpy(), ho), (shape, r, op)
    no_fail(("preprocess", shape, r, op))
# 2-D: summed-area search, brute force, window (random weights)
hs = np.zeros((3, 256, 256), np.int32)
for k in range(3):
    f = np.clip(rng.normal(90 + 40 * k, 20, 20000).astype(int), 0, 255)
    g = np.clip(f + rng.normal(0, 2, 20000).astype(int), 0, 255)
    np.add.at(hs[k], (f, g), 1)
h = torch.from_numpy(hs).cuda()
t0, _, _ = tg.tsallis_search(h, tg.tsallis_params(two_d=True))
for k in range(3):
    to, so, _, gap, _, _ = oracle.search2d(hs[k], float(np.float32(0.8)))
    if gap >= 1e-9:
        assert tuple(t0[k].tolist()) == (to, so)
no_fail("search2d")
tb, _, _ = tg.tsallis_search(h[:, :64, :64].contiguous(), tg.tsallis_params(two_d=True, nbins=64, shift=0,
                                                                            flags=tg.TSALLIS_FLAG_BRUTE_FORCE_2D))
no_fail("brute")
tg.proposer_select(1)
tg.proposer_set(np.random.default_rng(1).normal(0, 0.05, mlp.NPARAM).astype(np.float32))
tg.proposer_select(0)
tw, _, _ = tg.tsallis_search(h, tg.tsallis_params(two_d=True, topk=8))
assert torch.equal(tw, t0)
no_fail("window2d")
v = phantom.generate_cuda(phantom.chest_volume(3, 128, 96, 5))
m2, t2, _, _ = tg.tsallis_segment(v, tg.tsallis_params(two_d=True, mode="slice"))
no_fail("segment2d")
print("checked ok")
'''


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def test_checked_build_passes_every_check():
    from paper_2012_10684_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, TSALLIS_CHECKED="1", PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_normal_build_has_no_checks():
    import paper_2012_10684_gb300 as tg
    if os.environ.get("TSALLIS_CHECKED") == "1":
        pytest.skip("this process loaded the checked build")
    with pytest.raises(tg.TsallisError):
        tg.check_status()
