"""CPU-side checks of the C-ABI library: it builds, loads, exports every
function include/tsallis.h declares, and rejects bad arguments on the host
before touching the GPU. No kernel runs here."""
import ctypes
import glob
import os
import re

import pytest

import paper_2012_10684_gb300 as tg
from paper_2012_10684_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return tg.lib()


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith("tsallis_"):
                names.add(name)
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("tsallis_histogram", "tsallis_search", "tsallis_binarize", "tsallis_segment_batch"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(L):
    for code in range(8):
        assert tg.tsallis_status_string(code) not in ("", "unknown status")
    assert tg.tsallis_status_string(tg.TSALLIS_ERR_TIMEOUT | tg.TSALLIS_STATUS_RERANKED) == "device wait timed out"


def _seg(L, p, vol=16, mask=16, nx=8, ny=8, nz=2, ctx=None):
    t = ctypes.c_void_p(4096)
    return L.tsallis_segment(ctx, vol, nx, ny, nz, ctypes.byref(p), mask, t, t, t, None)


def test_host_argument_validation(L):
    p = tg.tsallis_params()
    # bad q
    for q in (0.0, -1.0, float("nan"), float("inf")):
        p.q = q
        assert _seg(L, p) == tg.TSALLIS_ERR_INVALID_ARG
    p = tg.tsallis_params()
    for field, bad in (("nbins", 1), ("nbins", 4097), ("mode", 2), ("polarity", 5), ("two_d", 3),
                       ("lo", 10 ** 6), ("flags", 0x80)):
        q = tg.tsallis_params()
        setattr(q, field, bad)
        assert _seg(L, q) == tg.TSALLIS_ERR_INVALID_ARG, field
    q = tg.tsallis_params(two_d=True, shift=3)   # 4096 >> 3 = 512 levels > 256
    assert _seg(L, q) == tg.TSALLIS_ERR_INVALID_ARG
    # shapes
    assert _seg(L, p, nx=0) == tg.TSALLIS_ERR_INVALID_ARG
    assert _seg(L, p, nz=-1) == tg.TSALLIS_ERR_INVALID_ARG
    assert _seg(L, p, nx=1 << 21) == tg.TSALLIS_ERR_INVALID_ARG
    # empty volume is a no-op
    assert _seg(L, p, nz=0) == tg.TSALLIS_OK
    # pointers: null, then misaligned volume or mask
    assert _seg(L, p, vol=None) == tg.TSALLIS_ERR_INVALID_ARG
    assert _seg(L, p, vol=18) == tg.TSALLIS_ERR_ALIGNMENT
    assert _seg(L, p, mask=20) == tg.TSALLIS_ERR_ALIGNMENT
    # well-formed arguments but no context
    assert _seg(L, p) == tg.TSALLIS_ERR_INVALID_ARG


def test_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert L.tsallis_create(ctypes.byref(h), 0) == tg.TSALLIS_ERR_CUDA
    assert L.tsallis_create(ctypes.byref(h), -1) == tg.TSALLIS_ERR_INVALID_ARG
    L.tsallis_destroy(None)


def test_python_binding_refuses_cpu_tensors(L):
    import torch
    v = torch.zeros((2, 4, 4), dtype=torch.int16)
    with pytest.raises(TypeError):
        tg.tsallis_segment(v)


def test_autotune_cache_file_round_trip(tmp_path):
    """The cache file format (no GPU): entries are added and replaced, the
    file is JSON with a format tag, and a foreign file is refused."""
    path = str(tmp_path / "tune.json")
    assert tg.autotune_cache_load(path) == {}
    tg.autotune_cache_store(path, "gpu|a", 65536, 2, 1.5)
    tg.autotune_cache_store(path, "gpu|b", 32768, 1, 2.5)
    tg.autotune_cache_store(path, "gpu|a", 131072, 2, 1.25)
    e = tg.autotune_cache_load(path)
    assert e == {"gpu|a": {"tile_vox": 131072, "blocks_per_sm": 2, "best_ms": 1.25},
                 "gpu|b": {"tile_vox": 32768, "blocks_per_sm": 1, "best_ms": 2.5}}
    bad = tmp_path / "bad.json"
    bad.write_text('{"something": 1}')
    with pytest.raises(ValueError):
        tg.autotune_cache_load(str(bad))
