"""GB300 maximum-Tsallis-entropy threshold segmentation.

Thin Python binding of the C ABI declared in ``include/tsallis.h``
(``libtsallis.so``, built in-tree by :mod:`paper_2012_10684_gb300.build`).
Functions carry the C names and only marshal arguments: torch tensors supply
device memory and the current CUDA stream; every step of the path runs in the
library's CUDA kernels. There is no CPU fallback: if the library is missing,
every call raises.

Method (Chang & Sheu, section II-C "Segmentation"): histogram of grey levels,
class masses and Tsallis class entropies for every threshold, the
pseudo-additive objective H1 + H2 + (1 - q) H1 H2 maximised over all
thresholds, then Algorithm 1 (thresholding kernel) on every voxel.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

__all__ = [
    "Params", "TsallisError", "lib", "tsallis_params", "tsallis_histogram", "tsallis_search",
    "tsallis_binarize", "tsallis_segment", "tsallis_segment_batch", "tsallis_status_string",
    "tsallis_preprocess", "preprocess_params",
    "TSALLIS_OK", "TSALLIS_ERR_NO_VALID_THRESHOLD", "TSALLIS_ERR_TIMEOUT", "TSALLIS_STATUS_RERANKED",
]

TSALLIS_OK = 0
TSALLIS_ERR_INVALID_ARG = 1
TSALLIS_ERR_ALIGNMENT = 2
TSALLIS_ERR_CUDA = 3
TSALLIS_ERR_NO_VALID_THRESHOLD = 4
TSALLIS_ERR_TIMEOUT = 5
TSALLIS_ERR_OOM = 6
TSALLIS_ERR_UNIMPLEMENTED = 7
TSALLIS_STATUS_RERANKED = 0x100
TSALLIS_STATUS_FIRST_PASS_EXACT = 0x200
TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL = 0x1
TSALLIS_FLAG_PREDICT_PROPOSER = 0x2
TSALLIS_FLAG_PREDICT_SUBSAMPLE = 0x4
TSALLIS_FLAG_BRUTE_FORCE_2D = 0x8
SLICE_KERNELS = {"auto": 0, "tiles": 1, "cluster": 2, "predict": 3, "pipeline": 4}

PER_SLICE, WHOLE_VOLUME = 0, 1
MASK_LOW, MASK_HIGH = 0, 1


class Params(ctypes.Structure):
    """Mirror of ``tsallis_params``."""
    _fields_ = [("lo", ctypes.c_int32), ("nbins", ctypes.c_int32), ("q", ctypes.c_float),
                ("mode", ctypes.c_int32), ("polarity", ctypes.c_int32), ("two_d", ctypes.c_int32),
                ("shift", ctypes.c_int32), ("topk", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class Volume(ctypes.Structure):
    """Mirror of ``tsallis_volume``."""
    _fields_ = [("vol", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64)]


class PreprocessParams(ctypes.Structure):
    """Mirror of ``tsallis_preprocess_params``."""
    _fields_ = [("background", ctypes.c_int32), ("hu_min", ctypes.c_int32), ("hu_max", ctypes.c_int32),
                ("radius", ctypes.c_int32), ("op", ctypes.c_int32), ("per_slice", ctypes.c_int32)]


MORPH_OPS = {"none": 0, "erode": 1, "dilate": 2, "open": 3, "close": 4, "chest_mask": 5, "black_tophat": 6}


class TsallisError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (fn, tsallis_status_string(code), code))


_lock = threading.Lock()
_lib = None
_ctx = {}

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "tsallis_params_default": ([ctypes.POINTER(Params)], ctypes.c_int),
    "tsallis_status_string": ([ctypes.c_int32], ctypes.c_char_p),
    "tsallis_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int], ctypes.c_int),
    "tsallis_destroy": ([_P], None),
    "tsallis_set_wait_timeout": ([_P, ctypes.c_uint64], ctypes.c_int),
    "tsallis_set_launch_shape": ([_P, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "tsallis_set_slice_kernel": ([_P, ctypes.c_int32], ctypes.c_int),
    "tsallis_set_speculation": ([_P, ctypes.c_int32], ctypes.c_int),
    "tsallis_set_prediction": ([_P, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "tsallis_test_withhold_predictions": ([_P, ctypes.c_int32], ctypes.c_int),
    "tsallis_histogram": ([_P, _P, _I64, _I64, _I64, ctypes.POINTER(Params), _P, _P], ctypes.c_int),
    "tsallis_search": ([_P, _P, _I64, ctypes.POINTER(Params), _P, _P, _P, _P, _P], ctypes.c_int),
    "tsallis_binarize": ([_P, _P, _I64, _I64, _I64, _P, ctypes.POINTER(Params), _P, _P], ctypes.c_int),
    "tsallis_segment": ([_P, _P, _I64, _I64, _I64, ctypes.POINTER(Params), _P, _P, _P, _P, _P], ctypes.c_int),
    "tsallis_segment_host": ([_P, _P, _I64, _I64, _I64, ctypes.POINTER(Params), _P, _P, _P, _P, _P], ctypes.c_int),
    "tsallis_segment_batch": ([_P, ctypes.POINTER(Volume), ctypes.c_int32, ctypes.POINTER(Params), _P, _P, _P, _P],
                              ctypes.c_int),
    "tsallis_autotune_batch": ([_P, ctypes.POINTER(Volume), ctypes.c_int32, ctypes.POINTER(Params), _P, _P, _P, _P,
                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "tsallis_proposer_set": ([_P, _P, _I64], ctypes.c_int),
    "tsallis_proposer_get": ([_P, _P, _I64], ctypes.c_int),
    "tsallis_proposer_load": ([_P, ctypes.c_char_p], ctypes.c_int),
    "tsallis_proposer_save": ([_P, ctypes.c_char_p], ctypes.c_int),
    "tsallis_proposer_features": ([_P, _P, _I64, _P, _P], ctypes.c_int),
    "tsallis_proposer_select": ([_P, ctypes.c_int32], ctypes.c_int),
    "tsallis_proposer_checkpoint_save": ([_P, ctypes.c_char_p, _P, _I64], ctypes.c_int),
    "tsallis_proposer_checkpoint_load": ([_P, ctypes.c_char_p, _P, _I64, ctypes.POINTER(ctypes.c_int64)],
                                         ctypes.c_int),
    "tsallis_proposer_forward": ([_P, _P, ctypes.c_int32, _P, _P], ctypes.c_int),
    "tsallis_proposer_train_step": ([_P, _P, _P, ctypes.c_int32, ctypes.c_float, ctypes.c_int32, _P, _P, _P],
                                    ctypes.c_int),
    "tsallis_preprocess_params_default": ([ctypes.POINTER(PreprocessParams)], ctypes.c_int),
    "tsallis_preprocess": ([_P, _P, _I64, _I64, _I64, ctypes.POINTER(PreprocessParams), _P, _P, _P], ctypes.c_int),
    "tsallis_check_status": ([_P, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "tsallis_probe_topk": ([_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P], ctypes.c_int),
    "tsallis_probe_dfmath": ([_P, _P, _I64, ctypes.c_uint32, ctypes.c_float, _P, _P, _P], ctypes.c_int),
}


def library_path() -> str:
    """The library this process loads: the checked build when the
    environment sets TSALLIS_CHECKED=1, else the normal one."""
    return _build.LIB_CHECKED if os.environ.get("TSALLIS_CHECKED") == "1" else _build.LIB


def lib():
    """The loaded C-ABI library. Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(library_path()):
                raise RuntimeError("libtsallis.so is not built (run paper_2012_10684_gb300.build.build()); "
                                   "there is no CPU fallback")
            L = ctypes.CDLL(library_path())
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def tsallis_status_string(code: int) -> str:
    try:
        return lib().tsallis_status_string(int(code)).decode()
    except RuntimeError:
        return "status %d" % code


def _check(fn, rc):
    if rc != TSALLIS_OK:
        raise TsallisError(fn, rc)


def context(device=None) -> int:
    """Handle of the per-device context (created on first use)."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    if dev is None:
        dev = torch.cuda.current_device()
    with _lock:
        h = _ctx.get(dev)
    if h is None:
        p = ctypes.c_void_p()
        _check("tsallis_create", lib().tsallis_create(ctypes.byref(p), dev))
        with _lock:
            _ctx[dev] = p.value
        h = p.value
    return h


def set_wait_timeout(ns: int, device=None) -> None:
    _check("tsallis_set_wait_timeout", lib().tsallis_set_wait_timeout(context(device), int(ns)))


DEFAULT_TILE_VOX = 131072   # a context's voxels per work tile until set_launch_shape changes it


def set_launch_shape(tile_vox: int = DEFAULT_TILE_VOX, blocks_per_sm: int = 0, device=None) -> None:
    """Launch shape of the persistent kernels (see tsallis_set_launch_shape);
    without arguments, the defaults."""
    _check("tsallis_set_launch_shape",
           lib().tsallis_set_launch_shape(context(device), int(tile_vox), int(blocks_per_sm)))


def set_slice_kernel(kind: str = "auto", device=None) -> None:
    """Kernel for per-slice 1-D segmentation: "auto", "tiles", "cluster" or
    "predict" (see tsallis_set_slice_kernel)."""
    _check("tsallis_set_slice_kernel", lib().tsallis_set_slice_kernel(context(device), SLICE_KERNELS[kind]))


def set_speculation(on: bool = False, device=None) -> None:
    """First-pass binarisation with a predicted threshold in the tile kernel
    (see tsallis_set_speculation)."""
    _check("tsallis_set_speculation", lib().tsallis_set_speculation(context(device), 1 if on else 0))


def set_prediction(row_stride: int = 8, window: int = 8, device=None) -> None:
    """Prediction row stride and list window of the predicted first-pass
    kernel (see tsallis_set_prediction)."""
    _check("tsallis_set_prediction", lib().tsallis_set_prediction(context(device), int(row_stride), int(window)))


def withhold_predictions(on: bool, device=None) -> None:
    """Test hook: the predicted first-pass kernel publishes no predictions
    (see tsallis_test_withhold_predictions)."""
    _check("tsallis_test_withhold_predictions",
           lib().tsallis_test_withhold_predictions(context(device), 1 if on else 0))


def tsallis_probe_dfmath(h: torch.Tensor, N: int, q: float):
    """Test hook: ((h/N)^q, log2 h) as computed by the search's double-float math."""
    if not h.is_cuda or h.dtype != torch.int32 or not h.is_contiguous():
        raise TypeError("h must be a contiguous int32 CUDA tensor of counts")
    pw = torch.empty(h.numel(), dtype=torch.float64, device=h.device)
    lg = torch.empty(h.numel(), dtype=torch.float64, device=h.device)
    _check("tsallis_probe_dfmath", lib().tsallis_probe_dfmath(context(h.device), h.data_ptr(), h.numel(), int(N),
                                                              float(q), pw.data_ptr(), lg.data_ptr(), _stream(h)))
    return pw, lg


def tsallis_params(q: float = 0.8, lo: int = -1024, nbins: int = 4096, mode="slice", polarity="low",
                   two_d: bool = False, shift: int = 4, topk: int = 0, flags: int = 0) -> Params:
    p = Params()
    lib().tsallis_params_default(ctypes.byref(p))
    p.q, p.lo, p.nbins = float(q), int(lo), int(nbins)
    p.mode = {"slice": PER_SLICE, "volume": WHOLE_VOLUME, PER_SLICE: PER_SLICE, WHOLE_VOLUME: WHOLE_VOLUME}[mode]
    p.polarity = {"low": MASK_LOW, "high": MASK_HIGH, MASK_LOW: MASK_LOW, MASK_HIGH: MASK_HIGH}[polarity]
    p.two_d, p.shift, p.topk, p.flags = int(bool(two_d)), int(shift), int(topk), int(flags)
    return p


def _vol3(vol: torch.Tensor):
    if not isinstance(vol, torch.Tensor) or not vol.is_cuda:
        raise TypeError("volume must be a CUDA tensor")
    if vol.dtype != torch.int16 or not vol.is_contiguous():
        raise TypeError("volume must be a contiguous int16 tensor")
    if vol.dim() == 2:
        return vol.shape[1], vol.shape[0], 1
    if vol.dim() != 3:
        raise ValueError("volume must be [nz][ny][nx] or [ny][nx]")
    return vol.shape[2], vol.shape[1], vol.shape[0]


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def _nh(p: Params, nz: int) -> int:
    return nz if p.mode == PER_SLICE else 1


def _levels(p: Params) -> int:
    return (p.nbins >> p.shift) if p.two_d else p.nbins


def _hist_shape(p: Params, nh: int):
    L = _levels(p)
    return (nh, L, L) if p.two_d else (nh, L)


def tsallis_histogram(vol: torch.Tensor, p: Params | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Step 1: int32 histograms [nh][L] (2-D: [nh][L2][L2])."""
    p = p or tsallis_params()
    nx, ny, nz = _vol3(vol)
    nh = _nh(p, nz)
    if out is None:
        out = torch.empty(_hist_shape(p, nh), dtype=torch.int32, device=vol.device)
    _check("tsallis_histogram", lib().tsallis_histogram(context(vol.device), vol.data_ptr(), nx, ny, nz,
                                                        ctypes.byref(p), out.data_ptr(), _stream(vol)))
    return out


def tsallis_search(hist: torch.Tensor, p: Params | None = None, curve: bool = False):
    """Steps 2-3: (t, phi, status[, curve]) for each histogram."""
    p = p or tsallis_params()
    if not hist.is_cuda or hist.dtype != torch.int32 or not hist.is_contiguous():
        raise TypeError("hist must be a contiguous int32 CUDA tensor")
    L = _levels(p)
    per = L * L if p.two_d else L
    if hist.numel() % per:
        raise ValueError("histogram size does not match nbins")
    nh = hist.numel() // per
    dev = hist.device
    t = torch.empty((nh, 2) if p.two_d else (nh,), dtype=torch.int32, device=dev)
    phi = torch.empty(nh, dtype=torch.float32, device=dev)
    st = torch.empty(nh, dtype=torch.int32, device=dev)
    cv = None
    if curve:
        cv = torch.empty((nh, L - 1, L - 1) if p.two_d else (nh, L - 1), dtype=torch.float32, device=dev)
    _check("tsallis_search", lib().tsallis_search(context(dev), hist.data_ptr(), nh, ctypes.byref(p), t.data_ptr(),
                                                  phi.data_ptr(), st.data_ptr(),
                                                  cv.data_ptr() if cv is not None else None, _stream(hist)))
    return (t, phi, st, cv) if curve else (t, phi, st)


def tsallis_binarize(vol: torch.Tensor, t: torch.Tensor, p: Params | None = None,
                     out: torch.Tensor | None = None) -> torch.Tensor:
    """Step 4 (Algorithm 1): uint8 mask with the thresholds in t."""
    p = p or tsallis_params()
    nx, ny, nz = _vol3(vol)
    if not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous():
        raise TypeError("t must be a contiguous int32 CUDA tensor")
    if out is None:
        out = torch.empty(vol.shape, dtype=torch.uint8, device=vol.device)
    _check("tsallis_binarize", lib().tsallis_binarize(context(vol.device), vol.data_ptr(), nx, ny, nz, t.data_ptr(),
                                                      ctypes.byref(p), out.data_ptr(), _stream(vol)))
    return out


def tsallis_segment(vol: torch.Tensor, p: Params | None = None, mask: torch.Tensor | None = None,
                    t: torch.Tensor | None = None, phi: torch.Tensor | None = None,
                    status: torch.Tensor | None = None):
    """Steps 1-4 fused: (mask, t, phi, status)."""
    p = p or tsallis_params()
    nx, ny, nz = _vol3(vol)
    nh = _nh(p, nz)
    dev = vol.device
    if mask is None:
        mask = torch.empty(vol.shape, dtype=torch.uint8, device=dev)
    if t is None:
        t = torch.empty((nh, 2) if p.two_d else (nh,), dtype=torch.int32, device=dev)
    if phi is None:
        phi = torch.empty(nh, dtype=torch.float32, device=dev)
    if status is None:
        status = torch.empty(nh, dtype=torch.int32, device=dev)
    _check("tsallis_segment", lib().tsallis_segment(context(dev), vol.data_ptr(), nx, ny, nz, ctypes.byref(p),
                                                    mask.data_ptr(), t.data_ptr(), phi.data_ptr(),
                                                    status.data_ptr(), _stream(vol)))
    return mask, t, phi, status


def _batch_args(vols, p, masks, outs):
    vols = list(vols)
    if not vols:
        raise ValueError("empty batch")
    dev = vols[0].device
    if masks is None:
        masks = [torch.empty(v.shape, dtype=torch.uint8, device=dev) for v in vols]
    arr = (Volume * len(vols))()
    nh = 0
    for i, (v, m) in enumerate(zip(vols, masks)):
        if v.device != dev or m.device != dev or m.dtype != torch.uint8 or m.shape != v.shape:
            raise ValueError("volume %d: mask must be a uint8 tensor of the volume's shape on its device" % i)
        nx, ny, nz = _vol3(v)
        if not m.is_contiguous():
            raise ValueError("mask %d must be contiguous" % i)
        arr[i] = Volume(v.data_ptr(), m.data_ptr(), nx, ny, nz)
        nh += _nh(p, nz)
    if outs is None:
        t = torch.empty((nh, 2) if p.two_d else (nh,), dtype=torch.int32, device=dev)
        phi = torch.empty(nh, dtype=torch.float32, device=dev)
        st = torch.empty(nh, dtype=torch.int32, device=dev)
    else:
        t, phi, st = outs
    return vols, masks, arr, t, phi, st


def tsallis_segment_batch(vols, p: Params | None = None, masks=None, outs=None):
    """Steps 1-4 for a list of volumes in one persistent launch:
    (masks, t, phi, status), one threshold per volume (whole-volume mode) or
    per slice (per-slice mode, slices numbered across the batch)."""
    p = p or tsallis_params()
    vols, masks, arr, t, phi, st = _batch_args(vols, p, masks, outs)
    _check("tsallis_segment_batch", lib().tsallis_segment_batch(context(vols[0].device), arr, len(vols),
                                                                ctypes.byref(p), t.data_ptr(), phi.data_ptr(),
                                                                st.data_ptr(), _stream(vols[0])))
    return masks, t, phi, st


def autotune_key(vols, p: Params) -> str:
    """Cache key of a batch's launch shape: the GPU, the parameters that
    change the work, and the volumes' shapes."""
    import hashlib
    dev = vols[0].device
    props = torch.cuda.get_device_properties(dev)
    shapes = ",".join("%dx%dx%d" % tuple(int(d) for d in reversed(v.shape[-3:])) for v in vols)
    return "%s|sm%d|mode%d|2d%d|L%d|shift%d|topk%d|flags%d|%s" % (
        props.name, props.multi_processor_count, p.mode, p.two_d, p.nbins, p.shift, p.topk, p.flags,
        hashlib.sha1(shapes.encode()).hexdigest())


def autotune_cache_load(path: str) -> dict:
    """The entries of an autotune cache file ({} when it does not exist)."""
    import json
    try:
        with open(path) as f:
            d = json.load(f)
    except FileNotFoundError:
        return {}
    if not isinstance(d, dict) or d.get("format") != "tsallis-autotune-1":
        raise ValueError("not an autotune cache: %s" % path)
    return d.get("entries", {})


def autotune_cache_store(path: str, key: str, tile_vox: int, blocks_per_sm: int, best_ms: float) -> None:
    """Adds (or replaces) one entry; the file is replaced atomically."""
    import json
    entries = autotune_cache_load(path)
    entries[key] = {"tile_vox": int(tile_vox), "blocks_per_sm": int(blocks_per_sm), "best_ms": float(best_ms)}
    tmp = "%s.tmp%d" % (path, os.getpid())
    with open(tmp, "w") as f:
        json.dump({"format": "tsallis-autotune-1", "entries": entries}, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tsallis_autotune_batch(vols, p: Params | None = None, masks=None, outs=None, cache: str | None = None):
    """Times the batch over the launch shapes and keeps the fastest for the
    context: returns (tile_vox, blocks_per_sm, best_ms). With cache (a JSON
    file path), a shape found there for this GPU, parameters and volume
    shapes is applied without timing, and a newly timed one is stored."""
    p = p or tsallis_params()
    if cache is not None:
        key = autotune_key(vols, p)
        hit = autotune_cache_load(cache).get(key)
        if hit is not None:
            set_launch_shape(hit["tile_vox"], hit["blocks_per_sm"], vols[0].device)
            return hit["tile_vox"], hit["blocks_per_sm"], hit["best_ms"]
    vols, masks, arr, t, phi, st = _batch_args(vols, p, masks, outs)
    tv, bps, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check("tsallis_autotune_batch", lib().tsallis_autotune_batch(
        context(vols[0].device), arr, len(vols), ctypes.byref(p), t.data_ptr(), phi.data_ptr(), st.data_ptr(),
        _stream(vols[0]), ctypes.byref(tv), ctypes.byref(bps), ctypes.byref(ms)))
    if cache is not None:
        autotune_cache_store(cache, key, tv.value, bps.value, ms.value)
    return tv.value, bps.value, ms.value


# ---------------------------------------------------------------- proposer

PROPOSER_PARAMS = 1184256
TSALLIS_STATUS_WINDOW_HIT = 0x400
TSALLIS_STATUS_FALLBACK_SHIFT = 16


def proposer_set(params, device=None) -> None:
    """Parameters of the learned proposer (flat float vector W1, b1, W2, b2,
    W3, b3); clears the optimiser state."""
    import numpy as np
    a = np.ascontiguousarray(params, np.float32).reshape(-1)
    if a.size != PROPOSER_PARAMS:
        raise ValueError("expected %d parameters" % PROPOSER_PARAMS)
    _check("tsallis_proposer_set", lib().tsallis_proposer_set(context(device), a.ctypes.data, a.size))


def proposer_get(device=None):
    import numpy as np
    a = np.empty(PROPOSER_PARAMS, np.float32)
    _check("tsallis_proposer_get", lib().tsallis_proposer_get(context(device), a.ctypes.data, a.size))
    return a


def proposer_load(path: str, device=None) -> None:
    _check("tsallis_proposer_load", lib().tsallis_proposer_load(context(device), os.fsencode(path)))


def proposer_save(path: str, device=None) -> None:
    _check("tsallis_proposer_save", lib().tsallis_proposer_save(context(device), os.fsencode(path)))


_selected = {}


def proposer_features(hist: torch.Tensor) -> torch.Tensor:
    """x [nh][256] from int32 histograms [nh][4096] (slot 1 selected:
    2-D histograms [nh][256][256])."""
    per = 65536 if _selected.get(hist.device.index, 0) == 1 else 4096
    if not hist.is_cuda or hist.dtype != torch.int32 or not hist.is_contiguous() or hist.numel() % per:
        raise TypeError("hist must be a contiguous int32 CUDA tensor of %d-cell histograms" % per)
    nh = hist.numel() // per
    x = torch.empty((nh, 256), dtype=torch.float32, device=hist.device)
    _check("tsallis_proposer_features", lib().tsallis_proposer_features(context(hist.device), hist.data_ptr(), nh,
                                                                        x.data_ptr(), _stream(hist)))
    return x


def proposer_forward(x: torch.Tensor) -> torch.Tensor:
    """Logits [B][4096] from features x [B][256] (float32, CUDA)."""
    x = x.contiguous()
    z = torch.empty((x.shape[0], 4096), dtype=torch.float32, device=x.device)
    _check("tsallis_proposer_forward", lib().tsallis_proposer_forward(context(x.device), x.data_ptr(), x.shape[0],
                                                                      z.data_ptr(), _stream(x)))
    return z


def proposer_train_step(x: torch.Tensor, y: torch.Tensor, lr: float = 1e-3, update: bool = True,
                        want_grad: bool = False):
    """One training step on a batch: returns (loss tensor [1], gradient or None)."""
    x, y = x.contiguous(), y.contiguous()
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    g = torch.empty(PROPOSER_PARAMS, dtype=torch.float32, device=x.device) if want_grad else None
    _check("tsallis_proposer_train_step", lib().tsallis_proposer_train_step(
        context(x.device), x.data_ptr(), y.data_ptr(), x.shape[0], float(lr), 1 if update else 0, loss.data_ptr(),
        g.data_ptr() if g is not None else None, _stream(x)))
    return loss, g


def proposer_checkpoint_save(path: str, user: bytes = b"", device=None) -> None:
    """Parameters, Adam state and step count, plus the caller's own bytes."""
    buf = ctypes.create_string_buffer(user, len(user)) if user else None
    _check("tsallis_proposer_checkpoint_save", lib().tsallis_proposer_checkpoint_save(
        context(device), os.fsencode(path), buf, len(user)))


def proposer_checkpoint_load(path: str, user_cap: int = 1 << 20, device=None) -> bytes:
    """Restores a checkpoint; returns the caller's bytes saved with it."""
    buf = ctypes.create_string_buffer(max(user_cap, 1))
    n = ctypes.c_int64(0)
    _check("tsallis_proposer_checkpoint_load", lib().tsallis_proposer_checkpoint_load(
        context(device), os.fsencode(path), buf, user_cap, ctypes.byref(n)))
    return buf.raw[: n.value]


def preprocess_params(op="chest_mask", radius: int = 10, background: int = -2000, hu_min: int = -2000,
                      hu_max: int = 2500, per_slice: bool = True) -> PreprocessParams:
    pp = PreprocessParams()
    _check("tsallis_preprocess_params_default", lib().tsallis_preprocess_params_default(ctypes.byref(pp)))
    pp.op = MORPH_OPS[op] if isinstance(op, str) else int(op)
    pp.radius, pp.background, pp.hu_min, pp.hu_max = int(radius), int(background), int(hu_min), int(hu_max)
    pp.per_slice = int(bool(per_slice))
    return pp


def tsallis_preprocess(vol: torch.Tensor, pp: PreprocessParams | None = None, out: torch.Tensor | None = None,
                       hist: torch.Tensor | None = None, want_out: bool = True, want_hist: bool = True):
    """8-bit pre-processing and chest-mask morphology of a CT volume:
    (levels int16 [nz][ny][nx] or None, int32 histograms [nh][256] or None)."""
    pp = pp or preprocess_params()
    nx, ny, nz = _vol3(vol)
    if want_out and out is None:
        out = torch.empty(vol.shape, dtype=torch.int16, device=vol.device)
    if want_hist and hist is None:
        hist = torch.empty((nz if pp.per_slice else 1, 256), dtype=torch.int32, device=vol.device)
    _check("tsallis_preprocess", lib().tsallis_preprocess(
        context(vol.device), vol.data_ptr(), nx, ny, nz, ctypes.byref(pp),
        out.data_ptr() if want_out else None, hist.data_ptr() if want_hist else None, _stream(vol)))
    return (out if want_out else None), (hist if want_hist else None)


def proposer_select(slot: int, device=None) -> None:
    """Slot the proposer_* calls act on: 0 (1-D searches) or 1 (2-D search)."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    _check("tsallis_proposer_select", lib().tsallis_proposer_select(context(dev), int(slot)))
    _selected[dev] = int(slot)


def check_status(device=None) -> int:
    """Checked build: the first failing index check's site since the last
    call (0: none); raises in a normal build."""
    v = ctypes.c_uint32(0)
    _check("tsallis_check_status", lib().tsallis_check_status(context(device), ctypes.byref(v)))
    return v.value


def probe_topk(z: torch.Tensor, k: int) -> torch.Tensor:
    """Test hook: the proposer's top-k indices [B][k] of logits [B][4096]."""
    if not z.is_cuda or z.dtype != torch.float32 or not z.is_contiguous() or z.shape[-1] != 4096:
        raise TypeError("logits must be a contiguous float32 CUDA tensor [B][4096]")
    B = z.numel() // 4096
    out = torch.empty((B, k), dtype=torch.int32, device=z.device)
    _check("tsallis_probe_topk", lib().tsallis_probe_topk(context(z.device), z.data_ptr(), B, int(k), out.data_ptr(),
                                                          _stream(z)))
    return out


def tsallis_segment_host(vol: torch.Tensor, p: Params | None = None, mask: torch.Tensor | None = None,
                         t: torch.Tensor | None = None, phi: torch.Tensor | None = None,
                         status: torch.Tensor | None = None, device=None, sync: bool = True):
    """Steps 1-4 from and to host memory (CPU tensors; page-locked ones let
    the copies overlap the kernels): (mask, t, phi, status) on the host.
    With sync=False the call returns once the work is enqueued on the
    device's current stream; the outputs are valid after synchronising it."""
    p = p or tsallis_params()
    if not isinstance(vol, torch.Tensor) or vol.is_cuda or vol.dtype != torch.int16 or not vol.is_contiguous():
        raise TypeError("volume must be a contiguous int16 CPU tensor")
    nz, ny, nx = (1,) + tuple(vol.shape) if vol.dim() == 2 else tuple(vol.shape)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
    nh = nz if p.mode == PER_SLICE else 1
    pin = vol.is_pinned()
    if mask is None:
        mask = torch.empty(vol.shape, dtype=torch.uint8, pin_memory=pin)
    if t is None:
        t = torch.empty((nh, 2) if p.two_d else (nh,), dtype=torch.int32, pin_memory=pin)
    if phi is None:
        phi = torch.empty(nh, dtype=torch.float32, pin_memory=pin)
    if status is None:
        status = torch.empty(nh, dtype=torch.int32, pin_memory=pin)
    stream = torch.cuda.current_stream(dev)
    _check("tsallis_segment_host", lib().tsallis_segment_host(
        context(dev), vol.data_ptr(), nx, ny, nz, ctypes.byref(p), mask.data_ptr(), t.data_ptr(), phi.data_ptr(),
        status.data_ptr(), stream.cuda_stream))
    if sync:
        stream.synchronize()
    return mask, t, phi, status
