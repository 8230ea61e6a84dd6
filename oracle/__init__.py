"""CPU oracle (FP64) for maximum-Tsallis-entropy thresholding.

TEST INFRASTRUCTURE ONLY: this package is the slow reference that the GPU path
is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` leg import it. The product package never imports
it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, double precision, plain loops);
this module only compiles it with gcc and marshals numpy arrays to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
F64 = ctypes.c_double

_SIGS = {
    "oracle_hist1d": [P, I64, I32, I32, P],
    "oracle_hist2d": [P, I64, I64, I64, I32, I32, I32, P, P, P],
    "oracle_objective1d_def": [P, I32, F64, P, P],
    "oracle_objective1d_prefix": [P, I32, F64, P, P],
    "oracle_objective2d_def": [P, I32, F64, P, P],
    "oracle_objective2d_prefix": [P, I32, F64, P, P],
    "oracle_argmax1d": [P, P, P, I32, P, P, P],
    "oracle_argmax2d": [P, P, P, I32, P, P, P, P],
    "oracle_binarize": [P, I64, I32, I32, I32, I32, I32, P],
    "oracle_segment1d": [P, I64, I64, I32, I32, F64, I32, I32, I32, P, P, P, P],
    "oracle_rescale8": [P, I64, I32, I32, I32, P],
    "oracle_morph2d": [P, I64, I64, I64, I32, I32, P],
}


def build(verbose: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           _SRC, "-o", _SO + ".tmp", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stdout + r.stderr)
    os.replace(_SO + ".tmp", _SO)
    if verbose:
        print("built", _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            for name, args in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None else None


def _check(rc, name):
    if rc != 0:
        raise RuntimeError("%s returned %d" % (name, rc))


# ------------------------------------------------------------------ API

def hist1d(vol, lo: int = -1024, L: int = 4096) -> np.ndarray:
    """Counts per level of b = clamp(v - lo, 0, L-1) (Fig. 2 measurement space)."""
    v = np.ascontiguousarray(vol, np.int16)
    h = np.zeros(L, np.int64)
    _check(lib().oracle_hist1d(_ptr(v), v.size, lo, L, _ptr(h)), "oracle_hist1d")
    return h


def hist2d(vol, lo: int = -1024, L1: int = 4096, shift: int = 4, return_levels: bool = False):
    """2-D histogram h(i, j) of grey level and floor-mean level (section II-C).

    ``vol`` is [nz][ny][nx]; nz == 1 uses the 3x3 window, nz > 1 the 3x3x3 one.
    """
    v = np.ascontiguousarray(vol, np.int16)
    if v.ndim == 2:
        v = v[None]
    nz, ny, nx = v.shape
    L2 = L1 >> shift
    h = np.zeros((L2, L2), np.int64)
    f = np.empty(v.shape, np.uint8) if return_levels else None
    m = np.empty(v.shape, np.uint8) if return_levels else None
    _check(lib().oracle_hist2d(_ptr(v), nx, ny, nz, lo, L1, shift, _ptr(h), _ptr(f), _ptr(m)), "oracle_hist2d")
    return (h, f, m) if return_levels else h


def objective1d(h, q: float, mode: str = "prefix"):
    """phi(t) for t in [0, L-2] and the validity mask (both classes non-empty)."""
    hh = np.ascontiguousarray(h, np.int64)
    L = hh.size
    phi = np.zeros(L - 1, np.float64)
    valid = np.zeros(L - 1, np.uint8)
    fn = lib().oracle_objective1d_def if mode == "definition" else lib().oracle_objective1d_prefix
    _check(fn(_ptr(hh), L, float(q), _ptr(phi), _ptr(valid)), "objective1d")
    return phi, valid.astype(bool)


def objective2d(h, q: float, mode: str = "prefix"):
    """phi(t, s) on [0, L-2]^2 and validity, for an L x L histogram."""
    hh = np.ascontiguousarray(h, np.int64)
    L = hh.shape[0]
    phi = np.zeros((L - 1, L - 1), np.float64)
    valid = np.zeros((L - 1, L - 1), np.uint8)
    fn = lib().oracle_objective2d_def if mode == "definition" else lib().oracle_objective2d_prefix
    _check(fn(_ptr(hh), L, float(q), _ptr(phi), _ptr(valid)), "objective2d")
    return phi, valid.astype(bool)


def argmax1d(phi, valid, h):
    """(t*, phi*, gap): smallest maximiser and relative gap to the next partition."""
    p = np.ascontiguousarray(phi, np.float64)
    v = np.ascontiguousarray(valid, np.uint8)
    hh = np.ascontiguousarray(h, np.int64)
    t = ctypes.c_int32()
    best = ctypes.c_double()
    gap = ctypes.c_double()
    _check(lib().oracle_argmax1d(_ptr(p), _ptr(v), _ptr(hh), hh.size, ctypes.byref(t), ctypes.byref(best),
                                 ctypes.byref(gap)), "argmax1d")
    return t.value, best.value, gap.value


def argmax2d(phi, valid, h):
    """(t*, s*, phi*, gap) with smallest t then s among equal maxima."""
    p = np.ascontiguousarray(phi, np.float64)
    v = np.ascontiguousarray(valid, np.uint8)
    hh = np.ascontiguousarray(h, np.int64)
    t = ctypes.c_int32()
    s = ctypes.c_int32()
    best = ctypes.c_double()
    gap = ctypes.c_double()
    _check(lib().oracle_argmax2d(_ptr(p), _ptr(v), _ptr(hh), hh.shape[0], ctypes.byref(t), ctypes.byref(s),
                                 ctypes.byref(best), ctypes.byref(gap)), "argmax2d")
    return t.value, s.value, best.value, gap.value


def search1d(h, q: float, mode: str = "prefix"):
    """Objective then maximiser: (t*, phi*, gap, phi curve, valid)."""
    phi, valid = objective1d(h, q, mode)
    t, best, gap = argmax1d(phi, valid, h)
    return t, best, gap, phi, valid


def search2d(h, q: float, mode: str = "prefix"):
    phi, valid = objective2d(h, q, mode)
    t, s, best, gap = argmax2d(phi, valid, h)
    return t, s, best, gap, phi, valid


def binarize(vol, t: int, lo: int = -1024, L: int = 4096, shift: int = 0, polarity: int = 0) -> np.ndarray:
    """Algorithm 1 on levels (polarity 1: level >= t+1; polarity 0: level <= t)."""
    v = np.ascontiguousarray(vol, np.int16)
    m = np.empty(v.shape, np.uint8)
    _check(lib().oracle_binarize(_ptr(v), v.size, lo, L, shift, int(t), int(polarity), _ptr(m)), "binarize")
    return m


def segment1d(vol, group_voxels: int, q: float, lo: int = -1024, L: int = 4096, polarity: int = 0,
              nthreads: int = 1, definition: bool = False, want_mask: bool = True):
    """Whole 1-D step over consecutive groups (slices or volumes).

    Returns (t[ngroups], phi[ngroups], gap[ngroups], mask or None).
    """
    v = np.ascontiguousarray(vol, np.int16).reshape(-1)
    if v.size % group_voxels:
        raise ValueError("volume size is not a multiple of the group size")
    ng = v.size // group_voxels
    t = np.zeros(ng, np.int32)
    phi = np.zeros(ng, np.float64)
    gap = np.zeros(ng, np.float64)
    mask = np.empty(v.size, np.uint8) if want_mask else None
    _check(lib().oracle_segment1d(_ptr(v), group_voxels, ng, lo, L, float(q), polarity, int(definition), nthreads,
                                  _ptr(t), _ptr(phi), _ptr(gap), _ptr(mask)), "segment1d")
    return t, phi, gap, mask


MORPH_OPS = {"copy": 0, "erode": 1, "dilate": 2, "open": 3, "close": 4, "chest_mask": 5, "black_tophat": 6}


def rescale8(vol, background: int = -2000, hu_min: int = -2000, hu_max: int = 2500) -> np.ndarray:
    """Section II-B pre-processing: CT numbers to 8-bit grey levels."""
    v = np.ascontiguousarray(vol, np.int16)
    g = np.empty(v.shape, np.uint8)
    _check(lib().oracle_rescale8(_ptr(v), v.size, background, hu_min, hu_max, _ptr(g)), "rescale8")
    return g


def morph2d(img, r: int = 10, op: str = "chest_mask") -> np.ndarray:
    """Section II-C morphology on each slice of a uint8 [nz][ny][nx] image
    with the disk of radius r."""
    a = np.ascontiguousarray(img, np.uint8)
    a3 = a.reshape((-1,) + a.shape[-2:])
    o = np.empty(a3.shape, np.uint8)
    _check(lib().oracle_morph2d(_ptr(a3), a3.shape[2], a3.shape[1], a3.shape[0], r, MORPH_OPS[op], _ptr(o)),
           "morph2d")
    return o.reshape(a.shape)


def preprocess(vol, r: int = 10, op: str = "chest_mask", background: int = -2000, hu_min: int = -2000,
               hu_max: int = 2500, per_slice: bool = True):
    """Pre-processing and morphology of a [nz][ny][nx] CT volume: the 8-bit
    image after the chest-mask step (as int16 levels 0..255) and its 256-level
    histograms, one per slice (per_slice) or one for the volume."""
    g = rescale8(vol, background, hu_min, hu_max)
    o = morph2d(g, r, op).astype(np.int16)
    o3 = o.reshape((-1,) + o.shape[-2:])
    groups = o3.reshape(o3.shape[0], -1) if per_slice else o3.reshape(1, -1)
    h = np.stack([hist1d(gr, lo=0, L=256) for gr in groups]).astype(np.int64)
    return o, h
