"""Seeded synthetic chest-CT phantoms (the input generator).

This module is shared by the oracle's tests, the GPU path's tests and the
benchmark. It holds none of the segmentation method's arithmetic: it only
builds a geometry (ellipses for body and lungs, a tree of capsules for the
airway) from a seeded numpy generator, and fills int16 Hounsfield volumes with
integer-only Gaussian noise, either on the host (plain C, threads over slices)
or on the GPU (a CUDA kernel compiled from the same header). Both builds give
bit-identical volumes for the same descriptor.

Workload recipes (sizes and value distributions of the paper's chest CT):
  * ``slice_phantom``   512x512 slice, body N(40,20), lungs N(-850,60), 6-10
    airway discs r=2..8 px N(-1000,15), outside air -1024, sensor sd 10.
  * ``chest_volume``    512x512xD, same classes extruded along z with a
    branching airway tree (trachea r=9 px, radius x0.79 and length x0.8 per
    generation, +-35 degree branches).
  * ``batch_specs``     uneven depths D ~ U[120,600], sensor sd ~ U[5,30],
    airway generations ~ U{4..8}.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_HOST_SO = os.path.join(_BUILD, "libphantom_host.so")
_CUDA_SO = os.path.join(_BUILD, "libphantom_cuda.so")
_lock = threading.Lock()


class _Capsule(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("ax", "ay", "az", "bx", "by", "bz", "r", "zlo", "zhi", "ylo", "yhi", "xlo", "xhi")]


class _Ellipse(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("cx", "cy", "a", "b")]


class _Desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
        ("seed", ctypes.c_uint64), ("vol_id", ctypes.c_uint32),
        ("air_hu", ctypes.c_int32),
        ("body_mu", ctypes.c_int32), ("body_sd", ctypes.c_int32),
        ("lung_mu", ctypes.c_int32), ("lung_sd", ctypes.c_int32),
        ("airway_mu", ctypes.c_int32), ("airway_sd", ctypes.c_int32),
        ("noise_sd", ctypes.c_int32),
        ("body", _Ellipse), ("lung", _Ellipse * 2),
        ("ncaps", ctypes.c_int32),
        ("caps", ctypes.c_void_p), ("slice_off", ctypes.c_void_p), ("slice_caps", ctypes.c_void_p),
    ]


CAPSULE_FIELDS = 13


@dataclass
class PhantomSpec:
    """Everything that determines one phantom volume."""
    nx: int
    ny: int
    nz: int
    seed: int
    vol_id: int = 0
    noise_sd: int = 10
    air_hu: int = -1024
    body_mu: int = 40
    body_sd: int = 20
    lung_mu: int = -850
    lung_sd: int = 60
    airway_mu: int = -1000
    airway_sd: int = 15
    body: tuple = (256, 256, 220, 160)
    lungs: tuple = ((161, 256, 75, 120), (351, 256, 75, 120))
    capsules: np.ndarray = field(default_factory=lambda: np.zeros((0, CAPSULE_FIELDS), np.int32))

    @property
    def nvox(self) -> int:
        return self.nx * self.ny * self.nz

    def slice_csr(self):
        """Per-slice lists of the capsules whose bounding box meets the slice."""
        caps = self.capsules
        off = np.zeros(self.nz + 1, np.int32)
        idx = []
        for z in range(self.nz):
            if len(caps):
                sel = np.nonzero((caps[:, 7] <= z) & (caps[:, 8] >= z))[0].astype(np.int32)
            else:
                sel = np.zeros(0, np.int32)
            idx.append(sel)
            off[z + 1] = off[z] + len(sel)
        flat = np.concatenate(idx) if idx else np.zeros(0, np.int32)
        if flat.size == 0:
            flat = np.zeros(1, np.int32)
        return off, flat.astype(np.int32)


def _capsule_row(a, b, r, nx, ny, nz):
    """Fixed-point capsule (1/16 voxel) with a conservative voxel bounding box."""
    A = [int(round(v * 16)) for v in a]
    B = [int(round(v * 16)) for v in b]
    R = max(1, int(round(r * 16)))

    def rng(lo16, hi16, n):
        lo = (lo16 - R - 8) // 16 - 1
        hi = -((-(hi16 + R - 8)) // 16) + 1
        return max(0, lo), min(n - 1, hi)

    zlo, zhi = rng(min(A[2], B[2]), max(A[2], B[2]), nz)
    ylo, yhi = rng(min(A[1], B[1]), max(A[1], B[1]), ny)
    xlo, xhi = rng(min(A[0], B[0]), max(A[0], B[0]), nx)
    return [A[0], A[1], A[2], B[0], B[1], B[2], R, zlo, zhi, ylo, yhi, xlo, xhi]


def _rotate(v, axis, ang):
    """Rodrigues rotation of vector v about a unit axis."""
    axis = axis / np.linalg.norm(axis)
    c, s = math.cos(ang), math.sin(ang)
    return v * c + np.cross(axis, v) * s + axis * np.dot(axis, v) * (1 - c)


def airway_tree(rng: np.random.Generator, nx, ny, nz, generations=6, r0=9.0,
                radius_ratio=0.79, length_ratio=0.8, angle_deg=35.0):
    """Capsules of a bifurcating airway tree starting at the top slice."""
    s = nx / 512.0
    start = np.array([nx / 2.0, ny * 0.45, -2.0])
    d0 = np.array([0.0, 0.0, 1.0])
    L0 = max(8.0, 0.30 * nz)
    segs = []

    def grow(p, d, length, r, gen, k):
        q = p + d * length
        segs.append((p.copy(), q.copy(), r))
        if gen >= generations:
            return
        # alternate the branching plane so the tree fills both lungs in 3-D
        perp = np.array([0.0, 1.0, 0.0]) if gen % 2 == 0 else np.cross(d, np.array([0.0, 1.0, 0.0]))
        if np.linalg.norm(perp) < 1e-6:
            perp = np.array([1.0, 0.0, 0.0])
        for sign in (-1.0, 1.0):
            jit = math.radians(rng.uniform(-5.0, 5.0))
            nd = _rotate(d, perp, sign * math.radians(angle_deg) + jit)
            nd = nd / np.linalg.norm(nd)
            grow(q, nd, length * length_ratio, r * radius_ratio, gen + 1, k * 2 + (sign > 0))

    grow(start, d0, L0, r0 * s, 0, 1)
    rows = [_capsule_row(a, b, r, nx, ny, nz) for a, b, r in segs]
    return np.array(rows, np.int32).reshape(-1, CAPSULE_FIELDS)


def _geometry(nx, ny):
    s = nx / 512.0
    t = ny / 512.0
    body = (int(round(nx / 2)), int(round(ny / 2)), max(1, int(round(220 * s))), max(1, int(round(160 * t))))
    lungs = ((int(round(nx / 2 - 95 * s)), int(round(ny / 2)), max(1, int(round(75 * s))), max(1, int(round(120 * t)))),
             (int(round(nx / 2 + 95 * s)), int(round(ny / 2)), max(1, int(round(75 * s))), max(1, int(round(120 * t)))))
    return body, lungs


def slice_phantom(seed: int, nx: int = 512, ny: int = 512, ndiscs=None, noise_sd: int = 10) -> PhantomSpec:
    """One slice with 6-10 airway discs of radius 2..8 px."""
    rng = np.random.default_rng(seed)
    body, lungs = _geometry(nx, ny)
    n = int(rng.integers(6, 11)) if ndiscs is None else ndiscs
    rows = []
    for i in range(n):
        if i == 0:   # trachea-like disc between the lungs
            cx, cy = nx / 2.0, ny * 0.45
        else:
            lx, ly, la, lb = lungs[i % 2]
            ang = rng.uniform(0, 2 * math.pi)
            rad = math.sqrt(rng.uniform(0, 0.6))
            cx, cy = lx + la * rad * math.cos(ang), ly + lb * rad * math.sin(ang)
        r = rng.uniform(2.0, 8.0) * nx / 512.0
        p = (cx, cy, 0.5)
        rows.append(_capsule_row(p, p, r, nx, ny, 1))
    caps = np.array(rows, np.int32).reshape(-1, CAPSULE_FIELDS)
    return PhantomSpec(nx, ny, 1, seed, noise_sd=noise_sd, body=body, lungs=lungs, capsules=caps)


def chest_volume(seed: int, nx: int = 512, ny: int = 512, nz: int = 400, generations: int = 6,
                 noise_sd: int = 10, vol_id: int = 0) -> PhantomSpec:
    """Chest volume with an airway tree of the given number of bifurcations."""
    rng = np.random.default_rng(seed)
    body, lungs = _geometry(nx, ny)
    caps = airway_tree(rng, nx, ny, nz, generations)
    return PhantomSpec(nx, ny, nz, seed, vol_id=vol_id, noise_sd=noise_sd, body=body, lungs=lungs,
                       capsules=caps)


def batch_specs(seed: int, nvol: int = 64, nx: int = 512, ny: int = 512, dmin: int = 120, dmax: int = 600):
    """Uneven batch: depths, sensor noise and tree depth drawn per volume."""
    rng = np.random.default_rng(seed)
    specs = []
    for v in range(nvol):
        nz = int(rng.integers(dmin, dmax + 1))
        sd = int(rng.integers(5, 31))
        gens = int(rng.integers(4, 9))
        specs.append(chest_volume(seed * 1000 + v, nx, ny, nz, gens, sd, vol_id=v))
    return specs


# ---------------------------------------------------------------- building

def build(verbose: bool = False, cuda: bool = True) -> None:
    """Compile the host generator (gcc) and, if asked, the CUDA one (nvcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "phantom.h")
    host_src = os.path.join(_HERE, "phantom_host.c")
    cu_src = os.path.join(_HERE, "phantom_cuda.cu")
    jobs = []
    if _stale(_HOST_SO, [hdr, host_src]):
        jobs.append(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", host_src, "-o", _HOST_SO])
    if cuda and _stale(_CUDA_SO, [hdr, cu_src]):
        jobs.append(["nvcc", "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                     "-Xcompiler", "-fPIC", "-shared", cu_src, "-o", _CUDA_SO])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("phantom build failed: %s\n%s" % (" ".join(j), out.decode()))
        if verbose and out:
            print(out.decode())


def _stale(target, srcs):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in srcs)


_host_lib = None
_cuda_lib = None


def _host():
    global _host_lib
    with _lock:
        if _host_lib is None:
            build(cuda=False)
            lib = ctypes.CDLL(_HOST_SO)
            lib.ph_generate_host.argtypes = [ctypes.POINTER(_Desc), ctypes.c_void_p, ctypes.c_int]
            lib.ph_generate_host.restype = ctypes.c_int
            _host_lib = lib
    return _host_lib


def _cuda():
    global _cuda_lib
    with _lock:
        if _cuda_lib is None:
            build(cuda=True)
            lib = ctypes.CDLL(_CUDA_SO)
            lib.ph_generate_cuda.argtypes = [ctypes.POINTER(_Desc), ctypes.c_void_p, ctypes.c_void_p]
            lib.ph_generate_cuda.restype = ctypes.c_int
            _cuda_lib = lib
    return _cuda_lib


def _desc(spec: PhantomSpec, caps_ptr, off_ptr, idx_ptr) -> _Desc:
    d = _Desc()
    d.nx, d.ny, d.nz = spec.nx, spec.ny, spec.nz
    d.seed = spec.seed & 0xFFFFFFFFFFFFFFFF
    d.vol_id = spec.vol_id
    d.air_hu = spec.air_hu
    d.body_mu, d.body_sd = spec.body_mu, spec.body_sd
    d.lung_mu, d.lung_sd = spec.lung_mu, spec.lung_sd
    d.airway_mu, d.airway_sd = spec.airway_mu, spec.airway_sd
    d.noise_sd = spec.noise_sd
    d.body = _Ellipse(*spec.body)
    d.lung[0] = _Ellipse(*spec.lungs[0])
    d.lung[1] = _Ellipse(*spec.lungs[1])
    d.ncaps = len(spec.capsules)
    d.caps, d.slice_off, d.slice_caps = caps_ptr, off_ptr, idx_ptr
    return d


def generate_host(spec: PhantomSpec, nthreads: int | None = None) -> np.ndarray:
    """int16 volume [nz][ny][nx] generated on the host."""
    caps = np.ascontiguousarray(spec.capsules, np.int32)
    if caps.size == 0:
        caps = np.zeros((1, CAPSULE_FIELDS), np.int32)
    off, idx = spec.slice_csr()
    out = np.empty((spec.nz, spec.ny, spec.nx), np.int16)
    d = _desc(spec, caps.ctypes.data, off.ctypes.data, idx.ctypes.data)
    n = nthreads or min(os.cpu_count() or 1, 32)
    rc = _host().ph_generate_host(ctypes.byref(d), out.ctypes.data, n)
    if rc != 0:
        raise RuntimeError("ph_generate_host failed with code %d" % rc)
    return out


def generate_cuda(spec: PhantomSpec, out=None, device="cuda"):
    """int16 volume generated on the GPU into a torch tensor (allocated if None)."""
    import torch
    caps = np.ascontiguousarray(spec.capsules, np.int32)
    if caps.size == 0:
        caps = np.zeros((1, CAPSULE_FIELDS), np.int32)
    off, idx = spec.slice_csr()
    dcaps = torch.from_numpy(caps).to(device)
    doff = torch.from_numpy(off).to(device)
    didx = torch.from_numpy(idx).to(device)
    if out is None:
        out = torch.empty((spec.nz, spec.ny, spec.nx), dtype=torch.int16, device=device)
    assert out.is_contiguous() and out.dtype == torch.int16 and out.numel() == spec.nvox
    d = _desc(spec, dcaps.data_ptr(), doff.data_ptr(), didx.data_ptr())
    stream = torch.cuda.current_stream(out.device).cuda_stream
    rc = _cuda().ph_generate_cuda(ctypes.byref(d), out.data_ptr(), stream)
    if rc != 0:
        raise RuntimeError("ph_generate_cuda failed with code %d" % rc)
    torch.cuda.current_stream(out.device).synchronize()  # keep capsule buffers alive until done
    return out
