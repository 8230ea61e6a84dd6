"""Benchmark of the maximum-Tsallis-entropy thresholding step on GB300.

Workload: synthetic chest CT volume 512x512x400 int16 (seeded phantom: body
N(40,20) HU, lungs N(-850,60), airway tree r=9 px with 6 bifurcations
N(-1000,15), outside air -1024, sensor noise sd 10), per-slice thresholds,
4096 levels over [-1024, 3071], 1-D Tsallis q = 0.8, uint8 mask. One step is
one pass of the whole path over the volume: histogram, exhaustive objective,
argmax (FP64 re-rank of near ties), binarise -- one launch of the fused
persistent kernel.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on
the same workload instead (bounded samples per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX, NY, NZ = 512, 512, 400
SEED = 2012106842
Q = 0.8
BYTES_PER_VOXEL = 3          # 2 B read + 1 B mask write; the re-read of a slice hits L2
BATCH_SEED = 2012106844
BATCH_BYTES_PER_VOXEL = 5    # per-volume thresholds: the volume is read twice (2 + 2) and the mask written
METRIC = "voxels/s segmented (hist+Tsallis search+binarize) on 1 GB300, % HBM roofline"
WORKLOAD = "chest phantom 512x512x400 int16, per-slice 1-D Tsallis q=0.8, 4096 levels, uint8 mask"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# the sources each per-slice kernel is built from (a profile's traffic figure
# is used only while they are unchanged)
KERNEL_SOURCES = {
    "k_segment1d": ("common.cuh", "dfmath.cuh", "top.cuh", "search1d.cuh", "seg1d.cu", "kernels.h"),
    "k_slice_pipe": ("common.cuh", "dfmath.cuh", "top.cuh", "search1d.cuh", "firstpass.cuh", "seg_pipe.cu",
                     "kernels.h"),
    "k_slice_spec": ("common.cuh", "dfmath.cuh", "top.cuh", "search1d.cuh", "firstpass.cuh", "seg_spec.cu",
                     "kernels.h"),
}
SLICE_KERNEL_NAMES = {"auto": "k_segment1d", "tiles": "k_segment1d", "pipeline": "k_slice_pipe",
                      "predict": "k_slice_spec"}


def _kernel_source_sha(kernel="k_segment1d"):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2012_10684_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _profiled_traffic(nvox, kernel="k_segment1d"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "%s_chest512x512x400.md" % kernel)
    try:
        text = open(path).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel source sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram bytes per launch:\s*([0-9.eE+]+)", text)
    m_v = re.search(r"voxels per launch:\s*([0-9]+)", text)
    if not (m_sha and m_b and m_v) or m_sha.group(1) != _kernel_source_sha(kernel):
        return None
    return float(m_b.group(1)) * nvox / float(m_v.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background (read-only
    queries). nvidia-smi writes the log itself (-f), which it flushes line by
    line; it is stopped with SIGINT so that it closes the file."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, uuid=None):
        self.index = index
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        sel = ("GPU-" + self.uuid) if self.uuid else str(self.index)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", sel, "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        if self.proc is not None:
            import signal
            time.sleep(0.25)   # at least one sample after the timed region
            self.proc.send_signal(signal.SIGINT)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        return rows

    @staticmethod
    def summarise(rows):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def _dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != n:
        if n > 1:
            raise SystemExit("--gpus %d needs torchrun with %d ranks (WORLD_SIZE=%d)" % (n, n, world))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity on one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    """The CPU oracle on the same workload: each step a bounded slab of slices."""
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import phantom

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    vol = phantom.generate_host(phantom.chest_volume(SEED, NX, NY, NZ))
    # size a step so that warm-up + timed steps take about a minute in total
    t0 = time.perf_counter()
    oracle.segment1d(vol[:cores], NX * NY, Q, nthreads=cores)
    per_slice = max((time.perf_counter() - t0) / cores, 1e-5)
    budget = 60.0 / max(args.steps + args.warmup, 1)
    nsl = int(max(1, min(NZ, budget / per_slice)))
    for i in range(args.warmup):
        z0 = (i * nsl) % (NZ - nsl + 1)
        oracle.segment1d(vol[z0:z0 + nsl], NX * NY, Q, nthreads=cores)
    t0 = time.perf_counter()
    for i in range(args.steps):
        z0 = (i * nsl) % (NZ - nsl + 1)
        oracle.segment1d(vol[z0:z0 + nsl], NX * NY, Q, nthreads=cores)
    dt = time.perf_counter() - t0
    value = args.steps * nsl * NX * NY / dt
    sample = "%d of %d slices per step (threads over slices), %d steps" % (nsl, NZ, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (CPU oracle, FP64)", "nx": NX, "ny": NY,
                                             "nz": NZ, "q": Q, "mode": "per-slice", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(vol_np, seconds=12.0):
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    passes = 0
    t0 = time.perf_counter()
    while True:
        oracle.segment1d(vol_np, NX * NY, Q, nthreads=cores)
        passes += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or passes >= 5000:
            break
    return {"value": passes * vol_np.size / dt, "unit": "voxels/s", "cores": cores, "kind": "oracle",
            "sample": "%d full passes over the 512x512x400 volume (per-slice, FP64 prefix mode, "
                      "threads over slices), %.1f s" % (passes, dt)}


def batch_leg(dev, steps=20, warmup=3, nvol=64, dmax=600):
    """The 64-volume batch (512x512xD chest phantoms, D uniform in [120, 600],
    noise sd in [5, 30] HU, 4-8 airway generations, q = 0.8, one threshold
    per volume): autotuned launch shape, one persistent launch per step,
    replayed from a CUDA graph. Returns the JSON object of this leg."""
    import torch

    import phantom
    import paper_2012_10684_gb300 as tg
    specs = phantom.batch_specs(BATCH_SEED, nvol=nvol, dmin=min(120, dmax), dmax=dmax)
    vols = [phantom.generate_cuda(sp, device=dev) for sp in specs]
    nvox = sum(v.numel() for v in vols)
    p = tg.tsallis_params(q=Q, mode="volume")
    masks = [torch.empty(v.shape, dtype=torch.uint8, device=dev) for v in vols]
    outs = (torch.empty(nvol, dtype=torch.int32, device=dev), torch.empty(nvol, dtype=torch.float32, device=dev),
            torch.empty(nvol, dtype=torch.int32, device=dev))
    tile, bps, tune_ms = tg.tsallis_autotune_batch(vols, p, masks, outs)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        tg.tsallis_segment_batch(vols, p, masks, outs)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            tg.tsallis_segment_batch(vols, p, masks, outs)
    torch.cuda.current_stream(dev).wait_stream(s)
    torch.cuda.synchronize(dev)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    for _ in range(steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    st = outs[2].cpu()
    assert bool(((st & 0xff) == 0).all()), "a volume failed"
    peak, _ = _peaks()
    achieved = BATCH_BYTES_PER_VOXEL * nvox / (ms / 1e3) / 1e9
    res = {"workload": "%d chest phantoms 512x512xD, D~U[%d,%d], noise sd U[5,30], q=0.8, per-volume thresholds"
                       % (nvol, min(120, dmax), dmax),
           "voxels": nvox, "value": nvox / (ms / 1e3), "unit": "voxels/s", "ms_per_step": ms, "steps": steps,
           "launch": "CUDA graph: group-table kernel + one persistent kernel",
           "autotuned": {"tile_vox": tile, "blocks_per_sm": bps, "ms": tune_ms},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "bytes_per_voxel": BATCH_BYTES_PER_VOXEL,
                        "basis": "algorithmic bytes (the volume read twice and the mask written); the tail of each "
                                 "volume's second read hits L2, so DRAM moves fewer bytes and frac can exceed 1"}}
    res["proposer"] = proposer_legs(dev, vols, masks, outs, outs[0].clone())
    tg.set_launch_shape()
    del vols, masks, g
    torch.cuda.empty_cache()
    return res


def _time_batch(dev, vols, p, masks, outs, steps, warmup):
    import torch

    import paper_2012_10684_gb300 as tg
    for _ in range(warmup):
        tg.tsallis_segment_batch(vols, p, masks, outs)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    for _ in range(steps):
        tg.tsallis_segment_batch(vols, p, masks, outs)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / steps


def proposer_legs(dev, vols, masks, outs, ref_t, steps=10, warmup=3):
    """The 64-volume batch with the trained proposer, two ways:
    - window: histograms, the proposer's top-64 window with its certificate
      and fallback, then Algorithm 1 (the volume read twice);
    - first pass: the proposer predicts each volume's threshold from the
      histogram of its middle sixteenth, the histogram pass binarises with
      it and lists voxels within 8 levels; volumes whose exact threshold is
      within 8 levels are finished by rewriting listed voxels, others are
      binarised again;
    and, for comparison, the first pass with the prediction taken from the
    exhaustive search of the same sixteenth (no proposer).
    Each reports voxels/s and the thresholds that differ from the exhaustive
    path's (must be none)."""
    import paper_2012_10684_gb300 as tg
    weights = os.path.join(ROOT, "paper_2012_10684_gb300", "proposer_weights.bin")
    if not os.path.exists(weights):
        return {"unavailable": "no trained proposer weights in the package"}
    tg.proposer_load(weights, dev)
    nvox = sum(v.numel() for v in vols)
    out = {}
    legs = (("window", tg.tsallis_params(q=Q, mode="volume", topk=64)),
            ("first_pass_proposer", tg.tsallis_params(q=Q, mode="volume", flags=tg.TSALLIS_FLAG_PREDICT_PROPOSER)),
            ("first_pass_subsample", tg.tsallis_params(q=Q, mode="volume",
                                                       flags=tg.TSALLIS_FLAG_PREDICT_SUBSAMPLE)))
    for name, p in legs:
        ms = _time_batch(dev, vols, p, masks, outs, steps, warmup)
        st = outs[2].cpu()
        r = {"value": nvox / (ms / 1e3), "unit": "voxels/s", "ms_per_step": ms, "steps": steps,
             "threshold_misses_after_fallback": int((outs[0] != ref_t).sum().item())}
        if name == "window":
            r["window_hit_rate"] = ((st & tg.TSALLIS_STATUS_WINDOW_HIT) != 0).float().mean().item()
            r["mean_blocks_searched_of_64"] = ((st >> tg.TSALLIS_STATUS_FALLBACK_SHIFT) & 0xff).float().mean().item()
        else:
            r["volumes_without_second_read"] = int(((st & tg.TSALLIS_STATUS_FIRST_PASS_EXACT) != 0).sum().item())
        out[name] = r
    return out


def two_d_leg(dev, steps=10, warmup=3):
    """The 2-D form on a 512x512x256 chest phantom: grey level (4096 levels
    >> 4) x 3x3x3 floor-mean level, 65,536-bin histogram, exhaustive (t, s)
    search over summed-area tables with an FP64 re-rank of near ties,
    Algorithm 1 on the grey level with t; one threshold pair for the volume.
    Algorithmic bytes: 5 per voxel (the histogram pass reads the volume,
    the binarise pass reads it again and writes the mask)."""
    import torch

    import phantom
    import paper_2012_10684_gb300 as tg
    vol = phantom.generate_cuda(phantom.chest_volume(2012106843, NX, NY, 256), device=dev)
    p = tg.tsallis_params(q=Q, mode="volume", two_d=True)
    mask = torch.empty(vol.shape, dtype=torch.uint8, device=dev)
    t = torch.empty((1, 2), dtype=torch.int32, device=dev)
    phi = torch.empty(1, dtype=torch.float32, device=dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    for _ in range(warmup):
        tg.tsallis_segment(vol, p, mask, t, phi, st)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    for _ in range(steps):
        tg.tsallis_segment(vol, p, mask, t, phi, st)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    assert int(st[0].item()) & 0xff == 0
    peak, _ = _peaks()
    achieved = 5 * vol.numel() / (ms / 1e3) / 1e9
    # the search alone on this volume's histogram: summed-area tables against
    # the paper's organisation (one thread per pair, quadrants summed directly)
    h = tg.tsallis_histogram(vol, p)
    search = {}
    for name, pf in (("summed_area", p), ("brute_force", tg.tsallis_params(q=Q, mode="volume", two_d=True,
                                                                           flags=tg.TSALLIS_FLAG_BRUTE_FORCE_2D))):
        for _ in range(warmup):
            r = tg.tsallis_search(h, pf)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            r = tg.tsallis_search(h, pf)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        search[name] = {"ms": e0.elapsed_time(e1) / steps, "t_s": [int(x) for x in r[0][0].tolist()]}
    # brute force: sum over pairs of the quadrant cells each visits, 2 (sum_{a<L2} a)^2
    # for L2 = 256; each visit is one integer add and a six-flop FP32 two-sum;
    # peak 128 FP32 lanes per clock per SM at the maximum SM clock
    L2 = 256
    visits = 2 * (L2 * (L2 - 1) // 2) ** 2
    props = torch.cuda.get_device_properties(dev)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        mhz = 2070.0
    fp_peak = 128 * props.multi_processor_count * mhz * 1e6 / 1e12
    fp_ach = 6 * visits / (search["brute_force"]["ms"] / 1e3) / 1e12
    search["brute_force"]["roofline"] = {"bound": "fp32", "achieved": fp_ach, "peak": fp_peak, "unit": "TFLOP/s",
                                         "frac": fp_ach / fp_peak, "cell_visits": visits}
    # the learned proposer's certified window (16 candidate cells of 4 x 4
    # pairs), on this volume's histogram and on its 256 slice histograms
    w2d = os.path.join(ROOT, "paper_2012_10684_gb300", "proposer2d_weights.bin")
    if os.path.exists(w2d):
        tg.proposer_select(1, dev)
        tg.proposer_load(w2d, dev)
        tg.proposer_select(0, dev)
        hs = tg.tsallis_histogram(vol, tg.tsallis_params(q=Q, mode="slice", two_d=True))
        for label, hh in (("volume", h), ("slices", hs)):
            out = {}
            for name, pf in (("exhaustive", tg.tsallis_params(q=Q, two_d=True)),
                             ("window16", tg.tsallis_params(q=Q, two_d=True, topk=16))):
                for _ in range(warmup):
                    r = tg.tsallis_search(hh, pf)
                torch.cuda.synchronize(dev)
                e0.record(stream)
                for _ in range(steps):
                    r = tg.tsallis_search(hh, pf)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                out[name] = {"ms": e0.elapsed_time(e1) / steps}
                if name == "window16":
                    stw = r[2].cpu()
                    out[name]["hit_rate"] = float(((stw & tg.TSALLIS_STATUS_WINDOW_HIT) != 0).float().mean())
                    out[name]["mean_cells_searched"] = float(((stw >> tg.TSALLIS_STATUS_FALLBACK_SHIFT) & 0xff)
                                                             .float().mean())
                    out[name]["same_as_exhaustive"] = bool(torch.equal(r[0], ref_t))
                else:
                    ref_t = r[0]
            search["proposer_window_" + label] = dict(out, histograms=int(hh.shape[0]))
    return {"workload": "chest phantom 512x512x256, 2-D grey x 3x3x3 mean, q=0.8, one (t, s) for the volume",
            "value": vol.numel() / (ms / 1e3), "unit": "voxels/s", "ms_per_step": ms, "steps": steps,
            "t_s": [int(x) for x in t[0].tolist()], "search_only": search,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_voxel": 5}}


def preprocess_leg(dev, steps=10, warmup=3, nz=NZ):
    """The steps before the threshold (8-bit levels, chest-mask opening with
    the disk of radius 10 and subtraction, 256-level slice histograms) in
    one launch, and the paper's whole segmentation step (that launch, the
    per-slice Tsallis search on 256 levels, Algorithm 1) on the 512x512x400
    chest phantom. Algorithmic bytes of the fused kernel: 4 per voxel (read
    the CT number, write the level); of the whole step: 7 (plus the
    binarise pass: read the level, write the mask)."""
    import torch

    import phantom
    import paper_2012_10684_gb300 as tg
    vol = phantom.generate_cuda(phantom.chest_volume(2012106842, NX, NY, nz), device=dev)
    pp = tg.preprocess_params()
    lev = torch.empty(vol.shape, dtype=torch.int16, device=dev)
    hist = torch.empty((nz, 256), dtype=torch.int32, device=dev)
    mask = torch.empty(vol.shape, dtype=torch.uint8, device=dev)
    p = tg.tsallis_params(q=Q, lo=0, nbins=256, mode="slice")
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    ms_pre = timed(lambda: tg.tsallis_preprocess(vol, pp, out=lev, hist=hist))
    res = {}

    def step():
        tg.tsallis_preprocess(vol, pp, out=lev, hist=hist)
        t, _, st = tg.tsallis_search(hist, p)
        tg.tsallis_binarize(lev, t, p, out=mask)
        res["st"] = st
    ms_step = timed(step)
    assert int((res["st"] & 0xff).max().item()) == 0
    peak, _ = _peaks()
    n = vol.numel()
    achieved = 4 * n / (ms_pre / 1e3) / 1e9
    # ALU roofline: the chord method needs, per pixel and pass, 2R extremes
    # for the chords of half-width 1..R and 2R to fold the 2R+1 chords of the
    # disk: 4R scalar min/max, 2R fp16x2 instructions; two passes (opening).
    # Peak: 64 ALU lanes per clock per SM x SMs x maximum SM clock.
    r = pp.radius
    alu_ops = 2 * 2 * r * n
    props = torch.cuda.get_device_properties(dev)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
        src = "sm_max_mhz of MEASURED_PEAKS.json"
    except (OSError, KeyError, ValueError):
        mhz, src = 2070.0, "nominal max SM clock"
    alu_peak = 64 * props.multi_processor_count * mhz * 1e6 / 1e9
    alu_ach = alu_ops / (ms_pre / 1e3) / 1e9
    return {"workload": "chest phantom 512x512x%d: 8-bit levels, chest-mask opening (disk radius 10), "
                        "slice histograms; then per-slice Tsallis q=0.8 on 256 levels and Algorithm 1" % nz,
            "preprocess": {"value": n / (ms_pre / 1e3), "unit": "voxels/s", "ms": ms_pre,
                           "roofline": {"bound": "alu", "achieved": alu_ach, "peak": alu_peak,
                                        "unit": "G fp16x2 min/max per s", "frac": alu_ach / alu_peak,
                                        "ops_per_voxel": 4 * r, "peak_basis": "64 lanes/clk/SM, " + src},
                           "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                   "bytes_per_voxel": 4}},
            "segmentation_step": {"value": n / (ms_step / 1e3), "unit": "voxels/s", "ms": ms_step,
                                  "launches": 3},
            "steps": steps}


def _timed(dev, fn, steps, warmup):
    """CUDA-event time per call of fn(i), after warm-up."""
    import torch
    for i in range(warmup):
        fn(i)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        fn(i)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / steps


def _hbm(nvox, ms, bytes_per_voxel):
    peak, kind = _peaks()
    ach = bytes_per_voxel * nvox / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "bytes_per_voxel": bytes_per_voxel, "basis": "algorithmic bytes", "peak_source": kind}


def copy_bound(dev, h_vol, h_mask, d_vol, d_mask, reps=20):
    """The rate the host link allows the host-buffer call: plain
    page-locked copies of the step's bytes (the volume in, the mask out),
    the two directions overlapped on two streams."""
    import torch
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def once():
        with torch.cuda.stream(s1):
            d_vol.copy_(h_vol, non_blocking=True)
        with torch.cuda.stream(s2):
            h_mask.copy_(d_mask, non_blocking=True)
    for _ in range(3):
        once()
    torch.cuda.synchronize(dev)
    ev[0].record(s1)
    s2.wait_event(ev[0])
    for _ in range(reps):
        once()
    ev[1].record(s2)
    s1.wait_event(ev[1])
    ev[2].record(s1)
    torch.cuda.synchronize(dev)
    ms = ev[0].elapsed_time(ev[2]) / reps
    nvox = d_vol.numel()
    return {"value": nvox / (ms / 1e3), "unit": "voxels/s", "ms_per_step": ms,
            "h2d_GBps": 2 * nvox / (ms / 1e3) / 1e9, "d2h_GBps": nvox / (ms / 1e3) / 1e9,
            "method": "cudaMemcpyAsync of the 209.7 MB volume H2D and the 104.9 MB mask D2H, overlapped on two "
                      "streams, page-locked buffers, %d repetitions" % reps}


def per_slice_legs(dev, vols, masks, outs, args, steps=200, warmup=10):
    """The rest of the 512x512x400 workload (two alternated volumes): per-slice
    thresholds at q = 0.5 and 1.5, each per-slice kernel at q = 0.8, the
    same step as three calls (histogram, search and binarise; the volume read
    twice from HBM), whole-volume thresholds at every q, and the single
    512x512 slice."""
    import torch

    import phantom
    import paper_2012_10684_gb300 as tg
    nvox = vols[0].numel()
    res = {}

    def run(p):
        return lambda i: tg.tsallis_segment(vols[i & 1], p, masks[i & 1], *outs[i & 1])
    out = {}
    for q in (0.5, 1.5):
        ms = _timed(dev, run(tg.tsallis_params(q=q, mode="slice")), steps, warmup)
        out["q%g" % q] = {"value": nvox / (ms / 1e3), "unit": "voxels/s", "ms": ms, "roofline": _hbm(nvox, ms, 3)}
    res["per_slice_q"] = out
    out = {}
    for kind in ("tiles", "pipeline", "predict"):
        tg.set_slice_kernel(kind)
        ms = _timed(dev, run(tg.tsallis_params(q=Q, mode="slice")), steps, warmup)
        st = outs[0][2]
        out[kind] = {"value": nvox / (ms / 1e3), "unit": "voxels/s", "ms": ms, "roofline": _hbm(nvox, ms, 3),
                     "ok": bool(((st & 0xff) == 0).all().item())}
    tg.set_slice_kernel("auto")
    res["slice_kernels_q0.8"] = out
    # the step as three calls: every slice histogram, the 400 searches, the binarise pass
    p = tg.tsallis_params(q=Q, mode="slice")
    hs = [tg.tsallis_histogram(v, p) for v in vols]
    ts = [tg.tsallis_search(h, p)[0] for h in hs]

    def two_pass(i):
        k = i & 1
        tg.tsallis_histogram(vols[k], p, hs[k])
        t, _, _ = tg.tsallis_search(hs[k], p)
        tg.tsallis_binarize(vols[k], t, p, masks[k])
    ms = _timed(dev, two_pass, steps, warmup)
    res["two_pass"] = {"value": nvox / (ms / 1e3), "unit": "voxels/s", "ms": ms, "calls": 3,
                       "roofline": _hbm(nvox, ms, 5), "roofline_3B": _hbm(nvox, ms, 3),
                       "note": "histogram pass, 400 searches, binarise pass from HBM (5 B/voxel of traffic)"}
    del hs, ts
    out = {}
    o1 = [(torch.empty(1, dtype=torch.int32, device=dev), torch.empty(1, dtype=torch.float32, device=dev),
           torch.empty(1, dtype=torch.int32, device=dev)) for _ in vols]
    for q in (0.5, 0.8, 1.5):
        pv = tg.tsallis_params(q=q, mode="volume")
        ms = _timed(dev, lambda i: tg.tsallis_segment(vols[i & 1], pv, masks[i & 1], *o1[i & 1]), steps, warmup)
        out["q%g" % q] = {"value": nvox / (ms / 1e3), "unit": "voxels/s", "ms": ms, "roofline": _hbm(nvox, ms, 5),
                          "t": int(o1[0][0].item())}
    res["whole_volume"] = out
    # one 512x512 slice (the single-slice workload): latency of one call
    sl = phantom.generate_cuda(phantom.slice_phantom(SEED, NX, NY), device=dev)
    ps = tg.tsallis_params(q=Q, mode="slice")
    m1 = torch.empty(sl.shape, dtype=torch.uint8, device=dev)
    r1 = (torch.empty(1, dtype=torch.int32, device=dev), torch.empty(1, dtype=torch.float32, device=dev),
          torch.empty(1, dtype=torch.int32, device=dev))
    ms = _timed(dev, lambda i: tg.tsallis_segment(sl, ps, m1, *r1), 2000, 50)
    res["single_slice"] = {"workload": "one 512x512 phantom slice, q=0.8, 4096 levels", "latency_us": ms * 1e3,
                           "value": sl.numel() / (ms / 1e3), "unit": "voxels/s", "t": int(r1[0].item()),
                           "note": "back-to-back calls on one stream; one launch each"}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-volume batch leg")
    ap.add_argument("--no-legs", action="store_true", help="skip the per-slice / whole-volume / single-slice legs")
    ap.add_argument("--slice-kernel", default="auto", choices=sorted(SLICE_KERNEL_NAMES),
                    help="per-slice kernel of the headline step (default: the library's choice)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batch leg (for profiling; prints the leg's JSON object)")
    ap.add_argument("--batch-nvol", type=int, default=64)
    ap.add_argument("--batch-dmax", type=int, default=600)
    ap.add_argument("--preprocess-only", action="store_true",
                    help="print only the pre-processing / chest-mask leg (for profiling)")
    ap.add_argument("--preprocess-nz", type=int, default=NZ, help="slices of the pre-processing leg's volume")
    ap.add_argument("--two-d-only", action="store_true", help="print only the 2-D leg (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = _dist_setup(args.gpus)
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return rc

    import numpy as np
    import torch

    import phantom
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if args.two_d_only:
        torch.cuda.set_device(local)
        print(json.dumps(two_d_leg(torch.device("cuda", local))), flush=True)
        return 0
    if args.preprocess_only:
        torch.cuda.set_device(local)
        print(json.dumps(preprocess_leg(torch.device("cuda", local), nz=args.preprocess_nz)), flush=True)
        return 0
    if args.batch_only:
        torch.cuda.set_device(local)
        print(json.dumps(batch_leg(torch.device("cuda", local), nvol=args.batch_nvol, dmax=args.batch_dmax)),
              flush=True)
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    import paper_2012_10684_gb300 as tg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # two volumes alternated step by step (each larger than L2)
    vol_np = phantom.generate_host(phantom.chest_volume(SEED, NX, NY, NZ))
    vols = [torch.from_numpy(vol_np).to(dev), phantom.generate_cuda(phantom.chest_volume(SEED + 1, NX, NY, NZ), device=dev)]
    p = tg.tsallis_params(q=Q, mode="slice")
    nvox = vols[0].numel()
    masks = [torch.empty(v.shape, dtype=torch.uint8, device=dev) for v in vols]
    outs = [(torch.empty(NZ, dtype=torch.int32, device=dev), torch.empty(NZ, dtype=torch.float32, device=dev),
             torch.empty(NZ, dtype=torch.int32, device=dev)) for _ in vols]
    stream = torch.cuda.current_stream(dev)

    def step(i):
        tg.tsallis_segment(vols[i & 1], p, masks[i & 1], *outs[i & 1])

    tg.set_slice_kernel(args.slice_kernel)
    kernel = SLICE_KERNEL_NAMES[args.slice_kernel]
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except (AttributeError, RuntimeError):
        uuid = None
    sampler = ClockSampler(local, uuid)
    sampler.start()
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler.summarise(sampler.stop())
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, dev)
    status = np.concatenate([o[2].cpu().numpy() for o in outs])
    assert np.all((status & 0xff) == 0), "a slice failed: %s" % status[(status & 0xff) != 0][:5]

    # end to end through the host-buffer entry point: the volume is read from
    # page-locked host memory and the mask, thresholds, values and statuses
    # written back to it, the copies pipelined with the kernels by the call
    k_e2e = max(10, min(args.steps, 300))
    h_vol = torch.from_numpy(vol_np).pin_memory()
    h_mask = torch.empty(vols[0].shape, dtype=torch.uint8).pin_memory()
    h_t = torch.empty(NZ, dtype=torch.int32).pin_memory()
    h_phi = torch.empty(NZ, dtype=torch.float32).pin_memory()
    h_st = torch.empty(NZ, dtype=torch.int32).pin_memory()
    for _ in range(3):
        tg.tsallis_segment_host(h_vol, p, h_mask, h_t, h_phi, h_st, device=dev, sync=False)
    torch.cuda.synchronize(dev)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(k_e2e):
        tg.tsallis_segment_host(h_vol, p, h_mask, h_t, h_phi, h_st, device=dev, sync=False)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), world, dev)
    copy = copy_bound(dev, h_vol, h_mask, vols[0], masks[0])

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    value = world * nvox * args.steps / (ms_max / 1e3)
    peak, peak_kind = _peaks()
    per_launch_s = ms / 1e3 / args.steps
    achieved = BYTES_PER_VOXEL * nvox / per_launch_s / 1e9
    traffic = _profiled_traffic(nvox, kernel)
    e2e_value = world * nvox * k_e2e / (e2e_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "nz": NZ, "q": Q, "mode": "per-slice",
                   "levels": 4096, "slice_kernel": args.slice_kernel + " (" + kernel + ")",
                   "l2": "two 210 MB volumes (and their 105 MB masks) alternated step by step, each larger than L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                     "algorithmic_bytes_per_launch": BYTES_PER_VOXEL * nvox,
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s"},
        "e2e": {"value": e2e_value, "unit": "voxels/s",
                "h2d_bytes_per_step": nvox * 2, "d2h_bytes_per_step": nvox + NZ * 12, "steps": k_e2e,
                "call": "tsallis_segment_host (page-locked host buffers, copies pipelined with the kernels)",
                "copy_bound": dict(copy, frac=e2e_value / copy["value"])},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "rerank_slices": int(((status & tg.TSALLIS_STATUS_RERANKED) != 0).sum()),
    }
    if not args.no_legs:
        line.update(per_slice_legs(dev, vols, masks, outs, args))
    if not args.no_batch:
        line["two_d"] = two_d_leg(dev)
        line["preprocess"] = preprocess_leg(dev)
        line["batch"] = batch_leg(dev)
        line["gpu_launches_batch"] = 2 * line["batch"]["steps"]
    if not args.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline(vol_np)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
