"""tsallis_segment_static, the entry point for callers that cannot allocate
device memory (for example code whose device memory all belongs to a
framework's pool, or that must not allocate after start-up): through the C
ABI it must give the same thresholds, objective values, statuses and masks as
tsallis_segment, on two calls in a row (the second call reuses the fixed
scratch the first one left behind).

This file is named to be collected last, and it builds what it needs, so it
also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import phantom
import paper_2012_10684_gb300 as tg

pytestmark = pytest.mark.gpu

PHI_RTOL = 1e-5
GAP = 1e-9


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    L = tg.lib()
    f = L.tsallis_segment_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(tg.Params),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L


def _static_call(L, vol, p):
    nz, ny, nx = vol.shape
    nh = nz if p.mode == tg.PER_SLICE else 1
    mask = torch.full(vol.shape, 7, dtype=torch.uint8, device=vol.device)
    t = torch.full((nh,), -5, dtype=torch.int32, device=vol.device)
    phi = torch.full((nh,), float("nan"), dtype=torch.float32, device=vol.device)
    st = torch.full((nh,), -1, dtype=torch.int32, device=vol.device)
    rc = L.tsallis_segment_static(vol.data_ptr(), nx, ny, nz, ctypes.byref(p), mask.data_ptr(), t.data_ptr(),
                                  phi.data_ptr(), st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == tg.TSALLIS_OK, tg.tsallis_status_string(rc)
    return mask, t, phi, st


@pytest.mark.parametrize("mode,q", [("slice", 0.8), ("slice", 1.5), ("volume", 0.5)])
def test_static_entry_matches_context_entry_twice(lib, mode, q):
    vol_np = phantom.generate_host(phantom.chest_volume(2012106843, nz=48))
    vol = torch.from_numpy(vol_np).cuda()
    p = tg.tsallis_params(q=q, mode=mode)
    ref = [x.cpu().numpy() for x in tg.tsallis_segment(vol, p)]
    g = vol_np.shape[1] * vol_np.shape[2] if mode == "slice" else vol_np.size
    _, _, gap, _ = oracle.segment1d(vol_np, g, float(np.float32(q)), nthreads=8, want_mask=False)
    for call in range(2):
        mask, t, phi, st = (x.cpu().numpy() for x in _static_call(lib, vol, p))
        assert np.array_equal(st & 0xff, ref[3] & 0xff), call
        for i in range(len(t)):
            if gap[i] >= GAP:
                assert t[i] == ref[1][i], (call, i)
            assert abs(phi[i] - ref[2][i]) <= PHI_RTOL * max(abs(ref[2][i]), 1.0), (call, i)
        if np.array_equal(t, ref[1]):
            assert np.array_equal(mask, ref[0]), call
        _check_masks(vol_np, mode, t, mask)


def _check_masks(vol_np, mode, t, mask):
    """Every mask is Algorithm 1 at the returned threshold (the oracle's)."""
    groups = [vol_np[z] for z in range(vol_np.shape[0])] if mode == "slice" else [vol_np]
    masks = [mask[z] for z in range(vol_np.shape[0])] if mode == "slice" else [mask]
    for i, (g, m) in enumerate(zip(groups, masks)):
        assert np.array_equal(m, oracle.binarize(g, int(t[i]))), i


def test_static_entry_skipped_arrival_times_out_then_exact(lib):
    """The first histogram tile never arrives: its slice's wait (the static
    entry's fixed 1 s limit) runs out and that slice reports TIMEOUT; the
    scratch the call leaves is clean, so the next call equals the oracle
    everywhere, masks included."""
    vol_np = phantom.generate_host(phantom.chest_volume(2012106856, nz=12))
    vol = torch.from_numpy(vol_np).cuda()
    p = tg.tsallis_params(q=0.8, flags=tg.TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL)
    _, t, _, st = (x.cpu().numpy() for x in _static_call(lib, vol, p))
    assert (st[0] & 0xff) == tg.TSALLIS_ERR_TIMEOUT and t[0] == -1
    for call in range(2):
        mask, t, phi, st = (x.cpu().numpy() for x in _static_call(lib, vol, tg.tsallis_params(q=0.8)))
        t_o, phi_o, gap_o, _ = oracle.segment1d(vol_np, vol_np.shape[1] * vol_np.shape[2], float(np.float32(0.8)),
                                                nthreads=8, want_mask=False)
        assert np.all((st & 0xff) == 0), (call, st)
        for i in range(len(t)):
            if gap_o[i] >= GAP:
                assert t[i] == t_o[i], (call, i)
            assert abs(phi[i] - phi_o[i]) <= PHI_RTOL * max(abs(phi_o[i]), 1.0), (call, i)
        _check_masks(vol_np, "slice", t, mask)


def test_static_entry_rejects_a_proposer_window(lib):
    vol = torch.zeros((2, 8, 8), dtype=torch.int16, device="cuda")
    out = torch.empty(vol.shape, dtype=torch.uint8, device="cuda")
    t = torch.empty(2, dtype=torch.int32, device="cuda")
    phi = torch.empty(2, dtype=torch.float32, device="cuda")
    st = torch.empty(2, dtype=torch.int32, device="cuda")
    p = tg.tsallis_params(topk=64)
    rc = lib.tsallis_segment_static(vol.data_ptr(), 8, 8, 2, ctypes.byref(p), out.data_ptr(), t.data_ptr(),
                                    phi.data_ptr(), st.data_ptr(), None)
    assert rc == tg.TSALLIS_ERR_INVALID_ARG


def test_static_entry_rejects_sizes_beyond_its_scratch(lib):
    p = tg.tsallis_params()
    big = torch.zeros((513, 8, 8), dtype=torch.int16, device="cuda")    # 513 slices > 512 histograms
    out = torch.empty(big.shape, dtype=torch.uint8, device="cuda")
    t = torch.empty(513, dtype=torch.int32, device="cuda")
    phi = torch.empty(513, dtype=torch.float32, device="cuda")
    st = torch.empty(513, dtype=torch.int32, device="cuda")
    rc = lib.tsallis_segment_static(big.data_ptr(), 8, 8, 513, ctypes.byref(p), out.data_ptr(), t.data_ptr(),
                                    phi.data_ptr(), st.data_ptr(), None)
    assert rc == tg.TSALLIS_ERR_INVALID_ARG
    p2 = tg.tsallis_params(two_d=True)
    rc = lib.tsallis_segment_static(big.data_ptr(), 8, 8, 4, ctypes.byref(p2), out.data_ptr(), t.data_ptr(),
                                    phi.data_ptr(), st.data_ptr(), None)
    assert rc == tg.TSALLIS_ERR_INVALID_ARG
