"""The support-point entry point that allocates nothing
(elas_support_points_static) must give exactly the results of
elas_support_points, which takes a caller workspace.

It exists for callers that may not allocate device memory, such as a
real-time stereo loop that reserves everything at start-up, or a plug-in
whose host application owns all device buffers.  Its scratch is one static
device array shared by all calls, so the test calls it twice in a row on
different pairs: the second call must not see anything of the first.  It
also checks that sizes beyond the array are refused before any launch.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


def _static_call(B, descL, descR, prm):
    """Calls the C entry point directly through ctypes; only the outputs are
    allocated here, by the caller, as the entry point requires."""
    lib = B.lib()
    h, w = descL.shape[:2]
    step = prm.candidate_stepsize
    hc, wc = h // step, w // step
    cap = max(1, hc * wc)
    d_can = torch.empty((hc, wc), dtype=torch.int16, device="cuda")
    lst = torch.empty((cap, 3), dtype=torch.int16, device="cuda")
    count = torch.empty((1,), dtype=torch.int32, device="cuda")
    gL = torch.empty(B.grid_shape(w, h, prm), dtype=torch.int32, device="cuda")
    gR = torch.empty_like(gL)
    # poison the outputs so that nothing stale can pass for a result
    for t in (d_can, lst, count, gL, gR):
        t.fill_(0x5A)
    st = lib.elas_support_points_static(
        C.c_void_p(descL.data_ptr()), C.c_void_p(descR.data_ptr()), w, h, C.byref(prm),
        C.c_void_p(d_can.data_ptr()), C.c_void_p(lst.data_ptr()), cap, C.c_void_p(count.data_ptr()),
        C.c_void_p(gL.data_ptr()), C.c_void_p(gR.data_ptr()),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    B.check(st)
    return dict(d_can=d_can, list=lst, count=count, grid_L=gL, grid_R=gR)


def _same(a, b):
    n = int(host(a["count"])[0])
    assert n == int(host(b["count"])[0]) and n > 0
    np.testing.assert_array_equal(host(a["d_can"]), host(b["d_can"]))
    np.testing.assert_array_equal(host(a["list"])[:n], host(b["list"])[:n])
    np.testing.assert_array_equal(host(a["grid_L"]), host(b["grid_L"]))
    np.testing.assert_array_equal(host(a["grid_R"]), host(b["grid_R"]))


def test_static_scratch_matches_workspace_entry_point():
    require_gpu()
    from paper_1802_07210_gb300 import binding as B
    cases = [(synth.VGA_640, 2, 0), (synth.SMALL_320, 1, 5)]
    for wl, cfg, idx in cases:  # two calls in a row, different sizes and data
        L, R, _ = synth.workload_pair(wl, idx, cfg)
        prm = B.as_params(wl.params)
        descL, descR = B.elas_descriptors(dev(L), dev(R))
        ref = B.elas_support_points(descL, descR, prm)
        got = _static_call(B, descL, descR, prm)
        _same(got, ref)
    # and the first pair again, after the array holds the second pair's grids
    L, R, _ = synth.workload_pair(synth.VGA_640, 0, 2)
    prm = B.as_params(synth.VGA_640.params)
    descL, descR = B.elas_descriptors(dev(L), dev(R))
    _same(_static_call(B, descL, descR, prm), B.elas_support_points(descL, descR, prm))


def test_static_scratch_row_matcher_and_variants():
    """Sizes that take the row-organised support matcher (2048x1536 at step
    5: 307 lattice rows, 504,064 of the 524,288 scratch bytes) and the
    paper's variants (census records, support down-sampling) through the
    static entry point, each equal to elas_support_points."""
    require_gpu()
    from paper_1802_07210_gb300 import binding as B
    lib = B.lib()
    wl = synth.scaled_workload(2048, 1536, 128)
    L, R, _ = synth.workload_pair(wl, 0, 12)
    prm = B.as_params(wl.params)
    assert 500_000 < lib.elas_support_workspace_bytes(2048, 1536, C.byref(prm)) <= 512 * 1024
    descL, descR = B.elas_descriptors(dev(L), dev(R))
    _same(_static_call(B, descL, descR, prm), B.elas_support_points(descL, descR, prm))
    # the paper's census records (9x9, 32 bytes) and 1/8 down-sampling
    wl2 = synth.VGA_640
    L, R, _ = synth.workload_pair(wl2, 1, 2)
    prm_c = B.as_params(dict(wl2.params, census_support_w=9, census_dense_w=5))
    cL, cR = B.elas_census(dev(L), dev(R), 9, 32)
    _same(_static_call(B, cL, cR, prm_c), B.elas_support_points(cL, cR, prm_c))
    prm_d = B.as_params(dict(wl2.params, candidate_stepsize=1, support_downsample=8))
    descL, descR = B.elas_descriptors(dev(L), dev(R))
    if lib.elas_support_workspace_bytes(640, 480, C.byref(prm_d)) <= 512 * 1024:
        _same(_static_call(B, descL, descR, prm_d), B.elas_support_points(descL, descR, prm_d))
    prm_d = B.as_params(dict(wl2.params, support_downsample=8))
    _same(_static_call(B, descL, descR, prm_d), B.elas_support_points(descL, descR, prm_d))


def test_static_scratch_refuses_oversized_images():
    require_gpu()
    from paper_1802_07210_gb300 import binding as B
    lib = B.lib()
    prm = B.params(candidate_stepsize=1)
    w, h = 1024, 1024  # 1M candidates: 4 MB of scratch, above the 512 KiB array
    assert lib.elas_support_workspace_bytes(w, h, C.byref(prm)) > 512 * 1024
    dummy = torch.empty(16, dtype=torch.uint8, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = lib.elas_support_points_static(p, p, w, h, C.byref(prm), p, p, w * h, p, None, None, None)
    assert st == 3
    assert b"static scratch" in lib.elas_last_error()
