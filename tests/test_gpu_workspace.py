"""One device buffer of exactly elas_workspace_bytes serves every per-pair
call at that size: support points, the device triangulation of both sides,
the dense step (plane prior and argmin), post-processing and speckle removal
all accept it, one after the other on the same buffer, and their results
equal the oracle's (integer maps bit-exact, post-processing within 1e-4)."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _cases():
    ragged = synth.scaled_workload(203, 117, 48)
    ragged.params.update(disp_min=3, candidate_stepsize=3)
    census = dict(synth.VGA_640.params, census_support_w=9, census_dense_w=5, support_downsample=8)
    return [("small_320", synth.SMALL_320.params, synth.SMALL_320, 1),
            ("ragged_step3", ragged.params, ragged, 7),
            ("vga_census_ds8", census, synth.VGA_640, 2)]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_every_call_on_one_workspace(case):
    from paper_1802_07210_gb300 import binding as B
    lib = B.lib()
    name, prmd, wl, cfg = case
    prmd = dict(prmd, ipol_gap_width=3, filter_adaptive_mean=1)
    L, R, _ = synth.workload_pair(wl, 0, cfg)
    ref = oracle.pipeline(L, R, prmd, postprocess_on=True)
    h, w = L.shape
    prm = B.as_params(prmd)
    total = lib.elas_workspace_bytes(w, h, C.byref(prm))
    ws = torch.empty(total, dtype=torch.uint8, device="cuda")
    assert ws.data_ptr() % 256 == 0
    wsp = C.c_void_p(ws.data_ptr())
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if prm.census_support_w > 0:
        sL, sR = B.elas_census(dev(L), dev(R), prm.census_support_w, 32)
        dL_, dR_ = B.elas_census(dev(L), dev(R), prm.census_dense_w, 16)
        rec = 32
    else:
        dL_, dR_ = B.elas_descriptors(dev(L), dev(R))
        sL, sR = dL_, dR_
        rec = 16
    step = prm.candidate_stepsize
    hc, wc = h // step, w // step
    cap = max(1, hc * wc)
    d_can = torch.empty((hc, wc), dtype=torch.int16, device="cuda")
    lst = torch.empty((cap, 3), dtype=torch.int16, device="cuda")
    count = torch.empty((1,), dtype=torch.int32, device="cuda")
    gL = torch.empty(B.grid_shape(w, h, prm), dtype=torch.int32, device="cuda")
    gR = torch.empty_like(gL)
    assert sL.shape[-1] == rec
    B.check(lib.elas_support_points(C.c_void_p(sL.data_ptr()), C.c_void_p(sR.data_ptr()), w, h, C.byref(prm),
                                    C.c_void_p(d_can.data_ptr()), C.c_void_p(lst.data_ptr()), cap,
                                    C.c_void_p(count.data_ptr()), C.c_void_p(gL.data_ptr()),
                                    C.c_void_p(gR.data_ptr()), wsp, total, st))
    n = int(host(count)[0])
    assert n == len(ref["list"])
    np.testing.assert_array_equal(host(lst)[:n], ref["list"])
    cap_tri = 2 * cap + 8
    tris, nts = [], []
    for right in (0, 1):
        tri = torch.empty((cap_tri, 3), dtype=torch.int32, device="cuda")
        nt = torch.empty((1,), dtype=torch.int32, device="cuda")
        B.check(lib.elas_triangulate_device(C.c_void_p(lst.data_ptr()), C.c_void_p(count.data_ptr()), cap, w, h,
                                            right, C.c_void_p(tri.data_ptr()), cap_tri, C.c_void_p(nt.data_ptr()),
                                            wsp, total, st))
        tris.append(tri)
        nts.append(int(host(nt)[0]))
    assert nts == [len(ref["triL"]), len(ref["triR"])]
    outL = torch.empty((h, w), dtype=torch.int16, device="cuda")
    outR = torch.empty_like(outL)
    B.check(lib.elas_dense_match(C.c_void_p(dL_.data_ptr()), C.c_void_p(dR_.data_ptr()), w, h, C.byref(prm),
                                 C.c_void_p(lst.data_ptr()), n, C.c_void_p(tris[0].data_ptr()), nts[0],
                                 C.c_void_p(tris[1].data_ptr()), nts[1], C.c_void_p(gL.data_ptr()),
                                 C.c_void_p(gR.data_ptr()), C.c_void_p(outL.data_ptr()), C.c_void_p(outR.data_ptr()),
                                 wsp, total, st))
    np.testing.assert_array_equal(host(outL), ref["denseL"])
    np.testing.assert_array_equal(host(outR), ref["denseR"])
    B.elas_lr_check(outL, outR, prm.lr_threshold, masks=False)
    np.testing.assert_array_equal(host(outL), ref["lrL"])
    post = torch.empty((h, w), dtype=torch.float32, device="cuda")
    B.check(lib.elas_postprocess(C.c_void_p(outL.data_ptr()), w, h, C.byref(prm), C.c_void_p(post.data_ptr()),
                                 wsp, total, st))
    assert np.abs(host(post) - ref["post"]).max() <= 1e-4
    sp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    B.check(lib.elas_speckle(C.c_void_p(outL.data_ptr()), w, h, 1, 50, C.c_void_p(sp.data_ptr()), wsp, total, st))
    np.testing.assert_array_equal(host(sp), oracle.speckle(ref["lrL"], 1, 50))
