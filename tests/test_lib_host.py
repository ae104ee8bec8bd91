"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point include/elas_gb300.h declares, rejects bad arguments
synchronously, and its host Delaunay step (Sec. III.A) reproduces the
oracle's triangulation exactly."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1802_07210_gb300 import _lib, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(elas_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.SIGNATURES), "binding table must mirror the header"


def test_params_default_matches_oracle_defaults(orc):
    p = _lib.params()
    o = orc.params()
    for name, _ in _lib.Params._fields_:
        oname = "flags" if name == "test_flags" else name
        assert getattr(p, name) == pytest.approx(getattr(o, oname)), name


def test_invalid_arguments_are_rejected_on_the_host():
    L = _lib.lib()
    st = L.elas_descriptors(None, None, 0, 10, 10, None, None, None)
    assert st == 1 and b"image size" in L.elas_last_error()
    p = _lib.params(disp_max=2000)
    assert L.elas_support_workspace_bytes(64, 64, C.byref(p)) == 0
    nt = C.c_int32(-5)
    assert L.elas_triangulate(None, -1, 0, None, 0, C.byref(nt)) == 1
    # the median filter: radius, size, NULL and aliasing checks (no CUDA call)
    assert L.elas_median(C.c_void_p(16), 8, 8, 4, C.c_void_p(32), None) == 1
    assert b"radius" in L.elas_last_error()
    assert L.elas_median(C.c_void_p(16), 0, 8, 1, C.c_void_p(32), None) == 1
    assert L.elas_median(None, 8, 8, 1, C.c_void_p(32), None) == 1
    assert L.elas_median(C.c_void_p(16), 8, 8, 1, C.c_void_p(16), None) == 1
    assert b"alias" in L.elas_last_error()
    # speckle removal: size, threshold, NULL, alignment and workspace checks
    nb = L.elas_speckle_workspace_bytes(64, 48)
    assert nb >= 2 * 64 * 48 * 4 and L.elas_speckle_workspace_bytes(0, 48) == 0
    assert L.elas_speckle(C.c_void_p(16), 64, 48, -1, 10, C.c_void_p(16), C.c_void_p(256), nb, None) == 1
    assert L.elas_speckle(C.c_void_p(16), 0, 48, 1, 10, C.c_void_p(16), C.c_void_p(256), nb, None) == 1
    assert L.elas_speckle(None, 64, 48, 1, 10, C.c_void_p(16), C.c_void_p(256), nb, None) == 1
    assert L.elas_speckle(C.c_void_p(16), 64, 48, 1, 10, C.c_void_p(16), C.c_void_p(128), nb, None) == 1
    assert L.elas_speckle(C.c_void_p(16), 64, 48, 1, 10, C.c_void_p(16), C.c_void_p(256), nb - 1, None) == 3
    # census records: window parity, range and record size (no CUDA call)
    for window, nbytes in ((4, 32), (1, 32), (17, 32), (13, 16), (9, 24)):
        assert L.elas_census(C.c_void_p(16), None, 8, 8, 8, window, nbytes, C.c_void_p(32), None, None) == 1
        assert b"census" in L.elas_last_error()
    assert L.elas_census(C.c_void_p(16), C.c_void_p(64), 8, 8, 8, 9, 32, C.c_void_p(32), None, None) == 1
    # census windows in the parameters: both 0, or odd support 3..15 and dense 3..11
    for cs, cd in ((9, 0), (0, 5), (8, 5), (9, 13), (17, 5), (1, 1)):
        bad = _lib.params(census_support_w=cs, census_dense_w=cd)
        assert L.elas_support_workspace_bytes(64, 64, C.byref(bad)) == 0, (cs, cd)
    assert L.elas_support_workspace_bytes(64, 64, C.byref(_lib.params(support_downsample=-1))) == 0
    assert L.elas_support_workspace_bytes(64, 64, C.byref(_lib.params(support_downsample=14))) > 0
    good = _lib.params(census_support_w=15, census_dense_w=11)
    assert L.elas_support_workspace_bytes(64, 64, C.byref(good)) > 0


def test_batch_and_server_configs_are_checked_on_the_host():
    """Shape and configuration errors are reported before any device call."""
    L = _lib.lib()
    out = C.c_void_p()
    w = (C.c_int32 * 1)(64)
    h = (C.c_int32 * 1)(48)
    prm = (_lib.Params * 1)(_lib.params())
    assert L.elas_batch_create(0, w, h, prm, C.byref(out)) == 1 and not out.value
    assert L.elas_batch_create(300, w, h, prm, C.byref(out)) == 1
    assert L.elas_batch_create(1, None, h, prm, C.byref(out)) == 1
    cfg = _lib.ServerConfig()
    assert L.elas_server_config_default(C.byref(cfg)) == 0
    assert 1 <= cfg.lanes <= 8 and 1 <= cfg.max_wave <= 256 and cfg.plain == 0
    for field, bad in (("lanes", 0), ("lanes", 9), ("max_wave", 0), ("max_wave", 257), ("max_slots", 0)):
        c = _lib.ServerConfig()
        L.elas_server_config_default(C.byref(c))
        setattr(c, field, bad)
        assert L.elas_server_create(C.byref(c), C.byref(out)) == 1, field
        assert field.encode() in L.elas_last_error()
    # slot sizes: grow with the image and the disparity range; 0 when invalid
    p64, p256 = _lib.params(disp_max=63), _lib.params(disp_max=255)
    s1 = L.elas_slot_device_bytes(320, 240, C.byref(p64))
    s2 = L.elas_slot_device_bytes(640, 480, C.byref(p64))
    s3 = L.elas_slot_device_bytes(640, 480, C.byref(p256))
    assert 0 < s1 < s2 < s3
    assert s2 >= 640 * 480 * 36  # two descriptor planes alone are 32 bytes a pixel
    assert L.elas_slot_device_bytes(3, 3, C.byref(p64)) == 0
    assert L.elas_slot_device_bytes(640, 480, C.byref(_lib.params(disp_max=5000))) == 0


def _canon(t):
    return sorted(tuple(int(v) for v in np.roll(r, -int(np.argmin(r)))) for r in np.asarray(t).reshape(-1, 3))


@pytest.mark.parametrize("seed", range(10))
def test_triangulation_matches_oracle_on_lattice_subsets(orc, seed):
    rng = np.random.default_rng(seed)
    gx, gy = int(rng.integers(2, 30)), int(rng.integers(2, 20))
    pts = [(5 * i + 5, 5 * j + 5, int(rng.integers(0, 40)))
           for j in range(gy) for i in range(gx) if rng.random() < rng.uniform(0.2, 1.0)]
    lst = np.array(pts, np.int16).reshape(-1, 3)
    for right in (0, 1):
        cap = max(1, 2 * len(lst))
        tri = np.empty((cap, 3), np.int32)
        nt = C.c_int32(0)
        _lib.check(_lib.lib().elas_triangulate(_lib.np_ptr(lst), len(lst), right, _lib.np_ptr(tri), cap,
                                               C.byref(nt)))
        got = tri[:nt.value]
        exp = orc.triangulate(lst, right=bool(right))
        # identical triangles with identical (counter-clockwise) orientation
        assert _canon(got) == _canon(exp)


def test_triangulation_matches_oracle_on_real_support(orc):
    wl = synth.SMALL_320
    L, R, _ = synth.workload_pair(wl, 3, 1)
    dL, dR = orc.descriptors(L), orc.descriptors(R)
    lst = orc.support_list(orc.support_points(dL, dR, wl.params), wl.params)
    assert len(lst) > 300
    for right in (0, 1):
        cap = 2 * len(lst)
        tri = np.empty((cap, 3), np.int32)
        nt = C.c_int32(0)
        _lib.check(_lib.lib().elas_triangulate(_lib.np_ptr(lst), len(lst), right, _lib.np_ptr(tri), cap,
                                               C.byref(nt)))
        assert _canon(tri[:nt.value]) == _canon(orc.triangulate(lst, right=bool(right)))


def test_triangulation_capacity_error():
    lst = np.array([[5, 5, 0], [10, 5, 0], [5, 10, 0], [10, 10, 0]], np.int16)
    tri = np.empty((1, 3), np.int32)
    nt = C.c_int32(0)
    st = _lib.lib().elas_triangulate(_lib.np_ptr(lst), 4, 0, _lib.np_ptr(tri), 1, C.byref(nt))
    assert st == 3 and nt.value == 2


def test_one_workspace_for_every_call():
    """elas_workspace_bytes covers every per-pair call's own requirement for
    the arguments a caller passes at that size (support points, either
    side's device triangulation with the full candidate capacity, the plane
    prior with the triangle bound of a mesh, the dense step, post-processing
    and speckle removal), and is 0 for invalid parameters.  A GPU test runs
    every call on one buffer of exactly this size."""
    L = _lib.lib()
    for w, h, kw in ((640, 480, {}), (1242, 375, {}), (8, 8, {}), (203, 117, dict(candidate_stepsize=3)),
                     (320, 240, dict(census_support_w=9, census_dense_w=5, support_downsample=8)),
                     (1920, 1080, dict(disp_max=63)), (4, 4, {})):
        p = _lib.params(**kw)
        step = p.candidate_stepsize
        cap = max(1, (w // step) * (h // step))
        total = L.elas_workspace_bytes(w, h, C.byref(p))
        assert total > 0
        assert total >= L.elas_support_workspace_bytes(w, h, C.byref(p))
        assert total >= L.elas_triangulate_device_workspace_bytes(cap, w, h)
        assert total >= L.elas_plane_prior_workspace_bytes(2 * cap + 8)
        assert total >= L.elas_dense_workspace_bytes(w, h, C.byref(p))
        assert total >= L.elas_postprocess_workspace_bytes(w, h)
        assert total >= L.elas_speckle_workspace_bytes(w, h)
    assert L.elas_workspace_bytes(64, 64, C.byref(_lib.params(disp_max=-3))) == 0
