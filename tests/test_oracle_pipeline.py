"""Whole-pipeline pins of the oracle (Sec. III.A): exact recovery of a known
integer shift on a noise-free fronto-parallel textured pair, Delaunay
validity on real support sets, and an accuracy sanity bound on the
piecewise-planar workload (KITTI outlier definition of Sec. VII.A)."""
import numpy as np
import pytest

from paper_1802_07210_gb300 import synth


def _dt_valid_vectorised(xy, tri):
    xy = xy.astype(np.int64)
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    o = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert (o > 0).all()
    for k in range(len(tri)):
        ad, bd, cd = a[k] - xy, b[k] - xy, c[k] - xy
        al = (ad ** 2).sum(1)
        bl = (bd ** 2).sum(1)
        cl = (cd ** 2).sum(1)
        det = (ad[:, 0] * (bd[:, 1] * cl - bl * cd[:, 1]) - ad[:, 1] * (bd[:, 0] * cl - bl * cd[:, 0])
               + al * (bd[:, 0] * cd[:, 1] - bd[:, 1] * cd[:, 0]))
        assert (det <= 0).all(), "a point lies strictly inside a circumcircle"
    return True


@pytest.mark.parametrize("shift", [4, 9, 23])
def test_known_shift_recovered_exactly(orc, shift):
    w, h = 160, 100
    L, R = synth.fronto_parallel_pair(w, h, shift, seed=shift)
    prm = dict(disp_min=0, disp_max=31, ipol_gap_width=0, filter_adaptive_mean=0)
    r = orc.pipeline(L, R, prm, postprocess_on=False)
    assert len(r["list"]) > 0 and (r["list"][:, 2] == shift).all()
    for side, dp, dense, desc in (("L", r["dplaneL"], r["denseL"], r["descL"]),
                                  ("R", r["dplaneR"], r["denseR"], r["descR"])):
        assert set(np.unique(dense).tolist()) <= {-1, shift}
        uu = np.arange(w)[None, :].repeat(h, 0)
        vv = np.arange(h)[:, None].repeat(w, 1)
        uo = uu - shift if side == "L" else uu + shift
        tex = np.abs(desc.astype(np.int32) - 128).sum(-1)
        must = (dp >= 0) & (uo >= 2) & (uo <= w - 3) & (tex >= 1) \
            & (uu >= 2) & (uu <= w - 3) & (vv >= 2) & (vv <= h - 3)
        assert must.sum() > 0.5 * w * h
        assert (dense[must] == shift).all()
    # LR: a left pixel survives iff its partner was matched too
    partner_ok = np.zeros_like(r["denseL"], bool)
    for v in range(h):
        for u in range(shift, w):
            partner_ok[v, u] = r["denseR"][v, u - shift] == shift
    np.testing.assert_array_equal(r["maskL"] == 1, (r["denseL"] == shift) & partner_ok)


def test_small_workload_pipeline(orc):
    wl = synth.SMALL_320
    L, R, gt = synth.workload_pair(wl, 0, 1)
    r = orc.pipeline(L, R, wl.params, postprocess_on=False)
    lst = r["list"]
    assert 500 < len(lst) < wl.spec.w * wl.spec.h // 25
    # both meshes are valid Delaunay triangulations of their point sets
    _dt_valid_vectorised(lst[:, :2].astype(np.int64), r["triL"])
    xr = np.stack([lst[:, 0].astype(np.int64) - lst[:, 2], lst[:, 1]], 1)
    _dt_valid_vectorised(xr, r["triR"])
    # accuracy sanity (not parity): KITTI outliers (|err| >= 3 and >= 5 %)
    valid = r["lrL"] >= 0
    err = np.abs(r["lrL"].astype(np.int64) - gt)
    outl = (err >= 3) & (err >= 0.05 * np.maximum(gt, 1)) & valid
    assert valid.mean() > 0.5
    assert outl.sum() < 0.05 * valid.sum()
