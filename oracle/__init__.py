"""ctypes wrapper over the plain-C ELAS oracle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.

Every function takes and returns numpy arrays in the layouts documented in
``elas_oracle.h``.  Parameters are plain dicts with the field names of
``oracle_params``; unspecified fields take the default parameter set.
"""
import ctypes as C
import numpy as np

from . import build as _build

_lib = None

FLAG_PRIOR_OFF = 1
FLAG_FULL_RANGE = 2
FLAG_REDUNDANCY_OFF = 4
FLAG_SHIFT_SUM = 8
FLAG_PAST_REDUNDANCY = 16


class OracleParams(C.Structure):
    _fields_ = [
        ("disp_min", C.c_int32), ("disp_max", C.c_int32),
        ("support_threshold", C.c_float), ("support_texture", C.c_int32),
        ("candidate_stepsize", C.c_int32),
        ("incon_window_size", C.c_int32), ("incon_threshold", C.c_int32),
        ("incon_min_support", C.c_int32), ("redun_max_dist", C.c_int32),
        ("grid_size", C.c_int32),
        ("beta", C.c_float), ("gamma", C.c_float), ("sigma", C.c_float),
        ("sradius", C.c_int32), ("match_texture", C.c_int32), ("lr_threshold", C.c_int32),
        ("ipol_gap_width", C.c_int32), ("filter_adaptive_mean", C.c_int32),
        ("flags", C.c_uint32),
        ("census_support_w", C.c_int32), ("census_dense_w", C.c_int32),
        ("support_downsample", C.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        i = C.c_int
        L.oracle_params_default.argtypes = [P]
        L.oracle_sobel.argtypes = [P, i, i, P, P]
        L.oracle_descriptors.argtypes = [P, i, i, P]
        L.oracle_census.argtypes = [P, i, i, i, i, P]
        L.oracle_support_match.argtypes = [P, P, i, i, P, P]
        L.oracle_filter_consistency.argtypes = [P, i, i, P, P]
        L.oracle_filter_redundancy.argtypes = [P, i, i, P, P]
        L.oracle_support_points.argtypes = [P, P, i, i, P, P]
        L.oracle_support_list.argtypes = [P, i, i, i, P]
        L.oracle_support_list.restype = i
        L.oracle_grid_vectors.argtypes = [P, i, i, i, P, i, P]
        L.oracle_delaunay.argtypes = [P, P, i, P, i]
        L.oracle_delaunay.restype = i
        L.oracle_triangulate.argtypes = [P, i, i, P, i]
        L.oracle_triangulate.restype = i
        L.oracle_orient.argtypes = [C.c_int64] * 6
        L.oracle_orient.restype = C.c_int64
        L.oracle_incircle.argtypes = [C.c_int64] * 8
        L.oracle_incircle.restype = C.c_int64
        L.oracle_prior_table.argtypes = [P, P]
        L.oracle_plane_prior.argtypes = [P, i, P, i, i, i, i, P, P, P]
        L.oracle_dense.argtypes = [P, P, i, i, P, P, P, i, P]
        L.oracle_lr_check.argtypes = [P, P, i, i, i, P, P, P, P]
        L.oracle_postprocess.argtypes = [P, i, i, P, P]
        L.oracle_median.argtypes = [P, i, i, i, P]
        L.oracle_speckle.argtypes = [P, i, i, i, i, P]
        _lib = L
    return _lib


def params(**kw) -> OracleParams:
    p = OracleParams()
    lib().oracle_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(prm):
    if prm is None:
        prm = params()
    elif isinstance(prm, dict):
        prm = params(**prm)
    return prm


def sobel(img):
    img = _c(img, np.uint8)
    h, w = img.shape
    du = np.empty((h, w), np.int32)
    dv = np.empty((h, w), np.int32)
    lib().oracle_sobel(_ptr(img), w, h, _ptr(du), _ptr(dv))
    return du, dv


def descriptors(img):
    img = _c(img, np.uint8)
    h, w = img.shape
    out = np.empty((h, w, 16), np.uint8)
    lib().oracle_descriptors(_ptr(img), w, h, _ptr(out))
    return out


def census(img, W, nbytes):
    """Census transform over a W x W window, packed into nbytes bytes per
    pixel (Sec. VI.A; bit order and border rule in elas_oracle.h)."""
    img = _c(img, np.uint8)
    h, w = img.shape
    if W < 1 or W % 2 == 0 or W * W > 8 * nbytes:
        raise ValueError("census window %d does not fit %d bytes" % (W, nbytes))
    out = np.empty((h, w, nbytes), np.uint8)
    lib().oracle_census(_ptr(img), w, h, int(W), int(nbytes), _ptr(out))
    return out


def _grid_shape(w, h, prm):
    s = prm.candidate_stepsize
    return h // s, w // s


def support_match(descL, descR, prm=None):
    prm = _p(prm)
    descL, descR = _c(descL, np.uint8), _c(descR, np.uint8)
    h, w = descL.shape[:2]
    out = np.empty(_grid_shape(w, h, prm), np.int16)
    lib().oracle_support_match(_ptr(descL), _ptr(descR), w, h, C.byref(prm), _ptr(out))
    return out


def filter_consistency(dcan, prm=None):
    prm = _p(prm)
    dcan = _c(dcan, np.int16)
    hc, wc = dcan.shape
    out = np.empty_like(dcan)
    lib().oracle_filter_consistency(_ptr(dcan), wc, hc, C.byref(prm), _ptr(out))
    return out


def filter_redundancy(dcan, prm=None):
    prm = _p(prm)
    dcan = _c(dcan, np.int16)
    hc, wc = dcan.shape
    out = np.empty_like(dcan)
    lib().oracle_filter_redundancy(_ptr(dcan), wc, hc, C.byref(prm), _ptr(out))
    return out


def support_points(descL, descR, prm=None):
    prm = _p(prm)
    descL, descR = _c(descL, np.uint8), _c(descR, np.uint8)
    h, w = descL.shape[:2]
    out = np.empty(_grid_shape(w, h, prm), np.int16)
    lib().oracle_support_points(_ptr(descL), _ptr(descR), w, h, C.byref(prm), _ptr(out))
    return out


def support_list(dcan, prm=None):
    prm = _p(prm)
    dcan = _c(dcan, np.int16)
    hc, wc = dcan.shape
    out = np.empty((max(1, hc * wc), 3), np.int16)
    n = lib().oracle_support_list(_ptr(dcan), wc, hc, prm.candidate_stepsize, _ptr(out))
    return out[:n].copy()


def grid_vectors(lst, w, h, prm=None, right=False):
    prm = _p(prm)
    lst = _c(lst, np.int16).reshape(-1, 3)
    G = prm.grid_size
    nw = (prm.disp_max + 1 + 31) // 32
    out = np.empty(((h + G - 1) // G, (w + G - 1) // G, nw), np.uint32)
    lib().oracle_grid_vectors(_ptr(lst), len(lst), w, h, C.byref(prm), int(right), _ptr(out))
    return out


def delaunay(xy):
    xy = np.asarray(xy, np.int64).reshape(-1, 2)
    x = _c(xy[:, 0], np.int32)
    y = _c(xy[:, 1], np.int32)
    n = len(x)
    cap = max(1, 2 * n)
    tri = np.empty((cap, 3), np.int32)
    nt = lib().oracle_delaunay(_ptr(x), _ptr(y), n, _ptr(tri), cap)
    if nt < 0:
        raise RuntimeError("triangle capacity exceeded")
    return tri[:nt].copy()


def triangulate(lst, right=False):
    lst = _c(lst, np.int16).reshape(-1, 3)
    n = len(lst)
    cap = max(1, 2 * n)
    tri = np.empty((cap, 3), np.int32)
    nt = lib().oracle_triangulate(_ptr(lst), n, int(right), _ptr(tri), cap)
    if nt < 0:
        raise RuntimeError("triangle capacity exceeded")
    return tri[:nt].copy()


def orient(a, b, c):
    return lib().oracle_orient(int(a[0]), int(a[1]), int(b[0]), int(b[1]), int(c[0]), int(c[1]))


def incircle(a, b, c, d):
    return lib().oracle_incircle(*(int(v) for p in (a, b, c, d) for v in p))


def prior_table(prm=None):
    prm = _p(prm)
    P = np.empty(prm.sradius + 1, np.int32)
    lib().oracle_prior_table(C.byref(prm), _ptr(P))
    return P


def plane_prior(lst, tri, w, h, prm=None, right=False, with_owners=False):
    prm = _p(prm)
    lst = _c(lst, np.int16).reshape(-1, 3)
    tri = _c(tri, np.int32).reshape(-1, 3)
    dplane = np.empty((h, w), np.int16)
    owners = np.empty((h, w), np.int32) if with_owners else None
    lib().oracle_plane_prior(_ptr(lst), len(lst), _ptr(tri), len(tri), int(right), w, h,
                             C.byref(prm), _ptr(dplane), _ptr(owners))
    return (dplane, owners) if with_owners else dplane


def dense(descL, descR, dplane, grid, prm=None, right=False):
    prm = _p(prm)
    descL, descR = _c(descL, np.uint8), _c(descR, np.uint8)
    h, w = descL.shape[:2]
    dplane = _c(dplane, np.int16) if dplane is not None else None
    grid = _c(grid, np.uint32) if grid is not None else None
    out = np.empty((h, w), np.int16)
    lib().oracle_dense(_ptr(descL), _ptr(descR), w, h, C.byref(prm), _ptr(dplane),
                       _ptr(grid), int(right), _ptr(out))
    return out


def lr_check(dL, dR, thr):
    dL, dR = _c(dL, np.int16), _c(dR, np.int16)
    h, w = dL.shape
    oL, oR = np.empty_like(dL), np.empty_like(dR)
    mL, mR = np.empty((h, w), np.uint8), np.empty((h, w), np.uint8)
    lib().oracle_lr_check(_ptr(dL), _ptr(dR), w, h, int(thr), _ptr(oL), _ptr(oR),
                          _ptr(mL), _ptr(mR))
    return oL, oR, mL, mR


def postprocess(d, prm=None):
    prm = _p(prm)
    d = _c(d, np.int16)
    h, w = d.shape
    out = np.empty((h, w), np.float32)
    lib().oracle_postprocess(_ptr(d), w, h, C.byref(prm), _ptr(out))
    return out


def median(d, r=1):
    """Median filter of valid disparities (Sec. VII; the reading is stated in
    elas_oracle.h)."""
    d = _c(d, np.int16)
    h, w = d.shape
    out = np.empty((h, w), np.int16)
    lib().oracle_median(_ptr(d), w, h, int(r), _ptr(out))
    return out


def speckle(d, sim_threshold=1, min_size=200):
    """Small-segment removal (ELAS post-processing; the reading is stated in
    elas_oracle.h)."""
    d = _c(d, np.int16)
    h, w = d.shape
    out = np.empty((h, w), np.int16)
    lib().oracle_speckle(_ptr(d), w, h, int(sim_threshold), int(min_size), _ptr(out))
    return out


def pipeline(imgL, imgR, prm=None, postprocess_on=True):
    """All steps in order for one stereo pair; returns a dict of every
    intermediate (descriptors, candidate grid, list, grids, triangles, prior
    maps, dense maps, LR-checked maps and masks, postprocessed map)."""
    prm = _p(prm)
    h, w = np.asarray(imgL).shape
    r = {}
    if prm.census_support_w > 0:
        # Sec. VI.A: support census (32 bytes) and dense census (16 bytes)
        r["sdescL"] = census(imgL, prm.census_support_w, 32)
        r["sdescR"] = census(imgR, prm.census_support_w, 32)
        r["descL"] = census(imgL, prm.census_dense_w, 16)
        r["descR"] = census(imgR, prm.census_dense_w, 16)
        r["dcan"] = support_points(r["sdescL"], r["sdescR"], prm)
    else:
        r["descL"] = descriptors(imgL)
        r["descR"] = descriptors(imgR)
        r["dcan"] = support_points(r["descL"], r["descR"], prm)
    r["list"] = support_list(r["dcan"], prm)
    r["gridL"] = grid_vectors(r["list"], w, h, prm, right=False)
    r["gridR"] = grid_vectors(r["list"], w, h, prm, right=True)
    r["triL"] = triangulate(r["list"], right=False)
    r["triR"] = triangulate(r["list"], right=True)
    r["dplaneL"] = plane_prior(r["list"], r["triL"], w, h, prm, right=False)
    r["dplaneR"] = plane_prior(r["list"], r["triR"], w, h, prm, right=True)
    r["denseL"] = dense(r["descL"], r["descR"], r["dplaneL"], r["gridL"], prm, right=False)
    r["denseR"] = dense(r["descL"], r["descR"], r["dplaneR"], r["gridR"], prm, right=True)
    oL, oR, mL, mR = lr_check(r["denseL"], r["denseR"], prm.lr_threshold)
    r["lrL"], r["lrR"], r["maskL"], r["maskR"] = oL, oR, mL, mR
    if postprocess_on:
        r["post"] = postprocess(oL, prm)
    return r
