"""Torch-facing binding of the C-ABI: one function per entry point, same
names.  PyTorch supplies device memory and the current stream only; every
output tensor is allocated here and filled by the library.

Layouts follow include/elas_gb300.h: images uint8 [h, w]; descriptors uint8
[h, w, 16]; candidate grid int16 [h//step, w//step]; support list int16
[cap, 3]; grid vectors int32 [gh, gw, nw] (uint32 bit patterns); triangles
int32 [ntri, 3]; disparity maps int16 [h, w]; post-processed map float32.
"""
import ctypes as C

import numpy as np
import torch

from ._lib import (BatchConfig, ElasError, Params, PipelineStats, ServerConfig, ServerResult, ServerStats,  # noqa: F401
                   as_params, check, lib, np_ptr, params)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return C.c_void_p(t.data_ptr())


def _opt(t, dtype, name, shape=None):
    return None if t is None else _dev(t, dtype, name, shape)


def grid_shape(w, h, prm):
    G = prm.grid_size
    return ((h + G - 1) // G, (w + G - 1) // G, (prm.disp_max + 1 + 31) // 32)


def _workspace(nbytes, device):
    # 256-byte aligned device scratch (torch's allocator aligns to >= 512)
    return torch.empty(max(1, int(nbytes)), dtype=torch.uint8, device=device)


def elas_descriptors(imgL, imgR=None, stream=None):
    h, w = imgL.shape
    pL = _dev(imgL, torch.uint8, "imgL")
    descL = torch.empty((h, w, 16), dtype=torch.uint8, device=imgL.device)
    descR = None
    pR = None
    if imgR is not None:
        pR = _dev(imgR, torch.uint8, "imgR", (h, w))
        descR = torch.empty_like(descL)
    check(lib().elas_descriptors(pL, pR, w, h, w, C.c_void_p(descL.data_ptr()),
                                 None if descR is None else C.c_void_p(descR.data_ptr()), _stream(stream)))
    return (descL, descR) if imgR is not None else descL


def elas_census(imgL, imgR=None, window=9, nbytes=32, stream=None):
    """Census records of one or two images (Sec. VI.A): uint8 [h][w][nbytes]."""
    h, w = imgL.shape
    pL = _dev(imgL, torch.uint8, "imgL")
    outL = torch.empty((h, w, nbytes), dtype=torch.uint8, device=imgL.device)
    outR = None
    pR = None
    if imgR is not None:
        pR = _dev(imgR, torch.uint8, "imgR", (h, w))
        outR = torch.empty_like(outL)
    check(lib().elas_census(pL, pR, w, h, w, int(window), int(nbytes), C.c_void_p(outL.data_ptr()),
                            None if outR is None else C.c_void_p(outR.data_ptr()), _stream(stream)))
    return (outL, outR) if imgR is not None else outL


def elas_support_points(descL, descR, prm=None, grids=True, stream=None):
    prm = as_params(prm)
    h, w = descL.shape[:2]
    dev = descL.device
    step = prm.candidate_stepsize
    hc, wc = h // step, w // step
    cap = max(1, hc * wc)
    d_can = torch.empty((hc, wc), dtype=torch.int16, device=dev)
    lst = torch.empty((cap, 3), dtype=torch.int16, device=dev)
    count = torch.empty((1,), dtype=torch.int32, device=dev)
    gL = gR = None
    if grids:
        gL = torch.empty(grid_shape(w, h, prm), dtype=torch.int32, device=dev)
        gR = torch.empty_like(gL)
    nb = lib().elas_support_workspace_bytes(w, h, C.byref(prm))
    ws = _workspace(nb, dev)
    rec = 32 if prm.census_support_w > 0 else 16  # support census records or descriptors
    check(lib().elas_support_points(
        _dev(descL, torch.uint8, "descL", (h, w, rec)), _dev(descR, torch.uint8, "descR", (h, w, rec)), w, h,
        C.byref(prm), C.c_void_p(d_can.data_ptr()), C.c_void_p(lst.data_ptr()), cap,
        C.c_void_p(count.data_ptr()), _opt(gL, torch.int32, "grid_L"), _opt(gR, torch.int32, "grid_R"),
        C.c_void_p(ws.data_ptr()), nb, _stream(stream)))
    return dict(d_can=d_can, list=lst, count=count, grid_L=gL, grid_R=gR)


def elas_triangulate(lst, right=False):
    """Host call: lst is a numpy int16 [n, 3] support list."""
    lst = np.ascontiguousarray(lst, dtype=np.int16).reshape(-1, 3)
    n = len(lst)
    cap = max(1, 2 * n)
    tri = np.empty((cap, 3), np.int32)
    nt = C.c_int32(0)
    check(lib().elas_triangulate(np_ptr(lst), n, int(bool(right)), np_ptr(tri), cap, C.byref(nt)))
    return tri[:nt.value].copy()


def elas_triangulate_device(lst, count, w, h, right=False, stream=None):
    """lst: device int16 [cap, 3]; count: device int32 [1].  Returns the
    device triangle buffer [2*cap+8, 3] and the device count tensor [1]."""
    cap = lst.shape[0]
    cap_tri = 2 * cap + 8
    tri = torch.empty((cap_tri, 3), dtype=torch.int32, device=lst.device)
    nt = torch.empty((1,), dtype=torch.int32, device=lst.device)
    nb = lib().elas_triangulate_device_workspace_bytes(cap, w, h)
    ws = _workspace(nb, lst.device)
    check(lib().elas_triangulate_device(_dev(lst, torch.int16, "list"), _dev(count, torch.int32, "count"), cap, w,
                                        h, int(bool(right)), C.c_void_p(tri.data_ptr()), cap_tri,
                                        C.c_void_p(nt.data_ptr()), C.c_void_p(ws.data_ptr()), nb, _stream(stream)))
    return tri, nt


def elas_plane_prior(lst, tri, w, h, prm=None, right=False, stream=None):
    prm = as_params(prm)
    dev = lst.device
    out = torch.empty((h, w), dtype=torch.int16, device=dev)
    n = lst.shape[0]
    ntri = tri.shape[0]
    nb = lib().elas_plane_prior_workspace_bytes(ntri)
    ws = _workspace(nb, dev)
    check(lib().elas_plane_prior(_dev(lst, torch.int16, "list"), n, _dev(tri, torch.int32, "tri"), ntri,
                                 int(bool(right)), w, h, C.byref(prm), C.c_void_p(out.data_ptr()),
                                 C.c_void_p(ws.data_ptr()), nb, _stream(stream)))
    return out


def elas_dense_argmin(descL, descR, prm=None, d_plane=None, grid=None, right=False, stream=None):
    prm = as_params(prm)
    h, w = descL.shape[:2]
    out = torch.empty((h, w), dtype=torch.int16, device=descL.device)
    check(lib().elas_dense_argmin(
        _dev(descL, torch.uint8, "descL", (h, w, 16)), _dev(descR, torch.uint8, "descR", (h, w, 16)), w, h,
        C.byref(prm), _opt(d_plane, torch.int16, "d_plane", (h, w)),
        _opt(grid, torch.int32, "grid", grid_shape(w, h, prm)), int(bool(right)),
        C.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def elas_dense_match(descL, descR, prm, lst, n, triL, triR, grid_L, grid_R, stream=None):
    prm = as_params(prm)
    h, w = descL.shape[:2]
    dev = descL.device
    dL = torch.empty((h, w), dtype=torch.int16, device=dev)
    dR = torch.empty_like(dL)
    nb = lib().elas_dense_workspace_bytes(w, h, C.byref(prm))
    ws = _workspace(nb, dev)
    gs = grid_shape(w, h, prm)
    check(lib().elas_dense_match(
        _dev(descL, torch.uint8, "descL", (h, w, 16)), _dev(descR, torch.uint8, "descR", (h, w, 16)), w, h,
        C.byref(prm), _dev(lst, torch.int16, "list"), int(n), _dev(triL, torch.int32, "triL"), triL.shape[0],
        _dev(triR, torch.int32, "triR"), triR.shape[0], _dev(grid_L, torch.int32, "grid_L", gs),
        _dev(grid_R, torch.int32, "grid_R", gs), C.c_void_p(dL.data_ptr()), C.c_void_p(dR.data_ptr()),
        C.c_void_p(ws.data_ptr()), nb, _stream(stream)))
    return dL, dR


def elas_lr_check(dL, dR, lr_threshold, masks=True, stream=None):
    """In place on dL and dR; returns (maskL, maskR) or None."""
    h, w = dL.shape
    mL = mR = None
    if masks:
        mL = torch.empty((h, w), dtype=torch.uint8, device=dL.device)
        mR = torch.empty_like(mL)
    check(lib().elas_lr_check(_dev(dL, torch.int16, "dL"), _dev(dR, torch.int16, "dR", (h, w)), w, h,
                              int(lr_threshold), _opt(mL, torch.uint8, "maskL"), _opt(mR, torch.uint8, "maskR"),
                              _stream(stream)))
    return (mL, mR) if masks else None


def elas_postprocess(d, prm=None, stream=None):
    prm = as_params(prm)
    h, w = d.shape
    out = torch.empty((h, w), dtype=torch.float32, device=d.device)
    nb = lib().elas_postprocess_workspace_bytes(w, h)
    ws = _workspace(nb, d.device)
    check(lib().elas_postprocess(_dev(d, torch.int16, "d"), w, h, C.byref(prm), C.c_void_p(out.data_ptr()),
                                 C.c_void_p(ws.data_ptr()), nb, _stream(stream)))
    return out


def elas_median(d, radius=1, out=None, stream=None):
    h, w = d.shape
    if out is None:
        out = torch.empty((h, w), dtype=torch.int16, device=d.device)
    check(lib().elas_median(_dev(d, torch.int16, "d"), w, h, int(radius), _dev(out, torch.int16, "out"),
                            _stream(stream)))
    return out


def elas_speckle(d, sim_threshold=1, min_size=200, out=None, stream=None, with_status=False):
    """Small-segment removal; out may be d itself (in place)."""
    h, w = d.shape
    if out is None:
        out = torch.empty((h, w), dtype=torch.int16, device=d.device)
    nb = lib().elas_speckle_workspace_bytes(w, h)
    ws = _workspace(nb, d.device)
    check(lib().elas_speckle(_dev(d, torch.int16, "d"), w, h, int(sim_threshold), int(min_size),
                             _dev(out, torch.int16, "out"), C.c_void_p(ws.data_ptr()), nb, _stream(stream)))
    if with_status:
        return out, ws[:4].view(torch.int32)
    return out


class Pipeline:
    """Owner of an ``elas_pipeline`` handle for one image size."""

    def __init__(self, w, h, prm=None, gpu_triangulation=True):
        self.w, self.h = w, h
        self.prm = as_params(prm)
        self._h = C.c_void_p()
        check(lib().elas_pipeline_create(w, h, C.byref(self.prm), C.byref(self._h)))
        check(lib().elas_pipeline_set_triangulation(self._h, int(bool(gpu_triangulation))))

    def run(self, imgL, imgR, dL, dR=None, post=None, stream=None):
        """Device tensors in and out (dL/dR int16 [h, w], post float32)."""
        check(lib().elas_pipeline_run(
            self._h, _dev(imgL, torch.uint8, "imgL", (self.h, self.w)),
            _dev(imgR, torch.uint8, "imgR", (self.h, self.w)), self.w,
            _dev(dL, torch.int16, "dL", (self.h, self.w)), _opt(dR, torch.int16, "dR", (self.h, self.w)),
            _opt(post, torch.float32, "post", (self.h, self.w)), _stream(stream)))

    def run_host(self, imgL, imgR, dL, dR=None, post=None, stream=None):
        """Host (ideally pinned) CPU tensors in and out; returns when done."""
        def hp(t, dtype, name):
            if t is None:
                return None
            if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
                raise TypeError("%s must be a contiguous host %s tensor" % (name, dtype))
            return C.c_void_p(t.data_ptr())
        check(lib().elas_pipeline_run_host(self._h, hp(imgL, torch.uint8, "imgL"), hp(imgR, torch.uint8, "imgR"),
                                           hp(dL, torch.int16, "dL"), hp(dR, torch.int16, "dR"),
                                           hp(post, torch.float32, "post"), _stream(stream)))

    def set_profiling(self, on=True):
        check(lib().elas_pipeline_set_profiling(self._h, int(bool(on))))

    def set_graph(self, on=True):
        check(lib().elas_pipeline_set_graph(self._h, int(bool(on))))

    def stats(self):
        st = PipelineStats()
        check(lib().elas_pipeline_stats_get(self._h, C.byref(st)))
        names = ("descriptors", "support", "triangulation", "plane_prior", "dense_argmin", "lr_post")
        return dict(n_support=st.n_support, n_tri_left=st.n_tri_left, n_tri_right=st.n_tri_right,
                    triangulate_ms=st.triangulate_ms, stage_ms={k: float(v) for k, v in zip(names, st.stage_ms)})

    def close(self):
        if self._h:
            lib().elas_pipeline_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cfg_dict(cfg):
    return {k: int(getattr(cfg, k)) for k, _ in BatchConfig._fields_}


def _ptr_array(ptrs):
    arr = (C.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


class Batch:
    """Owner of an ``elas_batch`` handle: many pairs, any mix of sizes and
    parameters, run together through batched launches (one launch per
    kernel for the whole batch)."""

    def __init__(self, shapes, prms):
        """shapes: list of (w, h); prms: one parameter block (shared) or a
        list with one per pair."""
        n = len(shapes)
        if not isinstance(prms, (list, tuple)):
            prms = [prms] * n
        if len(prms) != n:
            raise ValueError("%d shapes but %d parameter blocks" % (n, len(prms)))
        self.shapes = [(int(w), int(h)) for w, h in shapes]
        self.prms = [as_params(p) for p in prms]
        ws = (C.c_int32 * n)(*[w for w, _ in self.shapes])
        hs = (C.c_int32 * n)(*[h for _, h in self.shapes])
        parr = (Params * n)(*self.prms)
        self._h = C.c_void_p()
        check(lib().elas_batch_create(n, ws, hs, parr, C.byref(self._h)))

    def __len__(self):
        return len(self.shapes)

    def config(self):
        cfg = BatchConfig()
        check(lib().elas_batch_get_config(self._h, C.byref(cfg)))
        return _cfg_dict(cfg)

    def set_config(self, **kw):
        cur = self.config()
        cur.update(kw)
        cfg = BatchConfig(cur["desc_tile_rows"], cur["support_warps"], cur["dense_threads_per_pixel"],
                          cur["use_graph"], cur["dense_pixels_per_thread"], cur.get("dense_fused", 0))
        check(lib().elas_batch_set_config(self._h, C.byref(cfg)))

    def _dev_arrays(self, imgL, imgR, dL, dR, post):
        n = len(self)
        if len(imgL) != n or len(imgR) != n or len(dL) != n:
            raise ValueError("expected %d pairs" % n)
        pl, pr, pd, pdr, pp = [], [], [], [], []
        for i, (w, h) in enumerate(self.shapes):
            pl.append(_dev(imgL[i], torch.uint8, "imgL[%d]" % i, (h, w)))
            pr.append(_dev(imgR[i], torch.uint8, "imgR[%d]" % i, (h, w)))
            pd.append(_dev(dL[i], torch.int16, "dL[%d]" % i, (h, w)))
            pdr.append(None if dR is None or dR[i] is None else _dev(dR[i], torch.int16, "dR[%d]" % i, (h, w)))
            pp.append(None if post is None or post[i] is None else _dev(post[i], torch.float32, "post[%d]" % i, (h, w)))
        return _ptr_array(pl), _ptr_array(pr), _ptr_array(pd), _ptr_array(pdr), _ptr_array(pp)

    def run(self, imgL, imgR, dL, dR=None, post=None, stream=None):
        """Lists of device tensors (dR/post may be None or hold None)."""
        aL, aR, aD, aDR, aP = self._dev_arrays(imgL, imgR, dL, dR, post)
        check(lib().elas_batch_run(self._h, aL, aR, None, aD, aDR, aP, _stream(stream)))

    def run_host(self, imgL, imgR, dL, dR=None, post=None, stream=None):
        """Lists of host (ideally pinned) tensors; returns when done."""
        def hp(t, dtype, name, shape):
            if t is None:
                return None
            if t.is_cuda or t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != shape:
                raise TypeError("%s must be a contiguous host %s tensor of shape %s" % (name, dtype, shape))
            return C.c_void_p(t.data_ptr())
        n = len(self)
        pl, pr, pd, pdr, pp = [], [], [], [], []
        for i, (w, h) in enumerate(self.shapes):
            pl.append(hp(imgL[i], torch.uint8, "imgL[%d]" % i, (h, w)))
            pr.append(hp(imgR[i], torch.uint8, "imgR[%d]" % i, (h, w)))
            pd.append(hp(dL[i], torch.int16, "dL[%d]" % i, (h, w)))
            pdr.append(None if dR is None else hp(dR[i], torch.int16, "dR[%d]" % i, (h, w)))
            pp.append(None if post is None else hp(post[i], torch.float32, "post[%d]" % i, (h, w)))
        assert len(pl) == n
        check(lib().elas_batch_run_host(self._h, _ptr_array(pl), _ptr_array(pr), _ptr_array(pd), _ptr_array(pdr),
                                        _ptr_array(pp), _stream(stream)))

    def stats(self):
        n = len(self)
        a, b, c = (C.c_int32 * n)(), (C.c_int32 * n)(), (C.c_int32 * n)()
        check(lib().elas_batch_stats(self._h, a, b, c))
        return dict(n_support=list(a), n_tri_left=list(b), n_tri_right=list(c))

    def tune(self, imgL, imgR, dL, stream=None):
        aL, aR, aD, _, _ = self._dev_arrays(imgL, imgR, dL, None, None)
        cfg = BatchConfig()
        check(lib().elas_batch_tune(self._h, aL, aR, None, aD, _stream(stream), C.byref(cfg)))
        return _cfg_dict(cfg)

    def profile(self, stream=None):
        """Device ms of each stage of one eager run on the last-bound buffers."""
        ms = (C.c_float * 6)()
        check(lib().elas_batch_profile(self._h, _stream(stream), ms))
        names = ("descriptors", "support", "triangulation", "plane_prior", "dense_argmin", "lr_post")
        return {k: float(v) for k, v in zip(names, ms)}

    def device_bytes(self):
        return int(lib().elas_batch_device_bytes(self._h))

    def close(self):
        if self._h:
            lib().elas_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owner of an ``elas_server`` handle: requests with host buffers are
    queued with ``submit`` and their results collected with ``poll``."""

    def __init__(self, lanes=None, max_wave=None, max_slots=None, plain=False, hbm_budget_bytes=None,
                 hbm_reserve_bytes=None):
        cfg = ServerConfig()
        check(lib().elas_server_config_default(C.byref(cfg)))
        for k, v in dict(lanes=lanes, max_wave=max_wave, max_slots=max_slots, hbm_budget_bytes=hbm_budget_bytes,
                         hbm_reserve_bytes=hbm_reserve_bytes).items():
            if v is not None:
                setattr(cfg, k, int(v))
        cfg.plain = 1 if plain else 0
        self._h = C.c_void_p()
        self._keep = {}  # request id -> buffers that must outlive the request
        check(lib().elas_server_create(C.byref(cfg), C.byref(self._h)))

    def submit(self, rid, imgL, imgR, dL, prm=None, post=None):
        """imgL/imgR: host uint8 tensors [h, w]; dL: host int16 [h, w];
        post: host float32 [h, w] or None.  Pinned tensors copy fastest."""
        prm = as_params(prm)
        h, w = imgL.shape
        for t, dt, name in ((imgL, torch.uint8, "imgL"), (imgR, torch.uint8, "imgR"), (dL, torch.int16, "dL"),
                            (post, torch.float32, "post")):
            if t is None:
                continue
            if t.is_cuda or t.dtype != dt or not t.is_contiguous() or tuple(t.shape) != (h, w):
                raise TypeError("%s must be a contiguous host %s tensor [%d, %d]" % (name, dt, h, w))
        check(lib().elas_server_submit(self._h, int(rid), w, h, C.byref(prm), C.c_void_p(imgL.data_ptr()),
                                       C.c_void_p(imgR.data_ptr()), C.c_void_p(dL.data_ptr()),
                                       None if post is None else C.c_void_p(post.data_ptr())))
        self._keep[int(rid)] = (imgL, imgR, dL, post)

    def poll(self, max_results=256, timeout_ms=0):
        buf = (ServerResult * max_results)()
        k = lib().elas_server_poll(self._h, buf, max_results, int(timeout_ms))
        if k < 0:
            raise ElasError(1, "poll")
        out = []
        for i in range(k):
            r = buf[i]
            self._keep.pop(int(r.id), None)
            out.append(dict(id=int(r.id), status=int(r.status), n_support=int(r.n_support),
                            wave_size=int(r.wave_size), t_submit_ms=r.t_submit_ms, t_start_ms=r.t_start_ms,
                            t_done_ms=r.t_done_ms))
        return out

    def now_ms(self):
        return float(lib().elas_server_now_ms(self._h))

    def drain(self, timeout_ms):
        """Waits for every submitted request's result; ElasError with
        ELAS_ERR_TIMEOUT when timeout_ms runs out first."""
        check(lib().elas_server_drain(self._h, int(timeout_ms)))

    def inject_alloc_failures(self, n):
        """Testing: the next n slot allocations report out of memory."""
        check(lib().elas_server_inject_alloc_failures(self._h, int(n)))

    def stats(self):
        st = ServerStats()
        check(lib().elas_server_stats_get(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            lib().elas_server_destroy(self._h)
            self._h = C.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
