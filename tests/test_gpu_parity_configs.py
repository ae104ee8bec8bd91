"""End-to-end parity with the oracle at the full sizes of the paper-shaped
workloads (Sec. VII: KITTI 1242x375; the 1280x720 and 1920x1080 camera
shapes of the mixed batch and the serving mix), through every route a user
takes: the per-pair pipeline, the batched path (mixed sizes and disparity
ranges in one launch per kernel; eight 1242x375 pairs, enough lattice rows
for the row-organised support matcher) and the serving loop.

Integer maps (LR-checked left and right disparities) must be bit-exact, the
support-point and triangle counts equal, and the post-processed map within
1e-4.  These sizes reach code the small cases never take: the row-organised
support matcher, long star chains in the triangulation, big-triangle splits
in the rasteriser and candidate lists near the full disparity range.

The oracle runs on the host in a thread pool (its C calls release the
interpreter lock), one pair per thread."""
import concurrent.futures as cf
import os
import time

import numpy as np
import pytest

import oracle
from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu

POST_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _B():
    from paper_1802_07210_gb300 import binding
    return binding


def _post(wl):
    return dict(wl.params, ipol_gap_width=3, filter_adaptive_mean=1)


# (name, workload, cfg id, pair index, post-process)
def _items():
    big = []
    for D in (64, 128, 256):
        big.append(("1280x720_D%d" % D, synth.scaled_workload(1280, 720, D), 4, D, D == 128))
        big.append(("1920x1080_D%d" % D, synth.scaled_workload(1920, 1080, D), 4, D, D == 256))
    kitti = [("kitti_%d" % i, synth.KITTI_1242, 3, i, i == 1) for i in range(8)]
    mixed = [("320x240_D64", synth.scaled_workload(320, 240, 64), 4, 0, False),
             ("640x480_D128", synth.scaled_workload(640, 480, 128), 4, 0, True),
             ("1242x375_D128", synth.scaled_workload(1242, 375, 128), 4, 0, False)]
    return big, kitti, mixed


BIG, KITTI, MIXED = _items()


def _oracle_job(item):
    name, wl, cfg, idx, post = item
    L, R, _ = synth.workload_pair(wl, idx, cfg)
    prm = _post(wl) if post else dict(wl.params)
    r = oracle.pipeline(L, R, prm, postprocess_on=post)
    return name, dict(name=name, L=L, R=R, prm=prm, post=post, lrL=r["lrL"], lrR=r["lrR"],
                      n_support=len(r["list"]), ntriL=len(r["triL"]), ntriR=len(r["triR"]),
                      postmap=r.get("post"))


@pytest.fixture(scope="module")
def ref():
    """Oracle results of every pair of this module, keyed by name."""
    oracle.lib()
    items = BIG + KITTI + MIXED
    t0 = time.time()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(items), os.cpu_count() or 1))) as ex:
        out = dict(ex.map(_oracle_job, sorted(items, key=lambda it: -it[1].spec.w * it[1].spec.h)))
    print("oracle: %d pairs in %.1f s" % (len(out), time.time() - t0))
    return out


def _check(it, dL, dR, post, what, stats=None):
    np.testing.assert_array_equal(dL, it["lrL"], err_msg="%s %s left" % (what, it["name"]))
    if dR is not None:
        np.testing.assert_array_equal(dR, it["lrR"], err_msg="%s %s right" % (what, it["name"]))
    if it["post"] and post is not None:
        err = float(np.abs(post - it["postmap"]).max())
        assert err <= POST_TOL, (what, it["name"], err)
        assert ((post < 0) == (it["postmap"] < 0)).all(), (what, it["name"])
    if stats is not None:
        assert stats == (it["n_support"], it["ntriL"], it["ntriR"]), (what, it["name"], stats)


def _run_pipeline(it):
    B = _B()
    h, w = it["L"].shape
    pl = B.Pipeline(w, h, it["prm"])
    dL = torch.full((h, w), -7, dtype=torch.int16, device="cuda")
    dR = torch.full_like(dL, -7)
    post = torch.empty((h, w), dtype=torch.float32, device="cuda") if it["post"] else None
    pl.run(dev(it["L"]), dev(it["R"]), dL, dR, post)
    st = pl.stats()
    res = host(dL), host(dR), (host(post) if post is not None else None), \
        (st["n_support"], st["n_tri_left"], st["n_tri_right"])
    pl.close()
    return res


@pytest.mark.parametrize("name", [it[0] for it in BIG] + ["kitti_0", "kitti_1"])
def test_per_pair_pipeline_full_size(ref, name):
    """The plain one-pair path at each full camera size and disparity range
    (and 1242x375 D=256 with the ground plane and noise sigma 3)."""
    it = ref[name]
    dL, dR, post, st = _run_pipeline(it)
    _check(it, dL, dR, post, "pipeline", st)


def test_batch_of_kitti_pairs(ref):
    """Eight distinct 1242x375 D=256 pairs in one batch: 600 lattice rows, so
    the batched support stage takes the row-organised matcher; run eagerly,
    then captured and replayed as a CUDA graph."""
    B = _B()
    items = [ref[it[0]] for it in KITTI]
    b = B.Batch([(it["L"].shape[1], it["L"].shape[0]) for it in items], [it["prm"] for it in items])
    dL = [torch.empty(it["L"].shape, dtype=torch.int16, device="cuda") for it in items]
    dR = [torch.empty_like(t) for t in dL]
    post = [torch.empty(it["L"].shape, dtype=torch.float32, device="cuda") if it["post"] else None
            for it in items]
    imgL = [dev(it["L"]) for it in items]
    imgR = [dev(it["R"]) for it in items]
    for run in range(3):
        for t in dL + dR:
            t.fill_(-7)
        b.run(imgL, imgR, dL, dR, post)
        st = b.stats()
        for i, it in enumerate(items):
            _check(it, host(dL[i]), host(dR[i]), host(post[i]) if post[i] is not None else None,
                   "batch run %d" % run, (st["n_support"][i], st["n_tri_left"][i], st["n_tri_right"][i]))
    b.close()


def test_mixed_batch_every_size(ref):
    """One batch holding every size of the mixed workload (320x240, 640x480,
    1242x375, 1280x720, 1920x1080) with disparity ranges 64, 128 and 256:
    each pair's maps equal the oracle's for that pair alone."""
    B = _B()
    names = [it[0] for it in MIXED] + ["kitti_0", "1280x720_D128", "1280x720_D256", "1920x1080_D64",
                                       "1920x1080_D256"]
    items = [ref[n] for n in names]
    b = B.Batch([(it["L"].shape[1], it["L"].shape[0]) for it in items], [it["prm"] for it in items])
    dL = [torch.full(it["L"].shape, -7, dtype=torch.int16, device="cuda") for it in items]
    dR = [torch.full_like(t, -7) for t in dL]
    post = [torch.empty(it["L"].shape, dtype=torch.float32, device="cuda") if it["post"] else None
            for it in items]
    for run in range(2):
        b.run([dev(it["L"]) for it in items], [dev(it["R"]) for it in items], dL, dR, post)
        st = b.stats()
        for i, it in enumerate(items):
            _check(it, host(dL[i]), host(dR[i]), host(post[i]) if post[i] is not None else None,
                   "mixed run %d" % run, (st["n_support"][i], st["n_tri_left"][i], st["n_tri_right"][i]))
    b.close()


def test_server_camera_shapes(ref):
    """The serving loop with the camera shapes of the serving mix (640x480
    D=128, 1242x375 D=256, 1920x1080 D=256), submitted as a burst and then
    one by one: every result equals the oracle's, with host buffers."""
    B = _B()
    names = ["640x480_D128", "kitti_0", "kitti_1", "kitti_2", "1920x1080_D256", "1920x1080_D128"]
    items = [ref[n] for n in names]
    for stagger in (0.0, 0.002):
        srv = B.Server(lanes=3, max_wave=8)
        bufs = []
        for i, it in enumerate(items):
            h, w = it["L"].shape
            bufs.append(dict(L=torch.from_numpy(it["L"]).pin_memory(), R=torch.from_numpy(it["R"]).pin_memory(),
                             dL=torch.full((h, w), -7, dtype=torch.int16).pin_memory(),
                             post=torch.zeros((h, w), dtype=torch.float32).pin_memory() if it["post"] else None))
        results = {}
        for i, it in enumerate(items):
            srv.submit(i, bufs[i]["L"], bufs[i]["R"], bufs[i]["dL"], it["prm"], bufs[i]["post"])
            if stagger:
                time.sleep(stagger)
        t0 = time.time()
        while len(results) < len(items):
            for res in srv.poll(64, 200):
                results[res["id"]] = res
            assert time.time() - t0 < 120, "server did not finish"
        for i, it in enumerate(items):
            res = results[i]
            assert res["status"] == 0, (it["name"], res)
            assert res["n_support"] == it["n_support"], it["name"]
            _check(it, bufs[i]["dL"].numpy(), None,
                   bufs[i]["post"].numpy() if bufs[i]["post"] is not None else None, "server")
        srv.close()
