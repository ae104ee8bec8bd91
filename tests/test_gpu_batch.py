"""Batched path (elas_batch_*): pairs of mixed sizes, disparity ranges and
parameters run through one launch per kernel.  Every pair's result in the
mix must equal the oracle's for that pair alone (integer maps bit-exact,
post-processed maps within 1e-4) and the per-pair path's result, for every
tile-shape setting the tuner can pick, eagerly and through the captured
CUDA graph, with device and with host buffers."""
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


def _mix():
    ragged = synth.scaled_workload(203, 117, 48)
    ragged.params["disp_min"] = 3
    ragged.params["ipol_gap_width"] = 3
    ragged.params["filter_adaptive_mean"] = 1
    tiny = synth.scaled_workload(48, 40, 16)
    wide = synth.scaled_workload(621, 188, 128)
    full = synth.scaled_workload(160, 120, 32)
    full.params["flags"] = 2  # every in-range d is a candidate, no prior
    # (name, workload, cfg id, pair index, post-process)
    return [
        ("small_320_a", synth.SMALL_320, 1, 0, False),
        ("small_320_b", synth.SMALL_320, 1, 1, True),
        ("ragged_203x117", ragged, 7, 0, True),
        ("vga_640", synth.VGA_640, 2, 0, True),
        ("wide_621x188", wide, 3, 0, False),
        ("tiny_48x40", tiny, 9, 0, False),
        ("full_range_160x120", full, 8, 0, True),
    ]


MIX = _mix()


@pytest.fixture(scope="module")
def mix():
    out = []
    for name, wl, cfg, idx, post in MIX:
        L, R, _ = synth.workload_pair(wl, idx, cfg)
        prm = dict(wl.params)
        if post and not prm.get("ipol_gap_width") and not prm.get("filter_adaptive_mean"):
            prm.update(ipol_gap_width=3, filter_adaptive_mean=1)
        ref = oracle.pipeline(L, R, prm, postprocess_on=post)
        out.append(dict(name=name, L=L, R=R, prm=prm, post=post, ref=ref))
    return out


def _alloc(items):
    dL = [torch.empty(it["L"].shape, dtype=torch.int16, device="cuda") for it in items]
    dR = [torch.empty_like(t) for t in dL]
    post = [torch.empty(it["L"].shape, dtype=torch.float32, device="cuda") if it["post"] else None
            for it in items]
    return dL, dR, post


def _check(items, dL, dR, post, what):
    for i, it in enumerate(items):
        ref = it["ref"]
        np.testing.assert_array_equal(host(dL[i]), ref["lrL"], err_msg="%s %s left" % (what, it["name"]))
        np.testing.assert_array_equal(host(dR[i]), ref["lrR"], err_msg="%s %s right" % (what, it["name"]))
        if it["post"]:
            out = host(post[i])
            assert np.abs(out - ref["post"]).max() <= POST_TOL, (what, it["name"])
            assert ((out < 0) == (ref["post"] < 0)).all(), (what, it["name"])


def _batch(items):
    B = _B()
    return B.Batch([(it["L"].shape[1], it["L"].shape[0]) for it in items], [it["prm"] for it in items])


def test_mixed_batch_matches_oracle(mix):
    b = _batch(mix)
    imgL = [dev(it["L"]) for it in mix]
    imgR = [dev(it["R"]) for it in mix]
    dL, dR, post = _alloc(mix)
    # run 1: eager; run 2: captures the graph; run 3: replays it
    for run in range(3):
        for t in dL + dR:
            t.fill_(-7)
        b.run(imgL, imgR, dL, dR, post)
        _check(mix, dL, dR, post, "run %d" % run)
    st = b.stats()
    for i, it in enumerate(mix):
        ref = it["ref"]
        assert st["n_support"][i] == len(ref["list"]), it["name"]
        assert st["n_tri_left"][i] == len(ref["triL"]), it["name"]
        assert st["n_tri_right"][i] == len(ref["triR"]), it["name"]
    # new output buffers (the tables are re-bound, the graph is kept)
    dL2, dR2, post2 = _alloc(mix)
    b.run(imgL, imgR, dL2, dR2, post2)
    _check(mix, dL2, dR2, post2, "rebound")
    # post-processing switched off for every pair (a new graph)
    dL3, dR3, _ = _alloc(mix)
    b.run(imgL, imgR, dL3, dR3, None)
    for i, it in enumerate(mix):
        np.testing.assert_array_equal(host(dL3[i]), it["ref"]["lrL"])
    b.close()


def test_mixed_batch_equals_per_pair_path(mix):
    """Each pair in the mix gives what the per-pair path gives for it alone."""
    B = _B()
    b = _batch(mix)
    dL, dR, post = _alloc(mix)
    b.run([dev(it["L"]) for it in mix], [dev(it["R"]) for it in mix], dL, dR, post)
    for i, it in enumerate(mix):
        h, w = it["L"].shape
        pl = B.Pipeline(w, h, it["prm"])
        aL = torch.empty((h, w), dtype=torch.int16, device="cuda")
        aR = torch.empty_like(aL)
        ap = torch.empty((h, w), dtype=torch.float32, device="cuda") if it["post"] else None
        pl.run(dev(it["L"]), dev(it["R"]), aL, aR, ap)
        np.testing.assert_array_equal(host(dL[i]), host(aL))
        np.testing.assert_array_equal(host(dR[i]), host(aR))
        if it["post"]:
            np.testing.assert_array_equal(host(post[i]), host(ap))
        pl.close()
    b.close()


KNOBS = [
    dict(desc_tile_rows=36, support_warps=4, dense_threads_per_pixel=1, dense_pixels_per_thread=1, dense_fused=0),
    dict(desc_tile_rows=24, support_warps=16, dense_threads_per_pixel=2, dense_pixels_per_thread=2, dense_fused=0),
    dict(desc_tile_rows=12, support_warps=8, dense_threads_per_pixel=4, dense_pixels_per_thread=1, dense_fused=0),
    dict(desc_tile_rows=24, support_warps=4, dense_threads_per_pixel=1, dense_pixels_per_thread=4, dense_fused=0),
    dict(desc_tile_rows=36, support_warps=8, dense_threads_per_pixel=4, dense_pixels_per_thread=4, dense_fused=0),
    dict(desc_tile_rows=12, support_warps=16, dense_threads_per_pixel=1, dense_pixels_per_thread=8, dense_fused=0),
    # the prior and the argmin as one persistent cooperative launch
    dict(desc_tile_rows=24, support_warps=8, dense_threads_per_pixel=1, dense_pixels_per_thread=16, dense_fused=1),
    dict(desc_tile_rows=24, support_warps=8, dense_threads_per_pixel=2, dense_pixels_per_thread=16, dense_fused=1),
    dict(desc_tile_rows=12, support_warps=4, dense_threads_per_pixel=4, dense_pixels_per_thread=4, dense_fused=1),
]


@pytest.mark.parametrize("knobs", KNOBS, ids=lambda k: "%d-%d-%d-%d-%d" % tuple(k.values()))
@pytest.mark.parametrize("graph", [0, 1])
def test_knob_settings_give_identical_results(mix, knobs, graph):
    b = _batch(mix)
    b.set_config(use_graph=graph, **knobs)
    assert b.config() == dict(knobs, use_graph=graph)
    dL, dR, post = _alloc(mix)
    for run in range(2):
        b.run([dev(it["L"]) for it in mix], [dev(it["R"]) for it in mix], dL, dR, post)
        _check(mix, dL, dR, post, "knobs %s graph %d run %d" % (knobs, graph, run))
    b.close()


def test_tuner_picks_valid_knobs(mix):
    b = _batch(mix)
    imgL = [dev(it["L"]) for it in mix]
    imgR = [dev(it["R"]) for it in mix]
    dL, dR, post = _alloc(mix)
    cfg = b.tune(imgL, imgR, dL)
    assert cfg["desc_tile_rows"] in (12, 24, 36)
    assert cfg["support_warps"] in (4, 8, 16)
    assert cfg["dense_threads_per_pixel"] in (1, 2, 4)
    assert cfg["dense_pixels_per_thread"] in (1, 2, 4, 8, 16)
    assert cfg["dense_fused"] in (0, 1)
    assert b.config()["desc_tile_rows"] == cfg["desc_tile_rows"]
    b.run(imgL, imgR, dL, dR, post)
    _check(mix, dL, dR, post, "tuned")
    # a second batch of the same shapes starts from the tuned setting
    b2 = _batch(mix)
    c2 = b2.config()
    assert c2 == cfg
    b2.close()
    b.close()


def test_run_host(mix):
    b = _batch(mix)
    hL = [torch.from_numpy(it["L"]).pin_memory() for it in mix]
    hR = [torch.from_numpy(it["R"]).pin_memory() for it in mix]
    oL = [torch.empty(it["L"].shape, dtype=torch.int16).pin_memory() for it in mix]
    oR = [torch.empty(it["L"].shape, dtype=torch.int16).pin_memory() for it in mix]
    op = [torch.empty(it["L"].shape, dtype=torch.float32).pin_memory() if it["post"] else None for it in mix]
    for _ in range(2):
        b.run_host(hL, hR, oL, oR, op)
        for i, it in enumerate(mix):
            np.testing.assert_array_equal(oL[i].numpy(), it["ref"]["lrL"])
            np.testing.assert_array_equal(oR[i].numpy(), it["ref"]["lrR"])
            if it["post"]:
                assert np.abs(op[i].numpy() - it["ref"]["post"]).max() <= POST_TOL
    b.close()


def test_uniform_batch_of_many_pairs():
    """A larger uniform batch (the shape of a camera batch): every pair equals
    the per-pair path, run alone."""
    B = _B()
    wl = synth.SMALL_320
    n = 24
    pairs = [synth.workload_pair(wl, i, 1)[:2] for i in range(n)]
    b = B.Batch([(320, 240)] * n, wl.params)
    dL = [torch.empty((240, 320), dtype=torch.int16, device="cuda") for _ in range(n)]
    dR = [torch.empty_like(t) for t in dL]
    b.run([dev(L) for L, _ in pairs], [dev(R) for _, R in pairs], dL, dR)
    b.run([dev(L) for L, _ in pairs], [dev(R) for _, R in pairs], dL, dR)
    pl = B.Pipeline(320, 240, wl.params)
    aL = torch.empty((240, 320), dtype=torch.int16, device="cuda")
    aR = torch.empty_like(aL)
    for i, (L, R) in enumerate(pairs):
        pl.run(dev(L), dev(R), aL, aR)
        np.testing.assert_array_equal(host(dL[i]), host(aL))
        np.testing.assert_array_equal(host(dR[i]), host(aR))
    # and the first pair against the oracle
    ref = oracle.pipeline(pairs[0][0], pairs[0][1], wl.params)
    np.testing.assert_array_equal(host(dL[0]), ref["lrL"])
    pl.close()
    b.close()


@pytest.mark.parametrize("idx", [2, 3, 6])
def test_batch_of_one_pair(mix, idx):
    """A batch of one pair takes the one-pair triangulation settings (wider
    groups, no warp pass): its maps still equal the oracle's."""
    it = mix[idx]
    b = _batch([it])
    dL, dR, post = _alloc([it])
    for run in range(3):
        b.run([dev(it["L"])], [dev(it["R"])], dL, dR, post)
        _check([it], dL, dR, post, "one pair run %d" % run)
    st = b.stats()
    assert st["n_tri_left"][0] == len(it["ref"]["triL"]) and st["n_tri_right"][0] == len(it["ref"]["triR"])
    b.close()


def test_batch_with_row_organised_support_matching():
    """Enough lattice rows (four 640x480 and four 1242x375 pairs) for the
    batched support stage to take the row-organised matcher: every pair's
    maps and support count equal the per-pair path's (the per-candidate
    matcher), and the first pair's support list equals the oracle's."""
    B = _B()
    items = [(synth.VGA_640, 2, i) for i in range(4)] + [(synth.KITTI_1242, 3, i) for i in range(4)]
    pairs = [synth.workload_pair(wl, idx, cfg)[:2] for wl, cfg, idx in items]
    shapes = [(wl.spec.w, wl.spec.h) for wl, _, _ in items]
    # two pairs take the paper's shift-sum threshold and past-only redundancy
    variants = oracle.FLAG_SHIFT_SUM | oracle.FLAG_PAST_REDUNDANCY
    prms = [dict(wl.params, flags=variants) if i in (1, 5) else dict(wl.params) for i, (wl, _, _) in enumerate(items)]
    b = B.Batch(shapes, prms)
    dL = [torch.empty((h, w), dtype=torch.int16, device="cuda") for w, h in shapes]
    dR = [torch.empty_like(t) for t in dL]
    b.run([dev(L) for L, _ in pairs], [dev(R) for _, R in pairs], dL, dR)
    st = b.stats()
    for i, ((wl, _, _), (L, R)) in enumerate(zip(items, pairs)):
        h, w = L.shape
        pl = B.Pipeline(w, h, prms[i])
        aL = torch.empty((h, w), dtype=torch.int16, device="cuda")
        aR = torch.empty_like(aL)
        pl.run(dev(L), dev(R), aL, aR)
        np.testing.assert_array_equal(host(dL[i]), host(aL), err_msg="pair %d left" % i)
        np.testing.assert_array_equal(host(dR[i]), host(aR), err_msg="pair %d right" % i)
        assert st["n_support"][i] == pl.stats()["n_support"], i
        pl.close()
    for i in (0, 1):
        L, R = pairs[i]
        ref = oracle.support_list(oracle.support_points(oracle.descriptors(L), oracle.descriptors(R), prms[i]),
                                  prms[i])
        assert st["n_support"][i] == len(ref)
    b.close()


def test_batch_of_the_maximum_size():
    """256 pairs, the most one batch takes: small pairs of varied sizes and
    disparity ranges (ragged widths and heights), every eighth one textureless
    (no support point, an empty triangulation, every pixel invalid). Each
    pair's maps equal the oracle's for that pair alone."""
    B = _B()
    shapes = [(48, 40, 16), (37, 29, 16), (64, 48, 32), (100, 30, 24), (29, 61, 8), (80, 20, 48)]
    items = []
    for i in range(256):
        w, h, D = shapes[i % len(shapes)]
        wl = synth.scaled_workload(w, h, D)
        if i % 8 == 7:
            L = np.full((h, w), 40 + i % 100, np.uint8)
            R = L.copy()
        else:
            L, R, _ = synth.workload_pair(wl, i, 11)
        items.append(dict(name="pair%d_%dx%d" % (i, w, h), L=L, R=R, prm=dict(wl.params), post=False,
                          ref=oracle.pipeline(L, R, wl.params, postprocess_on=False)))
    b = _batch(items)
    dL, dR, post = _alloc(items)
    for run in range(2):
        for t in dL + dR:
            t.fill_(-7)
        b.run([dev(it["L"]) for it in items], [dev(it["R"]) for it in items], dL, dR)
        _check(items, dL, dR, post, "256 pairs run %d" % run)
    st = b.stats()
    for i, it in enumerate(items):
        assert st["n_support"][i] == len(it["ref"]["list"]), it["name"]
        if i % 8 == 7:
            assert st["n_support"][i] == 0 and (host(dL[i]) == -1).all()
    b.close()


def test_invalid_batches():
    B = _B()
    prm = synth.SMALL_320.params
    with pytest.raises(B.ElasError):
        B.Batch([(4, 4)], prm)  # no lattice candidate at step 5
    with pytest.raises(B.ElasError):
        B.Batch([(320, 240)] * 257, prm)  # above 256 pairs
    b = B.Batch([(64, 48)], prm)
    with pytest.raises(B.ElasError):
        b.set_config(desc_tile_rows=5)
    with pytest.raises(ValueError):
        b.run([], [], [])
    b.close()
