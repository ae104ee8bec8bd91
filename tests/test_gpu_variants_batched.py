"""The paper's own variant in batches and in the serving loop: census
descriptors over full windows with Hamming costs (Sec. VI.A, Table I window
sizes), the support down-sampling of Sec. VII, and the shift-sum threshold
(Eq. 3) with the past-only redundancy rule (Sec. VI.C), mixed in one batch
with Sobel/SAD pairs of other sizes.  Every pair's maps must equal the
oracle's for that pair alone (integer maps bit-exact, post-processing within
1e-4), eagerly and from the captured graph, and so must every result of the
server."""
import time

import numpy as np
import pytest

import oracle
from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _B():
    from paper_1802_07210_gb300 import binding
    return binding


def _mix():
    flags = oracle.FLAG_SHIFT_SUM | oracle.FLAG_PAST_REDUNDANCY
    vga, small = synth.VGA_640, synth.SMALL_320
    kitti = synth.KITTI_1242
    return [
        ("census_9_5", vga, 2, 0, dict(vga.params, census_support_w=9, census_dense_w=5), True),
        ("census_13_7", small, 1, 1, dict(small.params, census_support_w=13, census_dense_w=7), False),
        ("census_9_5_b", small, 1, 2, dict(small.params, census_support_w=9, census_dense_w=5, beta=0.1), False),
        ("downsample_8", vga, 2, 1, dict(vga.params, support_downsample=8), True),
        ("every_pixel_ds14", small, 1, 3, dict(small.params, candidate_stepsize=1, support_downsample=14), False),
        ("census_ds8_flags", kitti, 3, 0,
         dict(kitti.params, census_support_w=9, census_dense_w=5, support_downsample=8, flags=flags), False),
        ("sobel_flags", kitti, 3, 1, dict(kitti.params, flags=flags), False),
        ("sobel_plain", small, 1, 4, dict(small.params), True),
    ]


MIX = _mix()


@pytest.fixture(scope="module")
def mix():
    out = []
    for name, wl, cfg, idx, prm, post in MIX:
        L, R, _ = synth.workload_pair(wl, idx, cfg)
        prm = dict(prm)
        if post:
            prm.update(ipol_gap_width=3, filter_adaptive_mean=1)
        out.append(dict(name=name, L=L, R=R, prm=prm, post=post,
                        ref=oracle.pipeline(L, R, prm, postprocess_on=post)))
    return out


def _check(it, dL, dR, post, what):
    ref = it["ref"]
    np.testing.assert_array_equal(dL, ref["lrL"], err_msg="%s %s left" % (what, it["name"]))
    if dR is not None:
        np.testing.assert_array_equal(dR, ref["lrR"], err_msg="%s %s right" % (what, it["name"]))
    if it["post"] and post is not None:
        assert np.abs(post - ref["post"]).max() <= 1e-4, (what, it["name"])


@pytest.mark.parametrize("fused", [0, 1])
def test_variant_mix_in_one_batch(mix, fused):
    """fused: the plane prior and the dense argmin (Sobel/SAD and census
    pairs alike) in one persistent cooperative launch."""
    B = _B()
    b = B.Batch([(it["L"].shape[1], it["L"].shape[0]) for it in mix], [it["prm"] for it in mix])
    b.set_config(dense_fused=fused)
    dL = [torch.empty(it["L"].shape, dtype=torch.int16, device="cuda") for it in mix]
    dR = [torch.empty_like(t) for t in dL]
    post = [torch.empty(it["L"].shape, dtype=torch.float32, device="cuda") if it["post"] else None for it in mix]
    imgL = [dev(it["L"]) for it in mix]
    imgR = [dev(it["R"]) for it in mix]
    for run in range(3):  # eager, captured, replayed
        for t in dL + dR:
            t.fill_(-7)
        b.run(imgL, imgR, dL, dR, post)
        for i, it in enumerate(mix):
            _check(it, host(dL[i]), host(dR[i]), host(post[i]) if post[i] is not None else None, "run %d" % run)
    st = b.stats()
    for i, it in enumerate(mix):
        assert st["n_support"][i] == len(it["ref"]["list"]), it["name"]
        assert st["n_tri_left"][i] == len(it["ref"]["triL"]), it["name"]
    b.close()


def test_variant_batch_of_one_census_kind(mix):
    """A batch of census pairs only (no descriptor launch at all) and a
    batch of down-sampled Sobel pairs only."""
    B = _B()
    for names in (("census_9_5", "census_13_7", "census_9_5_b"), ("downsample_8", "every_pixel_ds14")):
        items = [it for it in mix if it["name"] in names]
        b = B.Batch([(it["L"].shape[1], it["L"].shape[0]) for it in items], [it["prm"] for it in items])
        dL = [torch.empty(it["L"].shape, dtype=torch.int16, device="cuda") for it in items]
        dR = [torch.empty_like(t) for t in dL]
        b.run([dev(it["L"]) for it in items], [dev(it["R"]) for it in items], dL, dR)
        for i, it in enumerate(items):
            _check(it, host(dL[i]), host(dR[i]), None, "kind batch")
        b.close()


def test_variant_requests_served(mix):
    B = _B()
    srv = B.Server(lanes=2, max_wave=8)
    bufs = []
    for i, it in enumerate(mix):
        h, w = it["L"].shape
        bufs.append(dict(L=torch.from_numpy(it["L"]).pin_memory(), R=torch.from_numpy(it["R"]).pin_memory(),
                         dL=torch.full((h, w), -7, dtype=torch.int16).pin_memory(),
                         post=torch.zeros((h, w), dtype=torch.float32).pin_memory() if it["post"] else None))
        srv.submit(i, bufs[i]["L"], bufs[i]["R"], bufs[i]["dL"], it["prm"], bufs[i]["post"])
    results = {}
    t0 = time.time()
    while len(results) < len(mix):
        for r in srv.poll(64, 200):
            results[r["id"]] = r
        assert time.time() - t0 < 120, "server did not finish"
    for i, it in enumerate(mix):
        assert results[i]["status"] == 0, (it["name"], results[i])
        assert results[i]["n_support"] == len(it["ref"]["list"]), it["name"]
        _check(it, bufs[i]["dL"].numpy(), None, bufs[i]["post"].numpy() if bufs[i]["post"] is not None else None,
               "server")
    srv.close()
