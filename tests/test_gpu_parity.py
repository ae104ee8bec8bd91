"""Parity of the CUDA path (through the C-ABI) with the CPU oracle, step by
step and end to end, on seeded synthetic pairs shaped like the paper's
workloads (Sec. VII: KITTI 1242x375, New Tsukuba 640x480) and on edge cases.
Integer outputs must be bit-exact; the float post-processing must agree
within 1e-4 absolute."""
import numpy as np
import pytest

import oracle
from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, grid_as_i32, host, require_gpu, torch

pytestmark = pytest.mark.gpu

POST_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _B():
    from paper_1802_07210_gb300 import binding
    return binding


def _cases():
    small = synth.SMALL_320
    ragged = synth.scaled_workload(203, 117, 48)
    ragged.params["disp_min"] = 3
    return [
        ("small_320", small, 1),
        ("ragged_203x117", ragged, 7),
        ("vga_640", synth.VGA_640, 2),
    ]


CASES = _cases()


@pytest.fixture(scope="module")
def pairs():
    out = {}
    for name, wl, cfg in CASES:
        L, R, gt = synth.workload_pair(wl, 0, cfg)
        out[name] = (wl, L, R, oracle.pipeline(L, R, wl.params, postprocess_on=True))
    return out


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_descriptors(pairs, name):
    B = _B()
    wl, L, R, ref = pairs[name]
    dL, dR = B.elas_descriptors(dev(L), dev(R))
    np.testing.assert_array_equal(host(dL), ref["descL"])
    np.testing.assert_array_equal(host(dR), ref["descR"])
    # single-image form and a pitched image
    h, w = L.shape
    np.testing.assert_array_equal(host(B.elas_descriptors(dev(R))), ref["descR"])


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_support_points(pairs, name):
    B = _B()
    wl, L, R, ref = pairs[name]
    r = B.elas_support_points(dev(ref["descL"]), dev(ref["descR"]), wl.params)
    np.testing.assert_array_equal(host(r["d_can"]), ref["dcan"])
    n = int(host(r["count"])[0])
    assert n == len(ref["list"])
    np.testing.assert_array_equal(host(r["list"])[:n], ref["list"])
    np.testing.assert_array_equal(host(r["grid_L"]), grid_as_i32(ref["gridL"]))
    np.testing.assert_array_equal(host(r["grid_R"]), grid_as_i32(ref["gridR"]))


def test_support_raw_and_filters(pairs):
    """Each filter stage on its own: redundancy off exposes the consistency
    output; the raw matcher is checked through a window size of 0 with
    min_support 0 (every valid point kept)."""
    B = _B()
    wl, L, R, ref = pairs["small_320"]
    prm = dict(wl.params, incon_window_size=0, incon_min_support=0, flags=oracle.FLAG_REDUNDANCY_OFF)
    r = B.elas_support_points(dev(ref["descL"]), dev(ref["descR"]), prm)
    np.testing.assert_array_equal(host(r["d_can"]), oracle.support_match(ref["descL"], ref["descR"], wl.params))
    prm = dict(wl.params, flags=oracle.FLAG_REDUNDANCY_OFF)
    r = B.elas_support_points(dev(ref["descL"]), dev(ref["descR"]), prm)
    exp = oracle.filter_consistency(oracle.support_match(ref["descL"], ref["descR"], wl.params), wl.params)
    np.testing.assert_array_equal(host(r["d_can"]), exp)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_plane_prior(pairs, name):
    B = _B()
    wl, L, R, ref = pairs[name]
    h, w = L.shape
    lst = dev(ref["list"])
    for side, tri, exp in (("L", ref["triL"], ref["dplaneL"]), ("R", ref["triR"], ref["dplaneR"])):
        dp = B.elas_plane_prior(lst, dev(tri.astype(np.int32)), w, h, wl.params, right=(side == "R"))
        np.testing.assert_array_equal(host(dp), exp)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_dense_argmin(pairs, name):
    B = _B()
    wl, L, R, ref = pairs[name]
    dL, dR = dev(ref["descL"]), dev(ref["descR"])
    for right, dp, g, exp in ((False, ref["dplaneL"], ref["gridL"], ref["denseL"]),
                              (True, ref["dplaneR"], ref["gridR"], ref["denseR"])):
        out = B.elas_dense_argmin(dL, dR, wl.params, dev(dp), dev(grid_as_i32(g)), right=right)
        np.testing.assert_array_equal(host(out), exp)


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_dense_test_modes(pairs, flags):
    B = _B()
    wl, L, R, ref = pairs["ragged_203x117"]
    prm = dict(wl.params, flags=flags)
    for right, dp, g in ((False, ref["dplaneL"], ref["gridL"]), (True, ref["dplaneR"], ref["gridR"])):
        exp = oracle.dense(ref["descL"], ref["descR"], dp, g, prm, right=right)
        out = B.elas_dense_argmin(dev(ref["descL"]), dev(ref["descR"]), prm, dev(dp), dev(grid_as_i32(g)),
                                  right=right)
        np.testing.assert_array_equal(host(out), exp)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_dense_match_and_lr(pairs, name):
    B = _B()
    wl, L, R, ref = pairs[name]
    n = len(ref["list"])
    dL, dR = B.elas_dense_match(dev(ref["descL"]), dev(ref["descR"]), wl.params, dev(ref["list"]), n,
                                dev(ref["triL"].astype(np.int32)), dev(ref["triR"].astype(np.int32)),
                                dev(grid_as_i32(ref["gridL"])), dev(grid_as_i32(ref["gridR"])))
    np.testing.assert_array_equal(host(dL), ref["denseL"])
    np.testing.assert_array_equal(host(dR), ref["denseR"])
    mL, mR = B.elas_lr_check(dL, dR, wl.params["lr_threshold"])
    np.testing.assert_array_equal(host(dL), ref["lrL"])
    np.testing.assert_array_equal(host(dR), ref["lrR"])
    np.testing.assert_array_equal(host(mL), ref["maskL"])
    np.testing.assert_array_equal(host(mR), ref["maskR"])


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_postprocess(pairs, name):
    B = _B()
    wl, L, R, ref = pairs[name]
    prm = dict(wl.params, ipol_gap_width=3, filter_adaptive_mean=1)
    exp = oracle.postprocess(ref["lrL"], prm)
    out = host(B.elas_postprocess(dev(ref["lrL"]), prm))
    assert np.abs(out - exp).max() <= POST_TOL
    assert ((out < 0) == (exp < 0)).all()
    # widths up to 16 run the fused one-launch kernel, wider ones the four passes
    for gap, mean in ((0, 1), (3, 0), (0, 0), (16, 1), (17, 1), (40, 0), (1, 1)):
        prm = dict(wl.params, ipol_gap_width=gap, filter_adaptive_mean=mean)
        exp = oracle.postprocess(ref["lrL"], prm)
        out = host(B.elas_postprocess(dev(ref["lrL"]), prm))
        assert np.abs(out - exp).max() <= POST_TOL


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_pipeline_end_to_end(pairs, name):
    """The whole path through the pipeline handle (GPU kernels + the library's
    own host triangulation) against the oracle pipeline."""
    B = _B()
    wl, L, R, ref = pairs[name]
    h, w = L.shape
    pl = B.Pipeline(w, h, wl.params)
    dL = torch.empty((h, w), dtype=torch.int16, device="cuda")
    dR = torch.empty_like(dL)
    post = torch.empty((h, w), dtype=torch.float32, device="cuda")
    tL, tR = dev(L), dev(R)
    # run 1 eager, run 2 captured into a graph, runs 3-4 replayed, run 5 eager
    for graph in (True, True, True, True, False):
        pl.set_graph(graph)
        for t in (dL, dR):
            t.fill_(-7)
        pl.run(tL, tR, dL, dR, post)
        np.testing.assert_array_equal(host(dL), ref["lrL"])
        np.testing.assert_array_equal(host(dR), ref["lrR"])
        assert np.abs(host(post) - ref["post"]).max() <= POST_TOL
    st = pl.stats()
    assert st["n_support"] == len(ref["list"])
    assert st["n_tri_left"] == len(ref["triL"]) and st["n_tri_right"] == len(ref["triR"])
    # host-buffer path: repeated calls on the same pinned buffers (the step
    # replayed from its graph), new contents of those buffers, and pageable
    # buffers
    hL = torch.empty((h, w), dtype=torch.int16).pin_memory()
    hR = torch.empty((h, w), dtype=torch.int16).pin_memory()
    hpost = torch.empty((h, w), dtype=torch.float32).pin_memory()
    iL, iR = torch.from_numpy(L).pin_memory(), torch.from_numpy(R).pin_memory()
    for run in range(4):
        for t in (hL, hR):
            t.fill_(-7)
        hpost.fill_(-7.0)
        pl.run_host(iL, iR, hL, hR, hpost)
        np.testing.assert_array_equal(hL.numpy(), ref["lrL"], err_msg="host run %d" % run)
        np.testing.assert_array_equal(hR.numpy(), ref["lrR"], err_msg="host run %d" % run)
        assert np.abs(hpost.numpy() - ref["post"]).max() <= POST_TOL
    # the same buffers, the images swapped for a fronto-parallel pair
    L2, R2 = synth.fronto_parallel_pair(w, h, 7, seed=11, noise_sigma=1.0)
    ref2 = oracle.pipeline(L2, R2, wl.params, postprocess_on=True)
    iL.copy_(torch.from_numpy(L2))
    iR.copy_(torch.from_numpy(R2))
    pl.run_host(iL, iR, hL, hR, hpost)
    np.testing.assert_array_equal(hL.numpy(), ref2["lrL"])
    np.testing.assert_array_equal(hR.numpy(), ref2["lrR"])
    assert np.abs(hpost.numpy() - ref2["post"]).max() <= POST_TOL
    pL = torch.empty((h, w), dtype=torch.int16)
    ppost = torch.empty((h, w), dtype=torch.float32)
    for run in range(2):
        pl.run_host(torch.from_numpy(L), torch.from_numpy(R), pL, None, ppost)
        np.testing.assert_array_equal(pL.numpy(), ref["lrL"], err_msg="pageable run %d" % run)
        assert np.abs(ppost.numpy() - ref["post"]).max() <= POST_TOL
    pl.close()


def test_pipeline_graph_per_buffer_set():
    """A ring of ten input/output buffer sets (more than the eight graphs the
    handle keeps) cycled three times: every run, eager, captured or replayed,
    gives the eager result of its pair, and a buffer set's graph follows new
    contents of its buffers."""
    B = _B()
    wl = synth.SMALL_320
    h, w = wl.spec.h, wl.spec.w
    n = 10
    pairs = [synth.workload_pair(wl, 50 + i, 1)[:2] for i in range(n)]
    ref = B.Pipeline(w, h, wl.params)
    ref.set_graph(False)
    exp = []
    for L, R in pairs:
        eL = torch.empty((h, w), dtype=torch.int16, device="cuda")
        eR = torch.empty_like(eL)
        ref.run(dev(L), dev(R), eL, eR)
        exp.append((host(eL), host(eR)))
    ref.close()
    pl = B.Pipeline(w, h, wl.params)
    ins = [(dev(L), dev(R)) for L, R in pairs]
    outs = [(torch.empty((h, w), dtype=torch.int16, device="cuda"),
             torch.empty((h, w), dtype=torch.int16, device="cuda")) for _ in range(n)]
    order = list(range(n)) + list(range(n)) + [3, 1, 3, 1, 7, 7]
    for i in order:
        oL, oR = outs[i]
        oL.fill_(-7)
        oR.fill_(-7)
        pl.run(ins[i][0], ins[i][1], oL, oR)
        np.testing.assert_array_equal(host(oL), exp[i][0], err_msg="buffer set %d" % i)
        np.testing.assert_array_equal(host(oR), exp[i][1], err_msg="buffer set %d" % i)
    # new contents in buffer set 3 (its graph is replayed on them)
    ins[3][0].copy_(ins[5][0])
    ins[3][1].copy_(ins[5][1])
    for _ in range(2):
        pl.run(ins[3][0], ins[3][1], outs[3][0], outs[3][1])
        np.testing.assert_array_equal(host(outs[3][0]), exp[5][0])
    pl.close()


@pytest.mark.parametrize("size", [(37, 23), (64, 48), (203, 117)])
def test_median_filter(size):
    """Median filter of valid disparities (Sec. VII) against the oracle:
    random maps with invalid pixels, every radius, ragged sizes."""
    B = _B()
    w, h = size
    rng = np.random.default_rng(w * h)
    for top in (90, 1024):  # small values, and the whole range of disparities (kMaxDisp 1023)
        d = rng.integers(-1, top, size=(h, w)).astype(np.int16)
        d[rng.random((h, w)) < 0.2] = -1
        for r in range(4):
            out = host(B.elas_median(dev(d), r))
            np.testing.assert_array_equal(out, oracle.median(d, r), err_msg="radius %d values < %d" % (r, top))


def test_median_filter_on_a_disparity_map(pairs):
    B = _B()
    wl, L, R, ref = pairs["vga_640"]
    for r in (1, 2):
        np.testing.assert_array_equal(host(B.elas_median(dev(ref["lrL"]), r)), oracle.median(ref["lrL"], r))


@pytest.mark.parametrize("flags", [oracle.FLAG_SHIFT_SUM, oracle.FLAG_PAST_REDUNDANCY,
                                   oracle.FLAG_SHIFT_SUM | oracle.FLAG_PAST_REDUNDANCY])
@pytest.mark.parametrize("name", ["small_320", "vga_640"])
def test_support_points_paper_variants(pairs, name, flags):
    """The paper's shift-sum ambiguity threshold (Eq. 3) and past-only
    redundancy rule (Sec. VI.C) as flags: support output and grid vectors
    equal the oracle's."""
    B = _B()
    wl, L, R, ref = pairs[name]
    prm = dict(wl.params, flags=flags)
    r = B.elas_support_points(dev(ref["descL"]), dev(ref["descR"]), prm)
    exp = oracle.support_points(ref["descL"], ref["descR"], prm)
    np.testing.assert_array_equal(host(r["d_can"]), exp)
    lst = oracle.support_list(exp, prm)
    n = int(host(r["count"])[0])
    assert n == len(lst)
    np.testing.assert_array_equal(host(r["list"])[:n], lst)
    h, w = L.shape
    np.testing.assert_array_equal(host(r["grid_L"]), grid_as_i32(oracle.grid_vectors(lst, w, h, prm)))
    np.testing.assert_array_equal(host(r["grid_R"]), grid_as_i32(oracle.grid_vectors(lst, w, h, prm, right=True)))


def test_pipeline_with_paper_variants(pairs):
    """The whole one-pair path with both flags against the oracle pipeline."""
    B = _B()
    wl, L, R, _ = pairs["small_320"]
    prm = dict(wl.params, flags=oracle.FLAG_SHIFT_SUM | oracle.FLAG_PAST_REDUNDANCY)
    ref = oracle.pipeline(L, R, prm, postprocess_on=False)
    h, w = L.shape
    pl = B.Pipeline(w, h, prm)
    dL = torch.empty((h, w), dtype=torch.int16, device="cuda")
    dR = torch.empty_like(dL)
    for _ in range(2):
        pl.run(dev(L), dev(R), dL, dR)
        np.testing.assert_array_equal(host(dL), ref["lrL"])
        np.testing.assert_array_equal(host(dR), ref["lrR"])
    assert pl.stats()["n_support"] == len(ref["list"])
    pl.close()
