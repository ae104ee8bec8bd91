"""Parity of the census variant (Sec. VI.A: census descriptors over full
W x W windows, Hamming costs) with the CPU oracle through the C-ABI: the
census records bit for bit, the support points (both matchers), the dense
argmin and the whole one-pair pipeline (batches and the server: test_gpu_variants_batched.py)."""

import numpy as np
import pytest

import oracle
from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, grid_as_i32, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _B():
    from paper_1802_07210_gb300 import binding
    return binding


SUPPORT_W = [3, 5, 7, 9, 11, 13, 15]
DENSE_W = [3, 5, 7, 9, 11]


@pytest.mark.parametrize("size", [(37, 29), (203, 117), (1242, 375)])
def test_census_records(size):
    B = _B()
    w, h = size
    rng = np.random.default_rng(w)
    L = rng.integers(0, 256, (h, w)).astype(np.uint8)
    R = (L // 7 * 7).astype(np.uint8)  # many equal neighbours: ties decide bits too
    for W in SUPPORT_W:
        sL, sR = B.elas_census(dev(L), dev(R), W, 32)
        np.testing.assert_array_equal(host(sL), oracle.census(L, W, 32), err_msg="support W=%d" % W)
        np.testing.assert_array_equal(host(sR), oracle.census(R, W, 32), err_msg="support W=%d" % W)
    for W in DENSE_W:
        d = B.elas_census(dev(L), None, W, 16)
        np.testing.assert_array_equal(host(d), oracle.census(L, W, 16), err_msg="dense W=%d" % W)


def _census_params(wl, ws, wd):
    return dict(wl.params, census_support_w=ws, census_dense_w=wd)


CASES = [("small_320", synth.SMALL_320, 1, 9, 5),
         ("ragged_203x117", synth.scaled_workload(203, 117, 48), 7, 13, 7),
         ("vga_640", synth.VGA_640, 2, 7, 3)]


@pytest.fixture(scope="module")
def refs():
    out = {}
    for name, wl, cfg, ws, wd in CASES:
        L, R, _ = synth.workload_pair(wl, 0, cfg)
        prm = _census_params(wl, ws, wd)
        out[name] = (prm, L, R, oracle.pipeline(L, R, prm, postprocess_on=wl.postprocess))
    return out


def _check_support(r, ref, prm, w, h):
    np.testing.assert_array_equal(host(r["d_can"]), ref["dcan"])
    n = int(host(r["count"])[0])
    assert n == len(ref["list"])
    np.testing.assert_array_equal(host(r["list"])[:n], ref["list"])
    np.testing.assert_array_equal(host(r["grid_L"]), grid_as_i32(oracle.grid_vectors(ref["list"], w, h, prm)))
    np.testing.assert_array_equal(host(r["grid_R"]),
                                  grid_as_i32(oracle.grid_vectors(ref["list"], w, h, prm, right=True)))


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_census_support_points(refs, name):
    B = _B()
    prm, L, R, ref = refs[name]
    h, w = L.shape
    r = B.elas_support_points(dev(ref["sdescL"]), dev(ref["sdescR"]), prm)
    _check_support(r, ref, prm, w, h)
    assert len(ref["list"]) > 20


def test_census_support_row_matcher():
    """A pair tall enough (306 lattice rows) for the row-organised matcher."""
    B = _B()
    wl = synth.scaled_workload(160, 1530, 64)
    L, R, _ = synth.workload_pair(wl, 0, 3)
    prm = _census_params(wl, 11, 5)
    sL, sR = oracle.census(L, 11, 32), oracle.census(R, 11, 32)
    dcan = oracle.support_points(sL, sR, prm)
    ref = {"dcan": dcan, "list": oracle.support_list(dcan, prm)}
    r = B.elas_support_points(dev(sL), dev(sR), prm)
    _check_support(r, ref, prm, 160, 1530)
    assert len(ref["list"]) > 100


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_census_dense_argmin(refs, name):
    B = _B()
    prm, L, R, ref = refs[name]
    for right, key in ((False, "denseL"), (True, "denseR")):
        dp = ref["dplaneR" if right else "dplaneL"]
        grid = ref["gridR" if right else "gridL"]
        out = B.elas_dense_argmin(dev(ref["descL"]), dev(ref["descR"]), prm, dev(dp), dev(grid_as_i32(grid)),
                                  right=right)
        np.testing.assert_array_equal(host(out), ref[key])
    # every in-range disparity, no prior
    fr = dict(prm, flags=oracle.FLAG_FULL_RANGE | oracle.FLAG_PRIOR_OFF)
    out = B.elas_dense_argmin(dev(ref["descL"]), dev(ref["descR"]), fr)
    np.testing.assert_array_equal(host(out), oracle.dense(ref["descL"], ref["descR"], None, None, fr))


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_census_pipeline(refs, name):
    B = _B()
    prm, L, R, ref = refs[name]
    h, w = L.shape
    pl = B.Pipeline(w, h, prm)
    dL = torch.empty((h, w), dtype=torch.int16, device="cuda")
    dR = torch.empty_like(dL)
    post = torch.empty((h, w), dtype=torch.float32, device="cuda") if "post" in ref else None
    for _ in range(2):  # the second run replays the captured graph
        pl.run(dev(L), dev(R), dL, dR, post)
        np.testing.assert_array_equal(host(dL), ref["lrL"])
        np.testing.assert_array_equal(host(dR), ref["lrR"])
        if post is not None:
            assert np.abs(host(post) - ref["post"]).max() <= 1e-4
    assert pl.stats()["n_support"] == len(ref["list"])
    pl.close()
