"""Edge cases of the CUDA path against the oracle (Sec. III.A steps): a fan
mesh of long, wide triangles, unusual grid and lattice sizes, wide images,
tiny images and empty support."""
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


def _fan(w):
    """Apex (5,5) and a row of points at v = 60: long triangles whose rows are
    wider than a warp, all meeting at the apex."""
    rng = np.random.default_rng(9)
    xs = list(range(40, w - 5, 5))
    lst = [[5, 5, 3]] + [[x, 60, int(rng.integers(4, 30))] for x in xs]
    lst = np.array(lst, np.int16)
    tri = np.array([[0, i, i + 1] for i in range(1, len(xs))], np.int32)
    return lst, tri


def test_plane_prior_fan_mesh():
    B = _B()
    w, h = 800, 70
    lst, tri = _fan(w)
    assert len(tri) > 128
    prm = dict(disp_max=63)
    exp = oracle.plane_prior(lst, tri, w, h, prm)
    got = host(B.elas_plane_prior(dev(lst), dev(tri), w, h, prm))
    np.testing.assert_array_equal(got, exp)


def test_dense_match_fan_mesh():
    B = _B()
    w, h = 800, 70
    lst, triL = _fan(w)
    triR = oracle.triangulate(lst, right=True)
    rng = np.random.default_rng(4)
    L = rng.integers(0, 256, (h, w), dtype=np.uint8)
    R = rng.integers(0, 256, (h, w), dtype=np.uint8)
    prm = dict(disp_max=63)
    dL_, dR_ = oracle.descriptors(L), oracle.descriptors(R)
    gL, gR = oracle.grid_vectors(lst, w, h, prm), oracle.grid_vectors(lst, w, h, prm, right=True)
    expL = oracle.dense(dL_, dR_, oracle.plane_prior(lst, triL, w, h, prm), gL, prm)
    expR = oracle.dense(dL_, dR_, oracle.plane_prior(lst, triR, w, h, prm, right=True), gR, prm, right=True)
    oL, oR = B.elas_dense_match(dev(dL_), dev(dR_), prm, dev(lst), len(lst), dev(triL), dev(triR.astype(np.int32)),
                                dev(grid_as_i32(gL)), dev(grid_as_i32(gR)))
    np.testing.assert_array_equal(host(oL), expL)
    np.testing.assert_array_equal(host(oR), expR)


def _whole(wl, seed):
    B = _B()
    L, R, _ = synth.make_pair(wl.spec, seed)
    prm = dict(wl.params, ipol_gap_width=3, filter_adaptive_mean=1)
    ref = oracle.pipeline(L, R, prm, postprocess_on=True)
    h, w = L.shape
    pl = B.Pipeline(w, h, prm)
    dL = torch.empty((h, w), dtype=torch.int16, device="cuda")
    dR = torch.empty_like(dL)
    post = torch.empty((h, w), dtype=torch.float32, device="cuda")
    pl.run(dev(L), dev(R), dL, dR, post)
    np.testing.assert_array_equal(host(dL), ref["lrL"])
    np.testing.assert_array_equal(host(dR), ref["lrR"])
    assert np.abs(host(post) - ref["post"]).max() <= 1e-4
    st = pl.stats()
    pl.close()
    return ref, st


def test_small_grid_and_lattice():
    wl = synth.scaled_workload(161, 97, 32)
    wl.params.update(grid_size=7, candidate_stepsize=3, incon_window_size=3, redun_max_dist=4)
    ref, st = _whole(wl, 31)
    assert st["n_support"] == len(ref["list"]) > 50


@pytest.mark.parametrize("step", [7, 10, 14])
def test_sparse_candidate_lattices(step):
    """Coarser candidate lattices (sparser support, as in the accuracy sweep):
    the whole path still equals the oracle."""
    wl = synth.scaled_workload(400, 300, 96)
    wl.params.update(candidate_stepsize=step)
    ref, st = _whole(wl, 40 + step)
    assert st["n_support"] == len(ref["list"]) > 10


def test_wide_image_beyond_2048():
    """Pixels with x - 2 > 2047: the candidate list's padding value must
    never be admitted."""
    wl = synth.scaled_workload(2200, 40, 64)
    _whole(wl, 5)


@pytest.mark.parametrize("size", [(8, 8), (13, 11), (40, 9)])
def test_tiny_images(size):
    w, h = size
    wl = synth.scaled_workload(w, h, 16)
    ref, st = _whole(wl, 2)
    assert st["n_support"] == len(ref["list"])


def test_textureless_pair_gives_empty_support_and_invalid_maps():
    B = _B()
    w, h = 120, 80
    img = np.full((h, w), 77, np.uint8)
    pl = B.Pipeline(w, h, dict(disp_max=31))
    dL = torch.empty((h, w), dtype=torch.int16, device="cuda")
    pl.run(dev(img), dev(img), dL)
    assert (host(dL) == -1).all()
    assert pl.stats()["n_support"] == 0
    pl.close()


def test_disparity_range_near_image_width():
    wl = synth.scaled_workload(96, 60, 96)   # disparities up to 95 on a 96-wide image
    _whole(wl, 8)
