"""The GPU triangulation (elas_triangulate_device) must produce exactly the
oracle's Delaunay triangulation (Sec. III.A) -- the unique one under the
symbolic tie-break -- as a set of counter-clockwise triangles, on lattice
subsets, real support sets, degenerate inputs and meshes with very large
empty circles."""
import numpy as np
import pytest

import oracle
from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _canon(t):
    t = np.asarray(t).reshape(-1, 3)
    return sorted(tuple(int(v) for v in np.roll(r, -int(np.argmin(r)))) for r in t)


def _gpu_tri(lst, w, h, right):
    from paper_1802_07210_gb300 import binding as B
    lst = np.asarray(lst, np.int16).reshape(-1, 3)
    n = len(lst)
    buf = lst if n else np.zeros((1, 3), np.int16)
    tri, nt = B.elas_triangulate_device(dev(buf), dev(np.array([n], np.int32)), w, h, right=right)
    k = int(host(nt)[0])
    assert k >= 0, "device triangulation reported a failure"
    return host(tri)[:k]


def _check(lst, w, h):
    for right in (False, True):
        got = _gpu_tri(lst, w, h, right)
        exp = oracle.triangulate(np.asarray(lst, np.int16).reshape(-1, 3), right=right)
        assert len(got) == len(exp)
        assert _canon(got) == _canon(exp)


@pytest.mark.parametrize("seed", range(8))
def test_lattice_subsets(seed):
    rng = np.random.default_rng(seed)
    gx, gy = int(rng.integers(2, 60)), int(rng.integers(2, 40))
    pts = [(5 * i + 5, 5 * j + 5, int(rng.integers(0, 40)))
           for j in range(gy) for i in range(gx) if rng.random() < rng.uniform(0.1, 1.0)]
    _check(pts, 5 * gx + 10, 5 * gy + 10)


@pytest.mark.parametrize("wl_cfg", [(synth.SMALL_320, 1), (synth.VGA_640, 2), (synth.KITTI_1242, 3)])
def test_real_support_sets(wl_cfg):
    wl, cfg = wl_cfg
    L, R, _ = synth.workload_pair(wl, 0, cfg)
    lst = oracle.support_list(oracle.support_points(oracle.descriptors(L), oracle.descriptors(R), wl.params),
                              wl.params)
    _check(lst, wl.spec.w, wl.spec.h)


def test_degenerate_inputs():
    _check([], 50, 50)
    _check([(10, 10, 0)], 50, 50)
    _check([(10, 10, 0), (20, 10, 0)], 50, 50)
    _check([(5 * i + 5, 10, i % 3) for i in range(9)], 60, 30)       # collinear
    _check([(10, 10, 0), (20, 10, 0), (10, 20, 0)], 50, 50)
    _check([(5 * i + 5, 10, 0) for i in range(9)] + [(23, 37, 0)], 60, 50)


def test_big_empty_circles_and_fans():
    # only the border of a large square: the circumcircles span the image
    pts = [(x, 5, 1) for x in range(5, 500, 5)] + [(x, 495, 2) for x in range(5, 500, 5)]
    pts += [(5, y, 3) for y in range(10, 495, 5)] + [(495, y, 4) for y in range(10, 495, 5)]
    _check(pts, 510, 510)
    # a fan: one apex, a long row of points far away
    pts = [(5, 5, 3)] + [(x, 300, (x // 5) % 30) for x in range(40, 795, 5)]
    _check(pts, 800, 310)


def test_dense_sets_and_far_clusters():
    rng = np.random.default_rng(5)
    # a 2-pixel lattice with holes: every disc holds more points than the
    # passes list, so the stars take the unlisted steps
    pts = [(2 * i + 3, 2 * j + 3, int(rng.integers(0, 30))) for j in range(40) for i in range(60)
           if rng.random() < 0.6]
    _check(pts, 130, 90)
    # clusters far apart: long edges between them and circles far wider than
    # any listed disc (region steps clipped to the disc and the half-plane)
    seen, pts = set(), []
    for cx, cy in ((20, 20), (300, 40), (150, 200), (40, 280), (290, 290), (160, 30)):
        for _ in range(30):
            x, y = cx + int(rng.integers(0, 20)), cy + int(rng.integers(0, 20))
            if (x, y) not in seen:
                seen.add((x, y))
                pts.append((x, y, int(rng.integers(0, 12))))
    _check(pts, 320, 320)


def test_right_coordinates_with_many_duplicates():
    # all points of a row collapse onto a few right-image positions
    pts = [(u, v, u % 20) for v in range(10, 60, 5) for u in range(20, 200, 5)]
    _check(pts, 210, 70)


@pytest.mark.parametrize("gpu", [True, False])
def test_pipeline_both_triangulation_modes(gpu):
    from paper_1802_07210_gb300 import binding as B
    wl = synth.SMALL_320
    L, R, _ = synth.workload_pair(wl, 4, 1)
    ref = oracle.pipeline(L, R, wl.params, postprocess_on=False)
    h, w = L.shape
    pl = B.Pipeline(w, h, wl.params, gpu_triangulation=gpu)
    dL = torch.empty((h, w), dtype=torch.int16, device="cuda")
    dR = torch.empty_like(dL)
    pl.run(dev(L), dev(R), dL, dR)
    np.testing.assert_array_equal(host(dL), ref["lrL"])
    np.testing.assert_array_equal(host(dR), ref["lrR"])
    st = pl.stats()
    assert (st["n_support"], st["n_tri_left"], st["n_tri_right"]) == (len(ref["list"]), len(ref["triL"]),
                                                                        len(ref["triR"]))
    pl.close()
