"""Pins of the oracle's small-segment (speckle) removal, ELAS post-processing
that the paper names but does not describe (Sec. III.A): segments are the
connected components of 4-neighbouring valid pixels whose disparities differ
by at most sim_threshold, and segments below min_size pixels are removed.

Pinned by a hand-worked map, by the component structure that scipy's
labelling and graph routines compute independently, and by invariants."""
import numpy as np
import pytest

scipy_ndimage = pytest.importorskip("scipy.ndimage")
csgraph = pytest.importorskip("scipy.sparse.csgraph")
sparse = pytest.importorskip("scipy.sparse")


def test_hand_worked_map(orc):
    """Links with |dd| <= 1: 1-1, 1-2, 2-3, 3-4, 4-5, 5-5 chain the nine
    pixels 1 1 1 2 3 4 5 5 5 into one segment although its ends differ by 4;
    the 9 links to nothing (|9 - 1| and |9 - 3| > 1): a segment of one."""
    d = np.array([[1, 1, -1, 5],
                  [1, 2, -1, 5],
                  [9, 3, 4, 5]], np.int16)
    exp = d.copy()
    exp[2, 0] = -1
    np.testing.assert_array_equal(orc.speckle(d, 1, 2), exp)
    np.testing.assert_array_equal(orc.speckle(d, 1, 9), exp)     # 9 pixels: kept at min_size 9
    np.testing.assert_array_equal(orc.speckle(d, 1, 10), np.where(d >= 0, -1, d).astype(np.int16))
    # with threshold 0 the segments are {1,1,1}, {2}, {3}, {4}, {5,5,5}, {9}
    exp0 = np.full_like(d, -1)
    exp0[0, 0] = exp0[0, 1] = exp0[1, 0] = 1
    exp0[0, 3] = exp0[1, 3] = exp0[2, 3] = 5
    np.testing.assert_array_equal(orc.speckle(d, 0, 3), exp0)


def test_diagonals_do_not_link(orc):
    d = np.full((5, 5), -1, np.int16)
    d[1, 1] = d[2, 2] = d[3, 3] = 7
    assert (orc.speckle(d, 5, 2) == -1).all()
    d[2, 1] = 7   # now (1,1)-(2,1)-(2,2) is a 4-connected segment of three
    out = orc.speckle(d, 0, 3)
    assert out[1, 1] == out[2, 1] == out[2, 2] == 7 and out[3, 3] == -1


def _expected_by_labelling(d, thr, min_size):
    """The definition through scipy: build the graph of links explicitly and
    take its connected components."""
    h, w = d.shape
    idx = np.arange(h * w).reshape(h, w)
    valid = d >= 0
    rows, cols = [], []
    link_h = valid[:, :-1] & valid[:, 1:] & (np.abs(d[:, :-1].astype(int) - d[:, 1:]) <= thr)
    link_v = valid[:-1, :] & valid[1:, :] & (np.abs(d[:-1, :].astype(int) - d[1:, :]) <= thr)
    rows += list(idx[:, :-1][link_h]) + list(idx[:-1, :][link_v])
    cols += list(idx[:, 1:][link_h]) + list(idx[1:, :][link_v])
    g = sparse.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(h * w, h * w))
    _, lab = csgraph.connected_components(g, directed=False)
    sizes = np.bincount(lab[valid.ravel()], minlength=h * w)
    keep = valid.ravel() & (sizes[lab] >= min_size)
    return np.where(keep.reshape(h, w), d, -1).astype(np.int16)


@pytest.mark.parametrize("thr,min_size", [(0, 3), (1, 5), (2, 12), (4, 40)])
def test_equals_graph_components(orc, thr, min_size):
    rng = np.random.default_rng(thr * 100 + min_size)
    # a piecewise smooth map with noise and holes, like an LR-checked map
    base = np.add.outer(np.arange(40) // 6, np.arange(57) // 9) * 3
    d = (base + rng.integers(-2, 3, base.shape)).astype(np.int16)
    d[rng.random(d.shape) < 0.15] = -1
    np.testing.assert_array_equal(orc.speckle(d, thr, min_size), _expected_by_labelling(d, thr, min_size))


def test_threshold_zero_equals_ndimage_label(orc):
    """With threshold 0 a segment is a 4-connected region of one value:
    scipy.ndimage.label per value gives the same components."""
    rng = np.random.default_rng(9)
    d = rng.integers(-1, 4, (33, 47)).astype(np.int16)
    exp = np.full_like(d, -1)
    for val in range(4):
        lab, n = scipy_ndimage.label(d == val)   # default structure: 4-connectivity
        sizes = np.bincount(lab.ravel())
        big = (lab > 0) & (sizes[lab] >= 4)
        exp[big] = val
    np.testing.assert_array_equal(orc.speckle(d, 0, 4), exp)


def test_invariants(orc):
    rng = np.random.default_rng(2)
    d = rng.integers(-1, 60, (30, 41)).astype(np.int16)
    d[10:20, 10:30] = 25   # one large flat segment
    for thr, ms in ((1, 1), (1, 0)):
        np.testing.assert_array_equal(orc.speckle(d, thr, ms), d)   # nothing is smaller than 1
    out = orc.speckle(d, 1, 8)
    # only removals, never new values; removing segments splits no other segment
    assert ((out == d) | (out == -1)).all()
    np.testing.assert_array_equal(orc.speckle(out, 1, 8), out)
    assert (out[10:20, 10:30] == 25).all()
