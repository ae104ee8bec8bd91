"""Pins of the oracle's census variant (Sec. VI.A): the census transform over
full W x W windows and the Hamming cost in the support and dense stages.

The transform is pinned by hand-derived examples (tests/golden), by the
invariances a census has (strictly increasing intensity maps, transposition
and mirroring with the matching bit permutation), by the border rule against
numpy's edge padding, and by closed-form bit counts.  The Hamming cost is
pinned through whole stages: a pair related by one known shift must give
that shift with cost 0, and the census pipeline must not see a strictly
increasing change of one image's intensities."""
import json
import os

import numpy as np
import pytest

from paper_1802_07210_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "census_examples.json")


def _bits(rec, W):
    """(W*W,) array of the bits of one packed record."""
    return np.unpackbits(rec, bitorder="little")[:W * W]


def test_hand_derived_examples(orc):
    g = json.load(open(GOLDEN))
    for c in g["cases"]:
        out = orc.census(np.array(c["image"], np.uint8), c["W"], c["nbytes"])
        e = c["expected_bytes"]
        assert list(out[c["v"], c["u"], :len(e)]) == e, c["derivation"]
        assert not out[c["v"], c["u"], len(e):].any()


@pytest.mark.parametrize("W", [3, 5, 9, 13])
def test_constant_image_has_no_bits(orc, W):
    out = orc.census(np.full((12, 17), 77, np.uint8), W, 32)
    assert not out.any()


@pytest.mark.parametrize("W", [3, 7, 11])
def test_invariant_under_increasing_intensity_maps(orc, W):
    """The census compares intensities only: any strictly increasing map of
    the grey levels leaves it unchanged (the illumination invariance the
    paper chooses it for)."""
    rng = np.random.default_rng(5)
    img = rng.integers(0, 120, (23, 31)).astype(np.uint8)
    lut = np.cumsum(rng.integers(1, 3, 120)) + 10  # strictly increasing steps of 1 or 2, max <= 250
    assert np.all(np.diff(lut) > 0) and lut.max() <= 255
    mapped = lut[img].astype(np.uint8)
    assert np.array_equal(orc.census(img, W, 32), orc.census(mapped, W, 32))


@pytest.mark.parametrize("W", [3, 5, 9])
def test_transpose_and_mirror_permute_the_bits(orc, W):
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, (14, 19)).astype(np.uint8)
    h, w = img.shape
    r = W // 2
    a = orc.census(img, W, 32)
    t = orc.census(np.ascontiguousarray(img.T), W, 32)
    m = orc.census(np.ascontiguousarray(img[:, ::-1]), W, 32)
    idx = np.arange(W * W).reshape(W, W)   # idx[dy + r, dx + r] = k
    for v in range(h):
        for u in range(w):
            b = _bits(a[v, u], W).reshape(W, W)
            assert np.array_equal(_bits(t[u, v], W).reshape(W, W), b.T)
            assert np.array_equal(_bits(m[v, w - 1 - u], W).reshape(W, W), b[:, ::-1])
    assert idx[r, r] == (W * W) // 2


@pytest.mark.parametrize("W", [3, 5, 7])
def test_border_rule_is_edge_replication(orc, W):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (9, 13)).astype(np.uint8)
    r = W // 2
    padded = np.pad(img, r, mode="edge")
    a = orc.census(img, W, 16)
    p = orc.census(padded, W, 16)
    assert np.array_equal(a, p[r:r + img.shape[0], r:r + img.shape[1]])


@pytest.mark.parametrize("W", [3, 5, 9, 13, 15])
def test_bit_counts_of_extremes(orc, W):
    """A strict maximum of its window sets every bit but the centre's; a
    strict minimum sets none; all bits lie inside the first W*W."""
    rng = np.random.default_rng(W)
    img = rng.integers(10, 200, (2 * W + 3, 2 * W + 5)).astype(np.uint8)
    c = (W + 1, W + 2)
    img[c] = 255
    out = orc.census(img, W, 32)
    assert int(np.unpackbits(out[c]).sum()) == W * W - 1
    assert not np.unpackbits(out[c], bitorder="little")[W * W:].any()
    img[c] = 0
    assert not orc.census(img, W, 32)[c].any()


def _shift_pair(w, h, shift, seed):
    L, R = synth.fronto_parallel_pair(w, h, shift, seed)
    return L, R


@pytest.mark.parametrize("ws", [7, 9, 13])
def test_support_match_finds_the_shift(orc, ws):
    """R(u - s, v) = L(u, v) exactly: at every candidate whose windows see no
    clamped border the true disparity costs 0 and random texture gives every
    other disparity a positive Hamming cost, so the ratio test accepts s in
    both directions."""
    w, h, s = 96, 40, 9
    L, R = _shift_pair(w, h, s, 21)
    prm = dict(disp_min=0, disp_max=31, candidate_stepsize=5, support_threshold=0.85,
               lr_threshold=0, census_support_w=ws, census_dense_w=5)
    cL, cR = orc.census(L, ws, 32), orc.census(R, ws, 32)
    dcan = orc.support_match(cL, cR, prm)
    r = ws // 2
    checked = 0
    for ic in range(dcan.shape[0]):
        for jc in range(dcan.shape[1]):
            u, v = 5 * jc, 5 * ic
            inside = 4 <= v <= h - 5 and v - r >= 0 and v + r <= h - 1
            # left window and right window at u - s fully inside both images,
            # and the right-to-left search from u - s meets every d up to 31
            if inside and u - s - r >= 0 and u + r <= w - 1 - s and u - s + 31 <= w - 5 and u >= 4 + s:
                assert dcan[ic, jc] == s, (u, v)
                checked += 1
    assert checked >= 20


def test_texture_thresholds_do_not_apply(orc):
    L, R = _shift_pair(80, 30, 6, 4)
    L[:, :40] = 90   # a flat region as well
    R[:, :34] = 90
    base = dict(disp_min=0, disp_max=20, census_support_w=9, census_dense_w=5)
    cL, cR = orc.census(L, 9, 32), orc.census(R, 9, 32)
    a = orc.support_match(cL, cR, dict(base, support_texture=0))
    b = orc.support_match(cL, cR, dict(base, support_texture=10 ** 6))
    assert np.array_equal(a, b)
    assert (a >= 0).any()
    dL, dR = orc.census(L, 5, 16), orc.census(R, 5, 16)
    fr = dict(base, flags=orc.FLAG_FULL_RANGE | orc.FLAG_PRIOR_OFF)
    x = orc.dense(dL, dR, None, None, dict(fr, match_texture=0))
    y = orc.dense(dL, dR, None, None, dict(fr, match_texture=10 ** 6))
    assert np.array_equal(x, y)
    # flat windows cost 0 at every d: the least d wins
    assert (x[10, 10:30] == 0).all()


@pytest.mark.parametrize("wd", [5, 7])
def test_dense_hamming_finds_the_shift(orc, wd):
    w, h, s = 80, 24, 7
    L, R = _shift_pair(w, h, s, 8)
    prm = dict(disp_min=0, disp_max=31, census_support_w=9, census_dense_w=wd,
               flags=orc.FLAG_FULL_RANGE | orc.FLAG_PRIOR_OFF)
    dL, dR = orc.census(L, wd, 16), orc.census(R, wd, 16)
    out = orc.dense(dL, dR, None, None, prm)
    r = wd // 2
    # the right window at u - s is inside the image and equals the left one,
    # so the minimum cost is 0 and the least d reaching it wins: d <= s, the
    # two census strings at d agree bit for bit, and it is s almost everywhere
    sl = out[r:h - r, s + r:w - r]
    assert (sl >= 0).all() and (sl <= s).all()
    for v in range(r, h - r):
        for u in range(s + r, w - r):
            d = int(out[v, u])
            assert not np.unpackbits(dL[v, u] ^ dR[v, u - d]).any(), (u, v, d)
    assert (sl == s).mean() > 0.98
    # every left pixel with u - s < 2 has no admissible d >= s: never s
    assert not (out[:, 2:s + 2] == s).any()


def test_pipeline_is_blind_to_an_intensity_change_of_one_image(orc):
    """Census descriptors make the whole path independent of a strictly
    increasing map of one image's grey levels; the Sobel/SAD path is not.
    The pair is first halved in contrast (levels 0..127) so that a strongly
    non-affine increasing map, a gamma curve onto 0..255, exists."""
    wl = synth.SMALL_320
    L, R, _ = synth.workload_pair(wl, 0)
    L, R = L[:96, :160] // 2, R[:96, :160] // 2
    lut = np.rint(255.0 * (np.arange(128) / 127.0) ** 0.6).astype(np.int64)
    assert np.all(np.diff(lut) > 0) and lut[-1] == 255
    R2 = lut[R].astype(np.uint8)
    prm = dict(wl.params, census_support_w=9, census_dense_w=5)
    a = orc.pipeline(L, R, prm, postprocess_on=False)
    b = orc.pipeline(L, R2, prm, postprocess_on=False)
    for k in ("dcan", "denseL", "denseR", "lrL"):
        assert np.array_equal(a[k], b[k]), k
    assert int((a["dcan"] >= 0).sum()) > 20
    sad = orc.support_points(orc.descriptors(L), orc.descriptors(R2), wl.params)
    sad0 = orc.support_points(orc.descriptors(L), orc.descriptors(R), wl.params)
    assert not np.array_equal(sad, sad0)


def test_degenerate_images(orc):
    """A 1x1 image clamps every neighbour onto the centre: no bits.  A single
    row clamps every dy onto it, so each window row repeats the 1-D census of
    the row (bits for dy equal the bits for dy = 0)."""
    assert not orc.census(np.array([[200]], np.uint8), 15, 32).any()
    row = np.array([[5, 9, 1, 7, 3, 8, 2]], np.uint8)
    for W in (3, 5, 7):
        c = orc.census(row, W, 16)
        for u in range(row.shape[1]):
            b = np.unpackbits(c[0, u], bitorder="little")[:W * W].reshape(W, W)
            assert (b == b[W // 2]).all()
            r = W // 2
            exp = [int(row[0, min(max(u + dx, 0), row.shape[1] - 1)] < row[0, u]) for dx in range(-r, r + 1)]
            assert list(b[W // 2]) == exp
