"""Pins of the oracle's left-right check and post-processing (Sec. III.A,
Fig. 1(i): invalidate occluded pixels, then improve smoothness)."""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_consistent_constant_maps(orc):
    h, w, s = 4, 20, 6
    dL = np.full((h, w), s, np.int16)
    dR = np.full((h, w), s, np.int16)
    oL, oR, mL, mR = orc.lr_check(dL, dR, 2)
    uu = np.arange(w)[None, :].repeat(h, 0)
    np.testing.assert_array_equal(mL, (uu - s >= 0).astype(np.uint8))
    np.testing.assert_array_equal(mR, (uu + s <= w - 1).astype(np.uint8))
    np.testing.assert_array_equal(oL, np.where(mL == 1, s, -1))
    np.testing.assert_array_equal(oR, np.where(mR == 1, s, -1))


def test_occlusion_strip(orc):
    """Background d=5 and a foreground strip at u=10..12 with d=9 in the left
    image.  The strip lands on x=1..3 of the right image.  Background pixels of
    the left image at u=6..8 also map to x=1..3 (occluded: |5-9| = 4 > 2) and
    right pixels x=5..7 map back onto the strip (also occluded)."""
    w = 30
    dL = np.full((1, w), 5, np.int16)
    dL[0, 10:13] = 9
    dR = np.full((1, w), 5, np.int16)
    dR[0, 1:4] = 9
    oL, oR, mL, mR = orc.lr_check(dL, dR, 2)
    expL = np.ones(w, np.uint8)
    expL[:5] = 0          # u - d < 0
    expL[6:9] = 0         # occluded background
    expR = np.ones(w, np.uint8)
    expR[5:8] = 0         # partner is the strip
    expR[w - 5:] = 0      # u + d > w - 1
    np.testing.assert_array_equal(mL[0], expL)
    np.testing.assert_array_equal(mR[0], expR)


def test_threshold_and_invalid_inputs(orc):
    dL = np.array([[-1, 3, 4, 5, 6, 7, 8, 9]], np.int16)
    dR = np.full((1, 8), 3, np.int16)
    dR[0, 0] = -1
    oL, oR, mL, mR = orc.lr_check(dL, dR, 2)
    # u=0 is invalid; for u >= 1, d = u + 2 puts the partner at x = -2 (outside)
    assert (mL == 0).all()
    dL = np.array([[2, 2, 2, 3, 4, 5, 6, 7]], np.int16)   # partners x = u - d
    dR = np.array([[2, 2, 4, 0, 0, 0, 0, 0]], np.int16)
    oL, oR, mL, mR = orc.lr_check(dL, dR, 2)
    # u=2: x=0, |2-2|=0 keep; u=3: x=1, |2-2| keep; u=4: x=2,|2-4|=2 keep;
    # u=5: x=3 (0) -> |3-0|=3 reject; u=6..7: x=3,4 (0) reject; u=0,1 out of range
    np.testing.assert_array_equal(mL[0], [0, 0, 1, 1, 1, 0, 0, 0])


def test_huge_threshold_keeps_every_valid_pair(orc):
    rng = np.random.default_rng(0)
    h, w = 6, 40
    dL = rng.integers(-1, 20, (h, w)).astype(np.int16)
    dR = rng.integers(-1, 20, (h, w)).astype(np.int16)
    oL, oR, mL, mR = orc.lr_check(dL, dR, 1000)
    for v in range(h):
        for u in range(w):
            d = dL[v, u]
            ok = d >= 0 and u - d >= 0 and dR[v, u - d] >= 0
            assert mL[v, u] == ok


def _post(orc, row, gap, mean):
    d = np.array([row], np.int16) if np.ndim(row) == 1 else np.array(row, np.int16)
    return orc.postprocess(d, dict(ipol_gap_width=gap, filter_adaptive_mean=mean))


def test_gap_interpolation_golden(orc):
    g = json.load(open(os.path.join(GOLD, "gap_interpolation.json")))
    for c in g["cases"]:
        out = _post(orc, c["row"], g["ipol_gap_width"], 0)[0]
        np.testing.assert_array_equal(out, np.array(c["expected"], np.float32))


def test_column_pass_follows_row_pass(orc):
    # the centre gap is 5 wide in its row (too long) but 1 tall in its column
    d = np.full((3, 7), 20, np.int16)
    d[1, 1:6] = -1
    d[0, 3] = 21
    out = _post(orc, d, 3, 0)
    assert out[1, 3] == 20.5          # column: between 21 and 20
    assert out[1, 1] == 20.0


def test_adaptive_mean_golden_ramp(orc):
    g = json.load(open(os.path.join(GOLD, "adaptive_mean_ramp.json")))
    out = _post(orc, g["row"], 0, 1)[0]
    for k, v in g["expected"].items():
        assert abs(float(out[int(k)]) - v) < 1e-5


def test_adaptive_mean_invariants(orc):
    # constant map unchanged; a step of height >= 4 does not blur; invalid stays -1
    d = np.full((9, 12), 30, np.int16)
    np.testing.assert_array_equal(_post(orc, d, 0, 1), d.astype(np.float32))
    d[:, 6:] = 34
    np.testing.assert_array_equal(_post(orc, d, 0, 1), d.astype(np.float32))
    d[4, 4] = -1
    out = _post(orc, d, 0, 1)
    assert out[4, 4] == -1.0


# ---------------------------------------------------------------------------
# Median filter (Sec. VII; reading: median of the valid disparities in the
# window, the lower one for an even count, invalid pixels kept)
# ---------------------------------------------------------------------------

def test_median_hand_example(orc):
    d = np.array([[1, 2, 3], [4, 100, 6], [7, 8, -1]], np.int16)
    # (0,0): {1,2,4,100} -> 2; (0,1): {1,2,3,4,6,100} -> 3; (1,1): eight
    # valid values -> 4th smallest 4; (2,1): {4,6,7,8,100} -> 7
    exp = np.array([[2, 3, 3], [4, 4, 6], [7, 7, -1]], np.int16)
    np.testing.assert_array_equal(orc.median(d, 1), exp)


def test_median_invariants(orc):
    rng = np.random.default_rng(3)
    const = np.full((9, 11), 37, np.int16)
    np.testing.assert_array_equal(orc.median(const, 1), const)
    np.testing.assert_array_equal(orc.median(const, 2), const)
    spiky = const.copy()
    spiky[4, 5] = 200  # an isolated spike in a flat region disappears
    np.testing.assert_array_equal(orc.median(spiky, 1), const)
    d = rng.integers(-1, 60, size=(13, 17)).astype(np.int16)
    np.testing.assert_array_equal(orc.median(d, 0), d)  # a 1x1 window is the identity
    out = orc.median(d, 2)
    np.testing.assert_array_equal(out < 0, d < 0)  # invalid pixels, and only those, stay invalid
    # every output is one of the valid values of its window
    for v, u in [(0, 0), (6, 8), (12, 16), (3, 14)]:
        win = d[max(0, v - 2):v + 3, max(0, u - 2):u + 3]
        if d[v, u] >= 0:
            assert out[v, u] in win[win >= 0]


def test_median_interior_matches_a_library_filter(orc):
    """With every disparity valid, a window at least r pixels from the border
    holds (2r+1)^2 values and its median is the library's median filter."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(4)
    d = rng.integers(0, 256, (41, 47)).astype(np.int16)
    for r in (1, 2, 3):
        inner = (slice(r, -r), slice(r, -r))
        np.testing.assert_array_equal(orc.median(d, r)[inner], ndimage.median_filter(d, size=2 * r + 1)[inner])
