"""Pins of the oracle's support-point steps: matching with the ratio test of
Eq. 1-2 (Sec. VI.B restates the original criterion), the left-right and
texture checks, the consistency and redundancy filters (Sec. III.A) and the
grid vectors (Sec. III.A, Fig. 2, Sec. VI.D)."""
import numpy as np
import pytest

from paper_1802_07210_gb300 import synth

BASE = dict(disp_min=0, disp_max=8, candidate_stepsize=5, support_texture=10,
            lr_threshold=2, support_threshold=0.85)


def _worked_example(x, z, extra_rl=None):
    """A hand-built 48x10 descriptor pair with exactly one textured candidate,
    (u, v) = (30, 5).  Only byte 0 differs from 128.  The left window corners
    (columns 28, 32; rows 3, 7) hold 228; the right image holds 228 - e[c] in
    columns 20..32 of rows 3 and 7 with e = 50 except e[24] = 0, e[28] = x,
    e[20] = z.  Left-to-right window cost: cost(d) = 2 (e[28-d] + e[32-d]):
      d=4 -> 2x, d=8 -> 2z, d=0 -> 2(x+50), every other d -> 200.
    Right-to-left from u_r = 26: cost(4) = 2x, cost(8) = 2(100-x),
    cost(0) = 2(100+x), others 2(200-x)."""
    w, h = 48, 10
    dL = np.full((h, w, 16), 128, np.uint8)
    dR = np.full((h, w, 16), 128, np.uint8)
    for r in (3, 7):
        dL[r, 28, 0] = dL[r, 32, 0] = 228
        for c in range(20, 33):
            e = 50
            if c == 24:
                e = 0
            elif c == 28:
                e = x
            elif c == 20:
                e = z
            dR[r, c, 0] = 228 - e
        if extra_rl is not None:
            for c, val in extra_rl.items():
                dL[r, c, 0] = val
    return dL, dR


def _the_candidate(dcan):
    # (u, v) = (30, 5) -> (jc, ic) = (6, 1)
    other = dcan.copy()
    other[1, 6] = -1
    assert (other == -1).all(), "only the hand-built candidate can be textured"
    return int(dcan[1, 6])


def test_ratio_test_boundary_is_inclusive(orc):
    # m1 = 34, m2 = 40: m1/m2 = 0.85 exactly -> accepted (Eq. 2 uses <=)
    dL, dR = _worked_example(17, 20)
    assert _the_candidate(orc.support_match(dL, dR, BASE)) == 4


def test_ratio_test_rejects_above_threshold(orc):
    # m1 = 36, m2 = 40 -> 0.9 > 0.85 -> rejected; with threshold 0.9 accepted
    dL, dR = _worked_example(18, 20)
    assert _the_candidate(orc.support_match(dL, dR, BASE)) == -1
    assert _the_candidate(orc.support_match(dL, dR, dict(BASE, support_threshold=0.9))) == 4


def test_ratio_direction_and_tie(orc):
    # m1 = m2 (two disparities share the minimum) is ambiguous -> rejected
    dL, dR = _worked_example(17, 17)
    assert _the_candidate(orc.support_match(dL, dR, dict(BASE, support_threshold=0.99))) == -1
    # a clear winner (m1 = 0, m2 = 40) is accepted even at a strict threshold
    dL, dR = _worked_example(0, 20)
    assert _the_candidate(orc.support_match(dL, dR, dict(BASE, support_threshold=0.05))) == 4


def test_shift_sum_threshold(orc):
    """Eq. 3 (ORACLE_FLAG_SHIFT_SUM): accept iff m1 <= m2/2 + m2/4 + m2/8 +
    m2/32 with integer shifts, in place of the float ratio test."""
    ss = dict(BASE, flags=orc.FLAG_SHIFT_SUM)
    # m2 = 40: T = 20 + 10 + 5 + 1 = 36.  m1 = 36 is accepted (the float test
    # at 0.85 rejects it), m1 = 38 is not
    dL, dR = _worked_example(18, 20)
    assert _the_candidate(orc.support_match(dL, dR, BASE)) == -1
    assert _the_candidate(orc.support_match(dL, dR, ss)) == 4
    dL, dR = _worked_example(19, 20)
    assert _the_candidate(orc.support_match(dL, dR, ss)) == -1
    # m2 = 70: T = 35 + 17 + 8 + 2 = 62 (below 0.90625 * 70 = 63.4 by the
    # truncations): m1 = 62 accepted, m1 = 64 rejected
    dL, dR = _worked_example(31, 35)
    assert _the_candidate(orc.support_match(dL, dR, ss)) == 4
    dL, dR = _worked_example(32, 35)
    assert _the_candidate(orc.support_match(dL, dR, ss)) == -1
    # the threshold parameter plays no part; a tie m1 = m2 stays rejected
    dL, dR = _worked_example(18, 20)
    assert _the_candidate(orc.support_match(dL, dR, dict(ss, support_threshold=0.01))) == 4
    dL, dR = _worked_example(17, 17)
    assert _the_candidate(orc.support_match(dL, dR, ss)) == -1


def test_left_right_recheck(orc):
    # make the right-to-left re-match prefer d = 7 (cost 0) over d = 4 (cost 34):
    # |4 - 7| = 3 > lr_threshold 2 -> rejected; lr_threshold 3 -> accepted
    x = 17
    dL, dR = _worked_example(x, 20, extra_rl={31: 228, 35: 228 - x})
    assert _the_candidate(orc.support_match(dL, dR, BASE)) == -1
    assert _the_candidate(orc.support_match(dL, dR, dict(BASE, lr_threshold=3))) == 4


def test_texture_threshold(orc):
    # left window texture = 4 * 100 = 400; right window at u_r = 26 (columns
    # 24 and 28 hold 228 and 211) = 2 * (100 + 83) = 366: both must pass
    dL, dR = _worked_example(17, 20)
    assert _the_candidate(orc.support_match(dL, dR, dict(BASE, support_texture=366))) == 4
    assert _the_candidate(orc.support_match(dL, dR, dict(BASE, support_texture=367))) == -1
    assert _the_candidate(orc.support_match(dL, dR, dict(BASE, support_texture=401))) == -1


def test_textureless_pair_has_no_support(orc):
    img = np.full((60, 80), 90, np.uint8)
    d = orc.descriptors(img)
    dcan = orc.support_points(d, d, dict(disp_max=31))
    assert (dcan == -1).all()


@pytest.mark.parametrize("shift", [0, 3, 7, 19])
def test_known_shift_support(orc, shift):
    L, R = synth.fronto_parallel_pair(120, 60, shift, seed=100 + shift)
    dL, dR = orc.descriptors(L), orc.descriptors(R)
    raw = orc.support_match(dL, dR, dict(disp_max=31))
    vv, uu = np.mgrid[0:raw.shape[0], 0:raw.shape[1]] * 5
    # the true disparity is searchable only where the right window fits (u - s >= 4)
    matchable = (uu - shift >= 4) & (uu <= 120 - 5) & (vv >= 4) & (vv <= 60 - 5)
    acc = raw[matchable & (raw >= 0)]
    assert acc.size >= 0.9 * matchable.sum()
    assert (acc == shift).all()


def _grid(hc, wc, pts):
    g = np.full((hc, wc), -1, np.int16)
    for (i, j), d in pts.items():
        g[i, j] = d
    return g


def test_consistency_filter(orc):
    prm = dict(incon_window_size=5, incon_threshold=5, incon_min_support=5)
    # 3x3 block: each point has 8 agreeing neighbours -> kept; isolated point removed
    pts = {(i, j): 10 for i in range(5, 8) for j in range(5, 8)}
    pts[(0, 14)] = 30
    out = orc.filter_consistency(_grid(15, 15, pts), prm)
    for (i, j), d in pts.items():
        assert out[i, j] == (d if (i, j) != (0, 14) else -1)
    # centre with exactly 5 supporters at window distance 5 and |dd| = 5 -> kept
    ring = [(2, 7), (12, 7), (7, 2), (7, 12), (2, 2)]
    g = _grid(15, 15, {**{p: 15 for p in ring}, (7, 7): 10})
    assert orc.filter_consistency(g, prm)[7, 7] == 10
    # |dd| = 6 -> not supporters
    g = _grid(15, 15, {**{p: 16 for p in ring}, (7, 7): 10})
    assert orc.filter_consistency(g, prm)[7, 7] == -1
    # one supporter at window distance 6 -> only 4 left
    ring6 = [(1, 7)] + ring[1:]
    g = _grid(15, 15, {**{p: 15 for p in ring6}, (7, 7): 10})
    assert orc.filter_consistency(g, prm)[7, 7] == -1


def test_redundancy_filter(orc):
    prm = dict(redun_max_dist=5)
    # full 7x7 block of one disparity: exactly the 5x5 interior is redundant
    pts = {(i, j): 10 for i in range(4, 11) for j in range(4, 11)}
    out = orc.filter_redundancy(_grid(15, 15, pts), prm)
    for (i, j) in pts:
        interior = 5 <= i <= 9 and 5 <= j <= 9
        assert out[i, j] == (-1 if interior else 10)
    # plus shape at distance 5 in all four directions -> centre removed
    arms = [(7, 2), (7, 12), (2, 7), (12, 7)]
    g = _grid(15, 15, {**{p: 10 for p in arms}, (7, 7): 10})
    assert orc.filter_redundancy(g, prm)[7, 7] == -1
    # one arm at distance 6 -> kept
    g = _grid(15, 15, {**{p: 10 for p in [(7, 1)] + arms[1:]}, (7, 7): 10})
    assert orc.filter_redundancy(g, prm)[7, 7] == 10
    # identical means identical: an arm at d = 11 -> kept
    g = _grid(15, 15, {**{p: 10 for p in arms[:3]}, arms[3]: 11, (7, 7): 10})
    assert orc.filter_redundancy(g, prm)[7, 7] == 10


def test_past_only_redundancy(orc):
    """Sec. VI.C (ORACLE_FLAG_PAST_REDUNDANCY): only the directions already
    passed in raster order count, left and up."""
    past = dict(redun_max_dist=3, flags=orc.FLAG_PAST_REDUNDANCY)
    four = dict(redun_max_dist=3)
    # identical values to the left and above: removed by the past-only rule,
    # kept by the four-direction rule (nothing to the right or below)
    g = _grid(9, 9, {(4, 4): 7, (4, 1): 7, (1, 4): 7})
    assert orc.filter_redundancy(g, past)[4, 4] == -1
    assert orc.filter_redundancy(g, four)[4, 4] == 7
    # the points that supplied them have no past partner: kept
    assert orc.filter_redundancy(g, past)[4, 1] == 7 and orc.filter_redundancy(g, past)[1, 4] == 7
    # identical values only to the right and below: kept by both rules
    g = _grid(9, 9, {(4, 4): 7, (4, 7): 7, (7, 4): 7})
    assert orc.filter_redundancy(g, past)[4, 4] == 7
    assert orc.filter_redundancy(g, four)[4, 4] == 7
    # left within reach, up beyond it (distance 4 > 3): kept
    g = _grid(9, 9, {(5, 4): 7, (5, 2): 7, (1, 4): 7})
    assert orc.filter_redundancy(g, past)[5, 4] == 7
    # the full 7x7 block: every point with a block point to its left and
    # above goes (a 6x6 corner), the top row and the left column stay
    pts = {(i, j): 10 for i in range(4, 11) for j in range(4, 11)}
    out = orc.filter_redundancy(_grid(15, 15, pts), dict(redun_max_dist=5, flags=orc.FLAG_PAST_REDUNDANCY))
    for (i, j) in pts:
        assert out[i, j] == (-1 if i > 4 and j > 4 else 10)


def _bits(cell):
    return {32 * k + b for k, word in enumerate(cell) for b in range(32) if (int(word) >> b) & 1}


def test_grid_vectors_single_point(orc):
    prm = dict(disp_min=0, disp_max=63, grid_size=20)
    w, h = 100, 60
    for d, want in [(31, {30, 31, 32}), (0, {0, 1}), (63, {62, 63})]:
        lst = np.array([[45, 25, d]], np.int16)
        g = orc.grid_vectors(lst, w, h, prm, right=False)
        assert g.shape == (3, 5, 2)
        for cy in range(3):
            for cx in range(5):
                exp = want if 1 <= cx <= 3 else set()
                assert _bits(g[cy, cx]) == exp
    # right-image grid uses u - d: (45 - 31) // 20 = cell 0
    g = orc.grid_vectors(np.array([[45, 25, 31]], np.int16), w, h, prm, right=True)
    for cy in range(3):
        for cx in range(5):
            assert _bits(g[cy, cx]) == ({30, 31, 32} if cx <= 1 else set())


def test_support_list_raster_order(orc):
    g = _grid(4, 5, {(0, 3): 7, (1, 0): 2, (1, 4): 9, (3, 2): 0})
    lst = orc.support_list(g, dict(candidate_stepsize=5))
    np.testing.assert_array_equal(lst, [[15, 0, 7], [0, 5, 2], [20, 5, 9], [10, 15, 0]])


@pytest.mark.parametrize("k", [2, 3, 8, 14, 32])
def test_support_downsampling(orc, k):
    """The paper's down-sampling of the extracted support points (Sec. VII):
    the points numbered 0, k, 2k, ... in raster order stay.  The down-sampled
    list is every k-th entry of the full one, its length ceil(n / k), the
    candidate grid keeps exactly those points, and the grid vectors of the
    smaller list are a subset of the full ones."""
    wl = synth.SMALL_320
    L, R, _ = synth.workload_pair(wl, 0, 1)
    dL, dR = orc.descriptors(L), orc.descriptors(R)
    full = orc.support_points(dL, dR, wl.params)
    prm = dict(wl.params, support_downsample=k)
    down = orc.support_points(dL, dR, prm)
    lf, ld = orc.support_list(full, wl.params), orc.support_list(down, prm)
    assert len(ld) == -(-len(lf) // k) and len(lf) > 10 * k
    np.testing.assert_array_equal(ld, lf[::k])
    assert ((down == full) | (down == -1)).all() and int((down >= 0).sum()) == len(ld)
    h, w = L.shape
    gf, gd = orc.grid_vectors(lf, w, h, prm), orc.grid_vectors(ld, w, h, prm)
    assert ((gd & ~gf) == 0).all() and (gd != gf).any()
    for k0 in (0, 1):
        np.testing.assert_array_equal(orc.support_points(dL, dR, dict(wl.params, support_downsample=k0)), full)


def test_downsampling_of_an_empty_support_set(orc):
    """A textureless pair has no support point: down-sampling keeps none and
    the list is empty for every k."""
    img = np.full((60, 80), 90, np.uint8)
    d = orc.descriptors(img)
    for k in (1, 2, 14):
        prm = dict(disp_max=31, support_downsample=k)
        assert len(orc.support_list(orc.support_points(d, d, prm), prm)) == 0
