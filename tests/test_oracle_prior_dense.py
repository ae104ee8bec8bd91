"""Pins of the oracle's slanted-plane prior (Sec. III.A; the prior matrix of
Sec. VI.D) and dense matching (Sec. III.A, Fig. 1(h))."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_prior_table_golden(orc):
    g = json.load(open(os.path.join(GOLD, "prior_table.json")))
    for c in g["cases"]:
        P = orc.prior_table(dict(gamma=c["gamma"], sigma=c["sigma"], beta=c["beta"],
                                 sradius=c["sradius"]))
        np.testing.assert_array_equal(P, c["P"])


def _lattice_list(xs, ys, dfun):
    return np.array([[x, y, dfun(x, y)] for y in ys for x in xs], np.int16)


def test_exact_plane_and_rectangle_coverage(orc):
    """Support points on d = (u + 2v)/5 over a rectangle: every pixel of the
    half-open rectangle [10,60) x [5,40) gets round-half-up((u+2v)/5) (the
    fraction is never .5) and exactly one owner; all other pixels stay -1."""
    xs, ys = range(10, 61, 5), range(5, 41, 5)
    lst = _lattice_list(xs, ys, lambda x, y: (x + 2 * y) // 5)
    tri = orc.triangulate(lst)
    w, h = 80, 50
    dp, own = orc.plane_prior(lst, tri, w, h, dict(disp_max=63), with_owners=True)
    vv, uu = np.mgrid[0:h, 0:w]
    inside = (uu >= 10) & (uu < 60) & (vv >= 5) & (vv < 40)
    exp = np.where(inside, np.floor((uu + 2 * vv) / 5 + 0.5), -1).astype(np.int16)
    np.testing.assert_array_equal(dp, exp)
    np.testing.assert_array_equal(own, inside.astype(np.int32))


def test_random_mesh_rational_and_ownership(orc):
    """Random support disparities on a jittered lattice subset: no pixel has
    two owners, and every pixel strictly inside a triangle carries
    round-half-up of the exact rational plane value (within 1e-4 of a .5
    boundary FP32 may round either way: there it is one of the two neighbours)."""
    rng = np.random.default_rng(7)
    xs, ys = range(5, 76, 5), range(5, 56, 5)
    lst = [[x, y, int(rng.integers(0, 60))] for y in ys for x in xs if rng.random() < 0.8]
    lst = np.array(lst, np.int16)
    w, h = 80, 60
    for right in (False, True):
        tri = orc.triangulate(lst, right=right)
        dp, own = orc.plane_prior(lst, tri, w, h, dict(disp_max=63), right=right, with_owners=True)
        assert own.max() <= 1
        checked = ties = 0
        for t in tri.tolist():
            ids = sorted(t)
            P = [(int(lst[i, 0]) - (int(lst[i, 2]) if right else 0), int(lst[i, 1]), int(lst[i, 2]))
                 for i in ids]
            (x0, y0, z0), (x1, y1, z1), (x2, y2, z2) = P
            det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
            a = Fraction((z1 - z0) * (y2 - y0) - (z2 - z0) * (y1 - y0), det)
            b = Fraction((x1 - x0) * (z2 - z0) - (x2 - x0) * (z1 - z0), det)
            c = z0 - a * x0 - b * y0
            for yy in range(min(y0, y1, y2), max(y0, y1, y2) + 1):
                for xx in range(min(x0, x1, x2), max(x0, x1, x2) + 1):
                    e = [(qx - px) * (yy - py) - (qy - py) * (xx - px)
                         for (px, py), (qx, qy) in (((x0, y0), (x1, y1)), ((x1, y1), (x2, y2)),
                                                    ((x2, y2), (x0, y0)))]
                    if not (all(v > 0 for v in e) or all(v < 0 for v in e)):
                        continue
                    if not (0 <= xx < w and 0 <= yy < h):
                        continue
                    mu = a * xx + b * yy + c
                    frac = mu - (mu.numerator // mu.denominator)
                    if abs(float(frac) - 0.5) < 1e-4:
                        # at (or next to) an exact .5 the FP32 value may round either way
                        assert dp[yy, xx] in (int(np.floor(float(mu))), int(np.floor(float(mu))) + 1)
                        ties += 1
                        continue
                    assert dp[yy, xx] == int(np.floor(float(mu) + 0.5))
                    assert own[yy, xx] == 1
                    checked += 1
        assert checked > 1000 and ties < 0.1 * checked


def _desc_from_image(orc, rng, h, w):
    return orc.descriptors(rng.integers(0, 256, (h, w), dtype=np.uint8))


@pytest.mark.parametrize("right", [False, True])
def test_full_range_prior_off_is_plain_winner_take_all(orc, right):
    """With the prior off and every disparity a candidate, dense matching is
    textbook winner-take-all block matching: argmin over d of the 16-byte
    SAD, first minimum on ties (computed here as a cost volume)."""
    rng = np.random.default_rng(2 + right)
    h, w, dmax = 12, 40, 15
    dL = _desc_from_image(orc, rng, h, w).astype(np.int32)
    dR = _desc_from_image(orc, rng, h, w).astype(np.int32)
    prm = dict(disp_min=0, disp_max=dmax, flags=1 | 2, match_texture=1)
    got = orc.dense(dL.astype(np.uint8), dR.astype(np.uint8), None, None, prm, right=right)
    ref, oth, sgn = (dR, dL, 1) if right else (dL, dR, -1)
    big = 1 << 30
    cost = np.full((dmax + 1, h, w), big, np.int64)
    for d in range(dmax + 1):
        for u in range(w):
            uo = u + sgn * d
            if 2 <= uo <= w - 3:
                cost[d, :, u] = np.abs(ref[:, u] - oth[:, uo]).sum(-1)
    exp = np.argmin(cost, axis=0).astype(np.int16)
    exp[cost.min(0) == big] = -1
    tex = np.abs(ref - 128).sum(-1)
    exp[tex < 1] = -1
    exp[:2], exp[h - 2:], exp[:, :2], exp[:, w - 2:] = -1, -1, -1, -1
    np.testing.assert_array_equal(got, exp)


def _hand_pixel(costs, w=40, h=5, u=20, v=2):
    """descL(u,v) holds byte0 = 178; descR(u-d, v) holds byte0 = 178 - cost[d],
    so SAD(d) = cost[d] exactly; every other descriptor is flat (128)."""
    dL = np.full((h, w, 16), 128, np.uint8)
    dR = np.full((h, w, 16), 128, np.uint8)
    dL[v, u, 0] = 178
    for d, c in costs.items():
        dR[v, u - d, 0] = 178 - c
    return dL, dR


def test_candidate_set_and_prior(orc):
    # SAD: 10 at d=5, 3 at d=7, 0 at d=12, 100 elsewhere in 0..15
    costs = {d: 100 for d in range(16)}
    costs.update({5: 10, 7: 3, 12: 0})
    dL, dR = _hand_pixel(costs)
    dplane = np.full((5, 40), -1, np.int16)
    dplane[2, 20] = 5
    G = 20
    grid = np.zeros((1, 2, 1), np.uint32)   # 1 x 2 cells, one 32-bit word (disp_max 15)
    prm = dict(disp_min=0, disp_max=15, grid_size=G, sradius=2, gamma=3.0, sigma=1.0, beta=0.02)
    # plane window {3..7} with P = [-14,-9,-2]: d=5 -> 10-14=-4, d=7 -> 3-2=1 -> 5
    out = orc.dense(dL, dR, dplane, grid, prm)
    assert out[2, 20] == 5
    assert (np.delete(out.ravel(), 2 * 40 + 20) == -1).all()
    # prior off: the plane window's raw SAD minimum d=7
    assert orc.dense(dL, dR, dplane, grid, dict(prm, flags=1))[2, 20] == 7
    # grid bit 12 joins the candidates (cost 0, no prior): 5 still wins (-4 < 0)
    grid[0, 1, 0] = 1 << 12
    assert orc.dense(dL, dR, dplane, grid, prm)[2, 20] == 5
    assert orc.dense(dL, dR, dplane, grid, dict(prm, flags=1))[2, 20] == 12
    # no plane (d_plane = -1): the pixel is not matched even with grid candidates
    dplane[2, 20] = -1
    assert orc.dense(dL, dR, dplane, grid, prm)[2, 20] == -1


def test_tie_breaks_to_smaller_disparity(orc):
    costs = {d: 100 for d in range(16)}
    costs.update({9: 4, 11: 4})
    dL, dR = _hand_pixel(costs)
    prm = dict(disp_min=0, disp_max=15, flags=1 | 2)
    assert orc.dense(dL, dR, None, None, prm)[2, 20] == 9
