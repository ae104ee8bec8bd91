"""Pins of the oracle's Delaunay triangulation (Sec. III.A: the support
points are triangulated with Delaunay to build the coarse mesh).

Checked against the definition (empty circumcircles), Euler's count and the
hull area, brute force in general position, and the closed form of the
symbolic tie-break on cocircular point sets."""
import itertools
import math

import numpy as np
import pytest


def _orient(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def _incircle(a, b, c, d):
    # plain 4x4 lifted determinant, Python big integers
    m = [[p[0] - d[0], p[1] - d[1], (p[0] - d[0]) ** 2 + (p[1] - d[1]) ** 2] for p in (a, b, c)]
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def _canon(tris):
    return sorted(tuple(sorted(t)) for t in np.asarray(tris).tolist())


def _hull_strict(pts):
    P = sorted(set(map(tuple, pts)))
    if len(P) < 3:
        return P
    lo, hi = [], []
    for p in P:
        while len(lo) >= 2 and _orient(lo[-2], lo[-1], p) <= 0:
            lo.pop()
        lo.append(p)
    for p in reversed(P):
        while len(hi) >= 2 and _orient(hi[-2], hi[-1], p) <= 0:
            hi.pop()
        hi.append(p)
    return lo[:-1] + hi[:-1]


def _on_boundary(pts, hull):
    cnt = 0
    for p in pts:
        on = False
        for a, b in zip(hull, hull[1:] + hull[:1]):
            if _orient(a, b, p) == 0 and min(a[0], b[0]) <= p[0] <= max(a[0], b[0]) \
                    and min(a[1], b[1]) <= p[1] <= max(a[1], b[1]):
                on = True
                break
        cnt += on
    return cnt


def _area2(poly):
    return sum(poly[i][0] * poly[(i + 1) % len(poly)][1] - poly[(i + 1) % len(poly)][0] * poly[i][1]
               for i in range(len(poly)))


def _check_valid_dt(pts, tris):
    pts = [tuple(map(int, p)) for p in pts]
    n = len(pts)
    hull = _hull_strict(pts)
    h = _on_boundary(pts, hull)
    assert len(tris) == 2 * n - h - 2, "Euler count"
    tot = 0
    edges = {}
    for t in tris:
        a, b, c = (pts[i] for i in t)
        o = _orient(a, b, c)
        assert o > 0, "triangles are counter-clockwise and non-degenerate"
        tot += o
        for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            assert e not in edges, "each directed edge once"
            edges[e] = True
        for k, p in enumerate(pts):
            if k in t:
                continue
            assert _incircle(a, b, c, p) <= 0, "empty circumcircle"
    assert tot == _area2(hull), "triangles tile the convex hull"


def test_general_position_matches_brute_force(orc):
    rng = np.random.default_rng(1)
    done = 0
    while done < 25:
        n = int(rng.integers(3, 11))
        pts = [tuple(map(int, p)) for p in rng.integers(0, 10000, (n, 2))]
        if len(set(pts)) < n:
            continue
        quads = itertools.combinations(range(n), 4)
        if any(_orient(pts[i], pts[j], pts[k]) == 0 for i, j, k in itertools.combinations(range(n), 3)):
            continue
        degenerate = False
        for q in quads:
            a, b, c, d = (pts[i] for i in q)
            if _orient(a, b, c) != 0 and _incircle(a, b, c, d) == 0:
                degenerate = True
        if degenerate:
            continue
        brute = []
        for i, j, k in itertools.combinations(range(n), 3):
            a, b, c = pts[i], pts[j], pts[k]
            if _orient(a, b, c) < 0:
                b, c = c, b
            if all(_incircle(a, b, c, pts[m]) < 0 for m in range(n) if m not in (i, j, k)):
                brute.append((i, j, k))
        got = orc.delaunay(pts)
        assert _canon(got) == sorted(brute)
        done += 1


def _incircle_all(P, T):
    """Exact incircle determinants of every point against every triangle
    (int64: coordinates below 2^14 keep each term below 2^58)."""
    out = []
    for t0 in range(0, len(T), 256):
        A, B, C = (P[T[t0:t0 + 256, i]][:, None, :] for i in range(3))
        m = [Q - P[None, :, :] for Q in (A, B, C)]
        lift = [q[..., 0] * q[..., 0] + q[..., 1] * q[..., 1] for q in m]
        det = (m[0][..., 0] * (m[1][..., 1] * lift[2] - lift[1] * m[2][..., 1])
               - m[0][..., 1] * (m[1][..., 0] * lift[2] - lift[1] * m[2][..., 0])
               + lift[0] * (m[1][..., 0] * m[2][..., 1] - m[1][..., 1] * m[2][..., 0]))
        out.append(det)
    return np.concatenate(out)


@pytest.mark.parametrize("seed", range(3))
def test_random_sets_match_qhull(orc, seed):
    """Sets of 1,500 points, far beyond what brute force reaches, against
    Qhull's Delaunay triangulation (a library routine), after checking
    exactly that Qhull's triangles have empty circumcircles with no fourth
    point on any of them: the triangulation is then the unique Delaunay one."""
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(300 + seed)
    P = np.unique(rng.integers(0, 16000, (1600, 2)), axis=0)[:1500]
    P = P[rng.permutation(len(P))].astype(np.int64)
    T = spatial.Delaunay(P.astype(np.float64)).simplices.astype(np.int64)
    # counter-clockwise, then every other point strictly outside each circle
    o = (P[T[:, 1], 0] - P[T[:, 0], 0]) * (P[T[:, 2], 1] - P[T[:, 0], 1]) \
        - (P[T[:, 1], 1] - P[T[:, 0], 1]) * (P[T[:, 2], 0] - P[T[:, 0], 0])
    assert np.all(o != 0)
    T[o < 0] = T[o < 0][:, [0, 2, 1]]
    det = _incircle_all(P, T)
    det[np.arange(len(T))[:, None], T] = -1  # a triangle's own vertices
    assert np.all(det < 0), "Qhull's triangulation is not strictly Delaunay for this seed"
    got = orc.delaunay([tuple(map(int, p)) for p in P])
    assert _canon(got) == _canon(T)


@pytest.mark.parametrize("seed", range(6))
def test_lattice_subsets_are_valid(orc, seed):
    rng = np.random.default_rng(seed)
    gx, gy = int(rng.integers(3, 14)), int(rng.integers(3, 10))
    lattice = [(5 * i, 5 * j) for j in range(gy) for i in range(gx)]
    keep = rng.random(len(lattice)) < rng.uniform(0.3, 1.0)
    pts = [p for p, k in zip(lattice, keep) if k]
    if len(pts) < 3 or len(_hull_strict(pts)) < 3:
        pytest.skip("degenerate subset")
    tris = orc.delaunay(pts)
    _check_valid_dt(pts, tris.tolist())


def test_row_sorted_lattice_is_valid(orc):
    """Points in raster order over many rows (the support list's order), so
    triangles whose circumcircles lie above every remaining row are set aside
    during the insertion: the result must still be the valid, unique
    triangulation (empty circumcircles, Euler count, hull area)."""
    rng = np.random.default_rng(11)
    lattice = [(5 * i, 5 * j) for j in range(18) for i in range(22)]
    pts = [p for p in lattice if rng.random() < 0.7]
    tris = orc.delaunay(pts)
    _check_valid_dt(pts, tris.tolist())


@pytest.mark.parametrize("seed", range(4))
def test_row_sorted_general_position_matches_brute_force(orc, seed):
    """Random points in general position inserted in ascending y: equal to the
    brute-force set of empty-circumcircle triangles."""
    rng = np.random.default_rng(100 + seed)
    while True:
        pts = sorted({tuple(map(int, p)) for p in rng.integers(0, 4000, (18, 2))}, key=lambda p: (p[1], p[0]))
        n = len(pts)
        if any(_orient(*(pts[i] for i in t)) == 0 for t in itertools.combinations(range(n), 3)):
            continue
        if any(_orient(*(pts[i] for i in q[:3])) != 0 and _incircle(*(pts[i] for i in q)) == 0
               for q in itertools.combinations(range(n), 4)):
            continue
        break
    brute = []
    for i, j, k in itertools.combinations(range(n), 3):
        a, b, c = pts[i], pts[j], pts[k]
        if _orient(a, b, c) < 0:
            b, c = c, b
        if all(_incircle(a, b, c, pts[m]) < 0 for m in range(n) if m not in (i, j, k)):
            brute.append((i, j, k))
    assert _canon(orc.delaunay(pts)) == sorted(brute)


def _ear_rule(poly_ids):
    """Closed form of the symbolic tie-break on a cocircular convex polygon:
    the vertex with the smallest index is lifted highest, so it is an ear;
    cut it off and recurse."""
    poly = list(poly_ids)
    out = []
    while len(poly) > 3:
        v = min(poly)
        k = poly.index(v)
        out.append(tuple(sorted((poly[k - 1], v, poly[(k + 1) % len(poly)]))))
        poly.pop(k)
    out.append(tuple(sorted(poly)))
    return sorted(out)


@pytest.mark.parametrize("seed", range(8))
def test_cocircular_tie_break_closed_form(orc, seed):
    # the 12 integer points on x^2 + y^2 = 25, shifted; input order = priority
    circ = [(x, y) for x in range(-5, 6) for y in range(-5, 6) if x * x + y * y == 25]
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(circ))
    pts = [(circ[i][0] + 10, circ[i][1] + 10) for i in perm]
    ang = [math.atan2(p[1] - 10, p[0] - 10) for p in pts]
    poly = sorted(range(len(pts)), key=lambda i: ang[i])
    assert _canon(orc.delaunay(pts)) == _ear_rule(poly)


def test_unit_square_takes_antidiagonal(orc):
    # raster order (0,0),(5,0),(0,5),(5,5): vertex 0 is an ear -> diagonal 1-2
    assert _canon(orc.delaunay([(0, 0), (5, 0), (0, 5), (5, 5)])) == [(0, 1, 2), (1, 2, 3)]


def test_degenerate_inputs(orc):
    assert len(orc.delaunay([])) == 0
    assert len(orc.delaunay([(0, 0), (5, 5)])) == 0
    assert len(orc.delaunay([(5 * i, 0) for i in range(7)])) == 0
    # collinear base + one apex: the only triangulation is the fan
    pts = [(5 * i, 0) for i in range(6)] + [(7, 9)]
    assert _canon(orc.delaunay(pts)) == sorted((i, i + 1, 6) for i in range(5))
    # the apex first in the input: same triangles, different indices
    pts2 = [(7, 9)] + [(5 * i, 0) for i in range(6)]
    assert _canon(orc.delaunay(pts2)) == sorted((0, i + 1, i + 2) for i in range(5))


def test_right_coordinates_drop_coincident_points(orc):
    # (20,0,5) and (25,0,10) both land on x = 15 in the right image: keep index 0
    lst = np.array([[20, 0, 5], [25, 0, 10], [40, 0, 3], [30, 10, 2], [10, 10, 1]], np.int16)
    tri = orc.triangulate(lst, right=True)
    assert 1 not in set(tri.ravel().tolist())
    assert len(tri) > 0
    tri_l = orc.triangulate(lst, right=False)
    assert 1 in set(tri_l.ravel().tolist())
