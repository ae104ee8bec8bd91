// Delaunay triangulation of the support points (Sec. III.A), host side.
//
// Incremental Bowyer-Watson over a triangle-adjacency structure with a
// vertex at infinity: every hull edge (a,b) carries a "ghost" triangle
// (a,b,INF) whose interior is the open half-plane left of a->b.  A new
// point is located by a visibility walk from the last created triangle
// (consecutive points are neighbours, so walks are short), its conflict region
// is grown by breadth-first search over neighbours, and the region's
// boundary is re-triangulated as a fan around the point.  Points are
// inserted along a Hilbert curve.
//
// Predicates are exact in 64-bit integers (coordinates < 2^14).  Cocircular
// ties are resolved by symbolically raising the lifted height of point i by
// eps_i, eps_0 >> eps_1 >> ... (the lowest index dominates): the resulting
// triangulation is the unique one of the perturbed set, independent of the
// insertion order or of the algorithm that computes it.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <unordered_set>
#include <vector>

#include "elas_gb300.h"

namespace elas {
elas_status fail(elas_status st, const char *fmt, ...);

namespace {

constexpr int kInf = -1;

struct Tri {
    int v[3];  // vertex ids; kInf only in slot 2
    int n[3];  // n[k]: triangle across edge (v[k], v[k+1])
    int mark;  // search stamp
    bool alive;
};

class Triangulation {
  public:
    Triangulation(const int32_t *x, const int32_t *y, int n) : X(x), Y(y), N(n) {}

    // Returns the number of finite triangles written (or the count needed).
    int64_t run(std::vector<int32_t> &out) {
        out.clear();
        if (N < 3) return 0;
        // Insertion order: along a Hilbert curve, so that every new point lies
        // next to the previous one and conflict regions stay small.  (Raster
        // order would insert each lattice row below a long collinear hull
        // edge and build a fan over the whole row per point.)  The result
        // does not depend on the order.
        std::vector<std::pair<uint32_t, int>> order(N);
        for (int i = 0; i < N; ++i) order[i] = {hilbert(X[i], Y[i]), i};
        std::stable_sort(order.begin(), order.end());
        const int p0 = order[0].second, p1 = order[1].second;
        int c = -1;
        for (int k = 2; k < N; ++k)
            if (orient(p0, p1, order[k].second) != 0) {
                c = order[k].second;
                break;
            }
        if (c < 0) return 0;
        int a = p0, b = p1;
        if (orient(a, b, c) < 0) std::swap(b, c);
        T.reserve(3 * (size_t)N + 16);
        const int f = make(a, b, c), g0 = make(b, a, kInf), g1 = make(c, b, kInf), g2 = make(a, c, kInf);
        const int ids[4] = {f, g0, g1, g2};
        link_group(ids, 4);
        hint = f;
        for (int k = 0; k < N; ++k) {
            const int p = order[k].second;
            if (p == a || p == b || p == c) continue;
            insert(p);
        }
        int64_t cnt = 0;
        for (const Tri &t : T)
            if (t.alive && t.v[2] != kInf) {
                out.push_back(t.v[0]);
                out.push_back(t.v[1]);
                out.push_back(t.v[2]);
                ++cnt;
            }
        return cnt;
    }

  private:
    const int32_t *X, *Y;
    int N;
    std::vector<Tri> T;
    std::vector<int> free_ids;
    int hint = 0;
    int stamp = 0;
    // scratch
    std::vector<int> stack, cavity;
    struct BEdge { int a, b, out; };
    std::vector<BEdge> bnd;
    std::vector<int> created;

    // Index of (x, y) along a Hilbert curve over [0, 2^15)^2.
    static uint32_t hilbert(int32_t xi, int32_t yi) {
        uint32_t x = (uint32_t)(xi + 8192), y = (uint32_t)(yi + 8192), d = 0;
        for (uint32_t s = 1u << 14; s > 0; s >>= 1) {
            const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
            d += s * s * ((3u * rx) ^ ry);
            if (ry == 0) {
                if (rx == 1) {
                    x = s - 1 - (x & (s - 1));
                    y = s - 1 - (y & (s - 1));
                }
                const uint32_t t = x;
                x = y;
                y = t;
            }
            x &= s - 1;
            y &= s - 1;
        }
        return d;
    }

    int64_t orient(int a, int b, int c) const {
        return (int64_t)(X[b] - X[a]) * (Y[c] - Y[a]) - (int64_t)(Y[b] - Y[a]) * (X[c] - X[a]);
    }

    // sign of the lifted 3x3 determinant: > 0 iff d inside circle(a,b,c), a,b,c CCW
    int incircle(int a, int b, int c, int d) const {
        const int64_t ax = X[a] - X[d], ay = Y[a] - Y[d];
        const int64_t bx = X[b] - X[d], by = Y[b] - Y[d];
        const int64_t cx = X[c] - X[d], cy = Y[c] - Y[d];
        const int64_t la = ax * ax + ay * ay, lb = bx * bx + by * by, lc = cx * cx + cy * cy;
        const int64_t det = la * (bx * cy - by * cx) - lb * (ax * cy - ay * cx) + lc * (ax * by - ay * bx);
        if (det != 0) return det > 0 ? 1 : -1;
        // perturbation: coefficient of eps_i for each of the four points
        const int who[4] = {a, b, c, d};
        const int64_t coef[4] = {orient(b, c, d), orient(c, a, d), orient(a, b, d), -orient(a, b, c)};
        int best = -1;
        for (int k = 0; k < 4; ++k)
            if (coef[k] != 0 && (best < 0 || who[k] < who[best])) best = k;
        if (best < 0) return 0;
        return coef[best] > 0 ? 1 : -1;
    }

    bool conflict(int t, int p) const {
        const Tri &tr = T[t];
        if (tr.v[2] == kInf) {
            const int a = tr.v[0], b = tr.v[1];
            const int64_t o = orient(a, b, p);
            if (o != 0) return o > 0;
            const int64_t dot = (int64_t)(X[p] - X[a]) * (X[b] - X[a]) + (int64_t)(Y[p] - Y[a]) * (Y[b] - Y[a]);
            const int64_t len = (int64_t)(X[b] - X[a]) * (X[b] - X[a]) + (int64_t)(Y[b] - Y[a]) * (Y[b] - Y[a]);
            return dot > 0 && dot < len;
        }
        return incircle(tr.v[0], tr.v[1], tr.v[2], p) > 0;
    }

    int make(int a, int b, int c) {
        int id;
        if (!free_ids.empty()) {
            id = free_ids.back();
            free_ids.pop_back();
        } else {
            id = (int)T.size();
            T.push_back(Tri());
        }
        Tri &t = T[id];
        t.v[0] = a;
        t.v[1] = b;
        t.v[2] = c;
        t.n[0] = t.n[1] = t.n[2] = -1;
        t.mark = 0;
        t.alive = true;
        return id;
    }

    // Connects the triangles of a group along their shared (reversed) edges.
    void link_group(const int *ids, int m) {
        for (int i = 0; i < m; ++i)
            for (int e = 0; e < 3; ++e) {
                const int a = T[ids[i]].v[e], b = T[ids[i]].v[(e + 1) % 3];
                for (int j = 0; j < m; ++j) {
                    if (j == i) continue;
                    for (int f = 0; f < 3; ++f)
                        if (T[ids[j]].v[f] == b && T[ids[j]].v[(f + 1) % 3] == a) T[ids[i]].n[e] = ids[j];
                }
            }
    }

    int locate(int p) {
        int t = hint;
        if (!T[t].alive) t = 0;
        while (!T[t].alive) ++t;
        if (T[t].v[2] == kInf) {
            if (conflict(t, p)) return t;
            t = T[t].n[0];  // the finite triangle across the hull edge
        }
        const int max_steps = 4 * (int)T.size() + 16;
        unsigned r = (unsigned)p * 2654435761u;
        for (int s = 0; s < max_steps; ++s) {
            const Tri &tr = T[t];
            if (tr.v[2] == kInf) {
                if (conflict(t, p)) return t;
                break;
            }
            r = r * 1103515245u + 12345u;
            const int off = (int)((r >> 16) % 3u);
            int next = -1;
            for (int k = 0; k < 3; ++k) {
                const int e = (k + off) % 3;
                if (orient(tr.v[e], tr.v[(e + 1) % 3], p) < 0) {
                    next = tr.n[e];
                    break;
                }
            }
            if (next < 0) return t;  // inside or on the boundary: in conflict
            t = next;
        }
        for (int i = 0; i < (int)T.size(); ++i)  // fallback, never expected
            if (T[i].alive && conflict(i, p)) return i;
        return -1;
    }

    void insert(int p) {
        const int t0 = locate(p);
        if (t0 < 0) return;
        ++stamp;
        stack.clear();
        cavity.clear();
        bnd.clear();
        T[t0].mark = stamp;
        stack.push_back(t0);
        while (!stack.empty()) {
            const int t = stack.back();
            stack.pop_back();
            cavity.push_back(t);
            for (int e = 0; e < 3; ++e) {
                const int nb = T[t].n[e];
                if (T[nb].mark == stamp) continue;
                if (conflict(nb, p)) {
                    T[nb].mark = stamp;
                    stack.push_back(nb);
                } else {
                    bnd.push_back({T[t].v[e], T[t].v[(e + 1) % 3], nb});
                }
            }
        }
        for (int t : cavity) {
            T[t].alive = false;
            T[t].mark = stamp;
            free_ids.push_back(t);
        }
        // new fan: triangle (a, b, p) per boundary edge (a, b), infinity last
        created.clear();
        const int m = (int)bnd.size();
        for (int i = 0; i < m; ++i) {
            const BEdge &be = bnd[i];
            int id;
            if (be.a == kInf)
                id = make(be.b, p, kInf);
            else if (be.b == kInf)
                id = make(p, be.a, kInf);
            else
                id = make(be.a, be.b, p);
            T[id].mark = stamp;
            created.push_back(id);
        }
        // The fan is a cycle around p: the twin of edge (b, p) of the triangle
        // built on boundary edge (a, b) is the one built on the edge leaving b,
        // the twin of (p, a) the one built on the edge entering a.
        for (int i = 0; i < m; ++i) {
            const BEdge &be = bnd[i];
            int next = -1, prev = -1;
            for (int j = 0; j < m; ++j) {
                if (bnd[j].a == be.b) next = created[j];
                if (bnd[j].b == be.a) prev = created[j];
            }
            Tri &nt = T[created[i]];
            for (int e = 0; e < 3; ++e) {
                const int a = nt.v[e], b = nt.v[(e + 1) % 3];
                if (a == be.a && b == be.b) {
                    nt.n[e] = be.out;
                    Tri &o = T[be.out];
                    for (int f = 0; f < 3; ++f)
                        if (o.v[f] == b && o.v[(f + 1) % 3] == a) o.n[f] = created[i];
                } else if (a == be.b) {
                    nt.n[e] = next;  // edge (b, p)
                } else {
                    nt.n[e] = prev;  // edge (p, a)
                }
            }
        }
        for (int id : created)
            if (T[id].v[2] != kInf) {
                hint = id;
                break;
            }
    }
};

}  // namespace

// Triangulates n points; triangles as index triples into the given arrays.
int64_t delaunay_points(const int32_t *x, const int32_t *y, int n, std::vector<int32_t> &tri) {
    Triangulation dt(x, y, n);
    return dt.run(tri);
}

}  // namespace elas

extern "C" elas_status elas_triangulate(const int16_t *list, int32_t n, int32_t right, int32_t *tri, int32_t cap,
                                        int32_t *ntri) {
    using namespace elas;
    if (!ntri) return fail(ELAS_ERR_INVALID_ARG, "ntri is NULL");
    *ntri = 0;
    if (n < 0) return fail(ELAS_ERR_INVALID_ARG, "negative point count");
    if (n > 0 && !list) return fail(ELAS_ERR_INVALID_ARG, "list is NULL");
    if (cap > 0 && !tri) return fail(ELAS_ERR_INVALID_ARG, "tri is NULL");
    std::vector<int32_t> x, y, idx;
    x.reserve(n);
    y.reserve(n);
    idx.reserve(n);
    std::unordered_set<int64_t> seen;
    if (right) seen.reserve(2 * (size_t)n + 1);
    for (int i = 0; i < n; ++i) {
        const int u = list[3 * i], v = list[3 * i + 1], d = list[3 * i + 2];
        const int px = right ? u - d : u;
        if (right) {
            const int64_t key = ((int64_t)v << 32) ^ (uint32_t)px;
            if (!seen.insert(key).second) continue;  // coincident: keep the lowest index
        }
        x.push_back(px);
        y.push_back(v);
        idx.push_back(i);
    }
    std::vector<int32_t> out;
    const int64_t nt = delaunay_points(x.data(), y.data(), (int)x.size(), out);
    *ntri = (int32_t)nt;
    if (nt > cap) return fail(ELAS_ERR_CAPACITY, "triangle capacity %d < %lld", cap, (long long)nt);
    for (int64_t k = 0; k < 3 * nt; ++k) tri[k] = idx[out[k]];
    return ELAS_OK;
}
