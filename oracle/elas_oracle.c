/*
 * ELAS oracle -- plain CPU reference, TEST INFRASTRUCTURE ONLY.
 *
 * Follows Sec. III.A of arXiv 1802.07210 (the original ELAS pipeline:
 * gradient descriptors, support points with ratio test, consistency and
 * redundancy filtering, Delaunay mesh, slanted-plane prior, dense argmin,
 * left-right check, smoothing) together with the project readings that fix
 * every point the paper leaves open (descriptor layout, texture checks,
 * tie-breaks, rounding, pixel ownership).  Each function is a direct loop
 * over its definition; speed is irrelevant here.
 *
 * Parity status: no function can be pinned to per-pixel values printed in
 * the paper (it prints none).  Each is pinned instead by closed forms,
 * hand-computed cases, invariants and textbook special cases in tests/.
 * The 16-byte sample pattern itself is a project convention ("parity
 * unpinned" against the paper).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared  (see build.py).
 */
#include "elas_oracle.h"
#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

void oracle_params_default(oracle_params *p)
{
    /* The "robotics" parameter set the workloads are quoted with. */
    memset(p, 0, sizeof(*p));
    p->disp_min = 0;
    p->disp_max = 255;
    p->support_threshold = 0.85f;
    p->support_texture = 10;
    p->candidate_stepsize = 5;
    p->incon_window_size = 5;
    p->incon_threshold = 5;
    p->incon_min_support = 5;
    p->redun_max_dist = 5;
    p->grid_size = 20;
    p->beta = 0.02f;
    p->gamma = 3.0f;
    p->sigma = 1.0f;
    p->sradius = 2;
    p->match_texture = 1;
    p->lr_threshold = 2;
    p->ipol_gap_width = 3;
    p->filter_adaptive_mean = 1;
    p->flags = 0;
    p->census_support_w = 0;
    p->census_dense_w = 0;
    p->support_downsample = 0;
}

static int iabs(int x) { return x < 0 ? -x : x; }

/* ------------------------------------------------------------------------ */
/* Sobel gradients and descriptors (Sec. III.A, Fig. 1(b-d); Sec. VI.A)      */
/* ------------------------------------------------------------------------ */

/* du: horizontal Sobel stencil (-1 0 1 / -2 0 2 / -1 0 1) applied as a
 * correlation (weight +1 on the right column); dv: its transpose (+1 on the
 * row below).  The one-pixel frame has response 0. */
void oracle_sobel(const uint8_t *img, int w, int h, int32_t *du, int32_t *dv)
{
    for (int v = 0; v < h; v++)
        for (int u = 0; u < w; u++) {
            int32_t gx = 0, gy = 0;
            if (u >= 1 && u <= w - 2 && v >= 1 && v <= h - 2) {
#define I(x, y) ((int32_t)img[(size_t)(y) * w + (x)])
                gx = (I(u + 1, v - 1) + 2 * I(u + 1, v) + I(u + 1, v + 1))
                   - (I(u - 1, v - 1) + 2 * I(u - 1, v) + I(u - 1, v + 1));
                gy = (I(u - 1, v + 1) + 2 * I(u, v + 1) + I(u + 1, v + 1))
                   - (I(u - 1, v - 1) + 2 * I(u, v - 1) + I(u + 1, v - 1));
#undef I
            }
            du[(size_t)v * w + u] = gx;
            dv[(size_t)v * w + u] = gy;
        }
}

/* q(s) = clamp(128 + trunc(s/4), 1, 255); the lower bound 1 makes
 * q(-s) = 256 - q(s) exactly. */
static int quantise(int32_t s)
{
    int q = 128 + s / 4; /* C division truncates toward zero */
    if (q < 1) q = 1;
    if (q > 255) q = 255;
    return q;
}

/* Sample offsets (x, y) inside the 5x5 window: 8 from du, then 8 from dv. */
static const int DU_SAMPLES[8][2] = {{-2, -2}, {2, -2}, {-1, 0}, {1, 0},
                                     {-2, 2},  {2, 2},  {0, -1}, {0, 1}};
static const int DV_SAMPLES[8][2] = {{0, -2},  {0, 2},  {-2, 0}, {2, 0},
                                     {-1, -1}, {1, -1}, {-1, 1}, {1, 1}};

void oracle_descriptors(const uint8_t *img, int w, int h, uint8_t *desc)
{
    int32_t *du = (int32_t *)malloc(sizeof(int32_t) * (size_t)w * h);
    int32_t *dv = (int32_t *)malloc(sizeof(int32_t) * (size_t)w * h);
    oracle_sobel(img, w, h, du, dv);
    for (int v = 0; v < h; v++)
        for (int u = 0; u < w; u++) {
            uint8_t *out = desc + ((size_t)v * w + u) * 16;
            for (int k = 0; k < 8; k++) {
                int x = u + DU_SAMPLES[k][0], y = v + DU_SAMPLES[k][1];
                int inside = x >= 0 && x < w && y >= 0 && y < h;
                out[k] = (uint8_t)(inside ? quantise(du[(size_t)y * w + x]) : 128);
            }
            for (int k = 0; k < 8; k++) {
                int x = u + DV_SAMPLES[k][0], y = v + DV_SAMPLES[k][1];
                int inside = x >= 0 && x < w && y >= 0 && y < h;
                out[8 + k] = (uint8_t)(inside ? quantise(dv[(size_t)y * w + x]) : 128);
            }
        }
    free(du);
    free(dv);
}

/* ------------------------------------------------------------------------ */
/* Census transform and Hamming distance (Sec. VI.A)                          */
/* ------------------------------------------------------------------------ */

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

void oracle_census(const uint8_t *img, int w, int h, int W, int nbytes, uint8_t *out)
{
    int r = W / 2;
    for (int v = 0; v < h; v++)
        for (int u = 0; u < w; u++) {
            uint8_t *o = out + ((size_t)v * w + u) * nbytes;
            memset(o, 0, (size_t)nbytes);
            int centre = img[(size_t)v * w + u];
            for (int dy = -r; dy <= r; dy++)
                for (int dx = -r; dx <= r; dx++) {
                    int qx = clampi(u + dx, 0, w - 1), qy = clampi(v + dy, 0, h - 1);
                    int k = (dy + r) * W + (dx + r);
                    if (img[(size_t)qy * w + qx] < centre) o[k >> 3] |= (uint8_t)(1u << (k & 7));
                }
        }
}

/* number of differing bits of two n-byte strings */
static int hamming(const uint8_t *a, const uint8_t *b, int n)
{
    int s = 0;
    for (int k = 0; k < n; k++)
        for (int bit = 0; bit < 8; bit++) s += ((a[k] ^ b[k]) >> bit) & 1;
    return s;
}

/* ------------------------------------------------------------------------ */
/* Support points (Sec. III.A; Eq. 1-2 of Sec. VI.B for the ratio test)      */
/* ------------------------------------------------------------------------ */

static const uint8_t *DESC(const uint8_t *desc, int w, int u, int v)
{
    return desc + ((size_t)v * w + u) * 16;
}

static int sad16(const uint8_t *a, const uint8_t *b)
{
    int s = 0;
    for (int k = 0; k < 16; k++) s += iabs((int)a[k] - (int)b[k]);
    return s;
}

static int texture16(const uint8_t *a)
{
    int s = 0;
    for (int k = 0; k < 16; k++) s += iabs((int)a[k] - 128);
    return s;
}

/* The support window: four descriptors at the corners (u+-2, v+-2), 64 bytes
 * covering a 9x9 neighbourhood. */
static const int CORNERS[4][2] = {{-2, -2}, {2, -2}, {-2, 2}, {2, 2}};

static int window_texture(const uint8_t *desc, int w, int u, int v)
{
    int s = 0;
    for (int c = 0; c < 4; c++)
        s += texture16(DESC(desc, w, u + CORNERS[c][0], v + CORNERS[c][1]));
    return s;
}

static int window_cost(const uint8_t *ref, const uint8_t *oth, int w, int u_ref,
                       int u_oth, int v, const oracle_params *p)
{
    if (p->census_support_w > 0) /* the 32-byte support census of each pixel */
        return hamming(ref + ((size_t)v * w + u_ref) * 32, oth + ((size_t)v * w + u_oth) * 32, 32);
    int s = 0;
    for (int c = 0; c < 4; c++)
        s += sad16(DESC(ref, w, u_ref + CORNERS[c][0], v + CORNERS[c][1]),
                   DESC(oth, w, u_oth + CORNERS[c][0], v + CORNERS[c][1]));
    return s;
}

/* Best disparity of the window at (u, v) of `ref` against `oth`, searching
 * u_oth = u + dir*d over [disp_min, disp_max] with the other window inside
 * [4, w-5].  d1 = smallest d reaching the minimum m1, m2 = minimum over all
 * other d.  Accepted iff at least two disparities were evaluated, m2 > 0 and
 * (float)m1 <= t * (float)m2 (Eq. 2: m1 <= 0.9 m2, t from the parameters).
 * Returns d1 or -1. */
static int best_disparity(const uint8_t *ref, const uint8_t *oth, int w, int u, int v,
                          int dir, const oracle_params *p)
{
    int n_eval = 0, m1 = INT_MAX, d1 = -1;
    for (int d = p->disp_min; d <= p->disp_max; d++) {
        int uo = u + dir * d;
        if (uo < 4 || uo > w - 5) continue;
        int c = window_cost(ref, oth, w, u, uo, v, p);
        n_eval++;
        if (c < m1) { m1 = c; d1 = d; }
    }
    if (n_eval < 2) return -1;
    int m2 = INT_MAX;
    for (int d = p->disp_min; d <= p->disp_max; d++) {
        int uo = u + dir * d;
        if (uo < 4 || uo > w - 5 || d == d1) continue;
        int c = window_cost(ref, oth, w, u, uo, v, p);
        if (c < m2) m2 = c;
    }
    if (m2 <= 0) return -1;
    if (p->flags & ORACLE_FLAG_SHIFT_SUM) {
        /* Eq. 3: T_err(m2) = m2/2 + m2/4 + m2/8 + m2/32, each term a right
         * shift of the integer m2 (the LUT shift-sum of Sec. VI.B) */
        int t = (m2 >> 1) + (m2 >> 2) + (m2 >> 3) + (m2 >> 5);
        return m1 <= t ? d1 : -1;
    }
    float lhs = (float)m1;
    float rhs = p->support_threshold * (float)m2;
    if (!(lhs <= rhs)) return -1;
    return d1;
}

void oracle_support_match(const uint8_t *descL, const uint8_t *descR, int w, int h,
                          const oracle_params *p, int16_t *dcan)
{
    int step = p->candidate_stepsize;
    int wc = w / step, hc = h / step;
    for (int ic = 0; ic < hc; ic++)
        for (int jc = 0; jc < wc; jc++) {
            int u = jc * step, v = ic * step;
            int16_t out = -1;
            int census = p->census_support_w > 0;
            if (u >= 4 && u <= w - 5 && v >= 4 && v <= h - 5 &&
                (census || window_texture(descL, w, u, v) >= p->support_texture)) {
                int d1 = best_disparity(descL, descR, w, u, v, -1, p);
                if (d1 >= 0) {
                    int ur = u - d1;
                    if (census || window_texture(descR, w, ur, v) >= p->support_texture) {
                        int d2 = best_disparity(descR, descL, w, ur, v, +1, p);
                        if (d2 >= 0 && iabs(d1 - d2) <= p->lr_threshold) out = (int16_t)d1;
                    }
                }
            }
            dcan[(size_t)ic * wc + jc] = out;
        }
}

/* Keep a point iff at least incon_min_support other valid points inside the
 * +-incon_window_size window (candidate units) differ by <= incon_threshold.
 * All decisions read the unfiltered input. */
void oracle_filter_consistency(const int16_t *in, int wc, int hc,
                               const oracle_params *p, int16_t *out)
{
    int r = p->incon_window_size;
    for (int ic = 0; ic < hc; ic++)
        for (int jc = 0; jc < wc; jc++) {
            int d = in[(size_t)ic * wc + jc];
            int16_t res = -1;
            if (d >= 0) {
                int cnt = 0;
                for (int di = -r; di <= r; di++)
                    for (int dj = -r; dj <= r; dj++) {
                        if (di == 0 && dj == 0) continue;
                        int i2 = ic + di, j2 = jc + dj;
                        if (i2 < 0 || i2 >= hc || j2 < 0 || j2 >= wc) continue;
                        int d2 = in[(size_t)i2 * wc + j2];
                        if (d2 >= 0 && iabs(d2 - d) <= p->incon_threshold) cnt++;
                    }
                if (cnt >= p->incon_min_support) res = (int16_t)d;
            }
            out[(size_t)ic * wc + jc] = res;
        }
}

/* Remove a point iff a point with the identical disparity lies within
 * redun_max_dist candidates in each of the four directions (left, right, up,
 * down); with ORACLE_FLAG_PAST_REDUNDANCY (Sec. VI.C) only the directions
 * already passed in raster order count: left and up.  All decisions read the
 * consistency-filtered input. */
void oracle_filter_redundancy(const int16_t *in, int wc, int hc,
                              const oracle_params *p, int16_t *out)
{
    /* left, up, right, down: the past-only rule takes the first two */
    static const int DIRS[4][2] = {{0, -1}, {-1, 0}, {0, 1}, {1, 0}};
    const int ndir = (p->flags & ORACLE_FLAG_PAST_REDUNDANCY) ? 2 : 4;
    for (int ic = 0; ic < hc; ic++)
        for (int jc = 0; jc < wc; jc++) {
            int d = in[(size_t)ic * wc + jc];
            int16_t res = -1;
            if (d >= 0) {
                int redundant = 1;
                for (int k = 0; k < ndir; k++) {
                    int found = 0;
                    for (int s = 1; s <= p->redun_max_dist; s++) {
                        int i2 = ic + s * DIRS[k][0], j2 = jc + s * DIRS[k][1];
                        if (i2 < 0 || i2 >= hc || j2 < 0 || j2 >= wc) break;
                        if (in[(size_t)i2 * wc + j2] == d) { found = 1; break; }
                    }
                    if (!found) redundant = 0;
                }
                if (!redundant) res = (int16_t)d;
            }
            out[(size_t)ic * wc + jc] = res;
        }
}

void oracle_support_points(const uint8_t *descL, const uint8_t *descR, int w, int h,
                           const oracle_params *p, int16_t *dcan)
{
    int step = p->candidate_stepsize;
    int wc = w / step, hc = h / step;
    size_t nc = (size_t)wc * hc;
    int16_t *raw = (int16_t *)malloc(sizeof(int16_t) * (nc ? nc : 1));
    int16_t *con = (int16_t *)malloc(sizeof(int16_t) * (nc ? nc : 1));
    oracle_support_match(descL, descR, w, h, p, raw);
    oracle_filter_consistency(raw, wc, hc, p, con);
    if (p->flags & ORACLE_FLAG_REDUNDANCY_OFF)
        memcpy(dcan, con, sizeof(int16_t) * nc);
    else
        oracle_filter_redundancy(con, wc, hc, p, dcan);
    if (p->support_downsample > 1) {
        /* keep the surviving points numbered 0, k, 2k, ... in raster order */
        size_t rank = 0;
        for (size_t i = 0; i < nc; i++) {
            if (dcan[i] < 0) continue;
            if (rank % (size_t)p->support_downsample != 0) dcan[i] = -1;
            rank++;
        }
    }
    free(raw);
    free(con);
}

int oracle_support_list(const int16_t *dcan, int wc, int hc, int step, int16_t *list)
{
    int n = 0;
    for (int ic = 0; ic < hc; ic++)
        for (int jc = 0; jc < wc; jc++) {
            int d = dcan[(size_t)ic * wc + jc];
            if (d < 0) continue;
            list[3 * n + 0] = (int16_t)(jc * step);
            list[3 * n + 1] = (int16_t)(ic * step);
            list[3 * n + 2] = (int16_t)d;
            n++;
        }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Grid vectors (Sec. III.A, Fig. 2; one-hot masks of Sec. VI.D)             */
/* ------------------------------------------------------------------------ */

void oracle_grid_vectors(const int16_t *list, int n, int w, int h,
                         const oracle_params *p, int right, uint32_t *grid)
{
    int G = p->grid_size;
    int gw = (w + G - 1) / G, gh = (h + G - 1) / G;
    int nw = (p->disp_max + 1 + 31) / 32;
    memset(grid, 0, sizeof(uint32_t) * (size_t)gw * gh * nw);
    for (int i = 0; i < n; i++) {
        int u = list[3 * i], v = list[3 * i + 1], d = list[3 * i + 2];
        int x = right ? u - d : u;
        int cx = x / G, cy = v / G;
        for (int cy2 = cy - 1; cy2 <= cy + 1; cy2++)
            for (int cx2 = cx - 1; cx2 <= cx + 1; cx2++) {
                if (cx2 < 0 || cx2 >= gw || cy2 < 0 || cy2 >= gh) continue;
                uint32_t *cell = grid + ((size_t)cy2 * gw + cx2) * nw;
                for (int dd = d - 1; dd <= d + 1; dd++) {
                    if (dd < p->disp_min || dd > p->disp_max) continue;
                    cell[dd >> 5] |= 1u << (dd & 31);
                }
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Delaunay triangulation (Sec. III.A)                                       */
/* ------------------------------------------------------------------------ */
/* Bowyer-Watson with a vertex at infinity ("ghost" triangles (a, b, INF),
 * whose outside half-plane is left of a->b), and exact integer predicates.
 * Cocircular ties are broken by perturbing the lifted heights
 * |p_i|^2 + eps_i with eps_0 >> eps_1 >> ... (the lowest index dominates), so
 * the triangulation is the unique one of the perturbed point set, whatever
 * algorithm builds it.  Every insertion scans all live triangles for
 * conflicts.  A finite triangle whose circumcircle lies wholly above the
 * lowest row any point still to come can occupy (every such point strictly
 * outside it, so no perturbation is ever consulted) can never be destroyed
 * again; it is set aside as final before the scan.  With the support list's
 * raster order this keeps the scanned set to the triangles near the current
 * row, and it changes no triangle: only triangles that could not conflict
 * are skipped. */

#define OINF (-1)

int64_t oracle_orient(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy)
{
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

/* > 0 iff d lies strictly inside the circle through a, b, c (a, b, c CCW). */
int64_t oracle_incircle(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                        int64_t cx, int64_t cy, int64_t dx, int64_t dy)
{
    int64_t adx = ax - dx, ady = ay - dy, bdx = bx - dx, bdy = by - dy;
    int64_t cdx = cx - dx, cdy = cy - dy;
    int64_t al = adx * adx + ady * ady, bl = bdx * bdx + bdy * bdy, cl = cdx * cdx + cdy * cdy;
    return adx * (bdy * cl - bl * cdy) - ady * (bdx * cl - bl * cdx) + al * (bdx * cdy - bdy * cdx);
}

static int64_t orient_i(const int32_t *x, const int32_t *y, int a, int b, int c)
{
    return oracle_orient(x[a], y[a], x[b], y[b], x[c], y[c]);
}

static int sign64(int64_t v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }

/* Sign of the perturbed in-circle determinant.  Raising lift i by eps_i adds
 *   eps_a*orient(b,c,d) + eps_b*orient(c,a,d) + eps_c*orient(a,b,d)
 *   - eps_d*orient(a,b,c)
 * so on an exact tie the sign is that of the first nonzero coefficient in
 * ascending index order. */
static int incircle_sos(const int32_t *x, const int32_t *y, int a, int b, int c, int d)
{
    int64_t det = oracle_incircle(x[a], y[a], x[b], y[b], x[c], y[c], x[d], y[d]);
    if (det != 0) return sign64(det);
    int ids[4] = {a, b, c, d};
    int64_t coef[4] = {orient_i(x, y, b, c, d), orient_i(x, y, c, a, d),
                       orient_i(x, y, a, b, d), -orient_i(x, y, a, b, c)};
    for (int i = 0; i < 4; i++) /* selection order by index */
        for (int j = i + 1; j < 4; j++)
            if (ids[j] < ids[i]) {
                int ti = ids[i]; ids[i] = ids[j]; ids[j] = ti;
                int64_t tc = coef[i]; coef[i] = coef[j]; coef[j] = tc;
            }
    for (int i = 0; i < 4; i++)
        if (coef[i] != 0) return sign64(coef[i]);
    return 0;
}

/* Does inserting point q destroy triangle t? */
static int in_conflict(const int32_t *x, const int32_t *y, const int *t, int q)
{
    if (t[2] == OINF) {
        int a = t[0], b = t[1];
        int64_t o = orient_i(x, y, a, b, q);
        if (o > 0) return 1;
        if (o < 0) return 0;
        /* collinear with the hull edge: in conflict iff strictly between a, b */
        int64_t dot = (int64_t)(x[q] - x[a]) * (x[b] - x[a]) + (int64_t)(y[q] - y[a]) * (y[b] - y[a]);
        int64_t len2 = (int64_t)(x[b] - x[a]) * (x[b] - x[a]) + (int64_t)(y[b] - y[a]) * (y[b] - y[a]);
        return dot > 0 && dot < len2;
    }
    return incircle_sos(x, y, t[0], t[1], t[2], q) > 0;
}

/* Is every point (x, y) with y >= ymin strictly outside the circumcircle
 * of the counter-clockwise finite triangle t?  With b', c' the vertices
 * relative to a, O = orient(a, b, c) > 0 and D = 2 O, the centre is
 * a + (Nx, Ny) / D with Nx = c'y |b'|^2 - b'y |c'|^2,
 * Ny = b'x |c'|^2 - c'x |b'|^2, and the radius is sqrt(Nx^2 + Ny^2) / D, so
 * the circle's lowest point lies above row ymin iff M = (ymin - ay) D - Ny > 0
 * and Nx^2 + Ny^2 < M^2 (exact in 128-bit integers for 16-bit coordinates). */
static int circle_above(const int32_t *x, const int32_t *y, const int *t, int64_t ymin)
{
    int64_t ax = x[t[0]], ay = y[t[0]];
    int64_t bx = x[t[1]] - ax, by = y[t[1]] - ay, cx = x[t[2]] - ax, cy = y[t[2]] - ay;
    int64_t O = bx * cy - by * cx;
    if (O <= 0) return 0;
    int64_t b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    __int128 Nx = (__int128)cy * b2 - (__int128)by * c2;
    __int128 Ny = (__int128)bx * c2 - (__int128)cx * b2;
    __int128 M = (__int128)(ymin - ay) * (2 * O) - Ny;
    if (M <= 0) return 0;
    return Nx * Nx + Ny * Ny < M * M;
}

static void put_tri(int *T, int k, int a, int b, int c)
{
    /* keep the infinite vertex (if any) in the last slot, rotation preserved */
    if (a == OINF) { int t0 = b, t1 = c; a = t0; b = t1; c = OINF; }
    else if (b == OINF) { int t0 = c, t1 = a; a = t0; b = t1; c = OINF; }
    T[3 * k] = a; T[3 * k + 1] = b; T[3 * k + 2] = c;
}

int oracle_delaunay(const int32_t *x, const int32_t *y, int n, int32_t *tri, int cap)
{
    if (n < 3) return 0;
    int a = 0, b = 1, c = -1;
    for (int k = 2; k < n; k++)
        if (orient_i(x, y, 0, 1, k) != 0) { c = k; break; }
    if (c < 0) return 0; /* all collinear: no triangle */
    if (orient_i(x, y, a, b, c) < 0) { int t = b; b = c; c = t; }

    int maxT = 3 * n + 16;
    int *T = (int *)malloc(sizeof(int) * 3 * (size_t)maxT);
    int nt = 0;
    put_tri(T, nt++, a, b, c);
    put_tri(T, nt++, b, a, OINF);
    put_tri(T, nt++, c, b, OINF);
    put_tri(T, nt++, a, c, OINF);

    char *inserted = (char *)calloc((size_t)n, 1);
    char *dead = (char *)malloc((size_t)maxT);
    int *edges = (int *)malloc(sizeof(int) * 2 * 3 * (size_t)maxT);
    int *F = (int *)malloc(sizeof(int) * 3 * (size_t)maxT); /* final (set-aside) triangles */
    int nf = 0;
    /* ylow[q] = lowest y among the points at positions q..n-1 */
    int32_t *ylow = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    ylow[n - 1] = y[n - 1];
    for (int k = n - 2; k >= 0; k--) ylow[k] = y[k] < ylow[k + 1] ? y[k] : ylow[k + 1];
    inserted[a] = inserted[b] = inserted[c] = 1;

    int64_t swept = INT64_MIN;
    for (int q = 0; q < n; q++) {
        if (inserted[q]) continue;
        inserted[q] = 1;
        if (ylow[q] > swept) {
            /* set aside the triangles no remaining point can destroy */
            swept = ylow[q];
            int w = 0;
            for (int k = 0; k < nt; k++) {
                if (T[3 * k + 2] != OINF && circle_above(x, y, &T[3 * k], swept)) {
                    F[3 * nf] = T[3 * k]; F[3 * nf + 1] = T[3 * k + 1]; F[3 * nf + 2] = T[3 * k + 2];
                    nf++;
                    continue;
                }
                if (w != k) { T[3 * w] = T[3 * k]; T[3 * w + 1] = T[3 * k + 1]; T[3 * w + 2] = T[3 * k + 2]; }
                w++;
            }
            nt = w;
        }
        for (int k = 0; k < nt; k++) dead[k] = (char)in_conflict(x, y, &T[3 * k], q);
        /* cavity boundary: directed edges of dead triangles whose reverse is
         * not an edge of another dead triangle */
        int ne = 0;
        for (int k = 0; k < nt; k++) {
            if (!dead[k]) continue;
            for (int e = 0; e < 3; e++) {
                int ea = T[3 * k + e], eb = T[3 * k + (e + 1) % 3];
                int shared = 0;
                for (int m = 0; m < nt && !shared; m++) {
                    if (m == k || !dead[m]) continue;
                    for (int f = 0; f < 3; f++)
                        if (T[3 * m + f] == eb && T[3 * m + (f + 1) % 3] == ea) { shared = 1; break; }
                }
                if (!shared) { edges[2 * ne] = ea; edges[2 * ne + 1] = eb; ne++; }
            }
        }
        /* drop dead triangles */
        int w = 0;
        for (int k = 0; k < nt; k++)
            if (!dead[k]) {
                if (w != k) { T[3 * w] = T[3 * k]; T[3 * w + 1] = T[3 * k + 1]; T[3 * w + 2] = T[3 * k + 2]; }
                w++;
            }
        nt = w;
        for (int e = 0; e < ne; e++) put_tri(T, nt++, edges[2 * e], edges[2 * e + 1], q);
    }

    int out = 0;
    for (int k = 0; k < nf && out >= 0; k++) {
        if (out >= cap) { out = -1; break; }
        tri[3 * out] = F[3 * k]; tri[3 * out + 1] = F[3 * k + 1]; tri[3 * out + 2] = F[3 * k + 2];
        out++;
    }
    for (int k = 0; k < nt && out >= 0; k++) {
        if (T[3 * k + 2] == OINF) continue;
        if (out >= cap) { out = -1; break; }
        tri[3 * out] = T[3 * k]; tri[3 * out + 1] = T[3 * k + 1]; tri[3 * out + 2] = T[3 * k + 2];
        out++;
    }
    free(T); free(F); free(ylow); free(inserted); free(dead); free(edges);
    return out;
}

int oracle_triangulate(const int16_t *list, int n, int right, int32_t *tri, int cap)
{
    int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *y = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int m = 0;
    for (int i = 0; i < n; i++) {
        int px = right ? list[3 * i] - list[3 * i + 2] : list[3 * i];
        int py = list[3 * i + 1];
        int dup = 0;
        for (int j = 0; j < m; j++)
            if (x[j] == px && y[j] == py) { dup = 1; break; }
        if (dup) continue;
        x[m] = px; y[m] = py; idx[m] = i; m++;
    }
    int nt = oracle_delaunay(x, y, m, tri, cap);
    for (int k = 0; nt > 0 && k < 3 * nt; k++) tri[k] = idx[tri[k]];
    free(x); free(y); free(idx);
    return nt;
}

/* ------------------------------------------------------------------------ */
/* Slanted-plane prior (Sec. III.A; prior matrix of Sec. VI.D)               */
/* ------------------------------------------------------------------------ */

/* P[delta] = trunc((log(gamma) - log(gamma + exp(-delta^2 / (2 sigma^2)))) / beta)
 * in double from the float parameters; delta = |d - d_plane| <= sradius. */
void oracle_prior_table(const oracle_params *p, int32_t *P)
{
    double g = (double)p->gamma, s = (double)p->sigma, b = (double)p->beta;
    for (int dlt = 0; dlt <= p->sradius; dlt++) {
        double e = exp(-((double)dlt * (double)dlt) / (2.0 * s * s));
        P[dlt] = (int32_t)((log(g) - log(g + e)) / b);
    }
}

/* Edge P->Q owns the pixels lying exactly on it iff it is a top edge
 * (horizontal, pointing +u) or a left edge (pointing -v), for triangles whose
 * edge functions are positive inside. */
static int edge_owned(int px, int py, int qx, int qy)
{
    return (qy == py && qx > px) || (qy < py);
}

static int64_t edge_fn(int px, int py, int qx, int qy, int x, int y)
{
    return (int64_t)(qx - px) * (y - py) - (int64_t)(qy - py) * (x - px);
}

void oracle_plane_prior(const int16_t *list, int n, const int32_t *tri, int ntri,
                        int right, int w, int h, const oracle_params *p,
                        int16_t *dplane, int32_t *owners)
{
    (void)n;
    for (size_t i = 0; i < (size_t)w * h; i++) dplane[i] = -1;
    if (owners) memset(owners, 0, sizeof(int32_t) * (size_t)w * h);
    for (int t = 0; t < ntri; t++) {
        int id[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        /* canonical vertex order: ascending support-list index */
        for (int i = 0; i < 3; i++)
            for (int j = i + 1; j < 3; j++)
                if (id[j] < id[i]) { int s = id[i]; id[i] = id[j]; id[j] = s; }
        int X[3], Y[3], Z[3];
        for (int k = 0; k < 3; k++) {
            int u = list[3 * id[k]], v = list[3 * id[k] + 1], d = list[3 * id[k] + 2];
            X[k] = right ? u - d : u;
            Y[k] = v;
            Z[k] = d;
        }
        int64_t det = (int64_t)(X[1] - X[0]) * (Y[2] - Y[0]) - (int64_t)(X[2] - X[0]) * (Y[1] - Y[0]);
        if (det == 0) continue;
        int64_t na = (int64_t)(Z[1] - Z[0]) * (Y[2] - Y[0]) - (int64_t)(Z[2] - Z[0]) * (Y[1] - Y[0]);
        int64_t nb = (int64_t)(X[1] - X[0]) * (Z[2] - Z[0]) - (int64_t)(X[2] - X[0]) * (Z[1] - Z[0]);
        float a = (float)na / (float)det;
        float b = (float)nb / (float)det;
        float c = (float)Z[0] - a * (float)X[0];
        c = c - b * (float)Y[0];
        /* positively oriented vertex order for the edge functions */
        int o0 = 0, o1 = 1, o2 = 2;
        if (det < 0) { o1 = 2; o2 = 1; }
        int ex[3] = {X[o0], X[o1], X[o2]}, ey[3] = {Y[o0], Y[o1], Y[o2]};
        int xmin = X[0], xmax = X[0], ymin = Y[0], ymax = Y[0];
        for (int k = 1; k < 3; k++) {
            if (X[k] < xmin) xmin = X[k];
            if (X[k] > xmax) xmax = X[k];
            if (Y[k] < ymin) ymin = Y[k];
            if (Y[k] > ymax) ymax = Y[k];
        }
        if (xmin < 0) xmin = 0;
        if (ymin < 0) ymin = 0;
        if (xmax > w - 1) xmax = w - 1;
        if (ymax > h - 1) ymax = h - 1;
        for (int yy = ymin; yy <= ymax; yy++)
            for (int xx = xmin; xx <= xmax; xx++) {
                int inside = 1;
                for (int e = 0; e < 3; e++) {
                    int px = ex[e], py = ey[e], qx = ex[(e + 1) % 3], qy = ey[(e + 1) % 3];
                    int64_t E = edge_fn(px, py, qx, qy, xx, yy);
                    if (!(E > 0 || (E == 0 && edge_owned(px, py, qx, qy)))) { inside = 0; break; }
                }
                if (!inside) continue;
                float t1 = a * (float)xx;
                float t2 = b * (float)yy;
                float mu = t1 + t2;
                mu = mu + c;
                int dp = (int)floorf(mu + 0.5f);
                if (dp < p->disp_min) dp = p->disp_min;
                if (dp > p->disp_max) dp = p->disp_max;
                dplane[(size_t)yy * w + xx] = (int16_t)dp;
                if (owners) owners[(size_t)yy * w + xx]++;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Dense matching (Sec. III.A, Fig. 1(h))                                     */
/* ------------------------------------------------------------------------ */

void oracle_dense(const uint8_t *descL, const uint8_t *descR, int w, int h,
                  const oracle_params *p, const int16_t *dplane,
                  const uint32_t *grid, int right, int16_t *out)
{
    int32_t P[64];
    int sr = p->sradius;
    oracle_prior_table(p, P);
    int full = (p->flags & ORACLE_FLAG_FULL_RANGE) != 0;
    int prior_off = (p->flags & ORACLE_FLAG_PRIOR_OFF) != 0;
    int G = p->grid_size, gw = (w + G - 1) / G;
    int nw = (p->disp_max + 1 + 31) / 32;
    const uint8_t *ref = right ? descR : descL;
    const uint8_t *oth = right ? descL : descR;
    int dir = right ? +1 : -1;
    for (int v = 0; v < h; v++)
        for (int u = 0; u < w; u++) {
            int16_t res = -1;
            out[(size_t)v * w + u] = res;
            if (u < 2 || u > w - 3 || v < 2 || v > h - 3) continue;
            const uint8_t *dr = DESC(ref, w, u, v);
            int census = p->census_dense_w > 0;
            if (!census && texture16(dr) < p->match_texture) continue;
            int dp = full ? -1 : dplane[(size_t)v * w + u];
            if (!full && dp < 0) continue;
            const uint32_t *cell = grid ? grid + ((size_t)(v / G) * gw + (u / G)) * nw : NULL;
            int best_c = INT_MAX, best_d = -1;
            for (int d = p->disp_min; d <= p->disp_max; d++) {
                int uo = u + dir * d;
                if (uo < 2 || uo > w - 3) continue;
                int in_plane = !full && iabs(d - dp) <= sr;
                int in_grid = !full && ((cell[d >> 5] >> (d & 31)) & 1u);
                if (!full && !in_plane && !in_grid) continue;
                int c = census ? hamming(dr, DESC(oth, w, uo, v), 16) : sad16(dr, DESC(oth, w, uo, v));
                if (in_plane && !prior_off) c += P[iabs(d - dp)];
                if (c < best_c) { best_c = c; best_d = d; }
            }
            out[(size_t)v * w + u] = (int16_t)best_d;
        }
}

/* ------------------------------------------------------------------------ */
/* Left-right check (Sec. III.A, Fig. 1(i))                                   */
/* ------------------------------------------------------------------------ */

void oracle_lr_check(const int16_t *dL, const int16_t *dR, int w, int h, int thr,
                     int16_t *outL, int16_t *outR, uint8_t *maskL, uint8_t *maskR)
{
    for (int v = 0; v < h; v++)
        for (int u = 0; u < w; u++) {
            size_t i = (size_t)v * w + u;
            int d = dL[i], keep = 0;
            if (d >= 0 && u - d >= 0) {
                int dr = dR[(size_t)v * w + (u - d)];
                if (dr >= 0 && iabs(d - dr) <= thr) keep = 1;
            }
            maskL[i] = (uint8_t)keep;
            outL[i] = keep ? (int16_t)d : (int16_t)-1;
            d = dR[i];
            keep = 0;
            if (d >= 0 && u + d <= w - 1) {
                int dl = dL[(size_t)v * w + (u + d)];
                if (dl >= 0 && iabs(d - dl) <= thr) keep = 1;
            }
            maskR[i] = (uint8_t)keep;
            outR[i] = keep ? (int16_t)d : (int16_t)-1;
        }
}

/* ------------------------------------------------------------------------ */
/* Post-processing (Sec. III.A, Fig. 1(i)): gap interpolation, adaptive mean */
/* ------------------------------------------------------------------------ */

#define AM_RADIUS 3

/* One gap-interpolation pass along lines of length `len`, `nl` lines,
 * element k of line l at in[l*ls + k*es]. */
static void gap_pass(const float *in, float *out, int nl, int len, size_t ls, size_t es,
                     int gap)
{
    for (int l = 0; l < nl; l++) {
        for (int k = 0; k < len; k++) out[l * ls + k * es] = in[l * ls + k * es];
        int k = 0;
        while (k < len) {
            if (in[l * ls + k * es] >= 0.0f) { k++; continue; }
            int s = k;
            while (k < len && in[l * ls + k * es] < 0.0f) k++;
            int e = k - 1; /* maximal invalid run [s, e] */
            if (s > 0 && e < len - 1 && e - s + 1 <= gap) {
                float d1 = in[l * ls + (s - 1) * es], d2 = in[l * ls + (e + 1) * es];
                float val = fabsf(d1 - d2) < 3.0f ? (d1 + d2) * 0.5f : (d1 < d2 ? d1 : d2);
                for (int m = s; m <= e; m++) out[l * ls + m * es] = val;
            }
        }
    }
}

static void mean_pass(const float *in, float *out, int nl, int len, size_t ls, size_t es)
{
    for (int l = 0; l < nl; l++)
        for (int k = 0; k < len; k++) {
            float d0 = in[l * ls + k * es];
            if (d0 < 0.0f) { out[l * ls + k * es] = d0; continue; }
            float sw = 0.0f, swd = 0.0f;
            for (int o = -AM_RADIUS; o <= AM_RADIUS; o++) {
                int m = k + o;
                if (m < 0 || m >= len) continue;
                float di = in[l * ls + m * es];
                if (di < 0.0f) continue;
                float wgt = 4.0f - fabsf(di - d0);
                if (wgt > 0.0f) {
                    sw = sw + wgt;
                    float t = wgt * di;
                    swd = swd + t;
                }
            }
            out[l * ls + k * es] = swd / sw;
        }
}

void oracle_postprocess(const int16_t *d, int w, int h, const oracle_params *p, float *out)
{
    size_t np = (size_t)w * h;
    float *A = (float *)malloc(sizeof(float) * (np ? np : 1));
    float *B = (float *)malloc(sizeof(float) * (np ? np : 1));
    for (size_t i = 0; i < np; i++) A[i] = (float)d[i];
    if (p->ipol_gap_width > 0) {
        gap_pass(A, B, h, w, (size_t)w, 1, p->ipol_gap_width); /* rows    */
        gap_pass(B, A, w, h, 1, (size_t)w, p->ipol_gap_width); /* columns */
    }
    if (p->filter_adaptive_mean) {
        mean_pass(A, B, h, w, (size_t)w, 1); /* horizontal */
        mean_pass(B, A, w, h, 1, (size_t)w); /* vertical   */
    }
    memcpy(out, A, sizeof(float) * np);
    free(A);
    free(B);
}

/* The median filter of Sec. VII with the reading stated in the header: a
 * window at a time, values collected in raster order and sorted by insertion
 * sort, the element (n-1)/2 taken. */
void oracle_median(const int16_t *d, int w, int h, int r, int16_t *out)
{
    int16_t vals[(2 * 16 + 1) * (2 * 16 + 1)];
    if (r < 0) r = 0;
    if (r > 16) r = 16;
    for (int v = 0; v < h; v++)
        for (int u = 0; u < w; u++) {
            const int16_t c = d[(size_t)v * w + u];
            if (c < 0) {
                out[(size_t)v * w + u] = -1;
                continue;
            }
            int n = 0;
            for (int y = v - r; y <= v + r; y++)
                for (int x = u - r; x <= u + r; x++) {
                    if (x < 0 || x >= w || y < 0 || y >= h) continue;
                    const int16_t q = d[(size_t)y * w + x];
                    if (q >= 0) vals[n++] = q;
                }
            for (int i = 1; i < n; i++) {
                const int16_t t = vals[i];
                int j = i - 1;
                while (j >= 0 && vals[j] > t) {
                    vals[j + 1] = vals[j];
                    j--;
                }
                vals[j + 1] = t;
            }
            out[(size_t)v * w + u] = vals[(n - 1) / 2];
        }
}

/* ------------------------------------------------------------------------ */
/* Small-segment removal (ELAS post-processing; reading in elas_oracle.h)     */
/* ------------------------------------------------------------------------ */

void oracle_speckle(const int16_t *d, int w, int h, int sim_threshold, int min_size, int16_t *out)
{
    size_t n = (size_t)w * h;
    int32_t *seg = (int32_t *)malloc(n * sizeof(int32_t));     /* segment id, -1 = none yet */
    int32_t *queue = (int32_t *)malloc(n * sizeof(int32_t));   /* breadth-first queue       */
    for (size_t i = 0; i < n; i++) seg[i] = -1;
    static const int NB[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    for (size_t s = 0; s < n; s++) {
        if (d[s] < 0 || seg[s] >= 0) continue;
        /* grow the segment of seed s breadth first */
        size_t head = 0, tail = 0;
        queue[tail++] = (int32_t)s;
        seg[s] = (int32_t)s;
        while (head < tail) {
            int32_t p = queue[head++];
            int u = p % w, v = p / w;
            for (int k = 0; k < 4; k++) {
                int x = u + NB[k][0], y = v + NB[k][1];
                if (x < 0 || x >= w || y < 0 || y >= h) continue;
                size_t q = (size_t)y * w + x;
                if (d[q] < 0 || seg[q] >= 0) continue;
                if (iabs((int)d[q] - (int)d[p]) > sim_threshold) continue;
                seg[q] = (int32_t)s;
                queue[tail++] = (int32_t)q;
            }
        }
        /* the queue now lists exactly the tail pixels of this segment */
        int16_t keep = (int64_t)tail >= (int64_t)min_size;
        for (size_t k = 0; k < tail; k++) out[queue[k]] = keep ? d[queue[k]] : (int16_t)-1;
    }
    for (size_t i = 0; i < n; i++)
        if (d[i] < 0) out[i] = -1;
    free(seg);
    free(queue);
}
