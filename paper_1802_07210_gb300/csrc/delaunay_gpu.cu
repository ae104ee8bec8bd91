// Delaunay triangulation of the support points on the GPU (Sec. III.A: the
// mesh of the support points; the paper keeps this step on a CPU and finds it
// dominates its run time, Sec. VII).
//
// The triangulation wanted is the unique one of the symbolically perturbed
// point set (lifted heights |p_i|^2 + eps_i, eps_0 >> eps_1 >> ..., i = list
// index), the same one the host routine builds.  Here every point builds its
// own star, one warp per point:
//   1. its nearest neighbour a0 (always a Delaunay edge: the circle with
//      diameter p-a0 holds no other point, not even on its boundary);
//   2. gift-wrapping counter-clockwise: the Delaunay triangle left of edge
//      (p, a) has as third vertex the point left of p->a that no other such
//      point lies inside the circle through p, a and it (exact predicate with
//      the symbolic tie-break: a strict total order, so a warp min-reduction
//      finds it); continue with (p, b) until the star closes at a0 or no
//      point is left of the edge (p on the hull), then wrap clockwise from a0.
// Pass 1 (a group of 16 lanes per point, 4 in batches) lists the points
// within R = 24 pixels (18 in batches) of p from a 16-pixel grid and wraps
// the star among them with the pencil key; it is accepted when every
// triangle's circumdisc lies inside that disc (4 r^2 <= R^2 in exact
// arithmetic, so no farther point can matter) and,
// where the star stays open (p on the hull), nothing lies beyond either open
// edge (checked against the extreme points of every image row).  In batches
// of two or more pairs the other stars go through the same group pass twice
// more: eight lanes and the points within 32 pixels, then one warp and the
// points within 64.  The rest are rebuilt by one CTA per point: each step
// takes the best of the points within 96 (then 192) pixels when its circle
// fits that disc, else scans the grid cells its circle (or, with no
// candidate, its half-plane) meets, which is exact.  Each triangle
// is emitted once, by its lowest-index vertex, at an offset from an
// exclusive scan of the per-point counts, so the output order is
// deterministic.
#include "launch.cuh"

namespace elas {

constexpr int kDtCell = 16;
constexpr int kDtMaxStar = 4096;  // wrap steps per star

__device__ __forceinline__ int dt_ncell(const DtArgs &a) { return a.gw * a.gh; }

__device__ __forceinline__ int dt_cell(const DtArgs &a, int x, int y) {
    const int cx = min(max(x, 0) / kDtCell, a.gw - 1), cy = min(max(y, 0) / kDtCell, a.gh - 1);
    return cy * a.gw + cx;
}

// -------------------------------------------------------------------------
// Exact predicates (coordinates below 2^15, products in 64 bits)
// -------------------------------------------------------------------------

__device__ __forceinline__ int64_t dt_orient(int ax, int ay, int bx, int by, int cx, int cy) {
    return (int64_t)(bx - ax) * (cy - ay) - (int64_t)(by - ay) * (cx - ax);
}

// Sign of "C strictly inside the circle through P, A, B" (P, A, B
// counter-clockwise), with the symbolic tie-break on the list indices.  T is
// the arithmetic type of the determinant: int is exact while every coordinate
// differs from P's by at most 64 (6 terms of at most 64*64*8192), int64_t
// always (differences below 2^15).
template <typename T>
__device__ __forceinline__ int dt_incircle(const int4 &P, const int4 &A, const int4 &B, const int4 &C) {
    const T ax = A.x - P.x, ay = A.y - P.y, bx = B.x - P.x, by = B.y - P.y, cx = C.x - P.x, cy = C.y - P.y;
    const T al = ax * ax + ay * ay, bl = bx * bx + by * by, cl = cx * cx + cy * cy;
    // value = -det[[a, |a|^2], [b, |b|^2], [c, |c|^2]] (relative to P)
    const T det = ax * (by * cl - bl * cy) - ay * (bx * cl - bl * cx) + al * (bx * cy - by * cx);
    if (det != 0) return det < 0 ? 1 : -1;
    // raising lift i by eps_i adds eps_P*orient(A,B,C) + eps_A*orient(B,P,C)
    // + eps_B*orient(P,A,C) - eps_C*orient(P,A,B); the lowest index decides
    const int who[4] = {P.z, A.z, B.z, C.z};
    const int64_t coef[4] = {dt_orient(A.x, A.y, B.x, B.y, C.x, C.y), dt_orient(B.x, B.y, P.x, P.y, C.x, C.y),
                             dt_orient(P.x, P.y, A.x, A.y, C.x, C.y), -dt_orient(P.x, P.y, A.x, A.y, B.x, B.y)};
    int best = -1;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (coef[k] != 0 && (best < 0 || who[k] < who[best])) best = k;
    return best < 0 ? 0 : (coef[best] > 0 ? 1 : -1);
}

// -------------------------------------------------------------------------
// Grid build
// -------------------------------------------------------------------------

__device__ __forceinline__ void dt_points_body(const DtArgs &a, const VB &vb) {
    const DtSide S = vb.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    for (int i = vb.x * blockDim.x + threadIdx.x; i < n; i += vb.gx * blockDim.x) {
        const int u = a.list[3 * i], v = a.list[3 * i + 1], d = a.list[3 * i + 2];
        const int x = S.right ? u - d : u;
        S.X[i] = x;
        S.Y[i] = v;
        S.status[i] = 0;
        S.owned[i] = 0;
        atomicAdd(S.cell_cnt + dt_cell(a, x, v), 1);
        if (v >= 0 && v < a.h) {
            atomicMin(S.rowmin + v, x);
            atomicMax(S.rowmax + v, x);
        }
    }
}

__global__ void dt_points_kernel(DtArgs a) { dt_points_body(a, vb_single()); }
__global__ void dt_points_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_points_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

// One CTA per side: exclusive scan of the cell counts, each thread taking
// kCellScanItems consecutive cells of a chunk (their loads go out together).
__device__ __forceinline__ void dt_cell_scan_body(const DtArgs &a, const VB &vb) {
    constexpr int kCellScanItems = 4;
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const DtSide S = vb.y ? a.s[1] : a.s[0];
    const int ncell = dt_ncell(a);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int chunk = kCellScanItems * (int)blockDim.x;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base <= ncell; base += chunk) {
        const int i0 = base + kCellScanItems * tid;
        int v[kCellScanItems];
#pragma unroll
        for (int k = 0; k < kCellScanItems; ++k) v[k] = i0 + k < ncell ? S.cell_cnt[i0 + k] : 0;
        int tot = 0;
#pragma unroll
        for (int k = 0; k < kCellScanItems; ++k) tot += v[k];
        int incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int x = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            s_w[lane] = x;
        }
        __syncthreads();
        int excl = s_carry + (wid ? s_w[wid - 1] : 0) + incl - tot;
#pragma unroll
        for (int k = 0; k < kCellScanItems; ++k) {
            if (i0 + k <= ncell) {  // entry ncell receives the total
                S.cell_start[i0 + k] = excl;
                S.cell_fill[i0 + k] = excl;
            }
            excl += v[k];
        }
        __syncthreads();
        if (tid == 0) s_carry += s_w[31];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) dt_cell_scan_kernel(DtArgs a) { dt_cell_scan_body(a, vb_single()); }
__global__ void __launch_bounds__(1024) dt_cell_scan_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_cell_scan_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

__device__ __forceinline__ void dt_scatter_body(const DtArgs &a, const VB &vb) {
    const DtSide S = vb.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    for (int i = vb.x * blockDim.x + threadIdx.x; i < n; i += vb.gx * blockDim.x) {
        const int x = S.X[i], y = S.Y[i];
        const int k = atomicAdd(S.cell_fill + dt_cell(a, x, y), 1);
        S.pts[k] = make_int4(x, y, i, 1);
        S.slot[i] = k;
    }
}

__global__ void dt_scatter_kernel(DtArgs a) { dt_scatter_body(a, vb_single()); }
__global__ void dt_scatter_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_scatter_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

// Coincident points (right coordinates only) keep the lowest list index.
__device__ __forceinline__ void dt_dedup_body(const DtArgs &a, const VB &vb) {
    const DtSide S = vb.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    for (int i = vb.x * blockDim.x + threadIdx.x; i < n; i += vb.gx * blockDim.x) {
        const int x = S.X[i], y = S.Y[i];
        const int c = dt_cell(a, x, y);
        bool dup = false;
        for (int k = S.cell_start[c]; k < S.cell_start[c + 1]; ++k) {
            const int4 q = S.pts[k];
            if (q.x == x && q.y == y && q.z < i) dup = true;
        }
        if (dup) {
            S.status[i] = -1;
            S.pts[S.slot[i]].w = 0;
        }
    }
}

__global__ void dt_dedup_kernel(DtArgs a) { dt_dedup_body(a, vb_single()); }
__global__ void dt_dedup_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_dedup_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

// -------------------------------------------------------------------------
// Stars
// -------------------------------------------------------------------------

constexpr int kDtRadius = 24;     // pass-1 search radius (one pair)
constexpr int kDtRadiusBatch = 18;  // pass-1 search radius in batched launches
constexpr int kDtSlots = 32;      // owned triangles kept per point

__device__ __forceinline__ int4 shfl4(const int4 &v, int src_xor) {
    return make_int4(__shfl_xor_sync(0xFFFFFFFFu, v.x, src_xor), __shfl_xor_sync(0xFFFFFFFFu, v.y, src_xor),
                     __shfl_xor_sync(0xFFFFFFFFu, v.z, src_xor), __shfl_xor_sync(0xFFFFFFFFu, v.w, src_xor));
}

__device__ __forceinline__ unsigned long long dt_nn_key(const int4 &p, const int4 &q) {
    const int64_t dx = q.x - p.x, dy = q.y - p.y;
    return ((unsigned long long)(dx * dx + dy * dy) << 32) | (unsigned)q.z;
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, k, o);
        k = other < k ? other : k;
    }
    return k;
}

// Is the circle through p, a, b no wider than R (2r <= R, r its radius)?
// With 4 r^2 = |pa|^2 |pb|^2 |ab|^2 / orient(p, a, b)^2 this is
// |pa|^2 |pb|^2 |ab|^2 <= R^2 orient^2, in exact integer arithmetic.  A point
// farther than R from p makes the diameter exceed R at once, so the products
// only see points within R: below R^4 * 4 R^2 < 2^63 for R <= 1024.
__device__ __forceinline__ bool dt_small_circle(const int4 &p, const int4 &a, const int4 &b, int R) {
    const int64_t R2 = (int64_t)R * R;
    const int64_t pa = (int64_t)(a.x - p.x) * (a.x - p.x) + (int64_t)(a.y - p.y) * (a.y - p.y);
    const int64_t pb = (int64_t)(b.x - p.x) * (b.x - p.x) + (int64_t)(b.y - p.y) * (b.y - p.y);
    if (pa > R2 || pb > R2) return false;
    const int64_t ab = (int64_t)(b.x - a.x) * (b.x - a.x) + (int64_t)(b.y - a.y) * (b.y - a.y);
    const int64_t ar = dt_orient(p.x, p.y, a.x, a.y, b.x, b.y);
    return pa * pb * ab <= R2 * ar * ar;
}

// The same test in 32-bit integers for discs of radius R <= 24: once pa and
// pb are at most R^2, pa * pb * ab <= 4 R^6 < 2^31 and R^2 * ar^2 <= R^6
// (|ar| <= sqrt(pa pb)); coordinate differences below 2^15 keep pa and pb
// themselves within 31 bits.
template <int R>
__device__ __forceinline__ bool dt_small_circle32(const int4 &p, const int4 &a, const int4 &b) {
    static_assert(R <= 24, "4 R^6 must fit in 31 bits");
    const int ax = a.x - p.x, ay = a.y - p.y, bx = b.x - p.x, by = b.y - p.y;
    const int pa = ax * ax + ay * ay, pb = bx * bx + by * by;
    if (pa > R * R || pb > R * R) return false;
    const int dx = bx - ax, dy = by - ay;
    const int ab = dx * dx + dy * dy;
    const int ar = ax * by - ay * bx;
    return pa * pb * ab <= R * R * ar * ar;
}

template <int R>
__device__ __forceinline__ bool dt_small_circle_r(const int4 &p, const int4 &a, const int4 &b) {
    if constexpr (R <= 24)
        return dt_small_circle32<R>(p, a, b);
    else
        return dt_small_circle(p, a, b, R);
}

// Records triangle (p, a, b) if p owns it (lowest index).
__device__ __forceinline__ void dt_record(const DtSide &S, int i, int &written, const int4 &p, const int4 &a,
                                          const int4 &b, bool leader) {
    if (p.z < a.z && p.z < b.z) {
        if (leader && written < kDtSlots) {
            int32_t *slot = S.slots + ((size_t)i * kDtSlots + written) * 2;
            slot[0] = a.z;
            slot[1] = b.z;
        }
        ++written;
    }
}

// The Delaunay third vertex of directed edge (p, e) on side s (+1 left,
// -1 right) is the candidate c with s*orient(p,e,c) > 0 that minimises the
// pencil parameter t(c) = N/D, N = |c-p|^2 - (e-p).(c-p), D = 2 s orient(p,e,c)
// (the circles through p and e are nested on each side in the order of t).
// Equal t means cocircular: the symbolic tie-break decides.  T: arithmetic
// type of the cross-multiplied comparison.
template <typename T>
struct DtKey {
    T N, D;
};

template <typename T>
__device__ __forceinline__ DtKey<T> dt_key(const int4 &p, const int4 &e, const int4 &c, int side) {
    const T ex = e.x - p.x, ey = e.y - p.y, cx = c.x - p.x, cy = c.y - p.y;
    DtKey<T> k;
    k.N = cx * cx + cy * cy - (ex * cx + ey * cy);
    k.D = 2 * side * (ex * cy - ey * cx);
    return k;
}

// Does c2 (key k2) beat c1 (key k1) for edge (p, e) on side s?
template <typename T>
__device__ __forceinline__ bool dt_key_better(const DtKey<T> &k1, const DtKey<T> &k2, const int4 &p, const int4 &e,
                                              const int4 &c1, const int4 &c2, int side) {
    const T l = k2.N * k1.D, r = k1.N * k2.D;
    if (l != r) return l < r;
    const int s = side > 0 ? dt_incircle<int64_t>(p, e, c1, c2) : dt_incircle<int64_t>(p, c1, e, c2);
    return s > 0 || (s == 0 && c2.z < c1.z);
}

// Pass 1: one group of kDtGroup lanes (kDtGroupOne for one pair) per point.
// The group lists the points within R of p (kDtRadius for one pair,
// kDtRadiusBatch in batches; indices into the grid-sorted array, in shared
// memory), then wraps the star: each lane keeps the best candidate of its
// share of the list under the pencil key (32-bit integers are exact: every
// difference is at most R <= 64) and the group reduces with shuffles.  A
// star is accepted when every triangle's circumdisc lies inside the radius
// (4 r^2 <= R^2, exact) and, for an open star (p on the hull), nothing lies
// beyond either open edge (checked against the extreme points of every image
// row).  Other stars are queued for the next pass.
constexpr int kDtGroup = 4;       // lanes per star in batched launches (issue-bound: less divergence waste)
constexpr int kDtGroupOne = 16;   // lanes per star for one pair (latency-bound: shorter star chains)
constexpr int kDtGroupThreads = 256;
constexpr int kDtListCap = 128;  // candidates per point (a radius-24 disc holds at most ~75 lattice points at step 5)
constexpr int kDtRadiusB = 64;   // warp pass (batches): one warp per star left by the middle pass
constexpr int kDtListCapB = 640; // the radius-64 disc holds at most ~520 lattice points

// Group reduction of (best, key) under the pencil order of edge (p, e).
template <int G>
__device__ __forceinline__ int4 dt_group_best(unsigned m, int4 best, DtKey<int> bk, const int4 &p, const int4 &e,
                                              int side) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        int4 ob;
        ob.x = __shfl_xor_sync(m, best.x, o);
        ob.y = __shfl_xor_sync(m, best.y, o);
        ob.z = __shfl_xor_sync(m, best.z, o);
        ob.w = __shfl_xor_sync(m, best.w, o);
        DtKey<int> ok;
        ok.N = __shfl_xor_sync(m, bk.N, o);
        ok.D = __shfl_xor_sync(m, bk.D, o);
        bool take = false;
        if (ob.w) {
            if (!best.w) {
                take = true;
            } else {
                // the same decision on both lanes of the pair: compare in a
                // fixed order (lower index first)
                const bool mine_first = best.z < ob.z;
                const bool second_wins = mine_first ? dt_key_better<int>(bk, ok, p, e, best, ob, side)
                                                    : dt_key_better<int>(ok, bk, p, e, ob, best, side);
                take = mine_first ? second_wins : !second_wins;
            }
        }
        if (take) {
            best = ob;
            bk = ok;
        }
    }
    return best;
}

// Star queues of a side: 1 = (pending, npending), 2 = (pending2,
// npending2), 3 = (pending, npending3) (batches: the third pass's output,
// written after the second pass has read `pending`).
__device__ __forceinline__ const int32_t *dt_queue(const DtSide &S, int q) { return q == 2 ? S.pending2 : S.pending; }
__device__ __forceinline__ int32_t *dt_queue_len(const DtSide &S, int q) {
    return q == 2 ? S.npending2 : (q == 3 ? S.npending3 : S.npending);
}

// G lanes per star, candidates within R (list capacity CAP).  QIN: 0 =
// every point, else the stars of that queue; failures go to queue QOUT.
template <int G, int R, int CAP, int QIN, int QOUT>
__device__ __forceinline__ void dt_group_pass_body(const DtArgs &a, const VB &vb) {
    constexpr bool QUEUE = QIN != 0;
    static_assert(2 * R / kDtCell + 2 <= G, "the group's lanes fetch the cell rows of the disc");
    static_assert(R <= 64, "32-bit pencil keys are exact for coordinates within 64 of p");
    __shared__ int s_list[kDtGroupThreads / G][CAP];
    const DtSide S = vb.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), gbase = lane & ~(G - 1);
    const unsigned gm = G == 32 ? 0xFFFFFFFFu : ((1u << (G & 31)) - 1u) << gbase;
    int *list = s_list[threadIdx.x / G];
    const int groups = vb.gx * (kDtGroupThreads / G);
    const int njobs = QUEUE ? *dt_queue_len(S, QIN) : n;
    const int32_t *qin = dt_queue(S, QIN);
    for (int j = vb.x * (kDtGroupThreads / G) + threadIdx.x / G; j < njobs; j += groups) {
        const int4 p = QUEUE ? S.pts[S.slot[qin[j]]] : S.pts[j];
        if (!p.w || (!QUEUE && S.status[p.z] != 0)) continue;
        // candidates: lanes fetch the cell rows' ranges, then stride over them
        const int cx0 = max(0, p.x - R) / kDtCell, cx1 = min(a.gw - 1, max(0, p.x + R) / kDtCell);
        const int cy0 = max(0, p.y - R) / kDtCell, cy1 = min(a.gh - 1, max(0, p.y + R) / kDtCell);
        const int nrows = cy1 - cy0 + 1;  // at most 2R/16 + 2
        int rs = 0, re = 0;
        if (gl < nrows) {
            rs = S.cell_start[(cy0 + gl) * a.gw + cx0];
            re = S.cell_start[(cy0 + gl) * a.gw + cx1 + 1];
        }
        int k = 0;
        unsigned long long key = ~0ull;
        int nn = -1;
        for (int r = 0; r < nrows; ++r) {
            const int s0 = __shfl_sync(gm, rs, gbase + r), e0 = __shfl_sync(gm, re, gbase + r);
            for (int c = s0; c < e0; c += G) {
                bool take = false;
                if (c + gl < e0) {
                    const int4 q = S.pts[c + gl];
                    const int dx = q.x - p.x, dy = q.y - p.y, d2 = dx * dx + dy * dy;
                    take = q.w && q.z != p.z && d2 <= R * R;
                    if (take) {
                        const unsigned long long kk = ((unsigned long long)d2 << 32) | (unsigned)q.z;
                        if (kk < key) {
                            key = kk;
                            nn = c + gl;
                        }
                    }
                }
                const unsigned b = __ballot_sync(gm, take) >> gbase;
                const int pos = k + __popc(b & ((1u << gl) - 1u));
                if (take && pos < CAP) list[pos] = c + gl;
                k += __popc(b);
            }
        }
        __syncwarp(gm);
        bool certified = k > 0 && k <= CAP;
        int written = 0;
        bool open_l = false, open_r = false;
        int4 e_l = p, e_r = p;
        if (certified) {
            // nearest neighbour of the group
            unsigned long long kmin = key;
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(gm, kmin, o);
                kmin = other < kmin ? other : kmin;
            }
            const int src = __ffs(__ballot_sync(gm, key == kmin) >> gbase) - 1;
            const int first_slot = __shfl_sync(gm, nn, gbase + src);
            const int4 first = S.pts[first_slot];
            int4 cur = first;
            bool closed = false;
            for (int step = 0; step <= k && certified; ++step) {  // counter-clockwise
                int4 best = make_int4(0, 0, 0, 0);
                DtKey<int> bk{0, 1};
                for (int c = gl; c < k; c += G) {
                    const int4 q = S.pts[list[c]];
                    if (q.z == cur.z) continue;
                    const DtKey<int> qk = dt_key<int>(p, cur, q, +1);
                    if (qk.D <= 0) continue;
                    if (!best.w || dt_key_better<int>(bk, qk, p, cur, best, q, +1)) {
                        best = q;
                        bk = qk;
                    }
                }
                best = dt_group_best<G>(gm, best, bk, p, cur, +1);
                if (!best.w) {
                    open_l = true;
                    e_l = cur;
                    break;
                }
                if (!dt_small_circle_r<R>(p, cur, best)) {
                    certified = false;
                    break;
                }
                dt_record(S, p.z, written, p, cur, best, gl == 0);
                if (best.z == first.z) {
                    closed = true;
                    break;
                }
                cur = best;
            }
            if (certified && !closed) {
                if (!open_l) certified = false;  // ran out of steps
                cur = first;
                for (int step = 0; step <= k && certified; ++step) {  // clockwise
                    int4 best = make_int4(0, 0, 0, 0);
                    DtKey<int> bk{0, 1};
                    for (int c = gl; c < k; c += G) {
                        const int4 q = S.pts[list[c]];
                        if (q.z == cur.z) continue;
                        const DtKey<int> qk = dt_key<int>(p, cur, q, -1);
                        if (qk.D <= 0) continue;
                        if (!best.w || dt_key_better<int>(bk, qk, p, cur, best, q, -1)) {
                            best = q;
                            bk = qk;
                        }
                    }
                    best = dt_group_best<G>(gm, best, bk, p, cur, -1);
                    if (!best.w) {
                        open_r = true;
                        e_r = cur;
                        break;
                    }
                    if (!dt_small_circle_r<R>(p, best, cur)) {
                        certified = false;
                        break;
                    }
                    dt_record(S, p.z, written, p, best, cur, gl == 0);
                    cur = best;
                }
                if (!open_r) certified = false;
            }
            // open edges (p on the hull): nothing may lie beyond them
            for (int side = 0; side < 2 && certified; ++side) {
                const bool open = side ? open_r : open_l;
                if (!open) continue;
                const int4 e = side ? e_r : e_l;
                bool bad = false;
                for (int y = gl; y < a.h && !bad; y += G) {
                    const int x0 = S.rowmin[y], x1 = S.rowmax[y];
                    if (x0 > x1) continue;
                    const int64_t o0 = dt_orient(p.x, p.y, e.x, e.y, x0, y);
                    const int64_t o1 = dt_orient(p.x, p.y, e.x, e.y, x1, y);
                    bad = side ? (o0 < 0 || o1 < 0) : (o0 > 0 || o1 > 0);
                }
                if (__ballot_sync(gm, bad) & gm) certified = false;
            }
        }
        if (gl == 0) {
            if (certified) {
                S.status[p.z] = 1;
                S.owned[p.z] = written;
                if (written > kDtSlots) atomicOr(S.err, 4);
            } else {
                const_cast<int32_t *>(dt_queue(S, QOUT))[atomicAdd(dt_queue_len(S, QOUT), 1)] = p.z;
            }
        }
        __syncwarp(gm);
    }
}


template <int G, int R> __device__ __forceinline__ void dt_pass1_body(const DtArgs &a, const VB &vb) {
    dt_group_pass_body<G, R, kDtListCap, 0, 1>(a, vb);
}

// Batches: the stars left by the first pass go through a middle pass (eight
// lanes, the 32-pixel disc) and those left again through the warp pass
// (the 64-pixel disc); the CTA pass takes the third queue.
constexpr int kDtRadiusM = 32;
constexpr int kDtListCapM = 192;  // the radius-32 disc holds at most ~130 lattice points
constexpr int kDtGroupM = 8;

__global__ void __launch_bounds__(kDtGroupThreads, 4) dt_pass1m_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_group_pass_body<kDtGroupM, kDtRadiusM, kDtListCapM, 1, 2>(slot_entry(tab, vm.stride, vb.slot), vb);
}
__global__ void __launch_bounds__(kDtGroupThreads, 3) dt_pass1b_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_group_pass_body<32, kDtRadiusB, kDtListCapB, 2, 3>(slot_entry(tab, vm.stride, vb.slot), vb);
}

__global__ void __launch_bounds__(kDtGroupThreads, 4) dt_pass1_kernel(DtArgs a) {
    dt_pass1_body<kDtGroupOne, kDtRadius>(a, vb_single());
}
// A batch of one pair takes the one-pair group pass (wider groups, larger disc).
__global__ void __launch_bounds__(kDtGroupThreads, 4) dt_pass1_kernel_b1(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_pass1_body<kDtGroupOne, kDtRadius>(slot_entry(tab, vm.stride, vb.slot), vb);
}
__global__ void __launch_bounds__(kDtGroupThreads, 4) dt_pass1_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_pass1_body<kDtGroup, kDtRadiusBatch>(slot_entry(tab, vm.stride, vb.slot), vb);
}

// CTA pass: one CTA per star left by the group passes.  The points within
// kDtRadius1 are cached in shared memory; every wrap step first takes the
// best cached candidate and keeps it when its circumdisc lies inside the
// cached disc (then no other point can beat it); the first step that does
// not fit refills the cache with the points within kDtRadius2, and a step
// that fits neither (large circle, no cached candidate on that side, or the
// cache overflowed) scans the grid cells its disc or half-plane meets, which
// is exact.  So every queued star comes out exact.
constexpr int kDtRadius1 = 96;     // first cache radius of the CTA pass
constexpr int kDtRadius2 = 192;    // its second, when a step's circle does not fit the first
constexpr int kDtCandCap2 = 3072;  // candidates cached per CTA (48 KB)
constexpr int kDtMaxRows = 64;     // cell rows a radius-192 disc spans, with margin
constexpr int kDtBlockThreads = 256;  // threads of a CTA-pass CTA (one pair: its longest star sets the pass)
constexpr int kDtBlocksPerSM = 3;     // CTA-pass CTAs resident per SM (85 registers a thread)
// batches of two or more pairs: smaller CTAs, one more per SM (more stars at
// once across the pairs; a step's selection takes a little longer)
constexpr int kDtBlockThreadsB = 192;
constexpr int kDtBlocksPerSMB = 4;
static_assert(2 * kDtRadius2 / kDtCell + 2 <= kDtMaxRows, "the CTA pass's disc must fit the row table");

// CTA reduction of the threads' (best, key) under the pencil order: each
// warp reduces with shuffles, warp 0 reduces the warps' results, and every
// thread reads the winner from shared memory.
template <int UNUSED = 0>
__device__ __forceinline__ int4 dt_warp_key_best(int4 best, DtKey<int64_t> &bk, const int4 &p, const int4 &e,
                                                 int side) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int4 ob = shfl4(best, o);
        DtKey<int64_t> ok;
        ok.N = __shfl_xor_sync(0xFFFFFFFFu, bk.N, o);
        ok.D = __shfl_xor_sync(0xFFFFFFFFu, bk.D, o);
        if (ob.w && (!best.w || dt_key_better<int64_t>(bk, ok, p, e, best, ob, side))) {
            best = ob;
            bk = ok;
        }
    }
    return best;
}

__device__ __forceinline__ int4 dt_block_best(int4 best, DtKey<int64_t> bk, const int4 &p, const int4 &e, int side,
                                              int4 *s_red, int64_t *s_n, int64_t *s_d) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    best = dt_warp_key_best(best, bk, p, e, side);
    __syncthreads();
    if (lane == 0) {
        s_red[warp] = best;
        s_n[warp] = bk.N;
        s_d[warp] = bk.D;
    }
    __syncthreads();
    if (warp == 0) {
        int4 b = lane < nw ? s_red[lane] : make_int4(0, 0, 0, 0);
        DtKey<int64_t> k{lane < nw ? s_n[lane] : 0, lane < nw ? s_d[lane] : 1};
        b = dt_warp_key_best(b, k, p, e, side);
        if (lane == 0) s_red[32] = b;
    }
    __syncthreads();
    return s_red[32];
}

struct DtBlockShared {
    int4 red[33];
    int64_t rn[32], rd[32];
    unsigned long long key[32];
    int rs[kDtMaxRows], rlen[kDtMaxRows + 1], cnt;
    unsigned fmin[3];  // least float key of a selection (three buffers, used in turn)
    int nband[3];      // band members listed by a selection
    int4 win;          // winner of an exactly ordered band
    int small;         // the first band member's circle fits the disc of radius R (selections with R > 0)
};

// Float filter of the pencil order (CTA pass).  With coordinates below 2^14
// the key (N, D) of every candidate fits in 32 bits (|N|, |D| < 2^31) and
// two keys compare exactly through 64-bit products.  The float
// f = fl(N) / fl(D) (two conversions rounded to nearest, one division within
// 2 ulp) is within 2^-21 |t| of t = N / D, so the exact winner w (least t)
// has f_w - f_min <= 2^-21 (|f_w| + |f_min|) + rounding, f_min the least f
// over the candidates: every candidate that can win lies in the band
// f - f_min <= 2^-17 (|f| + |f_min|).  A band of one is the winner; a larger
// band (cocircular candidates, or nearly) is ordered exactly.
constexpr int kDtBandCap = 32;

__device__ __forceinline__ unsigned dt_fbits(float f) {  // monotone in f (no NaN)
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float dt_fbits_value(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
__device__ __forceinline__ float dt_fkey(const DtKey<int> &k) { return __fdividef((float)k.N, (float)k.D); }
__device__ __forceinline__ bool dt_in_band(float f, float fmin) {
    return f - fmin <= 0x1p-17f * (fabsf(f) + fabsf(fmin));
}

// Does c2 (key k2) beat c1 (key k1)?  32-bit keys, 64-bit products.
__device__ __forceinline__ bool dt_key_better_w(const DtKey<int> &k1, const DtKey<int> &k2, const int4 &p,
                                                const int4 &e, const int4 &c1, const int4 &c2, int side) {
    const int64_t l = (int64_t)k2.N * k1.D, r = (int64_t)k1.N * k2.D;
    if (l != r) return l < r;
    const int s = side > 0 ? dt_incircle<int64_t>(p, e, c1, c2) : dt_incircle<int64_t>(p, c1, e, c2);
    return s > 0 || (s == 0 && c2.z < c1.z);
}

// CTA-wide Delaunay third vertex of edge (p, e) on `side`: each thread
// offers its candidates through each(visit) (called twice), thread 0 also
// the seed (w = 0: none).  Pass 1 finds the least float key (one warp
// reduction and a shared atomic), pass 2 has every thread take the exact
// best of its candidates in the band (its least one, unless its second
// least is in the band too) and list it; a single listed candidate
// is the winner, else warp 0 orders the list exactly (the whole CTA when it
// overflows).  par: the caller's turn counter (the same on every thread).
// With R > 0, small tells whether the winner's circumdisc lies inside the
// disc of radius R about p (dt_small_circle): the thread that lists the
// first band member tests it before the second barrier, which is the answer
// when the band has one member, so the other threads skip the 64-bit test.
// Thread 0 resets the next call's buffers before this call's first barrier:
// their last readers (two calls back) have passed the previous call's first
// barrier, and the next call writes them only after this call's.
template <typename Each>
__device__ int4 dt_block_select(Each each, const int4 &p, const int4 &e, int side, const int4 &seed,
                                DtBlockShared &sh, int &par, int R, bool &small) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int b = par, nxt = par == 2 ? 0 : par + 1;
    par = nxt;
    small = false;
    if (tid == 0) {
        sh.fmin[nxt] = 0xFFFFFFFFu;
        sh.nband[nxt] = 0;
    }
    auto usable = [&](const int4 &q) { return q.w && q.z != e.z && q.z != p.z; };
    // each thread keeps its least float key (with its candidate) and its
    // second least
    const float inf = __int_as_float(0x7F800000);
    float fl = inf, f2 = inf;
    int4 q1 = make_int4(0, 0, 0, 0);
    auto offer = [&](const int4 &q) {
        if (!usable(q)) return;
        const DtKey<int> k = dt_key<int>(p, e, q, side);
        if (k.D <= 0) return;
        const float f = dt_fkey(k);
        if (f < fl) {
            f2 = fl;
            fl = f;
            q1 = q;
        } else if (f < f2) {
            f2 = f;
        }
    };
    each(offer);
    if (tid == 0) offer(seed);
    const unsigned kb = __reduce_min_sync(0xFFFFFFFFu, fl == __int_as_float(0x7F800000) ? 0xFFFFFFFFu : dt_fbits(fl));
    if (lane == 0 && kb != 0xFFFFFFFFu) atomicMin(&sh.fmin[b], kb);
    __syncthreads();
    const unsigned kmin = sh.fmin[b];
    if (kmin == 0xFFFFFFFFu) return make_int4(0, 0, 0, 0);  // uniform: no candidate on this side
    const float fmin = dt_fbits_value(kmin);
    int4 best = make_int4(0, 0, 0, 0);
    DtKey<int> bk{0, 1};
    // the band test is increasing in f: with the second least key outside
    // the band only the least can be in it; else the thread offers again
    if (q1.w && dt_in_band(fl, fmin)) {
        if (f2 != inf && dt_in_band(f2, fmin)) {
            auto visit = [&](const int4 &q) {
                if (!usable(q)) return;
                const DtKey<int> k = dt_key<int>(p, e, q, side);
                if (k.D <= 0 || !dt_in_band(dt_fkey(k), fmin)) return;
                if (!best.w || dt_key_better_w(bk, k, p, e, best, q, side)) {
                    best = q;
                    bk = k;
                }
            };
            each(visit);
            if (tid == 0) visit(seed);
        } else {
            best = q1;
            bk = dt_key<int>(p, e, q1, side);
        }
    }
    auto fits = [&](const int4 &c) {
        return c.w && (side > 0 ? dt_small_circle(p, e, c, R) : dt_small_circle(p, c, e, R));
    };
    if (best.w) {
        const int pos = atomicAdd(&sh.nband[b], 1);
        if (pos < kDtBandCap) {
            sh.red[pos] = best;
            sh.rn[pos] = bk.N;
            sh.rd[pos] = bk.D;
            if (pos == 0 && R > 0) sh.small = fits(best);
        }
    }
    __syncthreads();
    const int nb = sh.nband[b];
    if (nb == 1) {
        small = R > 0 && sh.small;
        return sh.red[0];
    }
    int4 w;
    if (nb > kDtBandCap) {
        w = dt_block_best(best, DtKey<int64_t>{bk.N, bk.D}, p, e, side, sh.red, sh.rn, sh.rd);
    } else {
        if (tid < 32) {
            int4 c = lane < nb ? sh.red[lane] : make_int4(0, 0, 0, 0);
            DtKey<int64_t> k{lane < nb ? sh.rn[lane] : 0, lane < nb ? sh.rd[lane] : 1};
            c = dt_warp_key_best(c, k, p, e, side);
            if (lane == 0) sh.win = c;
        }
        __syncthreads();
        w = sh.win;
    }
    small = R > 0 && fits(w);
    return w;
}

// Best third vertex for edge (p, cur) on `side`, over the cache (cand, k) or,
// with cand == NULL, over every alive point.
__device__ __forceinline__ int4 dt_block_step(const DtSide &S, const int4 &p, const int4 &cur, int side,
                                              const int4 *cand, int k, int n, DtBlockShared &sh, int &par, int R,
                                              bool &small) {
    const int tid = threadIdx.x, nth = blockDim.x;
    const int4 none = make_int4(0, 0, 0, 0);
    if (cand)
        return dt_block_select(
            [&](auto &&v) {
                for (int j = tid; j < k; j += nth) v(cand[j]);
            },
            p, cur, side, none, sh, par, R, small);
    return dt_block_select(
        [&](auto &&v) {
            for (int j = tid; j < n; j += nth) v(S.pts[j]);
        },
        p, cur, side, none, sh, par, R, small);
}

// Exact step for edge (p, cur) on `side` without the radius limit.  Only
// points strictly inside the closed circumdisc of (p, cur, bc) can beat the
// cached best bc, and with no cached candidate only the open half-plane on
// that side matters; so the CTA scans the grid cells that meet that region,
// taking each cell row's cells as one contiguous range.  The region is
// widened so that float rounding cannot lose a cell: the circle's centre
// comes from exact integer numerators (one rounding each in the division),
// its radius is padded by 4 pixels plus 1e-4 of itself, each cell row band
// by 2 pixels and each x-range by a cell; a circle wider than 1e6 pixels is
// replaced by its half-plane (the part of the disc beyond the chord p-cur
// is then thinner than a pixel, and only that side's points are candidates).
__device__ int4 dt_block_region_step(const DtArgs &a, const DtSide &S, const int4 &p, const int4 &cur, int side,
                                     const int4 &bc, DtBlockShared &sh, int *r_start, int *r_len, int &par) {
    const int tid = threadIdx.x, nth = blockDim.x;
    float ccx = 0.0f, ccy = 0.0f, rad = 0.0f;
    bool disc = false;
    if (bc.w) {
        const int64_t ax = cur.x - p.x, ay = cur.y - p.y, bx = bc.x - p.x, by = bc.y - p.y;
        const int64_t d = 2 * (ax * by - ay * bx);  // nonzero: bc lies strictly on `side`
        const int64_t a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
        const float fd = (float)d;
        const float ux = (float)(by * a2 - ay * b2) / fd, uy = (float)(ax * b2 - bx * a2) / fd;
        const float r = sqrtf(ux * ux + uy * uy);
        if (r <= 1e6f) {
            disc = true;
            ccx = (float)p.x + ux;
            ccy = (float)p.y + uy;
            rad = r * 1.0001f + 4.0f;
        }
    }
    // half-plane: side * ((cur.x-p.x)(y-p.y) - (cur.y-p.y)(x-p.x)) > 0
    const int ex = cur.x - p.x, ey = cur.y - p.y;
    for (int cy = tid; cy < a.gh; cy += nth) {
        const int y0 = cy * kDtCell - 2, y1 = cy * kDtCell + kDtCell + 1;
        float xlo = -1e30f, xhi = 1e30f;
        bool any = true;
        if (disc) {
            const float dy = ccy < (float)y0 ? (float)y0 - ccy : (ccy > (float)y1 ? ccy - (float)y1 : 0.0f);
            if (dy > rad) {
                any = false;
            } else {
                const float hc = sqrtf(rad * rad - dy * dy) + 2.0f;
                xlo = ccx - hc;
                xhi = ccx + hc;
            }
        } else if (ey != 0) {
            // boundary x at the band's two edges (exact products, one rounding
            // in each division); the admissible side of x
            const float xa = (float)p.x + (float)(ex * (y0 - p.y)) / (float)ey;
            const float xb = (float)p.x + (float)(ex * (y1 - p.y)) / (float)ey;
            const float xm = fminf(xa, xb), xM = fmaxf(xa, xb);
            // side*(ex*(y-py) - ey*(x-px)) > 0  <=>  x < boundary if side*ey > 0
            if (side * ey > 0)
                xhi = xM + 2.0f;
            else
                xlo = xm - 2.0f;
        } else {
            // horizontal edge: the whole row is in or out
            any = side * ex * (y0 + y1 - 2 * p.y) > 0 || (y0 <= p.y && p.y <= y1);
        }
        int c0 = 0, c1 = a.gw - 1;
        if (any) {
            c0 = xlo < 0.0f ? 0 : (int)fminf((float)(a.gw - 1), floorf(xlo / kDtCell) - 1.0f);
            c1 = xhi >= 1e29f ? a.gw - 1 : (int)fmaxf(0.0f, fminf((float)(a.gw - 1), floorf(xhi / kDtCell) + 1.0f));
            c0 = max(0, c0);
        }
        const int s0 = any && c0 <= c1 ? S.cell_start[cy * a.gw + c0] : 0;
        const int e0 = any && c0 <= c1 ? S.cell_start[cy * a.gw + c1 + 1] : 0;
        r_start[cy] = s0;
        r_len[cy] = e0 - s0;  // the row's range length
    }
    __syncthreads();
    // each warp takes cell rows in turn; its lanes stride over the row's
    // contiguous range of the grid-sorted points
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    bool unused;
    return dt_block_select(
        [&](auto &&v) {
            for (int cy = warp; cy < a.gh; cy += nwarps) {
                const int s0 = r_start[cy], len = r_len[cy];
                int j = lane;
                for (; j + 96 < len; j += 128) {  // four loads in flight
                    const int4 q0 = S.pts[s0 + j], q1 = S.pts[s0 + j + 32], q2 = S.pts[s0 + j + 64],
                               q3 = S.pts[s0 + j + 96];
                    v(q0);
                    v(q1);
                    v(q2);
                    v(q3);
                }
                for (; j < len; j += 32) v(S.pts[s0 + j]);
            }
        },
        p, cur, side, bc, sh, par, 0, unused);
}

__device__ int dt_block_gather(const DtArgs &a, const DtSide &S, const int4 &p, int R, int4 *cand,
                               DtBlockShared &sh);

// Exact star of p, CTA-wide.  cand: shared cache (capacity kDtCandCap2)
// holding the k points within R of p (k > kDtCandCap2: unusable), or NULL.
// A step is taken from the cache when the winner's circle lies inside the
// disc of radius R (2r <= R: no point outside the cache can be inside it);
// otherwise the cache is refilled once at kDtRadius2 and, if that still does
// not hold the circle, the step scans the cells its disc or half-plane meets
// (every point without the region tables).  Writes the owned triangles to the
// slots or, with out != NULL, to out.  Returns 1, or -1 if it exceeded
// kDtMaxStar.
__device__ int dt_block_star(const DtArgs &a, const DtSide &S, int i, const int4 &p, int n, int4 *cand, int R, int k,
                             int *written, int32_t *out, DtBlockShared &sh, int *r_start, int *r_len) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nth = blockDim.x;
    int par = 0;  // selection buffers: cleared here, before the barriers below
    if (tid == 0) {
        sh.fmin[0] = sh.fmin[1] = sh.fmin[2] = 0xFFFFFFFFu;
        sh.nband[0] = sh.nband[1] = sh.nband[2] = 0;
    }
    // nearest neighbour: a cached point is nearer than every point outside
    // the cache, so a non-empty cache holds it; else one pass over all points
    unsigned long long key = ~0ull;
    const bool nn_cached = cand && k > 0 && k <= kDtCandCap2;
    const int nn_n = nn_cached ? k : n;
    for (int j = tid; j < nn_n; j += nth) {
        const int4 q = nn_cached ? cand[j] : S.pts[j];
        if (q.w && q.z != p.z) {
            const unsigned long long kk = dt_nn_key(p, q);
            key = kk < key ? kk : key;
        }
    }
    key = warp_min64(key);
    __syncthreads();
    if (lane == 0) sh.key[warp] = key;
    __syncthreads();
    key = lane < (nth >> 5) ? sh.key[lane] : ~0ull;
    key = warp_min64(key);
    *written = 0;
    if (key == ~0ull) return 1;  // p is the only point
    const int4 first = S.pts[S.slot[(int)(unsigned)(key & 0xFFFFFFFFu)]];
    int wr = 0;
    auto emit = [&](const int4 &u, const int4 &v) {  // triangle (p, u, v), ccw
        if (p.z < u.z && p.z < v.z) {
            if (tid == 0) {
                if (out) {
                    out[3 * wr] = p.z;
                    out[3 * wr + 1] = u.z;
                    out[3 * wr + 2] = v.z;
                } else if (wr < kDtSlots) {
                    int32_t *slot = S.slots + ((size_t)i * kDtSlots + wr) * 2;
                    slot[0] = u.z;
                    slot[1] = v.z;
                }
            }
            ++wr;
        }
    };
    auto next = [&](const int4 &cur, int side) {
        int4 b = make_int4(0, 0, 0, 0);
        for (;;) {
            if (!cand || k > kDtCandCap2) break;
            bool small;
            b = dt_block_step(S, p, cur, side, cand, k, n, sh, par, R, small);
            if (small) return b;
            if (R >= kDtRadius2) break;
            R = kDtRadius2;  // refill the cache once with the larger disc
            k = dt_block_gather(a, S, p, R, cand, sh);
        }
        if (r_start) return dt_block_region_step(a, S, p, cur, side, b, sh, r_start, r_len, par);
        bool unused;
        return dt_block_step(S, p, cur, side, nullptr, 0, n, sh, par, 0, unused);
    };
    int4 cur = first;
    bool closed = false;
    int step = 0;
    for (; step < kDtMaxStar; ++step) {  // counter-clockwise
        const int4 best = next(cur, +1);
        if (!best.w) break;  // hull edge
        emit(cur, best);
        if (best.z == first.z) {
            closed = true;
            break;
        }
        cur = best;
    }
    if (step >= kDtMaxStar) return -1;
    if (!closed) {  // clockwise from the first edge
        cur = first;
        for (step = 0; step < kDtMaxStar; ++step) {
            const int4 best = next(cur, -1);
            if (!best.w) break;
            emit(best, cur);
            cur = best;
        }
        if (step >= kDtMaxStar) return -1;
    }
    *written = wr;
    return 1;
}

// Gathers the points within R of p into the shared cache; returns their
// number (more than kDtCandCap2 means the cache overflowed).  The cell rows'
// ranges are fetched at once, the candidates read as one flat index space,
// and each warp places its hits with one atomic.
__device__ int dt_block_gather(const DtArgs &a, const DtSide &S, const int4 &p, int R, int4 *cand,
                               DtBlockShared &sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int cx0 = max(0, p.x - R) / kDtCell, cx1 = min(a.gw - 1, max(0, p.x + R) / kDtCell);
    const int cy0 = max(0, p.y - R) / kDtCell, cy1 = min(a.gh - 1, max(0, p.y + R) / kDtCell);
    const int nrows = min(kDtMaxRows, cy1 - cy0 + 1);
    __syncthreads();
    if (tid < nrows) {
        const int r0 = S.cell_start[(cy0 + tid) * a.gw + cx0], r1 = S.cell_start[(cy0 + tid) * a.gw + cx1 + 1];
        sh.rs[tid] = r0;
        sh.rlen[tid] = r1 - r0;
    }
    if (tid == 0) sh.cnt = 0;
    __syncthreads();
    // each warp takes cell rows in turn; its lanes stride over the row's
    // contiguous range and the warp places its hits with one atomic
    const int64_t R2 = (int64_t)R * R;
    for (int r = warp; r < nrows; r += nwarps) {
        const int s0 = sh.rs[r], len = sh.rlen[r];
        for (int j0 = 0; j0 < len; j0 += 32) {
            const int j = j0 + lane;
            bool take = false;
            int4 q = make_int4(0, 0, 0, 0);
            if (j < len) {
                q = S.pts[s0 + j];
                const int64_t dx = q.x - p.x, dy = q.y - p.y;
                take = q.w && q.z != p.z && dx * dx + dy * dy <= R2;
            }
            const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&sh.cnt, __popc(m));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            const int pos = base + __popc(m & ((1u << lane) - 1u));
            if (take && pos < kDtCandCap2) cand[pos] = q;
        }
    }
    __syncthreads();
    return sh.cnt;
}

// One queued star rebuilt by the whole CTA (exact): cached steps among the
// points within kDtRadius1 (then kDtRadius2), region scans otherwise.
__device__ __forceinline__ void dt_block_item(const DtArgs &a, const DtSide &S, int i, int n, int4 *s_cand,
                                              DtBlockShared &sh, int *r_start, int *r_len) {
    const int4 p = S.pts[S.slot[i]];
    const int k = dt_block_gather(a, S, p, kDtRadius1, s_cand, sh);
    int written = 0;
    const int r = dt_block_star(a, S, i, p, n, s_cand, kDtRadius1, k, &written, nullptr, sh, r_start, r_len);
    if (threadIdx.x == 0) {
        if (r == 1) {
            S.status[i] = 2;
            S.owned[i] = written;
            if (written > kDtSlots) atomicOr(S.err, 4);
        } else {
            atomicOr(S.err, 1);
        }
    }
    __syncthreads();
}

// One pair, persistent (every CTA resident): the CTAs take the stars of
// both sides' queues from one atomic counter, the two queues interleaved so
// that both sides' stars start in the first wave (the pass lasts as long as
// its longest star, so none should wait behind the other side's).  The
// counter is side 0's npending2, which dt_init_kernel zeroes and the one-pair
// passes leave unused.
__global__ void __launch_bounds__(kDtBlockThreads, kDtBlocksPerSM) dt_pass_block_kernel(DtArgs a, int nsides) {
    extern __shared__ int4 s_cand[];  // [kDtCandCap2], then the region rows
    __shared__ DtBlockShared sh;
    __shared__ int s_item;
    int *r_start = reinterpret_cast<int *>(s_cand + kDtCandCap2);
    int *r_len = r_start + a.gh;
    const int n = min(max(*a.count, 0), a.cap);
    const int nq0 = *a.s[0].npending, nq1 = nsides > 1 ? *a.s[1].npending : 0;
    const int m = min(nq0, nq1), total = nq0 + nq1;
    int32_t *counter = a.s[0].npending2;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= total) break;
        const bool two = item < 2 * m;
        const int side = two ? (item & 1) : (nq0 > nq1 ? 0 : 1);
        const int idx = two ? (item >> 1) : item - m;
        const DtSide S = side ? a.s[1] : a.s[0];
        dt_block_item(a, S, S.pending[idx], n, s_cand, sh, r_start, r_len);
    }
}

// Many pairs, persistent: the queues of every (pair, side) of the launch are
// concatenated in launch order and the CTAs take their entries one at a
// time from one atomic counter (zeroed by dt_init_kernel_b), so the long
// stars of one pair overlap the work of all the others.  queue_id 1: the
// warp pass's queues; 0: the group pass's (a batch of one pair, which skips
// the middle and warp passes).
template <int THREADS, int PER_SM>
__global__ void __launch_bounds__(THREADS, PER_SM)
    dt_pass_block_kernel_b(const DtArgs *__restrict__ tab, VMap vm, int nsides, int32_t *counter, int queue_id) {
    extern __shared__ int4 s_cand[];
    __shared__ DtBlockShared sh;
    __shared__ int s_pre[2 * kMaxBatch + 1];
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nq_all = vm.n * nsides;
    // exclusive prefix of the queue lengths (warp 0; nq_all <= 2 * kMaxBatch)
    if (tid < 32) {
        constexpr int kPer = (2 * kMaxBatch + 31) / 32;
        int v[kPer], sum = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int q = lane * kPer + j;
            v[j] = 0;
            if (q < nq_all) {
                const DtSide &Q = slot_entry(tab, vm.stride, vm.slot[q / nsides]).s[q % nsides];
                v[j] = max(0, *dt_queue_len(Q, queue_id ? 3 : 1));
            }
            sum += v[j];
        }
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        int run = incl - sum;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int q = lane * kPer + j;
            if (q <= nq_all) s_pre[q] = run;
            run += v[j];
        }
        if (lane == 31 && nq_all == 32 * kPer) s_pre[nq_all] = incl;
    }
    __syncthreads();
    const int total = s_pre[nq_all];
    int *r_start = reinterpret_cast<int *>(s_cand + kDtCandCap2);
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= total) break;
        // last queue whose start is <= item
        int lo = 0, hi = nq_all - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pre[mid] <= item)
                lo = mid;
            else
                hi = mid - 1;
        }
        const DtArgs &a = slot_entry(tab, vm.stride, vm.slot[lo / nsides]);
        const DtSide &S = a.s[lo % nsides];
        const int n = min(max(*a.count, 0), a.cap);
        dt_block_item(a, S, dt_queue(S, queue_id ? 3 : 1)[item - s_pre[lo]], n, s_cand, sh, r_start,
                      r_start + a.gh);
    }
}

// One CTA per side: exclusive scan of the owned counts, total = ntri.
__device__ __forceinline__ void dt_tri_scan_body(const DtArgs &a, const VB &vb) {
    // each thread scans kScanItems consecutive counts of a chunk (their loads
    // go out together), then the threads' totals are scanned across the CTA
    constexpr int kScanItems = 8;
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const DtSide S = vb.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int chunk = kScanItems * (int)blockDim.x;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += chunk) {
        const int i0 = base + kScanItems * tid;
        int v[kScanItems];
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = i0 + k < n ? S.owned[i0 + k] : 0;
        int tot = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) tot += v[k];
        int incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int x = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            s_w[lane] = x;
        }
        __syncthreads();
        int run = s_carry + (wid ? s_w[wid - 1] : 0) + incl - tot;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (i0 + k < n) S.offset[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 0) s_carry += s_w[31];
        __syncthreads();
    }
    if (tid == 0) {
        if (s_carry > a.cap_tri) atomicOr(S.err, 2);
        *S.ntri = (*S.err & 3) ? -1 : s_carry;  // -1: the triangulation failed
    }
}

__global__ void __launch_bounds__(1024) dt_tri_scan_kernel(DtArgs a) { dt_tri_scan_body(a, vb_single()); }
__global__ void __launch_bounds__(1024) dt_tri_scan_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_tri_scan_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

// One thread per point: copy the owned triangles to their offset.
__device__ __forceinline__ void dt_emit_body(const DtArgs &a, const VB &vb) {
    const DtSide S = vb.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    if (*S.ntri < 0) return;
    for (int i = vb.x * blockDim.x + threadIdx.x; i < n; i += vb.gx * blockDim.x) {
        const int m = min(S.owned[i], kDtSlots);
        int32_t *out = S.tri + 3 * (size_t)S.offset[i];
        const int32_t *sl = S.slots + (size_t)i * kDtSlots * 2;
        for (int k = 0; k < m; ++k) {
            out[3 * k + 0] = i;
            out[3 * k + 1] = sl[2 * k];
            out[3 * k + 2] = sl[2 * k + 1];
        }
    }
}

__global__ void dt_emit_kernel(DtArgs a) { dt_emit_body(a, vb_single()); }
__global__ void dt_emit_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_emit_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

// Points that own more than kDtSlots triangles (fan apexes): one CTA each
// rebuilds its star over every point and writes the owned triangles in order.
__device__ __forceinline__ void dt_emit_big_body(const DtArgs &a, const VB &vb) {
    __shared__ DtBlockShared sh;
    const DtSide S = vb.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    if (*S.ntri < 0 || !(*S.err & 4)) return;
    for (int i = vb.x; i < n; i += vb.gx) {
        if (S.owned[i] <= kDtSlots) continue;
        const int4 p = S.pts[S.slot[i]];
        int written = 0;
        dt_block_star(a, S, i, p, n, nullptr, 0, 0, &written, S.tri + 3 * (size_t)S.offset[i], sh, nullptr,
                      nullptr);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) dt_emit_big_kernel(DtArgs a) { dt_emit_big_body(a, vb_single()); }
__global__ void __launch_bounds__(256) dt_emit_big_kernel_b(const DtArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    dt_emit_big_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

// -------------------------------------------------------------------------
// Host side
// -------------------------------------------------------------------------

static void dt_geom(int w, int h, int &gw, int &gh) {
    gw = (w + kDtCell - 1) / kDtCell;
    gh = (h + kDtCell - 1) / kDtCell;
}

size_t dt_side_bytes(int cap, int w, int h) {
    int gw, gh;
    dt_geom(w, h, gw, gh);
    const size_t c = (size_t)(cap > 0 ? cap : 1);
    const size_t cells = (size_t)gw * gh + 1;
    return 2 * align_up(c * 4, 256) + align_up(c * 16, 256) + align_up(c * 4, 256) + 3 * align_up(cells * 4, 256) +
           3 * align_up(c * 4, 256) + align_up(c * kDtSlots * 8, 256) + 2 * align_up(c * 4, 256) +
           2 * align_up((size_t)h * 4, 256) + align_up(16, 256);
}

static DtSide dt_carve(void *ws, int cap, int w, int h) {
    int gw, gh;
    dt_geom(w, h, gw, gh);
    const size_t c = (size_t)(cap > 0 ? cap : 1);
    const size_t cells = (size_t)gw * gh + 1;
    char *b = reinterpret_cast<char *>(ws);
    DtSide s{};
    auto take = [&](size_t bytes) {
        char *r = b;
        b += align_up(bytes, 256);
        return r;
    };
    s.X = reinterpret_cast<int32_t *>(take(c * 4));
    s.Y = reinterpret_cast<int32_t *>(take(c * 4));
    s.pts = reinterpret_cast<int4 *>(take(c * 16));
    s.slot = reinterpret_cast<int32_t *>(take(c * 4));
    s.cell_cnt = reinterpret_cast<int32_t *>(take(cells * 4));
    s.cell_start = reinterpret_cast<int32_t *>(take(cells * 4));
    s.cell_fill = reinterpret_cast<int32_t *>(take(cells * 4));
    s.status = reinterpret_cast<int32_t *>(take(c * 4));
    s.owned = reinterpret_cast<int32_t *>(take(c * 4));
    s.offset = reinterpret_cast<int32_t *>(take(c * 4));
    s.slots = reinterpret_cast<int32_t *>(take(c * kDtSlots * 8));
    s.pending = reinterpret_cast<int32_t *>(take(c * 4));
    s.pending2 = reinterpret_cast<int32_t *>(take(c * 4));
    s.rowmin = reinterpret_cast<int32_t *>(take((size_t)h * 4));
    s.rowmax = reinterpret_cast<int32_t *>(take((size_t)h * 4));
    int32_t *small = reinterpret_cast<int32_t *>(take(16));
    s.err = small;
    s.npending = small + 1;
    s.npending2 = small + 2;
    s.npending3 = small + 3;
    return s;
}

__global__ void __launch_bounds__(256) dt_init_kernel(DtArgs a);

// Triangulates one or both sides.  sides[i] = right flag; tri/ntri per side.
elas_status launch_triangulate_device(const int16_t *list, const int32_t *count, int cap, int w, int h, int nsides,
                                      const int *rights, int32_t *const *tri, int32_t *const *ntri, int cap_tri,
                                      void *ws, cudaStream_t st) {
    DtArgs a{};
    a.list = list;
    a.count = count;
    a.cap = cap;
    a.cap_tri = cap_tri;
    a.w = w;
    a.h = h;
    dt_geom(w, h, a.gw, a.gh);
    const size_t side_bytes = dt_side_bytes(cap, w, h);
    for (int i = 0; i < nsides; ++i) {
        a.s[i] = dt_carve(reinterpret_cast<char *>(ws) + i * side_bytes, cap, w, h);
        a.s[i].right = rights[i];
        a.s[i].tri = tri[i];
        a.s[i].ntri = ntri[i];
    }
    // counters, cell counts and row extremes of both sides: one kernel
    const int nall = a.gw * a.gh + 1 + 2 * h + 4;
    dt_init_kernel<<<dim3((nall + 255) / 256, nsides), 256, 0, st>>>(a);
    const int tb = 256;
    const int pblocks = max(1, min((cap + tb - 1) / tb, sm_count() * 8));
    dt_points_kernel<<<dim3(pblocks, nsides), tb, 0, st>>>(a);
    dt_cell_scan_kernel<<<dim3(1, nsides), 1024, 0, st>>>(a);
    dt_scatter_kernel<<<dim3(pblocks, nsides), tb, 0, st>>>(a);
    dt_dedup_kernel<<<dim3(pblocks, nsides), tb, 0, st>>>(a);
    const int gblocks =
        max(1, min((cap + kDtGroupThreads / kDtGroupOne - 1) / (kDtGroupThreads / kDtGroupOne), sm_count() * 16));
    // one pair: the CTA pass takes the group pass's queue directly (its time
    // is that of the longest star, which the warp pass would not shorten)
    dt_pass1_kernel<<<dim3(gblocks, nsides), kDtGroupThreads, 0, st>>>(a);
    const int smem2 = kDtCandCap2 * (int)sizeof(int4);
    const int smem3 = smem2 + (2 * a.gh + 1) * (int)sizeof(int);
    if (smem3 > 227 * 1024) return fail(ELAS_ERR_INVALID_ARG, "image too tall for the triangulation grid");
    if (cudaFuncSetAttribute(dt_pass_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3) != cudaSuccess)
        return launch_status("dt_pass_block_kernel shared memory attribute");
    (void)smem2;
    dt_pass_block_kernel<<<sm_count() * kDtBlocksPerSM, kDtBlockThreads, smem3, st>>>(a, nsides);
    dt_tri_scan_kernel<<<dim3(1, nsides), 1024, 0, st>>>(a);
    dt_emit_kernel<<<dim3(pblocks, nsides), tb, 0, st>>>(a);
    dt_emit_big_kernel<<<dim3(sm_count(), nsides), 256, 0, st>>>(a);
    return launch_status("triangulation kernels");
}

// Batched launches keep no memsets: this kernel clears the counters and the
// row extremes of every (pair, side), and the CTA pass's queue counter.
__device__ __forceinline__ void dt_init_body(const DtArgs &a, const VB &vb, int32_t *counter) {
    const DtSide &S = a.s[vb.y];
    const int ncell1 = a.gw * a.gh + 1;
    const int nall = ncell1 + 2 * a.h + 4;
    if (counter && blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
    for (int k = vb.x * blockDim.x + threadIdx.x; k < nall; k += vb.gx * blockDim.x) {
        if (k < ncell1)
            S.cell_cnt[k] = 0;
        else if (k < ncell1 + a.h)
            S.rowmin[k - ncell1] = 0x7F7F7F7F;
        else if (k < ncell1 + 2 * a.h)
            S.rowmax[k - ncell1 - a.h] = (int32_t)0x80808080u;
        else
            S.err[k - ncell1 - 2 * a.h] = 0;  // err, npending, npending2, npending3
    }
}

__global__ void __launch_bounds__(256) dt_init_kernel(DtArgs a) { dt_init_body(a, vb_single(), nullptr); }
__global__ void __launch_bounds__(256) dt_init_kernel_b(const DtArgs *__restrict__ tab, VMap vm, int32_t *counter) {
    const VB vb = vb_batch(vm);
    dt_init_body(slot_entry(tab, vm.stride, vb.slot), vb, counter);
}

static int dt_point_blocks(int cap, int threads, int npairs) {
    // grid-stride kernels: about a third of the capacity per sweep in a
    // batch (the support list holds a fraction of the lattice), capped
    const int full = (cap + threads - 1) / threads;
    if (npairs <= 1) return max(1, min(full, sm_count() * 8));
    return max(1, min((full + 2) / 3, sm_count() * 8));
}

elas_status launch_triangulate_b(const DtArgs *tab, const DtArgs *host, const VMap &pairs, int nsides,
                                 int32_t *counter, cudaStream_t st) {
    if (pairs.n == 0) return ELAS_OK;
    if (nsides < 1 || nsides > 2) return fail(ELAS_ERR_INVALID_ARG, "nsides %d", nsides);
    VMap m_init, m_pts, m_scan, m_grp, m_grp2, m_big;
    vmap_clear(m_init, pairs.stride);
    vmap_clear(m_pts, pairs.stride);
    vmap_clear(m_scan, pairs.stride);
    vmap_clear(m_grp, pairs.stride);
    vmap_clear(m_grp2, pairs.stride);
    vmap_clear(m_big, pairs.stride);
    int max_gh = 1;
    for (int i = 0; i < pairs.n; ++i) {
        const int slot = pairs.slot[i];
        const DtArgs &a = slot_entry(host, pairs.stride, slot);
        const int nall = a.gw * a.gh + 1 + 2 * a.h + 4;
        vmap_add(m_init, slot, dim3((nall + 255) / 256, nsides));
        vmap_add(m_pts, slot, dim3(dt_point_blocks(a.cap, 256, pairs.n), nsides));
        vmap_add(m_scan, slot, dim3(1, nsides));
        const int gthreads = kDtGroupThreads / (pairs.n == 1 ? kDtGroupOne : kDtGroup);
        vmap_add(m_grp, slot, dim3(dt_point_blocks(a.cap, gthreads, pairs.n), nsides));
        // the middle and warp passes get their queues of a few percent of
        // the points (grid-stride over the queue)
        vmap_add(m_grp2, slot, dim3(max(1, min(sm_count(), a.cap / 256)), nsides));
        vmap_add(m_big, slot, dim3(pairs.n == 1 ? sm_count() : 64, nsides));
        max_gh = max(max_gh, a.gh);
    }
    const int smem3 = kDtCandCap2 * (int)sizeof(int4) + (2 * max_gh + 1) * (int)sizeof(int);
    if (smem3 > 200 * 1024) return fail(ELAS_ERR_INVALID_ARG, "image too tall for the triangulation grid");
    if (cudaFuncSetAttribute(dt_pass_block_kernel_b<kDtBlockThreads, kDtBlocksPerSM>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem3) != cudaSuccess ||
        cudaFuncSetAttribute(dt_pass_block_kernel_b<kDtBlockThreadsB, kDtBlocksPerSMB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem3) != cudaSuccess)
        return launch_status("dt_pass_block_kernel_b shared memory attribute");
    dt_init_kernel_b<<<vmap_total(m_init), 256, 0, st>>>(tab, m_init, counter);
    dt_points_kernel_b<<<vmap_total(m_pts), 256, 0, st>>>(tab, m_pts);
    dt_cell_scan_kernel_b<<<vmap_total(m_scan), 1024, 0, st>>>(tab, m_scan);
    dt_scatter_kernel_b<<<vmap_total(m_pts), 256, 0, st>>>(tab, m_pts);
    dt_dedup_kernel_b<<<vmap_total(m_pts), 256, 0, st>>>(tab, m_pts);
    // one pair: the one-pair group pass, then the CTA pass on its queue (as
    // in launch_triangulate_device); several: the batch group pass and the
    // warp pass
    const bool one = pairs.n == 1;
    if (one) {
        dt_pass1_kernel_b1<<<vmap_total(m_grp), kDtGroupThreads, 0, st>>>(tab, m_grp);
    } else {
        dt_pass1_kernel_b<<<vmap_total(m_grp), kDtGroupThreads, 0, st>>>(tab, m_grp);
        dt_pass1m_kernel_b<<<vmap_total(m_grp2), kDtGroupThreads, 0, st>>>(tab, m_grp2);
        dt_pass1b_kernel_b<<<vmap_total(m_grp2), kDtGroupThreads, 0, st>>>(tab, m_grp2);
    }
    const int nsm = sm_count();
    if (one)
        dt_pass_block_kernel_b<kDtBlockThreads, kDtBlocksPerSM>
            <<<nsm * kDtBlocksPerSM, kDtBlockThreads, smem3, st>>>(tab, pairs, nsides, counter, 0);
    else
        dt_pass_block_kernel_b<kDtBlockThreadsB, kDtBlocksPerSMB>
            <<<nsm * kDtBlocksPerSMB, kDtBlockThreadsB, smem3, st>>>(tab, pairs, nsides, counter, 1);
    dt_tri_scan_kernel_b<<<vmap_total(m_scan), 1024, 0, st>>>(tab, m_scan);
    dt_emit_kernel_b<<<vmap_total(m_pts), 256, 0, st>>>(tab, m_pts);
    dt_emit_big_kernel_b<<<vmap_total(m_big), 256, 0, st>>>(tab, m_big);
    return launch_status("batched triangulation kernels");
}

// Argument block of one pair's triangulation (both sides), for the tables
// of batched launches.
DtArgs triangulate_args(const int16_t *list, const int32_t *count, int cap, int w, int h, int32_t *const *tri,
                        int32_t *const *ntri, int cap_tri, void *ws) {
    DtArgs a{};
    a.list = list;
    a.count = count;
    a.cap = cap;
    a.cap_tri = cap_tri;
    a.w = w;
    a.h = h;
    dt_geom(w, h, a.gw, a.gh);
    const size_t side_bytes = dt_side_bytes(cap, w, h);
    for (int i = 0; i < 2; ++i) {
        a.s[i] = dt_carve(reinterpret_cast<char *>(ws) + i * side_bytes, cap, w, h);
        a.s[i].right = i;
        a.s[i].tri = tri[i];
        a.s[i].ntri = ntri[i];
    }
    return a;
}

size_t triangulate_device_workspace(int cap, int w, int h, int nsides) { return nsides * dt_side_bytes(cap, w, h); }

}  // namespace elas

extern "C" size_t elas_triangulate_device_workspace_bytes(int32_t cap, int32_t w, int32_t h) {
    if (cap < 0 || w < 1 || h < 1) return 0;
    return elas::triangulate_device_workspace(cap, w, h, 1);
}

extern "C" elas_status elas_triangulate_device(const int16_t *list, const int32_t *count, int32_t cap, int32_t w,
                                               int32_t h, int32_t right, int32_t *tri, int32_t cap_tri,
                                               int32_t *ntri, void *workspace, size_t workspace_bytes,
                                               elas_stream stream) {
    using namespace elas;
    if (w < 1 || h < 1 || w > 16383 || h > 16383) return fail(ELAS_ERR_INVALID_ARG, "image size %dx%d", w, h);
    if (!list || !count || !tri || !ntri || !workspace) return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (cap < 0 || cap_tri < 2 * cap + 8)
        return fail(ELAS_ERR_CAPACITY, "triangle capacity %d below 2*cap+8 = %d", cap_tri, 2 * cap + 8);
    if (!aligned(workspace, 256)) return fail(ELAS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (workspace_bytes < triangulate_device_workspace(cap, w, h, 1))
        return fail(ELAS_ERR_CAPACITY, "workspace %zu < %zu bytes", workspace_bytes,
                    triangulate_device_workspace(cap, w, h, 1));
    const int rights[1] = {right ? 1 : 0};
    int32_t *tris[1] = {tri};
    int32_t *nts[1] = {ntri};
    return launch_triangulate_device(list, count, cap, w, h, 1, rights, tris, nts, cap_tri, workspace,
                                     to_stream(stream));
}
