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
// Pass 1 (one warp per point) caches the points within 32 pixels of p, taken
// from a 16-pixel grid, in shared memory and wraps among them; the star is
// accepted when it closes and every triangle's circumdisc lies inside that
// disc (4 r^2 <= 32^2 in exact arithmetic), so no farther point can matter.
// Stars that stay open (hull points), or leave the disc, are redone in pass
// 2 by one CTA per point with every point as a candidate.  Each triangle is
// emitted once, by its lowest-index vertex, at an offset from an exclusive
// scan of the per-point counts, so the output order is deterministic.
#include "launch.cuh"

namespace elas {

constexpr int kDtCell = 16;
constexpr int kDtMaxStar = 4096;  // wrap steps per star

struct DtSide {
    int right;
    int32_t *X, *Y;        // [cap] coordinates per list index
    int4 *pts;             // [cap] (x, y, index, alive) sorted by grid cell
    int32_t *slot;         // [cap] position of each point in pts
    int32_t *cell_cnt;     // [ncell + 1]
    int32_t *cell_start;   // [ncell + 1]
    int32_t *cell_fill;    // [ncell + 1]
    int32_t *status;       // [cap] 0 pending, 1/2 certified in pass 1/2, -1 duplicate
    int32_t *owned;        // [cap] triangles owned (lowest-index vertex)
    int32_t *offset;       // [cap] exclusive scan of owned
    int32_t *slots;        // [cap][kDtSlots][2] owned triangles (the other two vertices)
    int32_t *pending;      // [cap] points queued for pass 2
    int32_t *npending;     // queue length
    int32_t *tri;          // output [cap_tri][3]
    int32_t *ntri;         // output count
    int32_t *err;          // bit 0: a star failed, bit 1: capacity, bit 2: slots overflowed
};

struct DtArgs {
    const int16_t *list;
    const int32_t *count;  // number of support points (device)
    int cap;               // capacity in points
    int cap_tri;
    int w, h, gw, gh;
    DtSide s[2];
};

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
// counter-clockwise), with the symbolic tie-break on the list indices.
__device__ __forceinline__ int dt_incircle(const int4 &P, const int4 &A, const int4 &B, const int4 &C) {
    const int64_t ax = A.x - P.x, ay = A.y - P.y, bx = B.x - P.x, by = B.y - P.y, cx = C.x - P.x, cy = C.y - P.y;
    const int64_t al = ax * ax + ay * ay, bl = bx * bx + by * by, cl = cx * cx + cy * cy;
    // value = -det[[a, |a|^2], [b, |b|^2], [c, |c|^2]] (relative to P)
    const int64_t det = ax * (by * cl - bl * cy) - ay * (bx * cl - bl * cx) + al * (bx * cy - by * cx);
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

__global__ void dt_points_kernel(DtArgs a) {
    const DtSide S = blockIdx.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int u = a.list[3 * i], v = a.list[3 * i + 1], d = a.list[3 * i + 2];
        const int x = S.right ? u - d : u;
        S.X[i] = x;
        S.Y[i] = v;
        S.status[i] = 0;
        S.owned[i] = 0;
        atomicAdd(S.cell_cnt + dt_cell(a, x, v), 1);
    }
}

// One CTA per side: exclusive scan of the cell counts.
__global__ void __launch_bounds__(1024) dt_cell_scan_kernel(DtArgs a) {
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const DtSide S = blockIdx.y ? a.s[1] : a.s[0];
    const int ncell = dt_ncell(a);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base <= ncell; base += 1024) {
        const int i = base + tid;
        const int v = i < ncell ? S.cell_cnt[i] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int x = s_w[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            s_w[lane] = x;
        }
        __syncthreads();
        const int excl = s_carry + (wid ? s_w[wid - 1] : 0) + incl - v;
        if (i <= ncell) {
            S.cell_start[i] = excl;
            S.cell_fill[i] = excl;
        }
        __syncthreads();
        if (tid == 0) s_carry += s_w[31];
        __syncthreads();
    }
}

__global__ void dt_scatter_kernel(DtArgs a) {
    const DtSide S = blockIdx.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = S.X[i], y = S.Y[i];
        const int k = atomicAdd(S.cell_fill + dt_cell(a, x, y), 1);
        S.pts[k] = make_int4(x, y, i, 1);
        S.slot[i] = k;
    }
}

// Coincident points (right coordinates only) keep the lowest list index.
__global__ void dt_dedup_kernel(DtArgs a) {
    const DtSide S = blockIdx.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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

// -------------------------------------------------------------------------
// Stars
// -------------------------------------------------------------------------

constexpr int kDtRadius = 32;     // pass-1 search radius
constexpr int kDtCandCap = 160;   // pass-1 candidates cached per warp
constexpr int kDtSlots = 32;      // owned triangles kept per point
constexpr int kDtWarps = 8;       // warps per CTA

__device__ __forceinline__ int4 shfl4(const int4 &v, int src_xor) {
    return make_int4(__shfl_xor_sync(0xFFFFFFFFu, v.x, src_xor), __shfl_xor_sync(0xFFFFFFFFu, v.y, src_xor),
                     __shfl_xor_sync(0xFFFFFFFFu, v.z, src_xor), __shfl_xor_sync(0xFFFFFFFFu, v.w, src_xor));
}

// Better of two third-vertex candidates in the pencil order of edge (p, e):
// ccw: triangles (p, e, c); else (p, c, e).  c2 beats c1 iff c2 lies inside
// the circle of c1's triangle.  w = 0 marks "no candidate".
__device__ __forceinline__ int4 dt_better(const int4 &c1, const int4 &c2, const int4 &p, const int4 &e, bool ccw) {
    if (!c2.w) return c1;
    if (!c1.w) return c2;
    const int s = ccw ? dt_incircle(p, e, c1, c2) : dt_incircle(p, c1, e, c2);
    return (s > 0 || (s == 0 && c2.z < c1.z)) ? c2 : c1;
}

__device__ __forceinline__ int4 dt_warp_best(int4 best, const int4 &p, const int4 &e, bool ccw) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = dt_better(best, shfl4(best, o), p, e, ccw);
    return best;
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

// Circumdisc of (p, a, b) inside the disc of radius R around p:
// |pa|^2 |pb|^2 |ab|^2 <= R^2 area2^2 (twice the circumradius <= R); the
// operands are integers below 2^53, so the double products are exact.
__device__ __forceinline__ bool dt_small_circle(const int4 &p, const int4 &a, const int4 &b, int R) {
    const double pa = (double)(a.x - p.x) * (a.x - p.x) + (double)(a.y - p.y) * (a.y - p.y);
    const double pb = (double)(b.x - p.x) * (b.x - p.x) + (double)(b.y - p.y) * (b.y - p.y);
    const double ab = (double)(b.x - a.x) * (b.x - a.x) + (double)(b.y - a.y) * (b.y - a.y);
    const double ar = (double)dt_orient(p.x, p.y, a.x, a.y, b.x, b.y);
    return pa * pb * ab <= (double)R * R * ar * ar;
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

// Pass 1: one warp per point, candidates within kDtRadius cached in shared
// memory.  Open stars (hull points), stars with too many candidates and
// stars whose circles leave the radius are queued for pass 2.
__global__ void __launch_bounds__(32 * kDtWarps) dt_pass1_kernel(DtArgs a) {
    __shared__ int4 s_cand[kDtWarps][kDtCandCap];
    const DtSide S = blockIdx.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int4 *cand = s_cand[warp];
    const int R = kDtRadius;
    const int64_t R2 = (int64_t)R * R;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
        if (S.status[i] < 0) continue;  // duplicate
        const int4 p = S.pts[S.slot[i]];
        // gather the candidates
        int k = 0;
        bool overflow = false;
        const int cx0 = max(0, p.x - R) / kDtCell, cx1 = min(a.gw - 1, (p.x + R) / kDtCell);
        const int cy0 = max(0, p.y - R) / kDtCell, cy1 = min(a.gh - 1, (p.y + R) / kDtCell);
        for (int cy = cy0; cy <= cy1; ++cy) {
            const int s0 = S.cell_start[cy * a.gw + cx0], e0 = S.cell_start[cy * a.gw + cx1 + 1];
            for (int j = s0; j < e0; j += 32) {
                bool take = false;
                int4 q = make_int4(0, 0, 0, 0);
                if (j + lane < e0) {
                    q = S.pts[j + lane];
                    const int64_t dx = q.x - p.x, dy = q.y - p.y;
                    take = q.w && q.z != p.z && dx * dx + dy * dy <= R2;
                }
                const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
                const int pos = k + __popc(m & ((1u << lane) - 1u));
                if (take && pos < kDtCandCap) cand[pos] = q;
                k += __popc(m);
            }
        }
        if (k > kDtCandCap) overflow = true;
        __syncwarp();
        bool certified = !overflow && k > 0;
        int written = 0;
        if (certified) {
            unsigned long long key = ~0ull;
            for (int j = lane; j < k; j += 32) {
                const unsigned long long kk = dt_nn_key(p, cand[j]);
                key = kk < key ? kk : key;
            }
            key = warp_min64(key);
            int4 first = make_int4(0, 0, (int)(unsigned)(key & 0xFFFFFFFFu), 1);
            for (int j = 0; j < k; ++j)  // coordinates of the nearest neighbour
                if (cand[j].z == first.z) first = cand[j];
            int4 cur = first;
            bool closed = false;
            for (int step = 0; step < k + 1 && certified; ++step) {
                int4 best = make_int4(0, 0, 0, 0);
                for (int j = lane; j < k; j += 32) {
                    const int4 q = cand[j];
                    if (q.z != cur.z && dt_orient(p.x, p.y, cur.x, cur.y, q.x, q.y) > 0)
                        best = dt_better(best, q, p, cur, true);
                }
                best = dt_warp_best(best, p, cur, true);
                if (!best.w || !dt_small_circle(p, cur, best, R)) {
                    certified = false;  // open side or large circle: pass 2
                    break;
                }
                dt_record(S, i, written, p, cur, best, lane == 0);
                if (best.z == first.z) {
                    closed = true;
                    break;
                }
                cur = best;
            }
            if (!closed) certified = false;
        }
        if (lane == 0) {
            if (certified) {
                S.status[i] = 1;
                S.owned[i] = written;
                if (written > kDtSlots) atomicOr(S.err, 4);
            } else {
                S.pending[atomicAdd(S.npending, 1)] = i;
            }
        }
    }
}

// Pass 2: one CTA per queued point, every point a candidate (so the star is
// exact and open sides are hull edges).
__device__ __forceinline__ int4 dt_block_best(int4 best, const int4 &p, const int4 &e, bool ccw, int4 *s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    best = dt_warp_best(best, p, e, ccw);
    __syncthreads();
    if (lane == 0) s_red[warp] = best;
    __syncthreads();
    int4 r = lane < (int)(blockDim.x >> 5) ? s_red[lane] : make_int4(0, 0, 0, 0);
    r = dt_warp_best(r, p, e, ccw);
    return r;  // every warp holds the same result
}

__global__ void __launch_bounds__(32 * kDtWarps) dt_pass2_kernel(DtArgs a) {
    __shared__ int4 s_red[kDtWarps];
    __shared__ unsigned long long s_key[kDtWarps];
    const DtSide S = blockIdx.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    const int np = *S.npending;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nth = blockDim.x;
    for (int q0 = blockIdx.x; q0 < np; q0 += gridDim.x) {
        const int i = S.pending[q0];
        const int4 p = S.pts[S.slot[i]];
        // nearest neighbour over all points
        unsigned long long key = ~0ull;
        for (int j = tid; j < n; j += nth) {
            const int4 q = S.pts[j];
            if (q.w && q.z != p.z) {
                const unsigned long long kk = dt_nn_key(p, q);
                key = kk < key ? kk : key;
            }
        }
        key = warp_min64(key);
        __syncthreads();
        if (lane == 0) s_key[warp] = key;
        __syncthreads();
        key = lane < (nth >> 5) ? s_key[lane] : ~0ull;
        key = warp_min64(key);
        int written = 0;
        bool ok = true;
        if (key != ~0ull) {
            const int4 first = S.pts[S.slot[(int)(unsigned)(key & 0xFFFFFFFFu)]];
            int4 cur = first;
            bool closed = false;
            int step = 0;
            for (; step < kDtMaxStar; ++step) {  // counter-clockwise
                int4 best = make_int4(0, 0, 0, 0);
                for (int j = tid; j < n; j += nth) {
                    const int4 q = S.pts[j];
                    if (q.w && q.z != p.z && q.z != cur.z && dt_orient(p.x, p.y, cur.x, cur.y, q.x, q.y) > 0)
                        best = dt_better(best, q, p, cur, true);
                }
                best = dt_block_best(best, p, cur, true, s_red);
                if (!best.w) break;  // hull edge
                dt_record(S, i, written, p, cur, best, tid == 0);
                if (best.z == first.z) {
                    closed = true;
                    break;
                }
                cur = best;
            }
            if (step >= kDtMaxStar) ok = false;
            if (!closed && ok) {  // clockwise from the first edge
                cur = first;
                for (step = 0; step < kDtMaxStar; ++step) {
                    int4 best = make_int4(0, 0, 0, 0);
                    for (int j = tid; j < n; j += nth) {
                        const int4 q = S.pts[j];
                        if (q.w && q.z != p.z && q.z != cur.z && dt_orient(p.x, p.y, cur.x, cur.y, q.x, q.y) < 0)
                            best = dt_better(best, q, p, cur, false);
                    }
                    best = dt_block_best(best, p, cur, false, s_red);
                    if (!best.w) break;
                    dt_record(S, i, written, p, best, cur, tid == 0);
                    cur = best;
                }
                if (step >= kDtMaxStar) ok = false;
            }
        }
        if (tid == 0) {
            if (ok) {
                S.status[i] = 2;
                S.owned[i] = written;
                if (written > kDtSlots) atomicOr(S.err, 4);
            } else {
                atomicOr(S.err, 1);
            }
        }
        __syncthreads();
    }
}

// One CTA per side: exclusive scan of the owned counts, total = ntri.
__global__ void __launch_bounds__(1024) dt_tri_scan_kernel(DtArgs a) {
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const DtSide S = blockIdx.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int i = base + tid;
        const int v = i < n ? S.owned[i] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int x = s_w[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            s_w[lane] = x;
        }
        __syncthreads();
        if (i < n) S.offset[i] = s_carry + (wid ? s_w[wid - 1] : 0) + incl - v;
        __syncthreads();
        if (tid == 0) s_carry += s_w[31];
        __syncthreads();
    }
    if (tid == 0) {
        if (s_carry > a.cap_tri) atomicOr(S.err, 2);
        *S.ntri = (*S.err & 3) ? -1 : s_carry;  // -1: the triangulation failed
    }
}

// One thread per point: copy the owned triangles to their offset.
__global__ void dt_emit_kernel(DtArgs a) {
    const DtSide S = blockIdx.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    if (*S.ntri < 0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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

// Points that own more than kDtSlots triangles (fan apexes): one CTA each
// rebuilds its star over all points and writes the owned triangles in order.
__global__ void __launch_bounds__(32 * kDtWarps) dt_emit_big_kernel(DtArgs a) {
    __shared__ int4 s_red[kDtWarps];
    __shared__ unsigned long long s_key[kDtWarps];
    const DtSide S = blockIdx.y ? a.s[1] : a.s[0];
    const int n = min(max(*a.count, 0), a.cap);
    if (*S.ntri < 0 || !(*S.err & 4)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nth = blockDim.x;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        if (S.owned[i] <= kDtSlots) continue;
        const int4 p = S.pts[S.slot[i]];
        int32_t *out = S.tri + 3 * (size_t)S.offset[i];
        unsigned long long key = ~0ull;
        for (int j = tid; j < n; j += nth) {
            const int4 q = S.pts[j];
            if (q.w && q.z != p.z) {
                const unsigned long long kk = dt_nn_key(p, q);
                key = kk < key ? kk : key;
            }
        }
        key = warp_min64(key);
        __syncthreads();
        if (lane == 0) s_key[warp] = key;
        __syncthreads();
        key = lane < (nth >> 5) ? s_key[lane] : ~0ull;
        key = warp_min64(key);
        const int4 first = S.pts[S.slot[(int)(unsigned)(key & 0xFFFFFFFFu)]];
        int written = 0;
        int4 cur = first;
        bool closed = false;
        for (int step = 0; step < kDtMaxStar; ++step) {
            int4 best = make_int4(0, 0, 0, 0);
            for (int j = tid; j < n; j += nth) {
                const int4 q = S.pts[j];
                if (q.w && q.z != p.z && q.z != cur.z && dt_orient(p.x, p.y, cur.x, cur.y, q.x, q.y) > 0)
                    best = dt_better(best, q, p, cur, true);
            }
            best = dt_block_best(best, p, cur, true, s_red);
            if (!best.w) break;
            if (p.z < cur.z && p.z < best.z) {
                if (tid == 0) {
                    out[3 * written] = i;
                    out[3 * written + 1] = cur.z;
                    out[3 * written + 2] = best.z;
                }
                ++written;
            }
            if (best.z == first.z) {
                closed = true;
                break;
            }
            cur = best;
        }
        if (!closed) {
            cur = first;
            for (int step = 0; step < kDtMaxStar; ++step) {
                int4 best = make_int4(0, 0, 0, 0);
                for (int j = tid; j < n; j += nth) {
                    const int4 q = S.pts[j];
                    if (q.w && q.z != p.z && q.z != cur.z && dt_orient(p.x, p.y, cur.x, cur.y, q.x, q.y) < 0)
                        best = dt_better(best, q, p, cur, false);
                }
                best = dt_block_best(best, p, cur, false, s_red);
                if (!best.w) break;
                if (p.z < cur.z && p.z < best.z) {
                    if (tid == 0) {
                        out[3 * written] = i;
                        out[3 * written + 1] = best.z;
                        out[3 * written + 2] = cur.z;
                    }
                    ++written;
                }
                cur = best;
            }
        }
        __syncthreads();
    }
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
           3 * align_up(c * 4, 256) + align_up(c * kDtSlots * 8, 256) + align_up(c * 4, 256) + align_up(16, 256);
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
    int32_t *small = reinterpret_cast<int32_t *>(take(16));
    s.err = small;
    s.npending = small + 1;
    return s;
}

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
        const size_t cells = (size_t)a.gw * a.gh + 1;
        if (cudaMemsetAsync(a.s[i].cell_cnt, 0, cells * 4, st) != cudaSuccess ||
            cudaMemsetAsync(a.s[i].err, 0, 16, st) != cudaSuccess)
            return launch_status("triangulation memsets");
    }
    const int tb = 256;
    const int pblocks = max(1, min((cap + tb - 1) / tb, 152 * 8));
    const int wblocks = max(1, min((cap + kDtWarps - 1) / kDtWarps, 152 * 16));
    dt_points_kernel<<<dim3(pblocks, nsides), tb, 0, st>>>(a);
    dt_cell_scan_kernel<<<dim3(1, nsides), 1024, 0, st>>>(a);
    dt_scatter_kernel<<<dim3(pblocks, nsides), tb, 0, st>>>(a);
    dt_dedup_kernel<<<dim3(pblocks, nsides), tb, 0, st>>>(a);
    dt_pass1_kernel<<<dim3(wblocks, nsides), 32 * kDtWarps, 0, st>>>(a);
    dt_pass2_kernel<<<dim3(152 * 4, nsides), 32 * kDtWarps, 0, st>>>(a);
    dt_tri_scan_kernel<<<dim3(1, nsides), 1024, 0, st>>>(a);
    dt_emit_kernel<<<dim3(pblocks, nsides), tb, 0, st>>>(a);
    dt_emit_big_kernel<<<dim3(152, nsides), 32 * kDtWarps, 0, st>>>(a);
    return launch_status("triangulation kernels");
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
