// Slanted-plane prior (Sec. III.A; image-sized prior matrix, Sec. VI.D) and
// dense per-pixel argmin of descriptor SAD plus tabulated prior over the
// grid-vector and plane-neighbourhood candidates (Sec. III.A, Fig. 1(h)).
//
// The prior is drawn in three launches:
// raster_setup_kernel  fills the maps with -1 and, one thread per triangle,
//                      writes a 64-byte record: the plane in the fixed FP32
//                      order, the three integer edge functions with the
//                      top-left rule folded into their constants, and the
//                      pixel bounding box; and the triangle's count of
//                      kUnitPx-pixel chunks of that box; it also clears the
//                      mesh's count of extra units;
// raster_list_kernel   one thread per triangle: the chunks after the first
//                      of a box go to the mesh's list of extra units (one
//                      atomicAdd per triangle of more than one chunk);
// raster_draw_kernel   one warp per unit (grid-stride; unit t < ntri is
//                      the first chunk of triangle t, the rest come from the
//                      list), its lanes on 32 pixels of the box at a time: a
//                      pixel owned by the triangle (at most one owner: the
//                      top-left rule) takes clamp(floor(plane + 0.5)).  A
//                      full list makes the warp of a triangle's first chunk
//                      draw the whole box instead.
// cell_kernel          one CTA per grid-vector cell (G x G pixels, which share
//                      one candidate mask) and per reference image.  It
//                      expands the cell's mask into an ascending candidate
//                      list in shared memory, then per pixel takes the
//                      minimum of the packed key (cost, d) over the list (no
//                      prior) and over the plane neighbourhood (with prior).
//                      A d in both sets is evaluated twice, without and with
//                      the prior; as P <= 0 the second never loses, so the
//                      result is the argmin over the union.  The list is
//                      uniform across the CTA: no divergence, broadcast
//                      shared loads.
#include <cooperative_groups.h>

#include "launch.cuh"

namespace elas {

constexpr int kKeyBias = 65536;  // keeps (cost + bias) positive; |P| <= 65535

__device__ __forceinline__ bool edge_owned(int px, int py, int qx, int qy) {
    return (qy == py && qx > px) || (qy < py);
}

__device__ __forceinline__ int side_ntri(const RasterSide &S) {
    return S.ntri_dev ? max(0, *S.ntri_dev) : S.ntri;
}

constexpr int kUnitPx = 256;  // pixels of a triangle's bounding box per work unit

// Rasteriser record of one triangle: pixel (x, y) is owned iff
// A[k] x + B[k] y + C[k] > 0 for k = 0, 1, 2 (the edge function of edge k,
// positively oriented, plus 1 on an owned edge, so E >= 0 there and E >= 1
// elsewhere), and then d_plane = clamp(floor((fa x + fb y) + fc + 0.5)).
// A degenerate triangle (det = 0) gets A = B = C = 0: it owns nothing.
struct TriBox {
    int xmin, xmax, ymin, ymax;
};
struct TriRec {
    int A[3], B[3], C[3];
    float fa, fb, fc;
};
constexpr int kRecWords = 4;  // 16-byte words of a stored record: edges, plane, box

// Plane and edge record of triangle t (vertices taken in ascending list
// index), and its pixel bounding box clipped to the image (empty: xmax <
// xmin).
__device__ __forceinline__ TriRec tri_record(const int16_t *__restrict__ list, const int32_t *__restrict__ tri, int t,
                                             int right, int w, int h, TriBox &box) {
    int i0 = __ldg(tri + 3 * t), i1 = __ldg(tri + 3 * t + 1), i2 = __ldg(tri + 3 * t + 2);
    // canonical vertex order: ascending list index
    if (i1 < i0) { const int q = i0; i0 = i1; i1 = q; }
    if (i2 < i1) { const int q = i1; i1 = i2; i2 = q; }
    if (i1 < i0) { const int q = i0; i0 = i1; i1 = q; }
    int X[3], Y[3], Z[3];
    const int id[3] = {i0, i1, i2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int u = __ldg(list + 3 * id[k]), v = __ldg(list + 3 * id[k] + 1);
        const int d = __ldg(list + 3 * id[k] + 2);
        X[k] = right ? u - d : u;
        Y[k] = v;
        Z[k] = d;
    }
    const int det = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]);
    const int na = (Z[1] - Z[0]) * (Y[2] - Y[0]) - (Z[2] - Z[0]) * (Y[1] - Y[0]);
    const int nb = (X[1] - X[0]) * (Z[2] - Z[0]) - (X[2] - X[0]) * (Z[1] - Z[0]);
    TriRec r;
    const float fdet = __int2float_rn(det == 0 ? 1 : det);
    r.fa = __fdiv_rn(__int2float_rn(na), fdet);
    r.fb = __fdiv_rn(__int2float_rn(nb), fdet);
    const float c = __fsub_rn(__int2float_rn(Z[0]), __fmul_rn(r.fa, __int2float_rn(X[0])));
    r.fc = __fsub_rn(c, __fmul_rn(r.fb, __int2float_rn(Y[0])));
    // positively oriented vertex cycle (v0, v1, v2)
    const int ex[3] = {X[0], det > 0 ? X[1] : X[2], det > 0 ? X[2] : X[1]};
    const int ey[3] = {Y[0], det > 0 ? Y[1] : Y[2], det > 0 ? Y[2] : Y[1]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1;
        // E(x, y) = (x1 - x0)(y - y0) - (y1 - y0)(x - x0) = A x + B y + C
        const int A = ey[k] - ey[k1], B = ex[k1] - ex[k];
        const int own = edge_owned(ex[k], ey[k], ex[k1], ey[k1]) ? 1 : 0;
        r.A[k] = det == 0 ? 0 : A;
        r.B[k] = det == 0 ? 0 : B;
        r.C[k] = det == 0 ? 0 : own - A * ex[k] - B * ey[k];
    }
    box.xmin = max(0, min(X[0], min(X[1], X[2])));
    box.xmax = min(w - 1, max(X[0], max(X[1], X[2])));
    box.ymin = max(0, min(Y[0], min(Y[1], Y[2])));
    box.ymax = min(h - 1, max(Y[0], max(Y[1], Y[2])));
    if (det == 0) box.xmax = box.xmin - 1;
    return r;
}

__device__ __forceinline__ void store_rec(int4 *__restrict__ rec, int t, const TriRec &r, const TriBox &b) {
    int4 *o = rec + kRecWords * (size_t)t;
    o[0] = make_int4(r.A[0], r.A[1], r.A[2], r.B[0]);
    o[1] = make_int4(r.B[1], r.B[2], r.C[0], r.C[1]);
    o[2] = make_int4(r.C[2], __float_as_int(r.fa), __float_as_int(r.fb), __float_as_int(r.fc));
    o[3] = make_int4(b.xmin, b.xmax, b.ymin, b.ymax);
}

__device__ __forceinline__ TriRec load_rec(const int4 *__restrict__ rec, int t) {
    const int4 p = rec[kRecWords * (size_t)t], q = rec[kRecWords * (size_t)t + 1], u = rec[kRecWords * (size_t)t + 2];
    TriRec r;
    r.A[0] = p.x, r.A[1] = p.y, r.A[2] = p.z, r.B[0] = p.w;
    r.B[1] = q.x, r.B[2] = q.y, r.C[0] = q.z, r.C[1] = q.w;
    r.C[2] = u.x, r.fa = __int_as_float(u.y), r.fb = __int_as_float(u.z), r.fc = __int_as_float(u.w);
    return r;
}

// Records, unit counts and the -1 fill of the maps (grid-stride; the maps
// of the sides need not be contiguous).
__device__ __forceinline__ void raster_setup_body(const RasterArgs &a, const VB &vb) {
    const int tid = vb.x * blockDim.x + threadIdx.x, stride = vb.gx * blockDim.x;
    const RasterSide &S = a.s[vb.y];
    // -1 fill: 16-byte stores between an unaligned head and tail
    const size_t npx = (size_t)a.w * a.h;
    int16_t *d = S.dplane;
    const size_t head = min(npx, (size_t)((16 - (reinterpret_cast<uintptr_t>(d) & 15)) & 15) / 2);
    const size_t n8 = (npx - head) / 8;
    uint4 *d8 = reinterpret_cast<uint4 *>(d + head);
    for (size_t i = tid; i < n8; i += stride) d8[i] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    if ((size_t)tid < head) d[tid] = -1;
    if ((size_t)tid < npx - head - 8 * n8) d[head + 8 * n8 + tid] = -1;
    if (tid == 0) *S.nunits = 0;
    const int ntri = side_ntri(S);
    for (int t = tid; t < ntri; t += stride) {
        TriBox b;
        const TriRec r = tri_record(a.list, S.tri, t, S.right, a.w, a.h, b);
        store_rec(S.rec, t, r, b);
        const long long area = b.xmax >= b.xmin && b.ymax >= b.ymin
                                   ? (long long)(b.xmax - b.xmin + 1) * (b.ymax - b.ymin + 1)
                                   : 0;
        S.ucnt[t] = (int)((area + kUnitPx - 1) / kUnitPx);
    }
}

__global__ void __launch_bounds__(256) raster_setup_kernel(RasterArgs a) { raster_setup_body(a, vb_single()); }
__global__ void __launch_bounds__(256) raster_setup_kernel_b(const RasterArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    raster_setup_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

constexpr int kListPad = 16;  // padding entries (2047) after a candidate list

// The candidate list of one grid-vector cell (Sec. III.A: the disparities
// of its mask within [dmin, dmax]), ascending, then kListPad entries of 2047
// (above every dmax); returns the count.  Warp collective.  The words are
// taken one at a time: lane l places bit l of the word after the set bits
// below it, so the list comes out sorted with no per-lane bit loop.
__device__ __forceinline__ int expand_cell_list(const uint32_t *__restrict__ g, int nw, int dmin, int dmax,
                                                uint16_t *out, int lane) {
    const uint32_t below = (1u << lane) - 1u;
    int base = 0;
    for (int w0 = 0; w0 < nw; w0 += 32) {
        const int wi = w0 + lane;
        uint32_t m = wi < nw ? __ldg(g + wi) : 0u;
        // keep the bits inside [dmin, dmax]
        const int lo = dmin - 32 * wi, hi = dmax - 32 * wi;
        if (lo > 0) m &= lo >= 32 ? 0u : (0xFFFFFFFFu << lo);
        if (hi < 31) m &= hi < 0 ? 0u : (0xFFFFFFFFu >> (31 - hi));
        const int nk = min(32, nw - w0);
        for (int k = 0; k < nk; ++k) {
            const uint32_t mk = __shfl_sync(0xFFFFFFFFu, m, k);
            if ((mk >> lane) & 1u) out[base + __popc(mk & below)] = (uint16_t)(32 * (w0 + k) + lane);
            base += __popc(mk);
        }
    }
    if (lane < kListPad) out[base + lane] = (uint16_t)2047;
    return base;
}

// Extra units (chunks 1.. of each box) of the mesh: ulist[k] = (t, chunk);
// *nunits counts them (64 bits: thin triangles' boxes can hold many), beyond
// unit_cap the list is incomplete.  With lstride > 0 it also expands the
// grid-vector masks of the mesh's side into the dense step's candidate
// lists.
__device__ __forceinline__ void raster_list_body(const RasterArgs &a, const VB &vb) {
    const RasterSide &S = a.s[vb.y];
    const int ntri = side_ntri(S);
    for (int t = vb.x * blockDim.x + threadIdx.x; t < ntri; t += vb.gx * blockDim.x) {
        const int n = S.ucnt[t] - 1;
        if (n <= 0) continue;
        const unsigned long long pos = atomicAdd(S.nunits, (unsigned long long)n);
        for (int j = 0; j < n && pos + j < (unsigned long long)a.unit_cap; ++j) S.ulist[pos + j] = make_int2(t, j + 1);
    }
    // the dense step's candidate lists: one warp per cell
    if (a.lstride > 0) {
        const int lane = threadIdx.x & 31;
        const int ncell = a.gw * a.gh;
        for (int c = vb.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncell; c += vb.gx * (blockDim.x >> 5)) {
            const int n = expand_cell_list(S.grid + (size_t)c * a.nw, a.nw, a.dmin, a.dmax,
                                           S.clist + (size_t)c * a.lstride, lane);
            if (lane == 0) S.ccount[c] = n;
        }
    }
}

__global__ void __launch_bounds__(256) raster_list_kernel(RasterArgs a) { raster_list_body(a, vb_single()); }
__global__ void __launch_bounds__(256) raster_list_kernel_b(const RasterArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    raster_list_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

// Pixels [p0, p1) of the box of record r (row-major in the box), 32 at a
// time across the warp.
__device__ __forceinline__ void raster_span(const RasterArgs &a, const RasterSide &S, const TriRec &r, const int4 &b,
                                            int p0, int p1, int lane) {
    const int bw = b.y - b.x + 1;
    int p = p0 + lane;
    int y = b.z + p / bw, x = b.x + (p - (p / bw) * bw);
    const int dy = 32 / bw, dx = 32 - dy * bw;
    for (; p < p1; p += 32) {
        if (r.A[0] * x + r.B[0] * y + r.C[0] > 0 && r.A[1] * x + r.B[1] * y + r.C[1] > 0 &&
            r.A[2] * x + r.B[2] * y + r.C[2] > 0) {
            const float t1 = __fmul_rn(r.fa, __int2float_rn(x));
            const float t2 = __fmul_rn(r.fb, __int2float_rn(y));
            const float mu = __fadd_rn(__fadd_rn(t1, t2), r.fc);
            const int dp = __float2int_rz(floorf(__fadd_rn(mu, 0.5f)));
            S.dplane[(size_t)y * a.w + x] = (int16_t)min(max(dp, a.dmin), a.dmax);
        }
        x += dx;
        y += dy;
        if (x > b.y) {
            x -= bw;
            ++y;
        }
    }
}

__device__ __forceinline__ void raster_draw_body(const RasterArgs &a, const VB &vb) {
    const RasterSide &S = a.s[vb.y];
    const int lane = threadIdx.x & 31;
    const int wid = vb.x * (blockDim.x >> 5) + (threadIdx.x >> 5), nwarps = vb.gx * (blockDim.x >> 5);
    const int ntri = side_ntri(S);
    const unsigned long long nextra = *S.nunits;
    const bool whole = nextra > (unsigned long long)a.unit_cap;  // the list is incomplete
    const int nunits = ntri + (whole ? 0 : (int)nextra);
    for (int u = wid; u < nunits; u += nwarps) {
        int t = u, c = 0;
        if (u >= ntri) {
            const int2 e = S.ulist[u - ntri];
            t = e.x;
            c = e.y;
        }
        const int4 b = S.rec[kRecWords * (size_t)t + 3];
        if (b.y < b.x || b.w < b.z) continue;
        const int area = (b.y - b.x + 1) * (b.w - b.z + 1);
        raster_span(a, S, load_rec(S.rec, t), b, c * kUnitPx, whole ? area : min(area, (c + 1) * kUnitPx), lane);
    }
}

__global__ void __launch_bounds__(256) raster_draw_kernel(RasterArgs a) { raster_draw_body(a, vb_single()); }
__global__ void __launch_bounds__(256) raster_draw_kernel_b(const RasterArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    raster_draw_body(slot_entry(tab, vm.stride, vb.slot), vb);
}


// Dense matching cost of two 16-byte descriptors added to acc: the SAD of
// Sobel descriptors, or the Hamming distance of dense census records
// (Sec. VI.A).  acc carries the key bias and, in the plane neighbourhood, the
// prior term, so the packed key is one multiply-add away.
template <bool CENSUS> __device__ __forceinline__ int dense_cost(const uint4 &a, const uint4 &b, int acc) {
    if (CENSUS) return acc + (int)ham16(a, b);
    uint32_t s = sad4_vacc(a.x, b.x, (uint32_t)acc);
    s = sad4_vacc(a.y, b.y, s);
    s = sad4_vacc(a.z, b.z, s);
    return (int)sad4_vacc(a.w, b.w, s);
}

// Packed key of a candidate: (cost + bias) * kKeyMul + d orders by (cost, d)
// as d <= kMaxDisp < kKeyMul; the multiplier is not a power of two so that
// the packing stays one integer multiply-add.
constexpr int kKeyMul = 2047;

// TPP = threads per pixel (1, 2 or 4): the TPP adjacent lanes of a pixel take
// every TPP-th candidate of its list and of its plane window and merge their
// keys with shuffles (min is order free, so every TPP gives the same result).
// GLIST: the cell's candidate list was expanded into global memory by the
// prior's list kernel (the CTA only waits for the prior table, at its
// start); else warp 0 expands the mask into shared memory first.
// PF: the reference descriptor and prior of a thread's next pixel are
// loaded while the current one is matched (batches, where a thread walks
// many pixels; one pair has one pixel per thread).
// WARPC: the cell belongs to one warp of the CTA (the persistent prior and
// argmin kernel runs kFusedCellWarps cells per CTA): the warp keeps its own
// list and prior table in shared memory and synchronises alone.
constexpr int kFusedThreads = 256;
constexpr int kFusedCellWarps = kFusedThreads / 32;

template <int TPP, bool CENSUS, bool GLIST, bool PF, bool WARPC = false>
__device__ __forceinline__ void cell_body(const CellArgs &a, const VB &vb) {
    constexpr int NG = WARPC ? kFusedCellWarps : 1;  // cell groups of the CTA
    __shared__ __align__(16) uint16_t s_list_g[NG][GLIST ? 1 : kMaxDisp + 1 + kListPad];
    __shared__ int s_P_g[NG][kMaxSradius + 1];
    __shared__ int s_nlist_g[NG];
    const int grp_of = WARPC ? (int)(threadIdx.x >> 5) : 0;
    uint16_t *s_list = s_list_g[grp_of];
    int *s_P = s_P_g[grp_of];
    int &s_nlist = s_nlist_g[grp_of];

    const CellSide &S = a.s[vb.z];
    const int W = a.w, H = a.h, G = a.G;
    const int dmin = a.dmin, dmax = a.dmax, sradius = a.sradius, full = a.full;
    const int cx = vb.x, cy = vb.y;
    const int x0 = cx * G, y0 = cy * G;
    const int cw = min(G, W - x0), ch = min(G, H - y0);
    const int npx = cw * ch;
    // threads of the cell: the CTA, or one warp
    const int tid = WARPC ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
    const int nthreads = WARPC ? 32 : (int)blockDim.x;
    const int lane = threadIdx.x & 31, warp = WARPC ? 0 : (int)(threadIdx.x >> 5);
    const int cell = cy * a.gw + cx;
    const uint4 *__restrict__ ref = S.ref;
    const uint4 *__restrict__ oth = S.oth;
    const int dir = S.dir;

    // the key bias with the prior term (none with the prior switched off)
    if (tid <= kMaxSradius) s_P[tid] = kKeyBias + (a.prior_off ? 0 : a.P[tid]);
    // ---- candidate list of the cell, ascending ---------------------------------
    const uint16_t *__restrict__ glist = GLIST ? S.clist + (size_t)cell * a.lstride : nullptr;
    if (!GLIST && !full && warp == 0) {
        const int n = expand_cell_list(S.grid + (size_t)cell * a.nw, a.nw, dmin, dmax, s_list, lane);
        if (lane == 0) s_nlist = n;
    }
    if (WARPC)
        __syncwarp();
    else
        __syncthreads();
    auto list_at = [&](int k) -> int { return GLIST ? (int)__ldg(glist + k) : (int)s_list[k]; };
    const int sub = TPP > 1 ? (tid & (TPP - 1)) : 0;

    // ---- per-pixel argmin -------------------------------------------------------
    // pixel p of the cell is (x0 + p % cw, y0 + p / cw); a thread's pixels
    // advance by ppb, so after one division the position steps incrementally
    const int ppb = nthreads / TPP;  // pixels per pass of the cell's threads
    const int sdy = ppb / cw, sdx = ppb - sdy * cw;
    int px = (tid / TPP) % cw, py = (tid / TPP) / cw;
    auto inner = [&](int qx, int qy) { return qx >= 2 && qx <= W - 3 && qy >= 2 && qy <= H - 3; };
    uint4 r_nx = make_uint4(0u, 0u, 0u, 0u);
    int dp_nx = -1;
    if (PF && tid / TPP < npx && inner(x0 + px, y0 + py)) {
        const size_t i0 = (size_t)(y0 + py) * W + x0 + px;
        r_nx = __ldg(ref + i0);
        if (!full) dp_nx = (int)__ldcg(S.dplane + i0);
    }
    for (int pb = 0; pb < npx; pb += ppb) {
        const int p = pb + tid / TPP;
        const bool live = p < npx;
        const int x = x0 + px, y = y0 + py;
        const size_t row = (size_t)y * W;
        const bool in = live && inner(x, y);
        uint4 r = r_nx;
        int dp = full ? -1 : dp_nx;
        if (!PF && in) {
            r = __ldg(ref + row + x);
            if (!full) dp = (int)__ldcg(S.dplane + row + x);
        }
        // the next pixel's position and loads
        px += sdx;
        py += sdy;
        if (px >= cw) {
            px -= cw;
            ++py;
        }
        if (PF && p + ppb < npx && inner(x0 + px, y0 + py)) {
            const size_t i1 = (size_t)(y0 + py) * W + x0 + px;
            r_nx = __ldg(ref + i1);
            if (!full) dp_nx = (int)__ldcg(S.dplane + i1);
        }
        int best = 0x7FFFFFFF;
        // the list length, read after the pixel's own loads so that they are
        // in flight together
        const int nlist = full ? 0 : (GLIST ? __ldg(S.ccount + cell) : s_nlist);
        // census records have no texture measure: no texture test
        if (in && (CENSUS || (int)texture16(r) >= a.match_texture) && (full || dp >= 0)) {
            // admissible d: 2 <= x + dir*d <= w-3 and d <= dmax, i.e. d <= dlim
            // (the lower bound of the first condition is <= 0; the list's
            // padding value 2047 exceeds every dmax)
            const int dlim = min(dmax, dir < 0 ? x - 2 : W - 3 - x);
            const uint4 *orow = oth + row + x;
            if (full) {
                for (int d = dmin + sub; d <= dlim; d += TPP) {  // no plane, so no prior term
                    best = min(best, dense_cost<CENSUS>(r, __ldg(orow + dir * d), kKeyBias) * kKeyMul + d);
                }
            } else {
                // the admissible entries are a prefix of the ascending list:
                // entries above dlim (only near the image border) are skipped
                // by a predicate, so the load of an inadmissible d never
                // issues; the batched census kernel finds the prefix's end by
                // bisection instead (the predicate costs it registers)
                constexpr bool kBisect = CENSUS && !GLIST;
                int cnt = nlist;
                if (kBisect && nlist > 0 && dlim < list_at(nlist - 1)) {
                    int lo = 0, hi = nlist;  // first entry above dlim
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (list_at(mid) <= dlim)
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    cnt = lo;
                }
#pragma unroll 8
                for (int k = sub; k < cnt; k += TPP) {
                    const int d = list_at(k);
                    if (kBisect || d <= dlim)
                        best = min(best, dense_cost<CENSUS>(r, __ldg(orow + dir * d), kKeyBias) * kKeyMul + d);
                }
                // the plane neighbourhood, the prior term in the accumulator
                const int lo = max(dmin, dp - sradius), hi = min(dlim, dp + sradius);
#pragma unroll 5
                for (int d = lo + sub; d <= hi; d += TPP)
                    best = min(best, dense_cost<CENSUS>(r, __ldg(orow + dir * d), s_P[abs(d - dp)]) * kKeyMul + d);
            }
        }
        if (TPP > 1) {
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
        }
        if (live && sub == 0) S.out[row + x] = (int16_t)(best != 0x7FFFFFFF ? (best % kKeyMul) : -1);
    }
}

template <bool CENSUS, bool GLIST> __global__ void __launch_bounds__(1024, 2) cell_kernel(CellArgs a) {
    cell_body<1, CENSUS, GLIST, false>(a, vb_single());
}

// Batched launches: one launch per cost kind among the pairs.
template <int TPP, bool CENSUS>
__global__ void __launch_bounds__(1024) cell_kernel_b(const CellArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    cell_body<TPP, CENSUS, false, true>(slot_entry(tab, vm.stride, vb.slot), vb);
}

template <bool CENSUS>
static void cell_launch_b(const CellArgs *tab, const VMap &m, int tpp, int threads, cudaStream_t st) {
    const int total = vmap_total(m);
    if (tpp == 1)
        cell_kernel_b<1, CENSUS><<<total, threads, 0, st>>>(tab, m);
    else if (tpp == 2)
        cell_kernel_b<2, CENSUS><<<total, threads, 0, st>>>(tab, m);
    else
        cell_kernel_b<4, CENSUS><<<total, threads, 0, st>>>(tab, m);
}

// ---------------------------------------------------------------------------
// Persistent prior + argmin for a batch (one cooperative launch): the CTAs
// walk the setup blocks of every pair, meet at a grid barrier, the list
// blocks, a barrier, the draw blocks, a barrier, then the cells, one warp
// per cell (kFusedCellWarps cells per item).  The bodies are those of the
// separate launches, so the maps are the same; every value one stage writes
// and a later one reads is read through L2 or with plain loads after the
// barrier.
// ---------------------------------------------------------------------------
struct DenseFusedArgs {
    const RasterArgs *rtab;
    const CellArgs *ctab;
    VMap setup, list, draw;
    VMap cells[2];  // Sobel/SAD and census pairs: items of kFusedCellWarps cells
};

// Cells of item b of `m`: warp k takes cell kFusedCellWarps * item + k of
// the pair's cells (both reference images, left first).
template <int TPP, bool CENSUS>
__device__ __forceinline__ void fused_cells(const DenseFusedArgs &f, const VMap &m, int b) {
    const VB vb = vb_at(m, b);
    const CellArgs &a = slot_entry(f.ctab, m.stride, vb.slot);
    const int gh = (a.h + a.G - 1) / a.G, per_side = a.gw * gh;
    const int c = vb.x * kFusedCellWarps + (int)(threadIdx.x >> 5);
    if (c >= 2 * per_side) return;
    VB w;
    w.slot = vb.slot;
    w.z = c / per_side;
    const int r = c - w.z * per_side;
    w.y = r / a.gw;
    w.x = r - w.y * a.gw;
    w.gx = a.gw;
    w.gy = gh;
    w.gz = 2;
    cell_body<TPP, CENSUS, false, true, true>(a, w);
}

template <int TPP> __global__ void __launch_bounds__(kFusedThreads, 4) dense_fused_kernel_b(DenseFusedArgs f) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    const int nb = gridDim.x;
    for (int b = blockIdx.x; b < vmap_total(f.setup); b += nb) {
        const VB vb = vb_at(f.setup, b);
        raster_setup_body(slot_entry(f.rtab, f.setup.stride, vb.slot), vb);
    }
    grid.sync();
    for (int b = blockIdx.x; b < vmap_total(f.list); b += nb) {
        const VB vb = vb_at(f.list, b);
        raster_list_body(slot_entry(f.rtab, f.list.stride, vb.slot), vb);
    }
    grid.sync();
    for (int b = blockIdx.x; b < vmap_total(f.draw); b += nb) {
        const VB vb = vb_at(f.draw, b);
        raster_draw_body(slot_entry(f.rtab, f.draw.stride, vb.slot), vb);
    }
    grid.sync();
    for (int b = blockIdx.x; b < vmap_total(f.cells[0]); b += nb) fused_cells<TPP, false>(f, f.cells[0], b);
    for (int b = blockIdx.x; b < vmap_total(f.cells[1]); b += nb) fused_cells<TPP, true>(f, f.cells[1], b);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

int max_triangles(int w, int h, const elas_params *p) {
    return 2 * (w / p->candidate_stepsize) * (h / p->candidate_stepsize) + 8;
}

static elas_status fill_prior_table(const elas_params *p, int *P) {
    for (int k = 0; k <= kMaxSradius; ++k) P[k] = 0;
    prior_table(p, P);
    for (int k = 0; k <= p->sradius; ++k)
        if (P[k] < -(kKeyBias - 1) || P[k] > kKeyBias - 1)
            return fail(ELAS_ERR_INVALID_ARG, "prior P[%d] = %d outside +-65535 (beta too small)", k, P[k]);
    return ELAS_OK;
}

// Entries of a mesh's list of extra units for at most tri_cap triangles:
// most boxes are one unit; very thin triangles near the hull have many.
static int raster_unit_cap(int tri_cap) { return 8 * (tri_cap > 0 ? tri_cap : 1) + 4096; }

// Scratch of one mesh: records, unit counts, list of extra units, its count.
static size_t raster_side_bytes(int tri_cap) {
    const size_t cap = (size_t)(tri_cap > 0 ? tri_cap : 1);
    return align_up(sizeof(int4) * kRecWords * cap, 256) + align_up(sizeof(int32_t) * cap, 256) +
           align_up(sizeof(int2) * (size_t)raster_unit_cap(tri_cap), 256) + 256;
}

size_t raster_scratch_bytes(int tri_cap, int nsides) { return (size_t)nsides * raster_side_bytes(tri_cap); }

// Argument block for nsides meshes of at most tri_cap triangles each, their
// scratch carved from `scratch` (raster_scratch_bytes bytes, 256-aligned).
static RasterArgs raster_args(const int16_t *list, const RasterSide *sides, int nsides, int w, int h,
                              const elas_params *p, void *scratch, int tri_cap) {
    RasterArgs a{};
    const size_t cap = (size_t)(tri_cap > 0 ? tri_cap : 1);
    a.list = list;
    a.nsides = nsides;
    a.w = w;
    a.h = h;
    a.dmin = p->disp_min;
    a.dmax = p->disp_max;
    a.unit_cap = raster_unit_cap(tri_cap);
    char *q = reinterpret_cast<char *>(scratch);
    for (int i = 0; i < nsides; ++i) {
        a.s[i] = sides[i];
        a.s[i].rec = reinterpret_cast<int4 *>(q);
        q += align_up(sizeof(int4) * kRecWords * cap, 256);
        a.s[i].ucnt = reinterpret_cast<int32_t *>(q);
        q += align_up(sizeof(int32_t) * cap, 256);
        a.s[i].ulist = reinterpret_cast<int2 *>(q);
        q += align_up(sizeof(int2) * (size_t)a.unit_cap, 256);
        a.s[i].nunits = reinterpret_cast<unsigned long long *>(q);
        q += 256;
    }
    return a;
}

static int raster_max_ntri(const RasterArgs &a) {
    int maxt = 0;
    for (int i = 0; i < a.nsides; ++i) maxt = max(maxt, a.s[i].ntri);
    return maxt;
}

// Grid of the setup kernel (per side: the larger of the pixel fill and the
// triangles, grid-stride) and of the draw kernel (warps over units).
static int raster_setup_blocks(const RasterArgs &a, int cap_blocks) {
    const long long n = max((long long)a.w * a.h, (long long)raster_max_ntri(a));
    return (int)max(1LL, min((n + 255) / 256, (long long)cap_blocks));
}

// Prior maps of one or two meshes.
static elas_status raster_meshes(const RasterArgs &a, cudaStream_t st) {
    raster_setup_kernel<<<dim3(raster_setup_blocks(a, sm_count() * 4), a.nsides), 256, 0, st>>>(a);
    raster_list_kernel<<<dim3(raster_setup_blocks(a, sm_count() * 4), a.nsides), 256, 0, st>>>(a);
    raster_draw_kernel<<<dim3(sm_count() * 4, a.nsides), 256, 0, st>>>(a);
    return launch_status("plane prior kernels");
}

static CellArgs cell_args(int w, int h, const elas_params *p, const int *P) {
    CellArgs a{};
    const GridGeom g = grid_geom(w, h, p);
    a.w = w;
    a.h = h;
    a.G = p->grid_size;
    a.gw = g.gw;
    a.nw = g.nw;
    a.dmin = p->disp_min;
    a.dmax = p->disp_max;
    a.sradius = p->sradius;
    a.match_texture = p->match_texture;
    a.full = (p->test_flags & ELAS_FLAG_FULL_RANGE) ? 1 : 0;
    a.prior_off = (p->test_flags & ELAS_FLAG_PRIOR_OFF) ? 1 : 0;
    a.census = p->census_dense_w > 0 ? 1 : 0;
    for (int k = 0; k <= kMaxSradius; ++k) a.P[k] = P[k];
    return a;
}

// Threads of a cell CTA: tpp per pixel of a G x G cell, each thread (group)
// taking ppt pixels in turn, at most 1024.
int cell_threads(int G, int tpp, int ppt) {
    const int t = ((G * G + ppt - 1) / ppt * tpp + 31) / 32 * 32;
    return t < 32 ? 32 : (t > 1024 ? 1024 : t);
}

dim3 cell_grid(const CellArgs &a, int nsides) {
    return dim3((a.w + a.G - 1) / a.G, (a.h + a.G - 1) / a.G, nsides);
}

static elas_status launch_cells(const CellArgs &a, int nsides, cudaStream_t st) {
    const dim3 grid = cell_grid(a, nsides);
    const int threads = cell_threads(a.G, 1, 1);
    if (a.lstride > 0) {
        if (a.census)
            cell_kernel<true, true><<<grid, threads, 0, st>>>(a);
        else
            cell_kernel<false, true><<<grid, threads, 0, st>>>(a);
    } else if (a.census) {
        cell_kernel<true, false><<<grid, threads, 0, st>>>(a);
    } else {
        cell_kernel<false, false><<<grid, threads, 0, st>>>(a);
    }
    return launch_status("cell_kernel");
}

elas_status launch_plane_prior(const int16_t *list, const int32_t *tri, int ntri, int right, int w, int h,
                               const elas_params *p, int16_t *dplane, void *scratch, cudaStream_t st) {
    RasterSide side{};
    side.tri = tri;
    side.ntri = ntri;
    side.right = right ? 1 : 0;
    side.dplane = dplane;
    return raster_meshes(raster_args(list, &side, 1, w, h, p, scratch, ntri), st);
}

elas_status launch_dense(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                         const int16_t *dplane, const uint32_t *grid, int right, int16_t *out, cudaStream_t st) {
    int P[kMaxSradius + 1];
    elas_status s = fill_prior_table(p, P);
    if (s != ELAS_OK) return s;
    CellArgs a = cell_args(w, h, p, P);
    CellSide &cs = a.s[0];
    cs.ref = reinterpret_cast<const uint4 *>(right ? descR : descL);
    cs.oth = reinterpret_cast<const uint4 *>(right ? descL : descR);
    cs.grid = grid;
    cs.dplane = dplane;
    cs.out = out;
    cs.dir = right ? +1 : -1;
    return launch_cells(a, 1, st);
}

// Stride of a cell's candidate list: every disparity of the mask and the padding.
static int cell_list_stride(const GridGeom &g) { return 32 * g.nw + kListPad; }

// The cells' candidate lists of both sides, then their counts.
static size_t cell_lists_bytes(int w, int h, const elas_params *p) {
    const GridGeom g = grid_geom(w, h, p);
    const size_t ncell = (size_t)g.gw * g.gh;
    return 2 * align_up(sizeof(uint16_t) * ncell * cell_list_stride(g), 256) +
           2 * align_up(sizeof(int32_t) * ncell, 256);
}

size_t dense_workspace(int w, int h, const elas_params *p) {
    return align_up(2 * (size_t)w * h * sizeof(int16_t), 256) + raster_scratch_bytes(max_triangles(w, h, p), 2) +
           cell_lists_bytes(w, h, p);
}

elas_status dense_args(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                       const int16_t *list, const int32_t *triL, int ntriL, const int32_t *triR, int ntriR,
                       const uint32_t *gridL, const uint32_t *gridR, int16_t *dL, int16_t *dR, void *ws,
                       const int32_t *ntri_dev, DenseStage *o, bool cell_lists) {
    int16_t *dpL = reinterpret_cast<int16_t *>(ws);
    int16_t *dpR = dpL + (size_t)w * h;
    RasterSide sides[2] = {};
    sides[0].tri = triL;
    sides[0].ntri = ntriL;
    sides[0].dplane = dpL;
    sides[0].ntri_dev = ntri_dev;
    sides[1].tri = triR;
    sides[1].ntri = ntriR;
    sides[1].right = 1;
    sides[1].dplane = dpR;
    sides[1].ntri_dev = ntri_dev ? ntri_dev + 1 : nullptr;
    char *scratch = reinterpret_cast<char *>(ws) + align_up(2 * (size_t)w * h * sizeof(int16_t), 256);
    // the cells' candidate lists after the rasteriser's scratch: with
    // cell_lists the prior's list kernel expands them and the argmin reads
    // them (one pair: no CTA waits for its list); batches keep the
    // expansion in each cell's CTA (one warp per cell there, so no wait)
    const GridGeom gg = grid_geom(w, h, p);
    const size_t ncell = (size_t)gg.gw * gg.gh;
    const int lstride = cell_list_stride(gg);
    char *lists = scratch + raster_scratch_bytes(max_triangles(w, h, p), 2);
    uint16_t *clist[2];
    int32_t *ccount[2];
    for (int i = 0; i < 2; ++i) {
        clist[i] = reinterpret_cast<uint16_t *>(lists);
        lists += align_up(sizeof(uint16_t) * ncell * lstride, 256);
    }
    for (int i = 0; i < 2; ++i) {
        ccount[i] = reinterpret_cast<int32_t *>(lists);
        lists += align_up(sizeof(int32_t) * ncell, 256);
    }
    for (int i = 0; i < 2; ++i) {
        sides[i].grid = i ? gridR : gridL;
        sides[i].clist = clist[i];
        sides[i].ccount = ccount[i];
    }
    o->raster = raster_args(list, sides, 2, w, h, p, scratch, max_triangles(w, h, p));
    o->raster.gw = gg.gw;
    o->raster.gh = gg.gh;
    o->raster.nw = gg.nw;
    o->raster.lstride = cell_lists ? lstride : 0;
    int P[kMaxSradius + 1];
    elas_status s = fill_prior_table(p, P);
    if (s != ELAS_OK) return s;
    o->cell = cell_args(w, h, p, P);
    o->cell.lstride = cell_lists ? lstride : 0;
    for (int i = 0; i < 2; ++i) {
        CellSide &cs = o->cell.s[i];
        cs.ref = reinterpret_cast<const uint4 *>(i ? descR : descL);
        cs.oth = reinterpret_cast<const uint4 *>(i ? descL : descR);
        cs.grid = i ? gridR : gridL;
        cs.dplane = i ? dpR : dpL;
        cs.out = i ? dR : dL;
        cs.dir = i ? +1 : -1;
        cs.clist = clist[i];
        cs.ccount = ccount[i];
    }
    return ELAS_OK;
}

elas_status launch_dense_both(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                              const int16_t *list, const int32_t *triL, int ntriL, const int32_t *triR, int ntriR,
                              const uint32_t *gridL, const uint32_t *gridR, int16_t *dL, int16_t *dR, void *ws,
                              cudaStream_t st, const int32_t *ntri_dev, cudaEvent_t after_prior) {
    DenseStage d;
    elas_status s = dense_args(descL, descR, w, h, p, list, triL, ntriL, triR, ntriR, gridL, gridR, dL, dR, ws,
                               ntri_dev, &d, true);
    if (s != ELAS_OK) return s;
    if ((s = raster_meshes(d.raster, st)) != ELAS_OK) return s;
    if (after_prior && record_mark(after_prior, st) != cudaSuccess) return launch_status("prior mark");
    return launch_cells(d.cell, 2, st);
}

// Batched plane prior and dense matching over the pairs of `pairs`; host
// is the host copy of the table.
// The persistent kernel for threads-per-pixel tpp: CTAs resident at once
// (every CTA of a cooperative launch must be), queried once per device.
template <int TPP> static int fused_blocks() {
    static int per_sm[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && per_sm[dev] == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dense_fused_kernel_b<TPP>, kFusedThreads, 0) !=
            cudaSuccess)
            n = 0;
        per_sm[dev] = n;
    }
    return (dev >= 0 && dev < 64 ? per_sm[dev] : 0) * sm_count();
}

template <int TPP> static elas_status launch_fused(DenseFusedArgs &f, cudaStream_t st) {
    const int blocks = fused_blocks<TPP>();
    if (blocks <= 0) return fail(ELAS_ERR_CUDA, "no resident CTA for the persistent dense kernel");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, dense_fused_kernel_b<TPP>, f) != cudaSuccess) return launch_status("dense_fused_kernel_b");
    return launch_status("dense_fused_kernel_b");
}

elas_status launch_dense_b(const DenseTables &t, const DenseStage *host, const VMap &pairs, int tpp, int ppt,
                           cudaStream_t st, cudaEvent_t after_prior, bool fused) {
    if (pairs.n == 0) return ELAS_OK;
    if (tpp != 1 && tpp != 2 && tpp != 4) return fail(ELAS_ERR_INVALID_ARG, "dense threads per pixel %d", tpp);
    if (ppt != 1 && ppt != 2 && ppt != 4 && ppt != 8 && ppt != 16)
        return fail(ELAS_ERR_INVALID_ARG, "dense pixels per thread %d", ppt);
    VMap m_setup, m_list, m_draw, m_cell[2];
    vmap_clear(m_setup, pairs.stride);
    vmap_clear(m_list, pairs.stride);
    vmap_clear(m_draw, pairs.stride);
    vmap_clear(m_cell[0], pairs.stride);
    vmap_clear(m_cell[1], pairs.stride);
    // per pair: the one-pair grids shared out among the pairs, at least 16 CTAs
    const int per_pair = max(16, sm_count() * 4 / pairs.n);
    int threads = 32;
    for (int i = 0; i < pairs.n; ++i) {
        const int slot = pairs.slot[i];
        const DenseStage &d = slot_entry(host, pairs.stride, slot);
        const RasterArgs &r = d.raster;
        vmap_add(m_setup, slot, dim3(raster_setup_blocks(r, per_pair), r.nsides));
        vmap_add(m_list, slot, dim3(raster_setup_blocks(r, per_pair), r.nsides));
        vmap_add(m_draw, slot, dim3(per_pair, r.nsides));
        vmap_add(m_cell[d.cell.census ? 1 : 0], slot, cell_grid(d.cell, 2));
        threads = max(threads, cell_threads(d.cell.G, tpp, ppt));
    }
    if (fused) {
        // one persistent launch: the prior and the argmin, one warp per cell
        DenseFusedArgs f;
        f.rtab = t.raster;
        f.ctab = t.cell;
        f.setup = m_setup;
        f.list = m_list;
        f.draw = m_draw;
        vmap_clear(f.cells[0], pairs.stride);
        vmap_clear(f.cells[1], pairs.stride);
        for (int i = 0; i < pairs.n; ++i) {
            const DenseStage &d = slot_entry(host, pairs.stride, pairs.slot[i]);
            const dim3 g = cell_grid(d.cell, 2);
            vmap_add(f.cells[d.cell.census ? 1 : 0], pairs.slot[i],
                     dim3((g.x * g.y * g.z + kFusedCellWarps - 1) / kFusedCellWarps));
        }
        elas_status s = tpp == 1 ? launch_fused<1>(f, st) : (tpp == 2 ? launch_fused<2>(f, st) : launch_fused<4>(f, st));
        if (s != ELAS_OK) return s;
        // the prior and the argmin share the launch: the mark follows it
        if (after_prior && record_mark(after_prior, st) != cudaSuccess) return launch_status("prior mark");
        return ELAS_OK;
    }
    raster_setup_kernel_b<<<vmap_total(m_setup), 256, 0, st>>>(t.raster, m_setup);
    raster_list_kernel_b<<<vmap_total(m_list), 256, 0, st>>>(t.raster, m_list);
    raster_draw_kernel_b<<<vmap_total(m_draw), 256, 0, st>>>(t.raster, m_draw);
    elas_status s = launch_status("batched plane prior");
    if (s != ELAS_OK) return s;
    if (after_prior && record_mark(after_prior, st) != cudaSuccess) return launch_status("prior mark");
    if (m_cell[0].n > 0) cell_launch_b<false>(t.cell, m_cell[0], tpp, threads, st);
    if (m_cell[1].n > 0) cell_launch_b<true>(t.cell, m_cell[1], tpp, threads, st);
    return launch_status("cell_kernel_b");
}

}  // namespace elas

extern "C" size_t elas_plane_prior_workspace_bytes(int32_t ntri) {
    return ntri < 0 ? 0 : elas::raster_scratch_bytes(ntri, 1);
}

extern "C" elas_status elas_plane_prior(const int16_t *list, int32_t n, const int32_t *tri, int32_t ntri,
                                        int32_t right, int32_t w, int32_t h, const elas_params *p,
                                        int16_t *d_plane, void *workspace, size_t workspace_bytes,
                                        elas_stream stream) {
    using namespace elas;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (!d_plane || !workspace || (ntri > 0 && (!list || !tri))) return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (n < 0 || ntri < 0) return fail(ELAS_ERR_INVALID_ARG, "negative count");
    if (ntri >= (1 << 30)) return fail(ELAS_ERR_INVALID_ARG, "too many triangles");
    if (!aligned(workspace, 256)) return fail(ELAS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (workspace_bytes < raster_scratch_bytes(ntri, 1))
        return fail(ELAS_ERR_CAPACITY, "workspace %zu < %zu bytes", workspace_bytes, raster_scratch_bytes(ntri, 1));
    return launch_plane_prior(list, tri, ntri, right, w, h, p, d_plane, workspace, to_stream(stream));
}

extern "C" elas_status elas_dense_argmin(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                                         const elas_params *p, const int16_t *d_plane, const uint32_t *grid,
                                         int32_t right, int16_t *out, elas_stream stream) {
    using namespace elas;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (!descL || !descR || !out) return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (!(p->test_flags & ELAS_FLAG_FULL_RANGE) && (!d_plane || !grid))
        return fail(ELAS_ERR_INVALID_ARG, "d_plane and grid are required without ELAS_FLAG_FULL_RANGE");
    if (!aligned(descL, 16) || !aligned(descR, 16)) return fail(ELAS_ERR_INVALID_ARG, "descriptors not 16-byte aligned");
    return launch_dense(descL, descR, w, h, p, d_plane, grid, right, out, to_stream(stream));
}

extern "C" size_t elas_dense_workspace_bytes(int32_t w, int32_t h, const elas_params *p) {
    if (elas::check_params(p, w, h) != ELAS_OK) return 0;
    return elas::dense_workspace(w, h, p);
}

extern "C" elas_status elas_dense_match(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                                        const elas_params *p, const int16_t *list, int32_t n, const int32_t *triL,
                                        int32_t ntriL, const int32_t *triR, int32_t ntriR,
                                        const uint32_t *grid_L, const uint32_t *grid_R, int16_t *dL, int16_t *dR,
                                        void *workspace, size_t workspace_bytes, elas_stream stream) {
    using namespace elas;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (!descL || !descR || !grid_L || !grid_R || !dL || !dR || !workspace)
        return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if ((ntriL > 0 || ntriR > 0) && !list) return fail(ELAS_ERR_INVALID_ARG, "NULL support list");
    if ((ntriL > 0 && !triL) || (ntriR > 0 && !triR)) return fail(ELAS_ERR_INVALID_ARG, "NULL triangles");
    if (n < 0 || ntriL < 0 || ntriR < 0) return fail(ELAS_ERR_INVALID_ARG, "negative count");
    if (ntriL > max_triangles(w, h, p) || ntriR > max_triangles(w, h, p))
        return fail(ELAS_ERR_CAPACITY, "triangle counts %d/%d above %d", ntriL, ntriR, max_triangles(w, h, p));
    if (!aligned(descL, 16) || !aligned(descR, 16)) return fail(ELAS_ERR_INVALID_ARG, "descriptors not 16-byte aligned");
    if (!aligned(workspace, 256)) return fail(ELAS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (workspace_bytes < dense_workspace(w, h, p))
        return fail(ELAS_ERR_CAPACITY, "workspace %zu < %zu bytes", workspace_bytes, dense_workspace(w, h, p));
    return launch_dense_both(descL, descR, w, h, p, list, triL, ntriL, triR, ntriR, grid_L, grid_R, dL, dR,
                             workspace, to_stream(stream), nullptr);
}
