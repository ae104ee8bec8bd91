// Slanted-plane prior (Sec. III.A; image-sized prior matrix, Sec. VI.D) and
// dense per-pixel argmin of descriptor SAD plus tabulated prior over the
// grid-vector and plane-neighbourhood candidates (Sec. III.A, Fig. 1(h)).
//
// plane_raster_kernel  eight lanes per triangle (four in batches of two or
//                      more pairs; grid-stride), both meshes in one launch.
//                      Every lane evaluates the FP32 plane in the fixed
//                      order.  The lanes tile the bounding box
//                      (up to eight across x, the rest over rows) and
//                      write a pixel when the three integer edge functions
//                      own it (E >= 0 on owned edges, E >= 1 otherwise), so
//                      ownership is exactly the top-left rule.  Triangles
//                      whose bounding box exceeds kBigAreaOne (one pair) or
//                      kBigAreaBatch pixels are listed
//                      instead (in up to kBigSplit parts) and drawn by
//                      plane_raster_big_kernel, one CTA per part (rows over
//                      warps, lanes across x; there the owned x-range of a
//                      row, widened by one, follows from the edge functions
//                      first), so they leave no tail.
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
#include "launch.cuh"

namespace elas {

constexpr int kKeyBias = 65536;  // keeps (cost + bias) positive; |P| <= 65535

__device__ __forceinline__ bool edge_owned(int px, int py, int qx, int qy) {
    return (qy == py && qx > px) || (qy < py);
}

__device__ __forceinline__ int floor_div(int n, int d) {  // d > 0
    const int q = n / d;
    return (n % d != 0 && n < 0) ? q - 1 : q;
}
__device__ __forceinline__ int ceil_div(int n, int d) {  // d > 0
    const int q = n / d;
    return (n % d != 0 && n > 0) ? q + 1 : q;
}

// Narrows [lo, hi] to the x where edge (px,py)->(qx,qy) admits row y.
__device__ __forceinline__ void edge_span(int px, int py, int qx, int qy, int own, int y, int &lo, int &hi) {
    const int A = py - qy;
    const int B = (qx - px) * (y - py) + (qy - py) * px;
    const int t = own ? 0 : 1;
    if (A > 0)
        lo = max(lo, ceil_div(t - B, A));
    else if (A < 0)
        hi = min(hi, floor_div(B - t, -A));
    else if (B < t)
        hi = lo - 1;
}


__device__ __forceinline__ int side_ntri(const RasterSide &S) {
    return S.ntri_dev ? max(0, *S.ntri_dev) : S.ntri;
}


// bounding-box pixels above which a triangle is "big": one pair (latency:
// shorter tails in the small-triangle kernel) and batches (throughput)
constexpr int kBigAreaOne = 384;
constexpr int kBigAreaBatch = 2048;

// Plane and positively oriented integer edges of one triangle.
struct TriGeom {
    float fa, fb, fc;
    int ex0, ey0, ex1, ey1, ex2, ey2, o0, o1, o2;
    int xmin, xmax, ymin, ymax;
    bool empty;
};

__device__ __forceinline__ TriGeom tri_geom(const int16_t *__restrict__ list, const int32_t *__restrict__ tri, int t,
                                            int right, int w, int h) {
    TriGeom g;
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
    g.empty = det == 0;
    const float fdet = __int2float_rn(det == 0 ? 1 : det);
    g.fa = __fdiv_rn(__int2float_rn(na), fdet);
    g.fb = __fdiv_rn(__int2float_rn(nb), fdet);
    const float c = __fsub_rn(__int2float_rn(Z[0]), __fmul_rn(g.fa, __int2float_rn(X[0])));
    g.fc = __fsub_rn(c, __fmul_rn(g.fb, __int2float_rn(Y[0])));
    g.ex0 = X[0];
    g.ey0 = Y[0];
    g.ex1 = det > 0 ? X[1] : X[2];
    g.ey1 = det > 0 ? Y[1] : Y[2];
    g.ex2 = det > 0 ? X[2] : X[1];
    g.ey2 = det > 0 ? Y[2] : Y[1];
    g.o0 = edge_owned(g.ex0, g.ey0, g.ex1, g.ey1);
    g.o1 = edge_owned(g.ex1, g.ey1, g.ex2, g.ey2);
    g.o2 = edge_owned(g.ex2, g.ey2, g.ex0, g.ey0);
    g.xmin = max(0, min(X[0], min(X[1], X[2])));
    g.xmax = min(w - 1, max(X[0], max(X[1], X[2])));
    g.ymin = max(0, min(Y[0], min(Y[1], Y[2])));
    g.ymax = min(h - 1, max(Y[0], max(Y[1], Y[2])));
    if (g.xmax < g.xmin || g.ymax < g.ymin) g.empty = true;
    return g;
}

// Writes the owned pixels of row y of a triangle, x from `first` in steps of
// `stride` (lanes of a warp stride 32, a single thread strides 1).
__device__ __forceinline__ void raster_row(const TriGeom &g, int y, int first, int stride, int w, int dmin, int dmax,
                                           int16_t *__restrict__ dplane) {
    int lo = g.xmin, hi = g.xmax;
    edge_span(g.ex0, g.ey0, g.ex1, g.ey1, g.o0, y, lo, hi);
    edge_span(g.ex1, g.ey1, g.ex2, g.ey2, g.o1, y, lo, hi);
    edge_span(g.ex2, g.ey2, g.ex0, g.ey0, g.o2, y, lo, hi);
    lo = max(g.xmin, lo - 1);
    hi = min(g.xmax, hi + 1);
    for (int x = lo + first; x <= hi; x += stride) {
        const int e0 = (g.ex1 - g.ex0) * (y - g.ey0) - (g.ey1 - g.ey0) * (x - g.ex0);
        const int e1 = (g.ex2 - g.ex1) * (y - g.ey1) - (g.ey2 - g.ey1) * (x - g.ex1);
        const int e2 = (g.ex0 - g.ex2) * (y - g.ey2) - (g.ey0 - g.ey2) * (x - g.ex2);
        if (!((e0 > 0 || (e0 == 0 && g.o0)) && (e1 > 0 || (e1 == 0 && g.o1)) && (e2 > 0 || (e2 == 0 && g.o2))))
            continue;
        const float t1 = __fmul_rn(g.fa, __int2float_rn(x));
        const float t2 = __fmul_rn(g.fb, __int2float_rn(y));
        const float mu = __fadd_rn(__fadd_rn(t1, t2), g.fc);
        const int dp = __float2int_rz(floorf(__fadd_rn(mu, 0.5f)));
        dplane[(size_t)y * w + x] = (int16_t)min(max(dp, dmin), dmax);
    }
}

// Writes the owned pixels of a small triangle: the group's G lanes tile the
// bounding box as LX x LY (LX the least power of two >= its width, at most
// G), consecutive x on consecutive lanes (their stores are contiguous), and
// every pixel is confirmed with the three edge functions as in raster_row.
template <int G>
__device__ __forceinline__ void raster_box(const TriGeom &g, int gl, int w, int dmin, int dmax,
                                           int16_t *__restrict__ dplane) {
    const int bw = g.xmax - g.xmin + 1;
    const int LX = bw >= G ? G : (bw > G / 2 ? G : (bw > G / 4 ? G / 2 : (bw > 1 ? 2 : 1)));
    const int LY = G / LX, lx = gl % LX, ly = gl / LX;
    for (int y = g.ymin + ly; y <= g.ymax; y += LY) {
        for (int x = g.xmin + lx; x <= g.xmax; x += LX) {
            const int e0 = (g.ex1 - g.ex0) * (y - g.ey0) - (g.ey1 - g.ey0) * (x - g.ex0);
            const int e1 = (g.ex2 - g.ex1) * (y - g.ey1) - (g.ey2 - g.ey1) * (x - g.ex1);
            const int e2 = (g.ex0 - g.ex2) * (y - g.ey2) - (g.ey0 - g.ey2) * (x - g.ex2);
            if (!((e0 > 0 || (e0 == 0 && g.o0)) && (e1 > 0 || (e1 == 0 && g.o1)) && (e2 > 0 || (e2 == 0 && g.o2))))
                continue;
            const float t1 = __fmul_rn(g.fa, __int2float_rn(x));
            const float t2 = __fmul_rn(g.fb, __int2float_rn(y));
            const float mu = __fadd_rn(__fadd_rn(t1, t2), g.fc);
            const int dp = __float2int_rz(floorf(__fadd_rn(mu, 0.5f)));
            dplane[(size_t)y * w + x] = (int16_t)min(max(dp, dmin), dmax);
        }
    }
}

constexpr int kRasterGroup = 8;       // lanes per small triangle (one pair: shorter chains)
constexpr int kRasterGroupBatch = 4;  // lanes per small triangle in batches (more triangles in flight)
constexpr int kBigSplit = 8;          // CTAs a big triangle is spread over, at most

template <int RG> __device__ __forceinline__ void plane_raster_body(const RasterArgs &a, const VB &vb, int big_area) {
    const int side = vb.y;
    const RasterSide S = side ? a.s[1] : a.s[0];
    const int gl = threadIdx.x & (RG - 1);
    const int gpb = blockDim.x / RG;  // triangles per CTA pass
    const int ntri = side_ntri(S);
    for (int t = vb.x * gpb + (int)threadIdx.x / RG; t < ntri; t += vb.gx * gpb) {
        const TriGeom g = tri_geom(a.list, S.tri, t, S.right, a.w, a.h);
        if (g.empty) continue;
        const int rows = g.ymax - g.ymin + 1;
        if ((g.xmax - g.xmin + 1) * rows > big_area) {
            // drawn by plane_raster_big_kernel, split over up to kBigSplit CTAs
            const int nsub = min(kBigSplit, (rows + 31) / 32);
            if (gl == 0) {
                const int k = atomicAdd(a.nbig, nsub);
                for (int j = 0; j < nsub; ++j) a.big[k + j] = make_int2((side << 8) | (j << 4) | nsub, t);
            }
            continue;
        }
        raster_box<RG>(g, gl, a.w, a.dmin, a.dmax, S.dplane);
    }
}

__global__ void __launch_bounds__(256) plane_raster_kernel(RasterArgs a) {
    plane_raster_body<kRasterGroup>(a, vb_single(), kBigAreaOne);
}
template <int RG>
__global__ void __launch_bounds__(256) plane_raster_kernel_b(const RasterArgs *__restrict__ tab, VMap vm,
                                                             int big_area) {
    const VB vb = vb_batch(vm);
    plane_raster_body<RG>(slot_entry(tab, vm.stride, vb.slot), vb, big_area);
}

// Big triangles: each list entry is one of the nsub parts of a triangle, one
// CTA each (grid-stride over the list); part j takes the 8-row groups
// j, j + nsub, j + 2 nsub, ... whose rows go to the CTA's warps, lanes
// striding across x.
__device__ __forceinline__ void plane_raster_big_body(const RasterArgs &a, const VB &vb) {
    const int n = *a.nbig;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    for (int k = vb.x; k < n; k += vb.gx) {
        const int2 e = a.big[k];
        const int side = e.x >> 8, part = (e.x >> 4) & 15, nsub = e.x & 15, t = e.y;
        const RasterSide S = side ? a.s[1] : a.s[0];
        const TriGeom g = tri_geom(a.list, S.tri, t, S.right, a.w, a.h);
        const int rows = g.ymax - g.ymin + 1;
        for (int r0 = part * wpb; r0 < rows; r0 += nsub * wpb) {
            const int r = r0 + warp;
            if (r < rows) raster_row(g, g.ymin + r, lane, 32, a.w, a.dmin, a.dmax, S.dplane);
        }
    }
}

__global__ void __launch_bounds__(256) plane_raster_big_kernel(RasterArgs a) { plane_raster_big_body(a, vb_single()); }
__global__ void __launch_bounds__(256) plane_raster_big_kernel_b(const RasterArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    plane_raster_big_body(slot_entry(tab, vm.stride, vb.slot), vb);
}



constexpr int kListPad = 16;  // padding entries (2047) after the candidate list

// TPP = threads per pixel (1, 2 or 4): the TPP adjacent lanes of a pixel take
// every TPP-th candidate of its list and of its plane window and merge their
// keys with shuffles (min is order free, so every TPP gives the same result).
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

template <int TPP, bool CENSUS> __device__ __forceinline__ void cell_body(const CellArgs &a, const VB &vb) {
    __shared__ __align__(16) uint16_t s_list[kMaxDisp + 1 + kListPad];
    __shared__ int s_P[kMaxSradius + 1];
    __shared__ int s_nlist;

    const CellSide &S = a.s[vb.z];
    const int W = a.w, H = a.h, G = a.G;
    const int dmin = a.dmin, dmax = a.dmax, sradius = a.sradius, full = a.full;
    const int cx = vb.x, cy = vb.y;
    const int x0 = cx * G, y0 = cy * G;
    const int cw = min(G, W - x0), ch = min(G, H - y0);
    const int npx = cw * ch;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cell = cy * a.gw + cx;
    const uint4 *__restrict__ ref = S.ref;
    const uint4 *__restrict__ oth = S.oth;
    const int dir = S.dir;

    // the key bias with the prior term (none with the prior switched off)
    if (tid <= kMaxSradius) s_P[tid] = kKeyBias + (a.prior_off ? 0 : a.P[tid]);
    // ---- candidate list of the cell, ascending ---------------------------------
    if (!full && warp == 0) {
        const int nw = a.nw;
        const uint32_t *g = S.grid + (size_t)cell * nw;
        // the words are taken one at a time: lane l places bit l of the word
        // after the set bits below it, so the list comes out sorted with no
        // per-lane bit loop
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
                if ((mk >> lane) & 1u) s_list[base + __popc(mk & below)] = (uint16_t)(32 * (w0 + k) + lane);
                base += __popc(mk);
            }
        }
        // pad with a disparity above every dmax
        if (lane < kListPad) s_list[base + lane] = (uint16_t)2047;
        if (lane == 0) s_nlist = base;
    }
    __syncthreads();
    const int nlist = full ? 0 : s_nlist;
    const int dlast = nlist > 0 ? (int)s_list[nlist - 1] : -1;  // largest entry
    const int sub = TPP > 1 ? (tid & (TPP - 1)) : 0;

    // ---- per-pixel argmin -------------------------------------------------------
    // pixel p of the cell is (x0 + p % cw, y0 + p / cw); a thread's pixels
    // advance by ppb, so after one division the position steps incrementally
    const int ppb = blockDim.x / TPP;  // pixels per pass of the CTA
    const int sdy = ppb / cw, sdx = ppb - sdy * cw;
    int px = (tid / TPP) % cw, py = (tid / TPP) / cw;
    for (int pb = 0; pb < npx; pb += ppb) {
        const int p = pb + tid / TPP;
        int best = 0x7FFFFFFF;
        bool live = false;
        size_t row = 0;
        int x = 0;
        if (p < npx) {
            x = x0 + px;
            const int y = y0 + py;
            row = (size_t)y * W;
            live = true;
            if (x >= 2 && x <= W - 3 && y >= 2 && y <= H - 3) {
                const uint4 r = __ldg(ref + row + x);
                const int dp = full ? -1 : (int)__ldg(S.dplane + row + x);
                // census records have no texture measure: no texture test
                if ((CENSUS || (int)texture16(r) >= a.match_texture) && (full || dp >= 0)) {
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
                        // the admissible entries are a prefix of the ascending list
                        int cnt = nlist;
                        if (dlim < dlast) {
                            int lo = 0, hi = nlist;  // first entry above dlim
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if ((int)s_list[mid] <= dlim)
                                    lo = mid + 1;
                                else
                                    hi = mid;
                            }
                            cnt = lo;
                        }
#pragma unroll 8
                        for (int k = sub; k < cnt; k += TPP) {
                            const int d = s_list[k];
                            best = min(best, dense_cost<CENSUS>(r, __ldg(orow + dir * d), kKeyBias) * kKeyMul + d);
                        }
                        // the plane neighbourhood, the prior term in the accumulator
                        const int lo = max(dmin, dp - sradius), hi = min(dlim, dp + sradius);
#pragma unroll 5
                        for (int d = lo + sub; d <= hi; d += TPP)
                            best = min(best, dense_cost<CENSUS>(r, __ldg(orow + dir * d), s_P[abs(d - dp)]) * kKeyMul + d);
                    }
                }
            }
        }
        if (TPP > 1) {
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
        }
        if (live && sub == 0) S.out[row + x] = (int16_t)(best != 0x7FFFFFFF ? (best % kKeyMul) : -1);
        px += sdx;
        py += sdy;
        if (px >= cw) {
            px -= cw;
            ++py;
        }
    }
}

template <bool CENSUS> __global__ void __launch_bounds__(1024) cell_kernel(CellArgs a) {
    cell_body<1, CENSUS>(a, vb_single());
}

// Batched launches: one launch per cost kind among the pairs.
template <int TPP, bool CENSUS>
__global__ void __launch_bounds__(1024) cell_kernel_b(const CellArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    cell_body<TPP, CENSUS>(slot_entry(tab, vm.stride, vb.slot), vb);
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

// Scratch of the rasteriser: the big-triangle list (up to kBigSplit parts
// per triangle) and its counter.
size_t raster_scratch_bytes(int ntri_total) {
    return align_up(sizeof(int32_t) * 4, 256) +
           align_up(sizeof(int2) * kBigSplit * (size_t)(ntri_total > 0 ? ntri_total : 1), 256);
}

// Batched launches keep no memsets: this kernel fills the prior maps of a
// pair (both sides, contiguous) with -1 and clears its big-triangle count.
__device__ __forceinline__ void raster_init_body(const RasterArgs &a, const VB &vb) {
    const size_t n = (size_t)a.nsides * a.w * a.h;  // int16 entries
    int16_t *d = a.s[0].dplane;
    const size_t n8 = n / 8;
    uint4 *d8 = reinterpret_cast<uint4 *>(d);
    const size_t stride = (size_t)vb.gx * blockDim.x;
    const size_t t = (size_t)vb.x * blockDim.x + threadIdx.x;
    for (size_t i = t; i < n8; i += stride) d8[i] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    if (t < n - 8 * n8) d[8 * n8 + t] = -1;
    if (t == 0) *a.nbig = 0;
}

__global__ void __launch_bounds__(256) raster_init_kernel(RasterArgs a) { raster_init_body(a, vb_single()); }
__global__ void __launch_bounds__(256) raster_init_kernel_b(const RasterArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    raster_init_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

static RasterArgs raster_args(const int16_t *list, const RasterSide *sides, int nsides, int w, int h,
                              const elas_params *p, void *scratch) {
    RasterArgs a{};
    a.list = list;
    a.nsides = nsides;
    a.nbig = reinterpret_cast<int32_t *>(scratch);
    a.big = reinterpret_cast<int2 *>(reinterpret_cast<char *>(scratch) + align_up(sizeof(int32_t) * 4, 256));
    a.w = w;
    a.h = h;
    a.dmin = p->disp_min;
    a.dmax = p->disp_max;
    for (int i = 0; i < nsides; ++i) a.s[i] = sides[i];
    return a;
}

static int raster_max_ntri(const RasterArgs &a) {
    int maxt = 0;
    for (int i = 0; i < a.nsides; ++i) maxt = max(maxt, a.s[i].ntri);
    return maxt;
}

// Prior maps of one or two meshes.  With two, the maps must be contiguous
// (dplane1 == dplane0 + w*h) so that one pass clears both: raster_init_kernel
// (16-byte stores) when the maps are 16-byte aligned, else two memsets.
static elas_status raster_meshes(const RasterArgs &a, cudaStream_t st) {
    const size_t n = (size_t)a.w * a.h * a.nsides;  // int16 entries
    if (aligned(a.s[0].dplane, 16)) {
        const size_t blocks = (n / 8 + 255) / 256;
        const size_t cap_blocks = (size_t)sm_count() * 8;
        raster_init_kernel<<<(unsigned)(blocks < cap_blocks ? (blocks > 0 ? blocks : 1) : cap_blocks), 256, 0, st>>>(a);
        elas_status s0 = launch_status("raster_init_kernel");
        if (s0 != ELAS_OK) return s0;
    } else if (cudaMemsetAsync(a.s[0].dplane, 0xFF, n * sizeof(int16_t), st) != cudaSuccess ||
               cudaMemsetAsync(a.nbig, 0, sizeof(int32_t), st) != cudaSuccess) {
        return launch_status("memset d_plane");
    }
    const int maxt = raster_max_ntri(a);
    if (maxt == 0) return ELAS_OK;
    const int wpb = 256 / kRasterGroup;  // triangles per CTA pass
    int blocks = (maxt + wpb - 1) / wpb;
    if (blocks > sm_count() * 4) blocks = sm_count() * 4;
    plane_raster_kernel<<<dim3(blocks, a.nsides), 256, 0, st>>>(a);
    elas_status s = launch_status("plane_raster_kernel");
    if (s != ELAS_OK) return s;
    plane_raster_big_kernel<<<2 * sm_count(), 256, 0, st>>>(a);
    return launch_status("plane_raster_big_kernel");
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
    if (a.census)
        cell_kernel<true><<<cell_grid(a, nsides), cell_threads(a.G, 1, 1), 0, st>>>(a);
    else
        cell_kernel<false><<<cell_grid(a, nsides), cell_threads(a.G, 1, 1), 0, st>>>(a);
    return launch_status("cell_kernel");
}

elas_status launch_plane_prior(const int16_t *list, const int32_t *tri, int ntri, int right, int w, int h,
                               const elas_params *p, int16_t *dplane, void *scratch, cudaStream_t st) {
    RasterSide side{tri, ntri, right ? 1 : 0, dplane, nullptr};
    return raster_meshes(raster_args(list, &side, 1, w, h, p, scratch), st);
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

size_t dense_workspace(int w, int h, const elas_params *p) {
    return align_up(2 * (size_t)w * h * sizeof(int16_t), 256) + raster_scratch_bytes(2 * max_triangles(w, h, p));
}

elas_status dense_args(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                       const int16_t *list, const int32_t *triL, int ntriL, const int32_t *triR, int ntriR,
                       const uint32_t *gridL, const uint32_t *gridR, int16_t *dL, int16_t *dR, void *ws,
                       const int32_t *ntri_dev, DenseStage *o) {
    int16_t *dpL = reinterpret_cast<int16_t *>(ws);
    int16_t *dpR = dpL + (size_t)w * h;
    const RasterSide sides[2] = {{triL, ntriL, 0, dpL, ntri_dev ? ntri_dev : nullptr},
                                 {triR, ntriR, 1, dpR, ntri_dev ? ntri_dev + 1 : nullptr}};
    void *scratch = reinterpret_cast<char *>(ws) + align_up(2 * (size_t)w * h * sizeof(int16_t), 256);
    o->raster = raster_args(list, sides, 2, w, h, p, scratch);
    int P[kMaxSradius + 1];
    elas_status s = fill_prior_table(p, P);
    if (s != ELAS_OK) return s;
    o->cell = cell_args(w, h, p, P);
    for (int i = 0; i < 2; ++i) {
        CellSide &cs = o->cell.s[i];
        cs.ref = reinterpret_cast<const uint4 *>(i ? descR : descL);
        cs.oth = reinterpret_cast<const uint4 *>(i ? descL : descR);
        cs.grid = i ? gridR : gridL;
        cs.dplane = i ? dpR : dpL;
        cs.out = i ? dR : dL;
        cs.dir = i ? +1 : -1;
    }
    return ELAS_OK;
}

elas_status launch_dense_both(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                              const int16_t *list, const int32_t *triL, int ntriL, const int32_t *triR, int ntriR,
                              const uint32_t *gridL, const uint32_t *gridR, int16_t *dL, int16_t *dR, void *ws,
                              cudaStream_t st, const int32_t *ntri_dev, cudaEvent_t after_prior) {
    DenseStage d;
    elas_status s = dense_args(descL, descR, w, h, p, list, triL, ntriL, triR, ntriR, gridL, gridR, dL, dR, ws,
                               ntri_dev, &d);
    if (s != ELAS_OK) return s;
    if ((s = raster_meshes(d.raster, st)) != ELAS_OK) return s;
    if (after_prior && record_mark(after_prior, st) != cudaSuccess) return launch_status("prior mark");
    return launch_cells(d.cell, 2, st);
}

// Batched plane prior and dense matching over the pairs of `pairs`; host
// is the host copy of the table.
elas_status launch_dense_b(const DenseTables &t, const DenseStage *host, const VMap &pairs, int tpp, int ppt,
                           cudaStream_t st, cudaEvent_t after_prior) {
    if (pairs.n == 0) return ELAS_OK;
    if (tpp != 1 && tpp != 2 && tpp != 4) return fail(ELAS_ERR_INVALID_ARG, "dense threads per pixel %d", tpp);
    if (ppt != 1 && ppt != 2 && ppt != 4 && ppt != 8 && ppt != 16)
        return fail(ELAS_ERR_INVALID_ARG, "dense pixels per thread %d", ppt);
    VMap m_init, m_tri, m_big, m_cell[2];
    vmap_clear(m_init, pairs.stride);
    vmap_clear(m_tri, pairs.stride);
    vmap_clear(m_big, pairs.stride);
    vmap_clear(m_cell[0], pairs.stride);
    vmap_clear(m_cell[1], pairs.stride);
    int threads = 32;
    for (int i = 0; i < pairs.n; ++i) {
        const int slot = pairs.slot[i];
        const DenseStage &d = slot_entry(host, pairs.stride, slot);
        const size_t n8 = ((size_t)d.raster.nsides * d.raster.w * d.raster.h + 7) / 8;
        vmap_add(m_init, slot, dim3((unsigned)min((n8 + 255) / 256, (size_t)sm_count() * 4)));
        const int maxt = raster_max_ntri(d.raster);
        const int wpb = 256 / (pairs.n == 1 ? kRasterGroup : kRasterGroupBatch);
        int blocks = (maxt + wpb - 1) / wpb;
        if (pairs.n > 1) blocks = (blocks + 2) / 3;
        blocks = max(1, min(blocks, sm_count() * 16));
        vmap_add(m_tri, slot, dim3(blocks, d.raster.nsides));
        // big triangles: the one-pair launch's 2 CTAs per SM, shared by the pairs
        vmap_add(m_big, slot, dim3(max(32, 2 * sm_count() / pairs.n)));
        vmap_add(m_cell[d.cell.census ? 1 : 0], slot, cell_grid(d.cell, 2));
        threads = max(threads, cell_threads(d.cell.G, tpp, ppt));
    }
    raster_init_kernel_b<<<vmap_total(m_init), 256, 0, st>>>(t.raster, m_init);
    if (pairs.n == 1)
        plane_raster_kernel_b<kRasterGroup><<<vmap_total(m_tri), 256, 0, st>>>(t.raster, m_tri, kBigAreaOne);
    else
        plane_raster_kernel_b<kRasterGroupBatch><<<vmap_total(m_tri), 256, 0, st>>>(t.raster, m_tri, kBigAreaBatch);
    plane_raster_big_kernel_b<<<vmap_total(m_big), 256, 0, st>>>(t.raster, m_big);
    elas_status s = launch_status("batched plane prior");
    if (s != ELAS_OK) return s;
    if (after_prior && record_mark(after_prior, st) != cudaSuccess) return launch_status("prior mark");
    if (m_cell[0].n > 0) cell_launch_b<false>(t.cell, m_cell[0], tpp, threads, st);
    if (m_cell[1].n > 0) cell_launch_b<true>(t.cell, m_cell[1], tpp, threads, st);
    return launch_status("cell_kernel_b");
}

}  // namespace elas

extern "C" size_t elas_plane_prior_workspace_bytes(int32_t ntri) {
    return ntri < 0 ? 0 : elas::raster_scratch_bytes(ntri);
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
    if (workspace_bytes < raster_scratch_bytes(ntri))
        return fail(ELAS_ERR_CAPACITY, "workspace %zu < %zu bytes", workspace_bytes, raster_scratch_bytes(ntri));
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
