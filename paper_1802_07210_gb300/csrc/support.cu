// Support points (Sec. III.A; ratio test of Eq. 1-2), consistency and
// redundancy filtering (Sec. III.A), grid vectors (Sec. III.A, Fig. 2;
// one-hot masks, Sec. VI.D) and raster-order compaction.
//
// Kernels, in launch order:
//   support_match_row_kernel  one CTA per lattice row: warps hold 32 right
//                           windows each and walk the row's candidates
//                           (below); the re-match is one warp per candidate.
//   support_match_kernel    (rows too wide for the row kernel's shared
//                           memory) one warp per lattice candidate; lanes
//                           stride the disparity range, each lane keeps
//                           (best, second) and the warp merges them with two
//                           min-reductions; the right-to-left re-match runs
//                           in the same warp.
//   consistency_kernel      32x8 candidate tile with its halo in shared
//                           memory, window count per candidate; also clears
//                           the grid-vector masks.
//   redundancy_grid_kernel  one lattice row per CTA: four directional scans
//                           over the rows within maxd (staged in shared
//                           memory), atomicOr of the {d-1,d,d+1} bits of every
//                           surviving point into the 3x3 cells around it (in
//                           shared memory, then one global atomic per word;
//                           OR is order free, so the masks are
//                           deterministic), and the row's point count.
//   compact_rows_kernel     one lattice row per CTA: offset = points in the
//                           rows above, ballot-based placement; raster order.
#include "launch.cuh"

namespace elas {


// The ambiguity test of a best cost m1 against the second minimum m2 > 0:
// the ratio test m1 <= thr * m2 (Eq. 2, in FP32), or with shift_sum Eq. 3's
// m1 <= m2/2 + m2/4 + m2/8 + m2/32 in integer shifts.
__device__ __forceinline__ bool sup_unambiguous(uint32_t m1, uint32_t m2, float thr, int shift_sum) {
    if (shift_sum) return m1 <= (m2 >> 1) + (m2 >> 2) + (m2 >> 3) + (m2 >> 5);
    return __uint2float_rn(m1) <= __fmul_rn(thr, __uint2float_rn(m2));
}

// The matching window of pixel (u, v).  With Sobel descriptors (Sec. III.A)
// it is the four 16-byte descriptors at (u+-2, v+-2); with the census
// variant (Sec. VI.A) the pixel's own 32-byte support census record in q[0],
// q[1] (q[2], q[3] stay zero and take no part in the cost).
struct Win {
    uint4 q[4];
};

template <bool CENSUS>
__device__ __forceinline__ Win load_win(const uint4 *__restrict__ d, int w, int u, int v) {
    Win r;
    if (CENSUS) {
        const uint4 *p = d + 2 * ((size_t)v * w + u);
        r.q[0] = __ldg(p);
        r.q[1] = __ldg(p + 1);
        r.q[2] = r.q[3] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        const size_t rt = (size_t)(v - 2) * w, rb = (size_t)(v + 2) * w;
        r.q[0] = __ldg(d + rt + u - 2);
        r.q[1] = __ldg(d + rt + u + 2);
        r.q[2] = __ldg(d + rb + u - 2);
        r.q[3] = __ldg(d + rb + u + 2);
    }
    return r;
}

// Window cost: the SAD of the four descriptors (accumulating byte-SIMD
// absolute differences), or the Hamming distance of the census bits.  Both
// stay below 2^15.
template <bool CENSUS> __device__ __forceinline__ uint32_t win_cost(const Win &a, const Win &b) {
    if (CENSUS) return ham16(a.q[0], b.q[0]) + ham16(a.q[1], b.q[1]);
    return sad16_vacc(a.q[0], b.q[0]) + sad16_vacc(a.q[1], b.q[1]) + sad16_vacc(a.q[2], b.q[2]) +
           sad16_vacc(a.q[3], b.q[3]);
}

// The texture test of a window: Sobel windows need texture >= support_texture;
// census windows have no texture measure and always pass.
template <bool CENSUS> __device__ __forceinline__ bool win_textured(const Win &a, int support_texture) {
    if (CENSUS) return true;
    const uint32_t t = texture16(a.q[0]) + texture16(a.q[1]) + texture16(a.q[2]) + texture16(a.q[3]);
    return (int)t >= support_texture;
}

// Best disparity of window `a` of pixel (u, v) against `oth`, searching
// other position uo = u + dir*d with 4 <= uo <= w-5.  Warp collective;
// returns d1 or -1 (ambiguous / not enough disparities).
template <bool CENSUS>
__device__ __forceinline__ int warp_best_disparity(const uint4 *__restrict__ oth, int w, const Win &a, int u, int v,
                                                   int dir, int dmin, int dmax, float thr, int shift_sum, int lane) {
    int lo, hi;
    if (dir < 0) {
        lo = max(dmin, u - w + 5);
        hi = min(dmax, u - 4);
    } else {
        lo = max(dmin, 4 - u);
        hi = min(dmax, w - 5 - u);
    }
    if (hi - lo + 1 < 2) return -1;
    uint32_t m1 = 0xFFFFFFFFu, m2 = 0xFFFFFFFFu;
    int d1 = -1;
#pragma unroll 2
    for (int d = lo + lane; d <= hi; d += 32) {
        const uint32_t c = win_cost<CENSUS>(a, load_win<CENSUS>(oth, w, u + dir * d, v));
        if (c < m1) {
            m2 = m1;
            m1 = c;
            d1 = d;
        } else if (c < m2) {
            m2 = c;
        }
    }
    // cost < 2^15 and d < 2^16: (cost, d) packs into one ordered key
    const uint32_t key = d1 >= 0 ? ((m1 << 16) | (uint32_t)d1) : 0xFFFFFFFFu;
    const uint32_t kmin = __reduce_min_sync(0xFFFFFFFFu, key);
    const int gd1 = (int)(kmin & 0xFFFFu);
    const uint32_t gm1 = kmin >> 16;
    // second minimum over all d != d1: the winner lane offers its own second
    // best, every other lane its best
    const uint32_t mine = (d1 == gd1) ? m2 : m1;
    const uint32_t gm2 = __reduce_min_sync(0xFFFFFFFFu, mine);
    if (gm2 == 0u || gm2 == 0xFFFFFFFFu) return -1;
    return sup_unambiguous(gm1, gm2, thr, shift_sum) ? gd1 : -1;
}

template <bool CENSUS> __device__ __forceinline__ void support_match_body(const MatchArgs &m, const VB &vb) {
    const SupportArgs &a = m.a;
    const uint4 *__restrict__ dL = m.dL;
    const uint4 *__restrict__ dR = m.dR;
    const int warp = (vb.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int w = a.w, wc = a.wc;
    if (warp >= wc * a.hc) return;
    const int ic = warp / wc, jc = warp - ic * wc;
    const int u = jc * a.step, v = ic * a.step;
    int out = -1;
    if (u >= 4 && u <= w - 5 && v >= 4 && v <= a.h - 5) {
        const Win l = load_win<CENSUS>(dL, w, u, v);
        if (win_textured<CENSUS>(l, a.support_texture)) {
            const int d1 =
                warp_best_disparity<CENSUS>(dR, w, l, u, v, -1, a.dmin, a.dmax, a.thr, a.shift_sum, lane);
            if (d1 >= 0) {
                const int ur = u - d1;
                const Win r = load_win<CENSUS>(dR, w, ur, v);
                if (win_textured<CENSUS>(r, a.support_texture)) {
                    const int d2 =
                        warp_best_disparity<CENSUS>(dL, w, r, ur, v, +1, a.dmin, a.dmax, a.thr, a.shift_sum, lane);
                    if (d2 >= 0 && abs(d1 - d2) <= a.lr_threshold) out = d1;
                }
            }
        }
    }
    if (lane == 0) m.raw[warp] = (int16_t)out;
}

template <bool CENSUS> __global__ void __launch_bounds__(512) support_match_kernel(MatchArgs m) {
    support_match_body<CENSUS>(m, vb_single());
}

// The same matching with one CTA per lattice row, organised around the
// right-image positions: a right window s meets the candidates u = s + d of
// every disparity d, so a warp holds the windows of 32 consecutive s in
// registers and walks the row's candidates once: per candidate each lane
// costs its own d = u - s against the candidate's left window (shared
// memory, the same address on every lane), and two warp minimum-reductions
// give the best (cost, d) of those 32 disparities and the least other cost.
// Each candidate collects one such result per 32-disparity window in shared
// memory; their merge is the same (best, second) as a search over the whole
// range: the least key over the windows and, for the second, the least of
// the other windows' best costs and the winning window's second.  The
// right-to-left re-match of the candidates that pass runs with one warp per
// candidate as in support_match_kernel.  Keys are (cost << 16) | d: least
// cost, then least d.
struct SupRowSmem {
    int slots;  // windows a candidate's range can meet
    size_t desc, res, lohi, d1;  // byte offsets
    size_t total;
};

__host__ __device__ __forceinline__ SupRowSmem sup_row_smem(int wc, int dmin, int dmax) {
    SupRowSmem o;
    o.slots = (dmax - dmin + 1 + 31) / 32 + 1;
    o.desc = 0;
    o.res = o.desc + (size_t)wc * 4 * sizeof(uint4);
    o.lohi = o.res + (size_t)wc * o.slots * sizeof(uint2);
    o.d1 = o.lohi + (size_t)wc * sizeof(int2);
    o.total = o.d1 + (((size_t)wc * sizeof(int) + 15) & ~(size_t)15);
    return o;
}

template <bool CENSUS> __device__ __forceinline__ void support_match_row_body(const MatchArgs &m, const VB &vb) {
    const SupportArgs &a = m.a;
    const uint4 *__restrict__ dL = m.dL;
    const uint4 *__restrict__ dR = m.dR;
    const int w = a.w, wc = a.wc, step = a.step, dmin = a.dmin, dmax = a.dmax;
    const int ic = vb.x, v = ic * step;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char s_raw[];
    const SupRowSmem L = sup_row_smem(wc, dmin, dmax);
    uint4 *s_desc = reinterpret_cast<uint4 *>(s_raw + L.desc);
    uint2 *s_res = reinterpret_cast<uint2 *>(s_raw + L.res);
    int2 *s_lohi = reinterpret_cast<int2 *>(s_raw + L.lohi);
    int *s_d1 = reinterpret_cast<int *>(s_raw + L.d1);
    const bool row_ok = v >= 4 && v <= a.h - 5;
    // candidates: left windows, texture, disparity range (lo > hi: none)
    for (int k = tid; k < wc; k += blockDim.x) {
        const int u = k * step;
        int lo = 1, hi = 0;
        if (row_ok && u >= 4 && u <= w - 5) {
            const Win l = load_win<CENSUS>(dL, w, u, v);
#pragma unroll
            for (int i = 0; i < 4; ++i) s_desc[4 * k + i] = l.q[i];
            if (win_textured<CENSUS>(l, a.support_texture)) {
                lo = max(dmin, u - w + 5);
                hi = min(dmax, u - 4);
                if (hi - lo + 1 < 2) lo = 1, hi = 0;
            }
        }
        s_lohi[k] = make_int2(lo, hi);
        for (int j = 0; j < L.slots; ++j) s_res[k * L.slots + j] = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
    }
    __syncthreads();
    // right windows s = 4 + 32 j + lane, 4 <= s <= w - 5
    const int nwin = row_ok ? (w - 8 + 31) / 32 : 0;
    for (int j = warp; j < nwin; j += nwarps) {
        const int s0 = 4 + 32 * j, sl = s0 + lane;
        const bool s_ok = sl <= w - 5;
        Win r;
        if (s_ok) {
            r = load_win<CENSUS>(dR, w, sl, v);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) r.q[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        // candidates u = s + d with d in [dmin, dmax] for some s of the window
        const int k0 = max(0, (s0 + dmin + step - 1) / step), k1 = min(wc - 1, (s0 + 31 + dmax) / step);
        const int slot = j % L.slots;
        // two candidates per step: their chains (window load, cost, the two
        // reductions) are independent, so they overlap
        for (int k = k0; k <= k1; k += 2) {
            const bool has1 = k + 1 <= k1;
            const int2 lh0 = s_lohi[k], lh1 = has1 ? s_lohi[k + 1] : make_int2(1, 0);
            const int d0 = k * step - sl, d1 = d0 + step;
            const bool in0 = s_ok && d0 >= lh0.x && d0 <= lh0.y;
            const bool in1 = s_ok && d1 >= lh1.x && d1 <= lh1.y;
            Win lw0, lw1;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                lw0.q[i] = s_desc[4 * k + i];
                lw1.q[i] = has1 ? s_desc[4 * (k + 1) + i] : lw0.q[i];
            }
            const uint32_t c0 = win_cost<CENSUS>(lw0, r), c1 = win_cost<CENSUS>(lw1, r);
            const uint32_t key0 = in0 ? ((c0 << 16) | (uint32_t)d0) : 0xFFFFFFFFu;
            const uint32_t key1 = in1 ? ((c1 << 16) | (uint32_t)d1) : 0xFFFFFFFFu;
            const uint32_t kmin0 = __reduce_min_sync(0xFFFFFFFFu, key0);
            const uint32_t kmin1 = __reduce_min_sync(0xFFFFFFFFu, key1);
            const uint32_t m20 = __reduce_min_sync(0xFFFFFFFFu, (in0 && key0 != kmin0) ? c0 : 0xFFFFFFFFu);
            const uint32_t m21 = __reduce_min_sync(0xFFFFFFFFu, (in1 && key1 != kmin1) ? c1 : 0xFFFFFFFFu);
            // a candidate with an empty range (lo > hi) has no lane in it
            if (lane == 0 && kmin0 != 0xFFFFFFFFu) s_res[k * L.slots + slot] = make_uint2(kmin0, m20);
            if (lane == 0 && kmin1 != 0xFFFFFFFFu) s_res[(k + 1) * L.slots + slot] = make_uint2(kmin1, m21);
        }
    }
    __syncthreads();
    // merge the windows of each candidate; ratio test
    for (int k = tid; k < wc; k += blockDim.x) {
        uint32_t best = 0xFFFFFFFFu;
        int bj = -1;
        for (int j = 0; j < L.slots; ++j) {
            const uint32_t x = s_res[k * L.slots + j].x;
            if (x < best) {
                best = x;
                bj = j;
            }
        }
        int d1 = -1;
        if (bj >= 0) {
            uint32_t gm2 = s_res[k * L.slots + bj].y;
            for (int j = 0; j < L.slots; ++j) {
                const uint32_t x = s_res[k * L.slots + j].x;
                if (j != bj && x != 0xFFFFFFFFu) gm2 = min(gm2, x >> 16);
            }
            const uint32_t gm1 = best >> 16;
            if (gm2 != 0u && gm2 != 0xFFFFFFFFu &&
                sup_unambiguous(gm1, gm2, a.thr, a.shift_sum))
                d1 = (int)(best & 0xFFFFu);
        }
        s_d1[k] = d1;
        if (d1 < 0) m.raw[ic * wc + k] = (int16_t)-1;
    }
    __syncthreads();
    // right-to-left re-match, one warp per candidate that passed
    for (int k = warp; k < wc; k += nwarps) {
        const int d1 = s_d1[k];
        if (d1 < 0) continue;
        const int ur = k * step - d1;
        const Win r = load_win<CENSUS>(dR, w, ur, v);
        int out = -1;
        if (win_textured<CENSUS>(r, a.support_texture)) {
            const int d2 = warp_best_disparity<CENSUS>(dL, w, r, ur, v, +1, dmin, dmax, a.thr, a.shift_sum, lane);
            if (d2 >= 0 && abs(d1 - d2) <= a.lr_threshold) out = d1;
        }
        if (lane == 0) m.raw[ic * wc + k] = (int16_t)out;
    }
}

template <bool CENSUS> __global__ void __launch_bounds__(512) support_match_row_kernel(MatchArgs m) {
    support_match_row_body<CENSUS>(m, vb_single());
}
// Batched launches: one launch per cost kind among the pairs.
template <bool CENSUS>
__global__ void __launch_bounds__(512) support_match_row_kernel_b(const MatchArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    support_match_row_body<CENSUS>(slot_entry(tab, vm.stride, vb.slot), vb);
}
template <bool CENSUS>
__global__ void __launch_bounds__(512) support_match_kernel_b(const MatchArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    support_match_body<CENSUS>(slot_entry(tab, vm.stride, vb.slot), vb);
}

// Consistency filter on a 32x8 tile of candidates staged with its halo in
// shared memory; also zeroes the grid-vector masks (grid-stride) so that the
// next kernel can OR into them.
constexpr int kConsTX = 32, kConsTY = 8;

__device__ __forceinline__ void consistency_body(const ConsArgs &c, const VB &vb) {
    extern __shared__ int16_t s_g[];
    const int r = c.r, wc = c.wc, hc = c.hc;
    const int SW = kConsTX + 2 * r, SH = kConsTY + 2 * r;
    const int j0 = vb.x * kConsTX - r, i0 = vb.y * kConsTY - r;
    const int tid = threadIdx.y * kConsTX + threadIdx.x;
    constexpr int NT = kConsTX * kConsTY;
    for (int k = tid; k < SW * SH; k += NT) {
        const int gi = i0 + k / SW, gj = j0 + k % SW;
        s_g[k] = (gi >= 0 && gi < hc && gj >= 0 && gj < wc) ? c.in[gi * wc + gj] : (int16_t)-1;
    }
    const int nblk = vb.gx * vb.gy, bid = vb.y * vb.gx + vb.x;
    uint32_t *gL = c.gL, *gR = c.gR;
    for (int k = bid * NT + tid; k < c.gwords; k += nblk * NT) {
        if (gL) gL[k] = 0u;
        if (gR) gR[k] = 0u;
    }
    __syncthreads();
    const int jc = vb.x * kConsTX + threadIdx.x, ic = vb.y * kConsTY + threadIdx.y;
    if (jc >= wc || ic >= hc) return;
    const int16_t *cp = s_g + (threadIdx.y + r) * SW + threadIdx.x + r;
    const int d = cp[0];
    const int thr = c.thr;
    int res = -1;
    if (d >= 0) {
        int cnt = 0;
        for (int di = -r; di <= r; ++di) {
            const int16_t *rowp = cp + di * SW;
            for (int dj = -r; dj <= r; ++dj) {
                const int v = rowp[dj];
                cnt += (v >= 0) & (abs(v - d) <= thr);
            }
        }
        cnt -= (thr >= 0);  // the point itself
        if (cnt >= c.min_support) res = d;
    }
    c.out[ic * wc + jc] = (int16_t)res;
}

__global__ void __launch_bounds__(kConsTX *kConsTY) consistency_kernel(ConsArgs c) {
    consistency_body(c, vb_single());
}
__global__ void __launch_bounds__(kConsTX *kConsTY) consistency_kernel_b(const ConsArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    consistency_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

__device__ __forceinline__ void or_bits(uint32_t *cell, int d, int dmin, int dmax) {
    for (int dd = d - 1; dd <= d + 1; ++dd)
        if (dd >= dmin && dd <= dmax) atomicOr(cell + (dd >> 5), 1u << (dd & 31));
}


// Redundancy filter for one lattice row per CTA, the grid-vector bits of the
// surviving points and the row's point count.  Staged (when the shared
// memory fits): the consistency rows within maxd are read once into shared
// memory, and the bits go to a shared copy of the three cell rows the row's
// points reach (both sides), ORed into the grid with one atomic per non-zero
// word afterwards; else every read and OR goes to global memory.  OR is order
// free, so the masks are deterministic either way.
__host__ __device__ __forceinline__ size_t red_rows_bytes(int wc, int maxd) {
    return ((size_t)(2 * maxd + 1) * wc * sizeof(int16_t) + 15) & ~(size_t)15;
}
__host__ __device__ __forceinline__ size_t red_smem_bytes(int wc, int maxd, int gw, int nw) {
    return red_rows_bytes(wc, maxd) + 2 * (size_t)3 * gw * nw * sizeof(uint32_t);
}

__device__ __forceinline__ void redundancy_grid_body(const RedArgs &ra, const VB &vb, bool staged) {
    extern __shared__ __align__(16) unsigned char s_red[];
    __shared__ int s_cnt[4];
    const int16_t *__restrict__ con = ra.con;
    const int wc = ra.wc, hc = ra.hc, maxd = ra.maxd;
    const GridArgs g = ra.g;
    const int ic = vb.x, tid = threadIdx.x, nth = blockDim.x;
    const int r0 = max(0, ic - maxd), r1 = min(hc - 1, ic + maxd);
    int16_t *s_rows = reinterpret_cast<int16_t *>(s_red);
    uint32_t *s_or = reinterpret_cast<uint32_t *>(s_red + red_rows_bytes(wc, maxd));
    const int cy = ic * g.step / g.G, cy0 = max(0, cy - 1), ncy = min(g.gh - 1, cy + 1) - cy0 + 1;
    const int orw = 3 * g.gw * g.nw;  // shared words per side
    if (staged) {
        for (int k = tid; k < (r1 - r0 + 1) * wc; k += nth) s_rows[k] = con[(size_t)r0 * wc + k];
        for (int k = tid; k < 2 * orw; k += nth) s_or[k] = 0u;
        __syncthreads();
    }
    auto at = [&](int i, int j) -> int { return staged ? s_rows[(i - r0) * wc + j] : con[(size_t)i * wc + j]; };
    int mine = 0;
    for (int jc = tid; jc < wc; jc += nth) {
        const int d = at(ic, jc);
        int res = d;
        if (d >= 0 && ra.enabled) {
            // left, up, right, down: the past-only rule (Sec. VI.C) takes the first two
            const int di[4] = {0, -1, 0, 1}, dj[4] = {-1, 0, 1, 0};
            const int ndir = ra.past_only ? 2 : 4;
            bool redundant = true;
            for (int k = 0; k < ndir && redundant; ++k) {
                bool found = false;
                for (int st = 1; st <= maxd; ++st) {
                    const int i2 = ic + st * di[k], j2 = jc + st * dj[k];
                    if (i2 < 0 || i2 >= hc || j2 < 0 || j2 >= wc) break;
                    if (at(i2, j2) == d) {
                        found = true;
                        break;
                    }
                }
                redundant = found;
            }
            if (redundant) res = -1;
        }
        ra.dcan[(size_t)ic * wc + jc] = (int16_t)res;
        if (res >= 0) ++mine;
        if (res >= 0 && !ra.defer_grid) {
            const int u = jc * g.step;
            for (int side = 0; side < 2; ++side) {
                uint32_t *grid = side ? ra.gridR : ra.gridL;
                if (!grid) continue;
                const int cx = (side ? u - res : u) / g.G;
                for (int y = cy0; y < cy0 + ncy; ++y)
                    for (int x = max(0, cx - 1); x <= min(g.gw - 1, cx + 1); ++x) {
                        if (staged) {
                            uint32_t *cell = s_or + side * orw + ((y - cy0) * g.gw + x) * g.nw;
                            for (int dd = res - 1; dd <= res + 1; ++dd)
                                if (dd >= g.dmin && dd <= g.dmax) atomicOr(cell + (dd >> 5), 1u << (dd & 31));
                        } else {
                            or_bits(grid + ((size_t)y * g.gw + x) * g.nw, res, g.dmin, g.dmax);
                        }
                    }
            }
        }
    }
    if (staged) {
        __syncthreads();
        const int rw = ncy * g.gw * g.nw;  // words of the cell rows that exist
        for (int k = tid; k < 2 * rw; k += nth) {
            const int side = k / rw, rem = k - side * rw;
            const uint32_t word = s_or[side * orw + rem];
            uint32_t *grid = side ? ra.gridR : ra.gridL;
            if (word && grid) atomicOr(grid + (size_t)cy0 * g.gw * g.nw + rem, word);
        }
    }
    mine = __reduce_add_sync(0xFFFFFFFFu, mine);
    if ((tid & 31) == 0) s_cnt[tid >> 5] = mine;
    __syncthreads();
    if (tid == 0) ra.rowcount[ic] = s_cnt[0] + s_cnt[1] + s_cnt[2] + s_cnt[3];
}

__global__ void __launch_bounds__(128) redundancy_grid_kernel(RedArgs ra, int staged) {
    redundancy_grid_body(ra, vb_single(), staged != 0);
}
__global__ void __launch_bounds__(128) redundancy_grid_kernel_b(const RedArgs *__restrict__ tab, VMap vm, int staged) {
    const VB vb = vb_batch(vm);
    redundancy_grid_body(slot_entry(tab, vm.stride, vb.slot), vb, staged != 0);
}

// Raster-order compaction, one lattice row per CTA: the row's offset is the
// sum of the counts of the rows above; entries are placed with warp ballots.
__device__ __forceinline__ void compact_rows_body(const CompactArgs &ca, const VB &vb) {
    __shared__ int s_w[4];
    const int wc = ca.wc, hc = ca.hc, step = ca.step;
    const int ic = vb.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int part = 0;
    for (int k = tid; k < ic; k += 128) part += ca.rowcount[k];
    part = __reduce_add_sync(0xFFFFFFFFu, part);
    if (lane == 0) s_w[warp] = part;
    __syncthreads();
    int base = s_w[0] + s_w[1] + s_w[2] + s_w[3];
    __syncthreads();
    int16_t *list = ca.list;
    for (int j0 = 0; j0 < wc; j0 += 128) {
        const int jc = j0 + tid;
        const int d = jc < wc ? ca.dcan[ic * wc + jc] : -1;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, d >= 0);
        if (lane == 0) s_w[warp] = __popc(bal);
        __syncthreads();
        int off = base + __popc(bal & ((1u << lane) - 1u));
        for (int k = 0; k < warp; ++k) off += s_w[k];
        if (d >= 0) {
            // down-sampling keeps the points numbered 0, k, 2k, ... (raster order)
            const int ke = ca.keep_every;
            if (ke <= 1 || off % ke == 0) {
                const int o = ke > 1 ? off / ke : off;
                list[3 * o + 0] = (int16_t)(jc * step);
                list[3 * o + 1] = (int16_t)(ic * step);
                list[3 * o + 2] = (int16_t)d;
            } else {
                ca.dcan[ic * wc + jc] = -1;
            }
        }
        base += s_w[0] + s_w[1] + s_w[2] + s_w[3];
        __syncthreads();
    }
    if (ic == hc - 1 && tid == 0) *ca.count = ca.keep_every > 1 ? (base + ca.keep_every - 1) / ca.keep_every : base;
}

__global__ void __launch_bounds__(128) compact_rows_kernel(CompactArgs ca) { compact_rows_body(ca, vb_single()); }

// Grid vectors of a down-sampled list (the masks were cleared by the
// consistency kernel): each point ORs its {d-1, d, d+1} bits into the 3x3
// cells around its cell, as the redundancy kernel does for every point
// without down-sampling.
__device__ __forceinline__ void list_grid_body(const ListGridArgs &a, const VB &vb) {
    const int n = min(*a.count, a.cap);
    const GridArgs g = a.g;
    for (int k = vb.x * blockDim.x + threadIdx.x; k < n; k += vb.gx * blockDim.x) {
        const int u = a.list[3 * k], v = a.list[3 * k + 1], d = a.list[3 * k + 2];
        const int cy = v / g.G;
        for (int side = 0; side < 2; ++side) {
            uint32_t *grid = side ? a.gridR : a.gridL;
            if (!grid) continue;
            const int cx = (side ? u - d : u) / g.G;
            for (int y = max(0, cy - 1); y <= min(g.gh - 1, cy + 1); ++y)
                for (int x = max(0, cx - 1); x <= min(g.gw - 1, cx + 1); ++x)
                    or_bits(grid + ((size_t)y * g.gw + x) * g.nw, d, g.dmin, g.dmax);
        }
    }
}
__global__ void __launch_bounds__(128) list_grid_kernel(ListGridArgs a) { list_grid_body(a, vb_single()); }
__global__ void __launch_bounds__(128) list_grid_kernel_b(const ListGridArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    list_grid_body(slot_entry(tab, vm.stride, vb.slot), vb);
}
__global__ void __launch_bounds__(128) compact_rows_kernel_b(const CompactArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    compact_rows_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

size_t support_workspace(int w, int h, const elas_params *p) {
    const size_t hc = (size_t)(h / p->candidate_stepsize);
    const size_t nc = (size_t)(w / p->candidate_stepsize) * hc;
    return 2 * align_up(nc * sizeof(int16_t) + 16, 256) + align_up(hc * sizeof(int32_t) + 16, 256);
}

constexpr int kMaxConsistencyWindow = 64;

elas_status support_args(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                         int16_t *d_can, int16_t *list, int32_t *count, uint32_t *grid_L, uint32_t *grid_R,
                         void *ws, SupportStage *o) {
    if (p->incon_window_size > kMaxConsistencyWindow)
        return fail(ELAS_ERR_INVALID_ARG, "incon_window_size %d above %d", p->incon_window_size, kMaxConsistencyWindow);
    SupportArgs a;
    a.w = w;
    a.h = h;
    a.step = p->candidate_stepsize;
    a.wc = w / a.step;
    a.hc = h / a.step;
    a.dmin = p->disp_min;
    a.dmax = p->disp_max;
    a.thr = p->support_threshold;
    a.shift_sum = (p->test_flags & ELAS_FLAG_SHIFT_SUM) ? 1 : 0;
    a.census = p->census_support_w > 0 ? 1 : 0;
    a.support_texture = p->support_texture;
    a.lr_threshold = p->lr_threshold;
    const int nc = a.wc * a.hc;
    const GridGeom g = grid_geom(w, h, p);
    const size_t grid_bytes = align_up((size_t)nc * sizeof(int16_t) + 16, 256);
    int16_t *raw = reinterpret_cast<int16_t *>(ws);
    int16_t *con = reinterpret_cast<int16_t *>(reinterpret_cast<char *>(ws) + grid_bytes);
    int32_t *rowcount = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(ws) + 2 * grid_bytes);
    o->match = MatchArgs{reinterpret_cast<const uint4 *>(descL), reinterpret_cast<const uint4 *>(descR), a, raw};
    o->cons = ConsArgs{raw, a.wc, a.hc, p->incon_window_size, p->incon_threshold, p->incon_min_support, con,
                       grid_L, grid_R, g.gw * g.gh * g.nw};
    o->red = RedArgs{con, a.wc, a.hc, p->redun_max_dist, (p->test_flags & ELAS_FLAG_REDUNDANCY_OFF) ? 0 : 1,
                     (p->test_flags & ELAS_FLAG_PAST_REDUNDANCY) ? 1 : 0,
                     GridArgs{a.step, p->grid_size, g.gw, g.gh, g.nw, a.dmin, a.dmax}, d_can, grid_L, grid_R,
                     rowcount, p->support_downsample > 1 ? 1 : 0};
    o->compact = CompactArgs{d_can, a.wc, a.hc, a.step, rowcount, list, count, p->support_downsample};
    const int k = p->support_downsample > 1 ? p->support_downsample : 1;
    o->lg = ListGridArgs{list, count, (nc + k - 1) / k, o->red.g, grid_L, grid_R};
    return ELAS_OK;
}

size_t consistency_smem(int r) { return (size_t)(kConsTX + 2 * r) * (kConsTY + 2 * r) * sizeof(int16_t); }

static elas_status consistency_smem_attr(const void *fn, size_t smem) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return launch_status("consistency_kernel shared memory attribute");
    return ELAS_OK;
}

// Shared memory of the staged redundancy filter; more runs it unstaged.
constexpr size_t kRedSmemMax = 96 * 1024;

static elas_status red_smem_attr(const void *fn, size_t smem) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return launch_status("redundancy_grid_kernel shared memory attribute");
    return ELAS_OK;
}

// Shared memory of the row-organised matcher; wider rows take the
// per-candidate kernel, and so do launches of fewer lattice rows than two
// per SM (one CTA per row would leave SMs idle).
constexpr size_t kSupRowSmemMax = 160 * 1024;
inline int sup_row_min_rows() { return 2 * sm_count(); }

static elas_status sup_row_smem_attr(const void *fn, size_t smem) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return launch_status("support_match_row_kernel shared memory attribute");
    return ELAS_OK;
}

dim3 support_match_grid(const MatchArgs &m, int warps) {
    const int nc = m.a.wc * m.a.hc;
    return dim3((nc + warps - 1) / warps);
}
dim3 consistency_grid(const ConsArgs &c) { return dim3((c.wc + kConsTX - 1) / kConsTX, (c.hc + kConsTY - 1) / kConsTY); }
dim3 lattice_row_grid(int hc) { return dim3(hc); }

elas_status launch_support(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                           int16_t *d_can, int16_t *list, int32_t *count, uint32_t *grid_L, uint32_t *grid_R,
                           void *ws, cudaStream_t st) {
    SupportStage sa;
    elas_status s = support_args(descL, descR, w, h, p, d_can, list, count, grid_L, grid_R, ws, &sa);
    if (s != ELAS_OK) return s;
    const int nc = sa.match.a.wc * sa.match.a.hc;
    if (nc == 0) {
        const size_t gbytes = (size_t)sa.cons.gwords * 4;
        if ((grid_L && cudaMemsetAsync(grid_L, 0, gbytes, st) != cudaSuccess) ||
            (grid_R && cudaMemsetAsync(grid_R, 0, gbytes, st) != cudaSuccess) ||
            cudaMemsetAsync(count, 0, sizeof(int32_t), st) != cudaSuccess)
            return launch_status("memset empty support");
        return ELAS_OK;
    }
    const int warps_per_block = 8;
    const size_t row_smem = sup_row_smem(sa.match.a.wc, sa.match.a.dmin, sa.match.a.dmax).total;
    const bool census = sa.match.a.census != 0;
    if (row_smem <= kSupRowSmemMax && sa.match.a.hc >= sup_row_min_rows()) {
        const void *fn = census ? (const void *)support_match_row_kernel<true>
                                : (const void *)support_match_row_kernel<false>;
        if ((s = sup_row_smem_attr(fn, row_smem)) != ELAS_OK) return s;
        if (census)
            support_match_row_kernel<true><<<lattice_row_grid(sa.match.a.hc), 32 * warps_per_block, row_smem, st>>>(
                sa.match);
        else
            support_match_row_kernel<false><<<lattice_row_grid(sa.match.a.hc), 32 * warps_per_block, row_smem, st>>>(
                sa.match);
        if ((s = launch_status("support_match_row_kernel")) != ELAS_OK) return s;
    } else {
        const dim3 grid = support_match_grid(sa.match, warps_per_block);
        if (census)
            support_match_kernel<true><<<grid, 32 * warps_per_block, 0, st>>>(sa.match);
        else
            support_match_kernel<false><<<grid, 32 * warps_per_block, 0, st>>>(sa.match);
        if ((s = launch_status("support_match_kernel")) != ELAS_OK) return s;
    }
    const size_t smem = consistency_smem(sa.cons.r);
    if ((s = consistency_smem_attr((const void *)consistency_kernel, smem)) != ELAS_OK) return s;
    consistency_kernel<<<consistency_grid(sa.cons), dim3(kConsTX, kConsTY), smem, st>>>(sa.cons);
    if ((s = launch_status("consistency_kernel")) != ELAS_OK) return s;
    size_t red_smem = red_smem_bytes(sa.red.wc, sa.red.maxd, sa.red.g.gw, sa.red.g.nw);
    const int red_staged = red_smem <= kRedSmemMax;
    if (!red_staged) red_smem = 0;
    if ((s = red_smem_attr((const void *)redundancy_grid_kernel, red_smem)) != ELAS_OK) return s;
    redundancy_grid_kernel<<<lattice_row_grid(sa.red.hc), 128, red_smem, st>>>(sa.red, red_staged);
    if ((s = launch_status("redundancy_grid_kernel")) != ELAS_OK) return s;
    compact_rows_kernel<<<lattice_row_grid(sa.compact.hc), 128, 0, st>>>(sa.compact);
    if ((s = launch_status("compact_rows_kernel")) != ELAS_OK) return s;
    if (sa.compact.keep_every <= 1) return ELAS_OK;
    int blocks = (sa.lg.cap + 127) / 128;
    if (blocks > sm_count() * 4) blocks = sm_count() * 4;
    list_grid_kernel<<<blocks, 128, 0, st>>>(sa.lg);
    return launch_status("list_grid_kernel");
}

// Batched support stage: every pair of the launch must have at least one
// lattice candidate (w, h >= candidate_stepsize).
elas_status launch_support_b(const SupportTables &t, const SupportStage *host, const VMap &pairs, int match_warps,
                             cudaStream_t st) {
    if (match_warps != 4 && match_warps != 8 && match_warps != 16)
        return fail(ELAS_ERR_INVALID_ARG, "support warps per CTA %d", match_warps);
    // matching: the pairs of each cost kind (descriptor SAD, census Hamming)
    VMap m_match[2], m_krows[2], m_cons, m_rows, m_lg;
    size_t row_smem[2] = {0, 0}, red_smem = 0;
    for (int c = 0; c < 2; ++c) {
        vmap_clear(m_match[c], pairs.stride);
        vmap_clear(m_krows[c], pairs.stride);
    }
    vmap_clear(m_cons, pairs.stride);
    vmap_clear(m_rows, pairs.stride);
    vmap_clear(m_lg, pairs.stride);
    size_t cons_smem = 0;
    for (int i = 0; i < pairs.n; ++i) {
        const int slot = pairs.slot[i];
        const SupportStage &h = slot_entry(host, pairs.stride, slot);
        if (h.match.a.wc * h.match.a.hc == 0)
            return fail(ELAS_ERR_INVALID_ARG, "pair %d has no lattice candidate", i);
        const int c = h.match.a.census ? 1 : 0;
        vmap_add(m_match[c], slot, support_match_grid(h.match, match_warps));
        vmap_add(m_krows[c], slot, lattice_row_grid(h.red.hc));
        row_smem[c] = max(row_smem[c], sup_row_smem(h.match.a.wc, h.match.a.dmin, h.match.a.dmax).total);
        red_smem = max(red_smem, red_smem_bytes(h.red.wc, h.red.maxd, h.red.g.gw, h.red.g.nw));
        vmap_add(m_cons, slot, consistency_grid(h.cons));
        vmap_add(m_rows, slot, lattice_row_grid(h.red.hc));
        cons_smem = cons_smem > consistency_smem(h.cons.r) ? cons_smem : consistency_smem(h.cons.r);
        if (h.compact.keep_every > 1)
            vmap_add(m_lg, slot, dim3(max(1, min((h.lg.cap + 127) / 128, sm_count() * 4 / pairs.n + 1))));
    }
    if (pairs.n == 0) return ELAS_OK;
    elas_status s;
    for (int c = 0; c < 2; ++c) {
        if (m_match[c].n == 0) continue;
        if (row_smem[c] <= kSupRowSmemMax && vmap_total(m_krows[c]) >= sup_row_min_rows()) {
            const void *fn = c ? (const void *)support_match_row_kernel_b<true>
                               : (const void *)support_match_row_kernel_b<false>;
            if ((s = sup_row_smem_attr(fn, row_smem[c])) != ELAS_OK) return s;
            if (c)
                support_match_row_kernel_b<true>
                    <<<vmap_total(m_krows[c]), 32 * match_warps, row_smem[c], st>>>(t.match, m_krows[c]);
            else
                support_match_row_kernel_b<false>
                    <<<vmap_total(m_krows[c]), 32 * match_warps, row_smem[c], st>>>(t.match, m_krows[c]);
            if ((s = launch_status("support_match_row_kernel_b")) != ELAS_OK) return s;
        } else {
            if (c)
                support_match_kernel_b<true><<<vmap_total(m_match[c]), 32 * match_warps, 0, st>>>(t.match, m_match[c]);
            else
                support_match_kernel_b<false><<<vmap_total(m_match[c]), 32 * match_warps, 0, st>>>(t.match,
                                                                                                  m_match[c]);
            if ((s = launch_status("support_match_kernel_b")) != ELAS_OK) return s;
        }
    }
    if ((s = consistency_smem_attr((const void *)consistency_kernel_b, cons_smem)) != ELAS_OK) return s;
    consistency_kernel_b<<<vmap_total(m_cons), dim3(kConsTX, kConsTY), cons_smem, st>>>(t.cons, m_cons);
    if ((s = launch_status("consistency_kernel_b")) != ELAS_OK) return s;
    const int red_staged = red_smem <= kRedSmemMax;
    if (!red_staged) red_smem = 0;
    if ((s = red_smem_attr((const void *)redundancy_grid_kernel_b, red_smem)) != ELAS_OK) return s;
    redundancy_grid_kernel_b<<<vmap_total(m_rows), 128, red_smem, st>>>(t.red, m_rows, red_staged);
    if ((s = launch_status("redundancy_grid_kernel_b")) != ELAS_OK) return s;
    compact_rows_kernel_b<<<vmap_total(m_rows), 128, 0, st>>>(t.compact, m_rows);
    if ((s = launch_status("compact_rows_kernel_b")) != ELAS_OK) return s;
    // down-sampled pairs: grid vectors from the kept points
    if (m_lg.n == 0) return ELAS_OK;
    list_grid_kernel_b<<<vmap_total(m_lg), 128, 0, st>>>(t.lg, m_lg);
    return launch_status("list_grid_kernel_b");
}

}  // namespace elas

extern "C" size_t elas_support_workspace_bytes(int32_t w, int32_t h, const elas_params *p) {
    if (elas::check_params(p, w, h) != ELAS_OK) return 0;
    return elas::support_workspace(w, h, p);
}

extern "C" elas_status elas_support_points(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                                           const elas_params *p, int16_t *d_can, int16_t *list, int32_t cap,
                                           int32_t *count, uint32_t *grid_L, uint32_t *grid_R, void *workspace,
                                           size_t workspace_bytes, elas_stream stream) {
    using namespace elas;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (!descL || !descR || !d_can || !list || !count || !workspace)
        return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned(descL, 16) || !aligned(descR, 16)) return fail(ELAS_ERR_INVALID_ARG, "descriptors not 16-byte aligned");
    if (!aligned(workspace, 256)) return fail(ELAS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    const int64_t nc = (int64_t)(w / p->candidate_stepsize) * (h / p->candidate_stepsize);
    if (cap < nc) return fail(ELAS_ERR_CAPACITY, "list capacity %d < %lld candidates", cap, (long long)nc);
    if (workspace_bytes < support_workspace(w, h, p))
        return fail(ELAS_ERR_CAPACITY, "workspace %zu < %zu bytes", workspace_bytes, support_workspace(w, h, p));
    return launch_support(descL, descR, w, h, p, d_can, list, count, grid_L, grid_R, workspace, to_stream(stream));
}

// ---------------------------------------------------------------------------
// Support points without any allocation by the caller or the library.
//
// The scratch (the unfiltered and the consistency-filtered candidate grids)
// lives in one file-scope device array instead of a caller workspace.  Every
// GPU that loads this library holds the array until the process exits.  Host
// code cannot use the array's name as a device address, so its address is
// looked up with cudaGetSymbolAddress, once per device, on the first call
// made while that device is current.
// ---------------------------------------------------------------------------
#include <mutex>

namespace elas {

static __device__ __align__(256) unsigned char g_support_scratch[ELAS_STATIC_SUPPORT_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};
}  // namespace

static elas_status static_support_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ELAS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(ELAS_ERR_INTERNAL, "device ordinal %d above %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_support_scratch);
        if (e != cudaSuccess)
            return fail(ELAS_ERR_CUDA, "cudaGetSymbolAddress(support scratch): %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ELAS_OK;
}

}  // namespace elas

extern "C" elas_status elas_support_points_static(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                                                  const elas_params *p, int16_t *d_can, int16_t *list, int32_t cap,
                                                  int32_t *count, uint32_t *grid_L, uint32_t *grid_R,
                                                  elas_stream stream) {
    using namespace elas;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (!descL || !descR || !d_can || !list || !count) return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned(descL, 16) || !aligned(descR, 16)) return fail(ELAS_ERR_INVALID_ARG, "descriptors not 16-byte aligned");
    const int64_t nc = (int64_t)(w / p->candidate_stepsize) * (h / p->candidate_stepsize);
    if (cap < nc) return fail(ELAS_ERR_CAPACITY, "list capacity %d < %lld candidates", cap, (long long)nc);
    const size_t need = support_workspace(w, h, p);
    if (need > (size_t)ELAS_STATIC_SUPPORT_SCRATCH_BYTES)
        return fail(ELAS_ERR_CAPACITY,
                    "%dx%d with candidate step %d needs %zu scratch bytes; the static scratch holds %u "
                    "(use elas_support_points with a workspace)",
                    w, h, p->candidate_stepsize, need, (unsigned)ELAS_STATIC_SUPPORT_SCRATCH_BYTES);
    void *scratch = nullptr;
    if ((s = static_support_scratch(&scratch)) != ELAS_OK) return s;
    return launch_support(descL, descR, w, h, p, d_can, list, count, grid_L, grid_R, scratch, to_stream(stream));
}
