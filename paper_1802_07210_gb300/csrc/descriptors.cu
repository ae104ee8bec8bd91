// Descriptors: Sobel gradient images quantised to uint8 and sampled into a
// 16-byte descriptor per pixel (Sec. III.A, Fig. 1(b-d); Sec. VI.A); and the
// census transform of the paper's variant (Sec. VI.A, at the end).
//
// Sobel descriptors.  A warp walks down a strip of 128 image columns, four
// adjacent columns per lane, and writes the descriptors of the inner 120
// (lanes 1..30) for `rows` consecutive image rows.  The warp first copies the
// image rows it reads (its rows and three above and below) into shared
// memory with asynchronous 4-byte copies, 33 aligned words per row, in two
// groups so that the walk starts when the first group has landed.  Per image
// row a lane takes its word (funnel-shifted with the next one when the row
// does not start on a 4-byte boundary), the two border bytes from the lanes
// beside it, and forms the horizontal Sobel sums of its four columns, two
// columns per register (16-bit halves).  The vertical sums of the three
// latest image rows give a gradient row, quantised to bytes (four columns per
// word); the five latest gradient rows and the neighbour lanes' words of each
// stay in registers, and a descriptor row is assembled from them by byte
// permutes: the four pixels' bytes of one output word are a 4x4 byte
// transpose.  Four warps per CTA, one above the other; no block barriers.
#include "launch.cuh"

namespace elas {

constexpr int kDescWarps = 4;     // warps per CTA
constexpr int kDescStrip = 120;   // output columns of a warp
constexpr int kDescMaxRows = 36;  // rows a warp walks, at most (a multiple of 6)
constexpr int kDescFirst = 12;    // image rows of the first copy group (6 output rows)
constexpr uint32_t kFull = 0xFFFFFFFFu;

// Rows a warp walks: 6 in the one-pair launch; 12, 24 or 36 in batched
// launches (chosen by the tuner).
static bool valid_desc_rows(int r) { return r == 12 || r == 24 || r == 36; }

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint8_t *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// Stages the 32-bit word of an image row at byte offset `off` (4-byte
// aligned in memory) into shared memory: an asynchronous copy when the word
// lies in [0, w), else the bytes in [0, w) read one by one (zero outside).
__device__ __forceinline__ void desc_stage_word(uint32_t *dst, const uint8_t *row, int off, int w) {
    if (off >= 0 && off + 3 < w) {
        cp_async4(dst, row + off);
        return;
    }
    uint32_t v = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (off + b >= 0 && off + b < w) v |= (uint32_t)__ldg(row + off + b) << (8 * b);
    *dst = v;
}

// Horizontal Sobel sums of one image row for a lane's four columns, two
// columns per register (low half: column 0 or 1, high half: column 2 or 3):
// hs = I(c-1) + 2 I(c) + I(c+1) and hd = I(c+1) - I(c-1) + 256.
struct DescPart {
    uint32_t hse, hso, hde, hdo;
};

// One gradient row of a lane: quantised du and dv of its four columns (byte
// k = column k) and the same words of the lanes to its left and right.
struct DescGrad {
    uint32_t du, duL, duR, dv, dvL, dvR;
};

// Two quantised gradients from a register of two halves G = g + 1024,
// g in [-1020, 1020]: q = clamp(128 + trunc(g / 4), 1, 255), returned as
// S = q + 128 in lo and hi.  A negative g adds 3 before the division by 4
// (a shift), which rounds its quarter toward zero.
__device__ __forceinline__ void desc_quant2(uint32_t G, uint32_t &lo, uint32_t &hi) {
    const uint32_t neg = ((G >> 10) & 0x00010001u) ^ 0x00010001u;
    const uint32_t S = (G + 3u * neg) >> 2;
    lo = min(max(S & 0x1FFu, 129u), 383u);
    hi = min(max(S >> 16, 129u), 383u);
}

// The byte word of four columns from their even-column and odd-column
// gradient pairs; the low byte of S is q ^ 0x80.
__device__ __forceinline__ uint32_t desc_pack(uint32_t e, uint32_t o) {
    uint32_t elo, ehi, olo, ohi;
    desc_quant2(e, elo, ehi);
    desc_quant2(o, olo, ohi);
    const uint32_t a = __byte_perm(elo, olo, 0x0040), b = __byte_perm(ehi, ohi, 0x0040);
    return __byte_perm(a, b, 0x5410) ^ 0x80808080u;
}

// 4x4 byte transpose: from t0 = [a0 b0 a1 b1], t1 = [a2 b2 a3 b3],
// t2 = [c0 d0 c1 d1], t3 = [c2 d2 c3 d3] the words o[k] = [ak bk ck dk].
__device__ __forceinline__ void desc_transpose(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3,
                                               uint32_t (&o)[4]) {
    o[0] = __byte_perm(t0, t2, 0x5410);
    o[1] = __byte_perm(t0, t2, 0x7632);
    o[2] = __byte_perm(t1, t3, 0x5410);
    o[3] = __byte_perm(t1, t3, 0x7632);
}

// Per-warp shared memory: the staged image rows and one descriptor row on
// its way to global memory.
struct DescSmem {
    uint32_t img[kDescMaxRows + 6][33];
    uint4 out[kDescStrip];
};

// The walk of one warp.  EDGE: the strip touches the left or right image
// border (byte-wise staging of partial words, gradient column masks, store
// guards); otherwise every word and column of the strip is inside the image.
template <bool EDGE>
__device__ __forceinline__ void desc_walk(DescSmem &sm, const uint8_t *img, uint4 *desc, int w, int h, size_t pitch,
                                          int c0, int Y0, int n) {
    const int lane = threadIdx.x & 31;
    // byte offset of column c0 within a 4-byte word: c0 is a multiple of 4,
    // so it is the row start's, the same for every lane
    const uint32_t mis0 = (uint32_t)(((uintptr_t)img + (uintptr_t)(intptr_t)c0) & 3u);
    const uint32_t pm = (uint32_t)(pitch & 3u);
    // gradients are defined for 1 <= c <= w-2 (and 1 <= r <= h-2); 128 elsewhere
    uint32_t cm = 0xFFFFFFFFu;
    if (EDGE) {
        cm = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (c0 + k >= 1 && c0 + k <= w - 2) cm |= 0xFFu << (8 * k);
    }
    const int n6 = (n + 5) / 6 * 6;  // rows walked (those at or past n are not stored)
    const int nr = n6 + 6;           // image rows staged: Y0 - 3 .. Y0 + n6 + 2

    // image row Y0 - 3 + r in sm.img[r], words 0..32
    auto stage = [&](int r0, int r1) {
        for (int r = r0; r < r1; ++r) {
            const int i = Y0 - 3 + r;
            if (i < 0 || i >= h) {
                sm.img[r][lane] = 0u;
                if (lane == 31) sm.img[r][32] = 0u;
                continue;
            }
            const uint8_t *row = img + (size_t)i * pitch;
            const int off = c0 - (int)((mis0 + (uint32_t)i * pm) & 3u);
            if (EDGE) {
                desc_stage_word(&sm.img[r][lane], row, off, w);
                if (lane == 31) desc_stage_word(&sm.img[r][32], row, off + 4, w);
            } else {
                cp_async4(&sm.img[r][lane], row + off);
                if (lane == 31) cp_async4(&sm.img[r][32], row + off + 4);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    auto part = [&](int r, DescPart &p) {
        const uint32_t mis = (mis0 + (uint32_t)(Y0 - 3 + r) * pm) & 3u;
        const uint32_t lo = sm.img[r][lane], hi = sm.img[r][lane + 1];
        const uint32_t W = __funnelshift_r(lo, hi, 8u * mis);              // columns c0 .. c0+3
        const uint32_t im1 = __shfl_up_sync(kFull, W, 1) >> 24;           // column c0 - 1
        const uint32_t ip4 = __byte_perm(hi, 0u, 0x4440u | mis);          // column c0 + 4
        const uint32_t ce = __byte_perm(W, 0u, 0x4240), co = __byte_perm(W, 0u, 0x4341);
        const uint32_t le = __byte_perm(co, im1, 0x1054), ro = __byte_perm(ce, ip4, 0x5432);
        p.hse = le + 2u * ce + co;
        p.hde = co - le + 0x01000100u;
        p.hso = ce + 2u * co + ro;
        p.hdo = ro - ce + 0x01000100u;
    };
    // gradient row r from the sums of image rows r-1 (pa), r (pb), r+1 (pc):
    // du = hd(r-1) + 2 hd(r) + hd(r+1), dv = hs(r+1) - hs(r-1), each + 1024
    auto grad = [&](int r, const DescPart &pa, const DescPart &pb, const DescPart &pc, DescGrad &g) {
        uint32_t du = 0x80808080u, dv = 0x80808080u;
        if (r >= 1 && r <= h - 2) {
            du = desc_pack(pa.hde + 2u * pb.hde + pc.hde, pa.hdo + 2u * pb.hdo + pc.hdo);
            dv = desc_pack(pc.hse - pa.hse + 0x04000400u, pc.hso - pa.hso + 0x04000400u);
            if (EDGE) {
                du = (du & cm) | (0x80808080u & ~cm);
                dv = (dv & cm) | (0x80808080u & ~cm);
            }
        }
        g.du = du;
        g.dv = dv;
        g.duL = __shfl_up_sync(kFull, du, 1);
        g.duR = __shfl_down_sync(kFull, du, 1);
        g.dvL = __shfl_up_sync(kFull, dv, 1);
        g.dvR = __shfl_down_sync(kFull, dv, 1);
    };
    // descriptor row y from gradient rows y-2 .. y+2.  A permute of (left,
    // own) indexes columns -4..3 as bytes 0..7, of (own, right) columns 0..7.
    // The 120 descriptors go through shared memory (chunk k of lane l's 64
    // bytes at 16 ((k + (l-1)/2) & 3), which keeps both sides free of bank
    // conflicts) and leave as 512 contiguous bytes per store instruction.
    const int q = 4 * lane - 4;  // first output pixel of the lane (lanes 1..30)
    auto emit = [&](int y, const DescGrad &m2, const DescGrad &m1, const DescGrad &z, const DescGrad &p1,
                    const DescGrad &p2) {
        uint32_t ox[4], oy[4], oz[4], ow[4];
        // du(-2,-2) du(2,-2) du(-1,0) du(1,0)
        desc_transpose(__byte_perm(m2.duL, m2.du, 0x7362), __byte_perm(m2.du, m2.duR, 0x5140),
                       __byte_perm(z.duL, z.du, 0x6453), __byte_perm(z.du, z.duR, 0x4231), ox);
        // du(-2,2) du(2,2) du(0,-1) du(0,1)
        desc_transpose(__byte_perm(p2.duL, p2.du, 0x7362), __byte_perm(p2.du, p2.duR, 0x5140),
                       __byte_perm(m1.du, p1.du, 0x5140), __byte_perm(m1.du, p1.du, 0x7362), oy);
        // dv(0,-2) dv(0,2) dv(-2,0) dv(2,0)
        desc_transpose(__byte_perm(m2.dv, p2.dv, 0x5140), __byte_perm(m2.dv, p2.dv, 0x7362),
                       __byte_perm(z.dvL, z.dv, 0x7362), __byte_perm(z.dv, z.dvR, 0x5140), oz);
        // dv(-1,-1) dv(1,-1) dv(-1,1) dv(1,1)
        desc_transpose(__byte_perm(m1.dvL, m1.dv, 0x6453), __byte_perm(m1.dv, m1.dvR, 0x4231),
                       __byte_perm(p1.dvL, p1.dv, 0x6453), __byte_perm(p1.dv, p1.dvR, 0x4231), ow);
        if (lane >= 1 && lane <= 30) {
            const int sw = (lane - 1) >> 1;
#pragma unroll
            for (int k = 0; k < 4; ++k) sm.out[q + ((k + sw) & 3)] = make_uint4(ox[k], oy[k], oz[k], ow[k]);
        }
        __syncwarp();
        if (y < Y0 + n) {
            uint4 *o = desc + (size_t)y * w + (c0 + 4 - 4 * lane);  // the strip's first output column
            const int cols = EDGE ? min(kDescStrip, w - (c0 + 4 - 4 * lane)) : kDescStrip;
#pragma unroll
            for (int t = lane; t < kDescStrip; t += 32) {
                if (t < cols) o[t] = sm.out[(t & ~3) + (((t & 3) + (t >> 3)) & 3)];
            }
        }
        __syncwarp();
    };

    stage(0, min(nr, kDescFirst));
    stage(kDescFirst, nr);
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncwarp();
    // Rings indexed by row relative to Y0: sums of image row m in P[(m+3) % 3],
    // gradient row m in G[(m+2) % 6].
    DescPart P[3];
    DescGrad G[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        part(m, P[m % 3]);
        if (m >= 2) grad(Y0 - 4 + m, P[(m + 1) % 3], P[(m + 2) % 3], P[m % 3], G[m - 2]);
    }
    for (int j0 = 0; j0 < n6; j0 += 6) {
        if (j0 == kDescFirst - 6) {  // rows of the second copy group from here on
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int j = j0 + k;  // j % 6 == k
            part(j + 6, P[k % 3]);
            grad(Y0 + j + 2, P[(k + 1) % 3], P[(k + 2) % 3], P[k % 3], G[(k + 4) % 6]);
            emit(Y0 + j, G[k % 6], G[(k + 1) % 6], G[(k + 2) % 6], G[(k + 3) % 6], G[(k + 4) % 6]);
        }
    }
}

__device__ __forceinline__ void descriptor_body(const DescArgs &a, const VB &vb, int rows) {
    __shared__ DescSmem s_desc[kDescWarps];
    const int warp = (int)(threadIdx.x >> 5);
    const int X = vb.x * kDescStrip;
    const int Y0 = (vb.y * kDescWarps + warp) * rows;
    const int w = a.w, h = a.h;
    if (Y0 >= h) return;  // the whole warp
    const uint8_t *img = vb.z ? a.imgR : a.imgL;
    uint4 *desc = vb.z ? a.descR : a.descL;
    const int c0 = X - 4 + 4 * (int)(threadIdx.x & 31);  // the lane's first column
    const int n = min(rows, h - Y0);
    if (X >= kDescStrip && X + 128 <= w)
        desc_walk<false>(s_desc[warp], img, desc, w, h, (size_t)a.pitch, c0, Y0, n);
    else
        desc_walk<true>(s_desc[warp], img, desc, w, h, (size_t)a.pitch, c0, Y0, n);
}

__global__ void __launch_bounds__(32 * kDescWarps) descriptor_kernel(DescArgs a, int rows) {
    descriptor_body(a, vb_single(), rows);
}

__global__ void __launch_bounds__(32 * kDescWarps)
    descriptor_kernel_b(const DescArgs *__restrict__ tab, VMap vm, int rows) {
    const VB vb = vb_batch(vm);
    descriptor_body(slot_entry(tab, vm.stride, vb.slot), vb, rows);
}

dim3 descriptor_grid(int w, int h, int two, int rows) {
    const int groups = (h + rows - 1) / rows;
    return dim3((w + kDescStrip - 1) / kDescStrip, (groups + kDescWarps - 1) / kDescWarps, two ? 2 : 1);
}

constexpr int kDescRowsOnePair = 6;
static_assert(kDescRowsOnePair <= kDescMaxRows, "the one-pair rows must fit the staging buffer");

elas_status launch_descriptors(const uint8_t *imgL, const uint8_t *imgR, int w, int h, int pitch,
                               uint8_t *descL, uint8_t *descR, cudaStream_t st) {
    DescArgs a{imgL, imgR, w, h, pitch, reinterpret_cast<uint4 *>(descL), reinterpret_cast<uint4 *>(descR)};
    descriptor_kernel<<<descriptor_grid(w, h, imgR != nullptr, kDescRowsOnePair), 32 * kDescWarps, 0, st>>>(
        a, kDescRowsOnePair);
    return launch_status("descriptor_kernel");
}

elas_status launch_descriptors_b(const DescArgs *tab, const DescArgs *host, const VMap &pairs, int rows,
                                 cudaStream_t st) {
    if (!valid_desc_rows(rows)) return fail(ELAS_ERR_INVALID_ARG, "descriptor rows per warp %d", rows);
    VMap m;
    vmap_clear(m, pairs.stride);
    for (int i = 0; i < pairs.n; ++i) {
        const DescArgs &d = slot_entry(host, pairs.stride, pairs.slot[i]);
        vmap_add(m, pairs.slot[i], descriptor_grid(d.w, d.h, d.imgR != nullptr, rows));
    }
    const int total = vmap_total(m);
    if (total == 0) return ELAS_OK;
    descriptor_kernel_b<<<total, 32 * kDescWarps, 0, st>>>(tab, m, rows);
    return launch_status("descriptor_kernel_b");
}

// ---------------------------------------------------------------------------
// Census transform (Sec. VI.A).  Bit k = (dy + R) * W + (dx + R) of a pixel
// is set iff its neighbour at (dx, dy) is darker than the pixel (R = W/2);
// neighbours outside the image repeat the nearest border pixel, so every
// pixel has a full W x W census.  One CTA per 128x8 tile of one image: the
// tile and its halo are staged in shared memory with clamped coordinates
// (rows as 32-bit words, R4 = R rounded up to 4 bytes each side).  A thread
// takes four adjacent pixels of a row: for every offset the four neighbour
// bytes are one funnel shift of the row's words, the four comparisons one
// byte-wise "less than" (bytes_lt), and the four bits go to byte lanes of an
// accumulator (bit k & 7 of lane j for pixel j); four accumulators
// (k >> 3 & 3) make one 32-bit word of every pixel after a byte transpose.
// The loops are unrolled, so every position is a constant.  NW = 8 words
// for the 32-byte support record, 4 for the 16-byte dense record.
// ---------------------------------------------------------------------------
constexpr int kCensusPX = 4;                             // adjacent pixels of a thread
constexpr int kCensusTW = 32 * kCensusPX, kCensusTH = 8;  // tile: one warp per row

// Bit 7 of byte j is [n_j < c_j] for unsigned bytes (the other bits carry
// nothing).  (n_j | 0x80) - (c_j & 0x7F) lies in [1, 255], so it borrows
// nothing from the next byte, and its bit 7 is [n_j & 0x7F >= c_j & 0x7F];
// n < c iff the top bits are 0 < 1, or equal with the low bits n < c.
__device__ __forceinline__ uint32_t bytes_lt(uint32_t n, uint32_t c, uint32_t c_low) {
    const uint32_t d = (n | 0x80808080u) - c_low;
    return (~n & c) | (~(n ^ c) & ~d);
}

template <int W, int NW> __device__ __forceinline__ void census_body(const CensusArgs &a, const VB &vb) {
    constexpr int R = W / 2, R4 = (R + 3) & ~3;
    constexpr int SWB = kCensusTW + 2 * R4, SWW = SWB / 4, SH = kCensusTH + 2 * R;
    constexpr int RW0 = (R4 - R) / 4, NRW = (R4 + R + 3) / 4 - RW0 + 1;  // row words a thread reads
    static_assert(W * W <= 32 * NW, "census window does not fit the record");
    static_assert((R4 + R + 3) / 4 <= R4 / 2, "a thread's row words stay inside the staged row");
    __shared__ uint32_t s[SH][SWW];
    const uint8_t *img = vb.z ? a.imgR : a.imgL;
    uint4 *out = vb.z ? a.outR : a.outL;
    const int w = a.w, h = a.h;
    const int x0 = vb.x * kCensusTW, y0 = vb.y * kCensusTH;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    uint8_t *sb = reinterpret_cast<uint8_t *>(&s[0][0]);
    for (int i = tid; i < SH * SWB; i += blockDim.x * blockDim.y) {
        const int sy = i / SWB, sx = i - sy * SWB;
        const int x = min(max(x0 - R4 + sx, 0), w - 1), y = min(max(y0 - R + sy, 0), h - 1);
        sb[i] = img[(size_t)y * a.pitch + x];
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + kCensusPX * tx, y = y0 + ty;
    if (x >= w || y >= h) return;
    const uint32_t c = s[ty + R][R4 / 4 + tx];  // the four pixels
    const uint32_t c_low = c & 0x7F7F7F7Fu;
    uint32_t word[kCensusPX][NW];
#pragma unroll
    for (int j = 0; j < kCensusPX; ++j)
#pragma unroll
        for (int q = 0; q < NW; ++q) word[j][q] = 0u;
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
        uint32_t rw[NRW];
#pragma unroll
        for (int q = 0; q < NRW; ++q) rw[q] = s[ty + R + dy][tx + RW0 + q];
#pragma unroll
        for (int dx = -R; dx <= R; ++dx) {
            const int k = (dy + R) * W + (dx + R);
            const int off = R4 + dx, lo = off / 4 - RW0, sh = 8 * (off % 4);
            const uint32_t n = sh == 0 ? rw[lo] : __funnelshift_r(rw[lo], rw[lo + 1], sh);
            const int bit = k & 7;
            acc[(k >> 3) & 3] |= (bytes_lt(n, c, c_low) >> (7 - bit)) & (0x01010101u << bit);
            if ((k & 31) == 31 || k == W * W - 1) {
                // bytes 0..3 of word k >> 5 of the four pixels, transposed
                const uint32_t lo01 = __byte_perm(acc[0], acc[1], 0x5140), hi01 = __byte_perm(acc[0], acc[1], 0x7362);
                const uint32_t lo23 = __byte_perm(acc[2], acc[3], 0x5140), hi23 = __byte_perm(acc[2], acc[3], 0x7362);
                word[0][k >> 5] = __byte_perm(lo01, lo23, 0x5410);
                word[1][k >> 5] = __byte_perm(lo01, lo23, 0x7632);
                word[2][k >> 5] = __byte_perm(hi01, hi23, 0x5410);
                word[3][k >> 5] = __byte_perm(hi01, hi23, 0x7632);
                acc[0] = acc[1] = acc[2] = acc[3] = 0u;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kCensusPX; ++j) {
        if (x + j >= w) break;
        uint4 *o = out + ((size_t)y * w + x + j) * (NW / 4);
#pragma unroll
        for (int q = 0; q < NW / 4; ++q)
            o[q] = make_uint4(word[j][4 * q], word[j][4 * q + 1], word[j][4 * q + 2], word[j][4 * q + 3]);
    }
}

template <int W, int NW> __global__ void __launch_bounds__(32 * kCensusTH) census_kernel(CensusArgs a) {
    census_body<W, NW>(a, vb_single());
}
template <int W, int NW>
__global__ void __launch_bounds__(32 * kCensusTH) census_kernel_b(const CensusArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    census_body<W, NW>(slot_entry(tab, vm.stride, vb.slot), vb);
}

static dim3 census_grid(int w, int h, int two) {
    return dim3((w + kCensusTW - 1) / kCensusTW, (h + kCensusTH - 1) / kCensusTH, two ? 2 : 1);
}

template <int W, int NW>
static elas_status census_launch(const CensusArgs &a, int two, cudaStream_t st) {
    census_kernel<W, NW><<<census_grid(a.w, a.h, two), dim3(32, kCensusTH), 0, st>>>(a);
    return launch_status("census_kernel");
}

template <int W, int NW> static void census_launch_b(const CensusArgs *tab, const VMap &m, cudaStream_t st) {
    census_kernel_b<W, NW><<<vmap_total(m), dim3(32, kCensusTH), 0, st>>>(tab, m);
}

bool census_shape_ok(int window, int nbytes) {
    if (nbytes != 16 && nbytes != 32) return false;
    if (window < 3 || window % 2 == 0) return false;
    return window * window <= 8 * nbytes;
}

elas_status launch_census(const uint8_t *imgL, const uint8_t *imgR, int w, int h, int pitch, int window, int nbytes,
                          uint8_t *outL, uint8_t *outR, cudaStream_t st) {
    const CensusArgs a{imgL, imgR, w, h, pitch, reinterpret_cast<uint4 *>(outL), reinterpret_cast<uint4 *>(outR),
                       window};
    const int two = imgR != nullptr;
    if (nbytes == 32) {
        switch (window) {
        case 3: return census_launch<3, 8>(a, two, st);
        case 5: return census_launch<5, 8>(a, two, st);
        case 7: return census_launch<7, 8>(a, two, st);
        case 9: return census_launch<9, 8>(a, two, st);
        case 11: return census_launch<11, 8>(a, two, st);
        case 13: return census_launch<13, 8>(a, two, st);
        case 15: return census_launch<15, 8>(a, two, st);
        }
    } else if (nbytes == 16) {
        switch (window) {
        case 3: return census_launch<3, 4>(a, two, st);
        case 5: return census_launch<5, 4>(a, two, st);
        case 7: return census_launch<7, 4>(a, two, st);
        case 9: return census_launch<9, 4>(a, two, st);
        case 11: return census_launch<11, 4>(a, two, st);
        }
    }
    return fail(ELAS_ERR_INVALID_ARG, "census window %d with %d bytes per pixel", window, nbytes);
}

// Batched census records: one launch per window size among the pairs (a
// batch of the paper's variant normally has one), every pair's tiles in it.
elas_status launch_census_b(const CensusArgs *tab, const CensusArgs *host, const VMap &pairs, int nbytes,
                            cudaStream_t st) {
    bool done[16] = {};
    for (int i = 0; i < pairs.n; ++i) {
        const int win = slot_entry(host, pairs.stride, pairs.slot[i]).window;
        if (!census_shape_ok(win, nbytes)) return fail(ELAS_ERR_INVALID_ARG, "census window %d, %d bytes", win, nbytes);
        if (done[win]) continue;
        done[win] = true;
        VMap m;
        vmap_clear(m, pairs.stride);
        for (int j = i; j < pairs.n; ++j) {
            const CensusArgs &c = slot_entry(host, pairs.stride, pairs.slot[j]);
            if (c.window == win) vmap_add(m, pairs.slot[j], census_grid(c.w, c.h, c.imgR != nullptr));
        }
        if (nbytes == 32) {
            switch (win) {
            case 3: census_launch_b<3, 8>(tab, m, st); break;
            case 5: census_launch_b<5, 8>(tab, m, st); break;
            case 7: census_launch_b<7, 8>(tab, m, st); break;
            case 9: census_launch_b<9, 8>(tab, m, st); break;
            case 11: census_launch_b<11, 8>(tab, m, st); break;
            case 13: census_launch_b<13, 8>(tab, m, st); break;
            case 15: census_launch_b<15, 8>(tab, m, st); break;
            }
        } else {
            switch (win) {
            case 3: census_launch_b<3, 4>(tab, m, st); break;
            case 5: census_launch_b<5, 4>(tab, m, st); break;
            case 7: census_launch_b<7, 4>(tab, m, st); break;
            case 9: census_launch_b<9, 4>(tab, m, st); break;
            case 11: census_launch_b<11, 4>(tab, m, st); break;
            }
        }
        elas_status s = launch_status("census_kernel_b");
        if (s != ELAS_OK) return s;
    }
    return ELAS_OK;
}

}  // namespace elas

extern "C" elas_status elas_census(const uint8_t *imgL, const uint8_t *imgR, int32_t w, int32_t h, int32_t pitch,
                                   int32_t window, int32_t nbytes, uint8_t *outL, uint8_t *outR,
                                   elas_stream stream) {
    using namespace elas;
    if (w < 1 || h < 1 || w > 16383 || h > 16383) return fail(ELAS_ERR_INVALID_ARG, "image size %dx%d", w, h);
    if (pitch < w) return fail(ELAS_ERR_INVALID_ARG, "pitch %d < width %d", pitch, w);
    if (!census_shape_ok(window, nbytes))
        return fail(ELAS_ERR_INVALID_ARG, "census window %d with %d bytes per pixel (odd 3..15 in 32 bytes, 3..11 in 16)",
                    window, nbytes);
    if (!imgL || !outL) return fail(ELAS_ERR_INVALID_ARG, "NULL left image or census buffer");
    if ((imgR == nullptr) != (outR == nullptr))
        return fail(ELAS_ERR_INVALID_ARG, "imgR and outR must both be set or both be NULL");
    if (!aligned(outL, 16) || (outR && !aligned(outR, 16)))
        return fail(ELAS_ERR_INVALID_ARG, "census buffers must be 16-byte aligned");
    return launch_census(imgL, imgR, w, h, pitch, window, nbytes, outL, outR, to_stream(stream));
}

extern "C" elas_status elas_descriptors(const uint8_t *imgL, const uint8_t *imgR, int32_t w, int32_t h,
                                        int32_t pitch, uint8_t *descL, uint8_t *descR,
                                        elas_stream stream) {
    using namespace elas;
    if (w < 1 || h < 1 || w > 16383 || h > 16383) return fail(ELAS_ERR_INVALID_ARG, "image size %dx%d", w, h);
    if (pitch < w) return fail(ELAS_ERR_INVALID_ARG, "pitch %d < width %d", pitch, w);
    if (!imgL || !descL) return fail(ELAS_ERR_INVALID_ARG, "NULL left image or descriptor buffer");
    if ((imgR == nullptr) != (descR == nullptr))
        return fail(ELAS_ERR_INVALID_ARG, "imgR and descR must both be set or both be NULL");
    if (!aligned(descL, 16) || (descR && !aligned(descR, 16)))
        return fail(ELAS_ERR_INVALID_ARG, "descriptor buffers must be 16-byte aligned");
    return launch_descriptors(imgL, imgR, w, h, pitch, descL, descR, to_stream(stream));
}
