// Descriptors: Sobel gradient images quantised to uint8 and sampled into a
// 16-byte descriptor per pixel (Sec. III.A, Fig. 1(b-d); Sec. VI.A); and the
// census transform of the paper's variant (Sec. VI.A, at the end).
//
// One CTA produces up to four 32xTH tiles of descriptors, one above the other
// (TH = 8 for the one-pair launch; 4, 8 or 16 in batched launches, chosen by
// the tuner).  The image tile with a 3-pixel halo is staged in shared memory, the quantised du/dv
// planes of the tile with a 2-pixel halo are computed once into shared
// memory, and every thread assembles its pixel's 16 bytes and writes them as
// one 16-byte store (a warp writes 512 contiguous bytes).
#include "launch.cuh"

namespace elas {

constexpr int kDescTW = 32;

__device__ __forceinline__ int quantise(int s) {
    int q = 128 + s / 4;  // truncation toward zero
    return q < 1 ? 1 : (q > 255 ? 255 : q);
}

// TH = tile height (image rows of a tile): one of 4, 8, 16.  A CTA makes
// kDescTiles vertically adjacent tiles in turn; the image bytes of the next
// tile are loaded into registers while the current one is computed, so the
// loads of one tile overlap the work of the previous one.
constexpr int kDescTiles = 4;

template <int TH>
__device__ __forceinline__ void descriptor_body(const DescArgs &a, const VB &vb) {
    const uint8_t *img = vb.z ? a.imgR : a.imgL;
    uint4 *desc = vb.z ? a.descR : a.descL;
    const int w = a.w, h = a.h, pitch = a.pitch;

    constexpr int IW = kDescTW + 6, IH = TH + 6;  // image tile with halo 3
    constexpr int QW = kDescTW + 4, QH = TH + 4;  // gradient tile with halo 2
    constexpr int NT = kDescTW * TH, NI = IW * IH;
    constexpr int PER = (NI + NT - 1) / NT;  // image bytes a thread loads per tile
    __shared__ int16_t s_img[IH][IW];
    __shared__ uint8_t s_du[QH][QW];
    __shared__ uint8_t s_dv[QH][QW];

    const int x0 = vb.x * kDescTW;
    const int tid = threadIdx.y * kDescTW + threadIdx.x;
    const int nty = (h + TH - 1) / TH, ty0 = vb.y * kDescTiles;
    const int ntile = min(kDescTiles, nty - ty0);

    int v[PER];
    auto fetch = [&](int ty) {
        const int y0 = ty * TH;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = tid + u * NT;
            const int ix = i % IW, iy = i / IW;
            const int x = x0 - 3 + ix, y = y0 - 3 + iy;
            v[u] = i < NI && x >= 0 && x < w && y >= 0 && y < h ? img[(size_t)y * pitch + x] : 0;
        }
    };
    fetch(ty0);
    for (int t = 0; t < ntile; ++t) {
        const int y0 = (ty0 + t) * TH;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = tid + u * NT;
            if (i < NI) s_img[i / IW][i % IW] = (int16_t)v[u];
        }
        __syncthreads();
        if (t + 1 < ntile) fetch(ty0 + t + 1);  // in flight while this tile is computed

        for (int i = tid; i < QW * QH; i += NT) {
            const int qx = i % QW, qy = i / QW;
            const int x = x0 - 2 + qx, y = y0 - 2 + qy;
            int qdu = 128, qdv = 128;
            if (x >= 1 && x <= w - 2 && y >= 1 && y <= h - 2) {
                const int ix = qx + 1, iy = qy + 1;  // image-tile coordinates of (x, y)
                const int a0 = s_img[iy - 1][ix - 1], b = s_img[iy - 1][ix], c = s_img[iy - 1][ix + 1];
                const int d = s_img[iy][ix - 1], f = s_img[iy][ix + 1];
                const int g = s_img[iy + 1][ix - 1], hh = s_img[iy + 1][ix], k = s_img[iy + 1][ix + 1];
                const int gx = (c + 2 * f + k) - (a0 + 2 * d + g);
                const int gy = (g + 2 * hh + k) - (a0 + 2 * b + c);
                qdu = quantise(gx);
                qdv = quantise(gy);
            }
            s_du[qy][qx] = (uint8_t)qdu;
            s_dv[qy][qx] = (uint8_t)qdv;
        }
        __syncthreads();

        const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
        if (x < w && y < h) {
            const int cx = threadIdx.x + 2, cy = threadIdx.y + 2;
#define DU(ox, oy) ((uint32_t)s_du[cy + (oy)][cx + (ox)])
#define DV(ox, oy) ((uint32_t)s_dv[cy + (oy)][cx + (ox)])
            uint4 o;
            o.x = DU(-2, -2) | (DU(2, -2) << 8) | (DU(-1, 0) << 16) | (DU(1, 0) << 24);
            o.y = DU(-2, 2) | (DU(2, 2) << 8) | (DU(0, -1) << 16) | (DU(0, 1) << 24);
            o.z = DV(0, -2) | (DV(0, 2) << 8) | (DV(-2, 0) << 16) | (DV(2, 0) << 24);
            o.w = DV(-1, -1) | (DV(1, -1) << 8) | (DV(-1, 1) << 16) | (DV(1, 1) << 24);
#undef DU
#undef DV
            desc[(size_t)y * w + x] = o;
        }
        __syncthreads();  // the next tile overwrites the shared tiles
    }
}

template <int TH> __global__ void __launch_bounds__(kDescTW *TH) descriptor_kernel(DescArgs a) {
    descriptor_body<TH>(a, vb_single());
}

template <int TH>
__global__ void __launch_bounds__(kDescTW *TH) descriptor_kernel_b(const DescArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    descriptor_body<TH>(slot_entry(tab, vm.stride, vb.slot), vb);
}

dim3 descriptor_grid(int w, int h, int two, int tile_rows) {
    const int nty = (h + tile_rows - 1) / tile_rows;
    return dim3((w + kDescTW - 1) / kDescTW, (nty + kDescTiles - 1) / kDescTiles, two ? 2 : 1);
}

static bool valid_tile_rows(int th) { return th == 4 || th == 8 || th == 16; }

elas_status launch_descriptors(const uint8_t *imgL, const uint8_t *imgR, int w, int h, int pitch,
                               uint8_t *descL, uint8_t *descR, cudaStream_t st) {
    DescArgs a{imgL, imgR, w, h, pitch, reinterpret_cast<uint4 *>(descL), reinterpret_cast<uint4 *>(descR)};
    descriptor_kernel<8><<<descriptor_grid(w, h, imgR != nullptr, 8), dim3(kDescTW, 8), 0, st>>>(a);
    return launch_status("descriptor_kernel");
}

elas_status launch_descriptors_b(const DescArgs *tab, const DescArgs *host, const VMap &pairs, int tile_rows,
                                 cudaStream_t st) {
    if (!valid_tile_rows(tile_rows)) return fail(ELAS_ERR_INVALID_ARG, "descriptor tile rows %d", tile_rows);
    VMap m;
    vmap_clear(m, pairs.stride);
    for (int i = 0; i < pairs.n; ++i) {
        const DescArgs &d = slot_entry(host, pairs.stride, pairs.slot[i]);
        vmap_add(m, pairs.slot[i], descriptor_grid(d.w, d.h, d.imgR != nullptr, tile_rows));
    }
    const int total = vmap_total(m);
    if (total == 0) return ELAS_OK;
    const dim3 block(kDescTW, tile_rows);
    if (tile_rows == 4)
        descriptor_kernel_b<4><<<total, block, 0, st>>>(tab, m);
    else if (tile_rows == 8)
        descriptor_kernel_b<8><<<total, block, 0, st>>>(tab, m);
    else
        descriptor_kernel_b<16><<<total, block, 0, st>>>(tab, m);
    return launch_status("descriptor_kernel_b");
}

// ---------------------------------------------------------------------------
// Census transform (Sec. VI.A).  Bit k = (dy + R) * W + (dx + R) of a pixel
// is set iff its neighbour at (dx, dy) is darker than the pixel (R = W/2);
// neighbours outside the image repeat the nearest border pixel, so every
// pixel has a full W x W census.  One CTA per 32x8 tile of one image: the
// tile and its R-pixel halo are staged in shared memory with clamped
// coordinates, then each thread compares its W*W neighbours (the loops are
// unrolled, so the bit positions are constants) and stores its NW 32-bit
// words as 16-byte vectors: NW = 8 for the 32-byte support record, 4 for the
// 16-byte dense record.
// ---------------------------------------------------------------------------
constexpr int kCensusTW = 32, kCensusTH = 8;

template <int W, int NW> __device__ __forceinline__ void census_body(const CensusArgs &a, const VB &vb) {
    constexpr int R = W / 2, SW = kCensusTW + 2 * R, SH = kCensusTH + 2 * R;
    static_assert(W * W <= 32 * NW, "census window does not fit the record");
    __shared__ uint8_t s[SH][SW];
    const uint8_t *img = vb.z ? a.imgR : a.imgL;
    uint4 *out = vb.z ? a.outR : a.outL;
    const int w = a.w, h = a.h;
    const int x0 = vb.x * kCensusTW, y0 = vb.y * kCensusTH;
    const int tid = threadIdx.y * kCensusTW + threadIdx.x;
    for (int i = tid; i < SW * SH; i += kCensusTW * kCensusTH) {
        const int sx = i % SW, sy = i / SW;
        const int x = min(max(x0 - R + sx, 0), w - 1), y = min(max(y0 - R + sy, 0), h - 1);
        s[sy][sx] = img[(size_t)y * a.pitch + x];
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= w || y >= h) return;
    const int cx = threadIdx.x + R, cy = threadIdx.y + R;
    const uint32_t c = s[cy][cx];
    uint32_t word[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) word[j] = 0u;
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
#pragma unroll
        for (int dx = -R; dx <= R; ++dx) {
            const int k = (dy + R) * W + (dx + R);
            word[k >> 5] |= (uint32_t)((uint32_t)s[cy + dy][cx + dx] < c) << (k & 31);
        }
    }
    uint4 *o = out + ((size_t)y * w + x) * (NW / 4);
#pragma unroll
    for (int j = 0; j < NW / 4; ++j) o[j] = make_uint4(word[4 * j], word[4 * j + 1], word[4 * j + 2], word[4 * j + 3]);
}

template <int W, int NW> __global__ void __launch_bounds__(kCensusTW *kCensusTH) census_kernel(CensusArgs a) {
    census_body<W, NW>(a, vb_single());
}
template <int W, int NW>
__global__ void __launch_bounds__(kCensusTW *kCensusTH) census_kernel_b(const CensusArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    census_body<W, NW>(slot_entry(tab, vm.stride, vb.slot), vb);
}

static dim3 census_grid(int w, int h, int two) {
    return dim3((w + kCensusTW - 1) / kCensusTW, (h + kCensusTH - 1) / kCensusTH, two ? 2 : 1);
}

template <int W, int NW>
static elas_status census_launch(const CensusArgs &a, int two, cudaStream_t st) {
    census_kernel<W, NW><<<census_grid(a.w, a.h, two), dim3(kCensusTW, kCensusTH), 0, st>>>(a);
    return launch_status("census_kernel");
}

template <int W, int NW> static void census_launch_b(const CensusArgs *tab, const VMap &m, cudaStream_t st) {
    census_kernel_b<W, NW><<<vmap_total(m), dim3(kCensusTW, kCensusTH), 0, st>>>(tab, m);
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
