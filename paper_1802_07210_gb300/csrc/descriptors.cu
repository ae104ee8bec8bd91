// Descriptors: Sobel gradient images quantised to uint8 and sampled into a
// 16-byte descriptor per pixel (Sec. III.A, Fig. 1(b-d); Sec. VI.A).
//
// One CTA produces a 32x8 tile of descriptors.  The image tile with a 3-pixel
// halo is staged in shared memory, the quantised du/dv planes of the tile
// with a 2-pixel halo are computed once into shared memory, and every thread
// assembles its pixel's 16 bytes and writes them as one 16-byte store
// (a warp writes 512 contiguous bytes).
#include "launch.cuh"

namespace elas {

constexpr int kDescTW = 32;
constexpr int kDescTH = 8;

__device__ __forceinline__ int quantise(int s) {
    int q = 128 + s / 4;  // truncation toward zero
    return q < 1 ? 1 : (q > 255 ? 255 : q);
}

__global__ void __launch_bounds__(kDescTW *kDescTH)
descriptor_kernel(const uint8_t *__restrict__ imgL, const uint8_t *__restrict__ imgR, int w, int h,
                  int pitch, uint4 *__restrict__ descL, uint4 *__restrict__ descR) {
    const uint8_t *img = blockIdx.z ? imgR : imgL;
    uint4 *desc = blockIdx.z ? descR : descL;

    constexpr int IW = kDescTW + 6, IH = kDescTH + 6;  // image tile with halo 3
    constexpr int QW = kDescTW + 4, QH = kDescTH + 4;  // gradient tile with halo 2
    __shared__ int16_t s_img[IH][IW];
    __shared__ uint8_t s_du[QH][QW];
    __shared__ uint8_t s_dv[QH][QW];

    const int x0 = blockIdx.x * kDescTW, y0 = blockIdx.y * kDescTH;
    const int tid = threadIdx.y * kDescTW + threadIdx.x;
    constexpr int NT = kDescTW * kDescTH;

    for (int i = tid; i < IW * IH; i += NT) {
        const int ix = i % IW, iy = i / IW;
        const int x = x0 - 3 + ix, y = y0 - 3 + iy;
        int val = 0;
        if (x >= 0 && x < w && y >= 0 && y < h) val = img[(size_t)y * pitch + x];
        s_img[iy][ix] = (int16_t)val;
    }
    __syncthreads();

    for (int i = tid; i < QW * QH; i += NT) {
        const int qx = i % QW, qy = i / QW;
        const int x = x0 - 2 + qx, y = y0 - 2 + qy;
        int qdu = 128, qdv = 128;
        if (x >= 1 && x <= w - 2 && y >= 1 && y <= h - 2) {
            const int ix = qx + 1, iy = qy + 1;  // image-tile coordinates of (x, y)
            const int a = s_img[iy - 1][ix - 1], b = s_img[iy - 1][ix], c = s_img[iy - 1][ix + 1];
            const int d = s_img[iy][ix - 1], f = s_img[iy][ix + 1];
            const int g = s_img[iy + 1][ix - 1], hh = s_img[iy + 1][ix], k = s_img[iy + 1][ix + 1];
            const int gx = (c + 2 * f + k) - (a + 2 * d + g);
            const int gy = (g + 2 * hh + k) - (a + 2 * b + c);
            qdu = quantise(gx);
            qdv = quantise(gy);
        }
        s_du[qy][qx] = (uint8_t)qdu;
        s_dv[qy][qx] = (uint8_t)qdv;
    }
    __syncthreads();

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= w || y >= h) return;
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

elas_status launch_descriptors(const uint8_t *imgL, const uint8_t *imgR, int w, int h, int pitch,
                               uint8_t *descL, uint8_t *descR, cudaStream_t st) {
    dim3 block(kDescTW, kDescTH, 1);
    dim3 grid((w + kDescTW - 1) / kDescTW, (h + kDescTH - 1) / kDescTH, imgR ? 2 : 1);
    descriptor_kernel<<<grid, block, 0, st>>>(imgL, imgR, w, h, pitch, reinterpret_cast<uint4 *>(descL),
                                              reinterpret_cast<uint4 *>(descR));
    return launch_status("descriptor_kernel");
}

}  // namespace elas

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
