// Left-right consistency check and post-processing (Sec. III.A, Fig. 1(i)).
//
// lr_check_kernel   one CTA per image row; both rows are staged in shared
//                   memory before any write, so the in-place update reads
//                   only unmodified values (rows are independent).
// gap_kernel        gap interpolation along rows or columns, one thread per
//                   pixel: the maximal invalid run through a pixel is found
//                   by scanning at most ipol_gap_width steps each way.
// mean_kernel       adaptive mean along rows or columns, one thread per
//                   pixel, taps in ascending offset order, FP32 without
//                   contraction.
#include "launch.cuh"

namespace elas {

__global__ void lr_check_kernel(int16_t *__restrict__ dL, int16_t *__restrict__ dR, int w, int thr,
                                uint8_t *__restrict__ maskL, uint8_t *__restrict__ maskR) {
    extern __shared__ int16_t s_rows[];
    int16_t *sL = s_rows, *sR = s_rows + w;
    const size_t row = (size_t)blockIdx.x * w;
    for (int u = threadIdx.x; u < w; u += blockDim.x) {
        sL[u] = dL[row + u];
        sR[u] = dR[row + u];
    }
    __syncthreads();
    for (int u = threadIdx.x; u < w; u += blockDim.x) {
        int d = sL[u], keep = 0;
        if (d >= 0 && u - d >= 0) {
            const int dr = sR[u - d];
            keep = dr >= 0 && abs(d - dr) <= thr;
        }
        dL[row + u] = keep ? (int16_t)d : (int16_t)-1;
        if (maskL) maskL[row + u] = (uint8_t)keep;
        d = sR[u];
        keep = 0;
        if (d >= 0 && u + d <= w - 1) {
            const int dl = sL[u + d];
            keep = dl >= 0 && abs(d - dl) <= thr;
        }
        dR[row + u] = keep ? (int16_t)d : (int16_t)-1;
        if (maskR) maskR[row + u] = (uint8_t)keep;
    }
}

// Value of element k along a line: from the int16 map or the float buffer.
struct LineIn {
    const int16_t *i16;
    const float *f32;
    __device__ __forceinline__ float at(size_t idx) const { return i16 ? (float)i16[idx] : f32[idx]; }
};

__global__ void gap_kernel(LineIn in, float *__restrict__ out, int w, int h, int vertical, int gap) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= w || v >= h) return;
    const int len = vertical ? h : w;
    const int k = vertical ? v : u;
    const size_t base = vertical ? (size_t)u : (size_t)v * w;
    const size_t es = vertical ? (size_t)w : 1;
    const float x = in.at(base + (size_t)k * es);
    float res = x;
    if (x < 0.0f) {
        // nearest valid element on each side within gap steps
        int l = -1, r = -1;
        for (int s = 1; s <= gap && k - s >= 0; ++s)
            if (in.at(base + (size_t)(k - s) * es) >= 0.0f) { l = k - s; break; }
        for (int s = 1; s <= gap && k + s < len; ++s)
            if (in.at(base + (size_t)(k + s) * es) >= 0.0f) { r = k + s; break; }
        if (l >= 0 && r >= 0 && r - l - 1 <= gap) {
            const float d1 = in.at(base + (size_t)l * es), d2 = in.at(base + (size_t)r * es);
            res = fabsf(__fsub_rn(d1, d2)) < 3.0f ? __fmul_rn(__fadd_rn(d1, d2), 0.5f) : fminf(d1, d2);
        }
    }
    out[(size_t)v * w + u] = res;
}

constexpr int kMeanRadius = 3;

__global__ void mean_kernel(LineIn in, float *__restrict__ out, int w, int h, int vertical) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= w || v >= h) return;
    const int len = vertical ? h : w;
    const int k = vertical ? v : u;
    const size_t base = vertical ? (size_t)u : (size_t)v * w;
    const size_t es = vertical ? (size_t)w : 1;
    const float d0 = in.at(base + (size_t)k * es);
    float res = d0;
    if (d0 >= 0.0f) {
        float sw = 0.0f, swd = 0.0f;
#pragma unroll
        for (int o = -kMeanRadius; o <= kMeanRadius; ++o) {
            const int m = k + o;
            if (m < 0 || m >= len) continue;
            const float di = in.at(base + (size_t)m * es);
            if (di < 0.0f) continue;
            const float wgt = __fsub_rn(4.0f, fabsf(__fsub_rn(di, d0)));
            if (wgt > 0.0f) {
                sw = __fadd_rn(sw, wgt);
                swd = __fadd_rn(swd, __fmul_rn(wgt, di));
            }
        }
        res = __fdiv_rn(swd, sw);
    }
    out[(size_t)v * w + u] = res;
}

__global__ void to_float_kernel(const int16_t *__restrict__ in, float *__restrict__ out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

size_t post_workspace(int w, int h) { return 2 * align_up((size_t)w * h * sizeof(float), 256); }

elas_status launch_lr_check(int16_t *dL, int16_t *dR, int w, int h, int thr, uint8_t *maskL, uint8_t *maskR,
                            cudaStream_t st) {
    const size_t smem = 2 * (size_t)w * sizeof(int16_t);
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(lr_check_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return launch_status("lr_check smem attribute");
    }
    lr_check_kernel<<<h, 256, smem, st>>>(dL, dR, w, thr, maskL, maskR);
    return launch_status("lr_check_kernel");
}

elas_status launch_post(const int16_t *d, int w, int h, const elas_params *p, float *out, void *ws, cudaStream_t st) {
    float *A = reinterpret_cast<float *>(ws);
    float *B = reinterpret_cast<float *>(reinterpret_cast<char *>(ws) + align_up((size_t)w * h * sizeof(float), 256));
    dim3 blk(32, 8), grd((w + 31) / 32, (h + 7) / 8);
    // ordered list of passes; the last one writes `out`
    int passes[4], np = 0;
    if (p->ipol_gap_width > 0) { passes[np++] = 0; passes[np++] = 1; }
    if (p->filter_adaptive_mean) { passes[np++] = 2; passes[np++] = 3; }
    if (np == 0) {
        const size_t n = (size_t)w * h;
        to_float_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, out, n);
        return launch_status("to_float_kernel");
    }
    LineIn in{d, nullptr};
    for (int i = 0; i < np; ++i) {
        float *dst = (i == np - 1) ? out : ((i & 1) ? B : A);
        const int kind = passes[i];
        if (kind < 2)
            gap_kernel<<<grd, blk, 0, st>>>(in, dst, w, h, kind == 1, p->ipol_gap_width);
        else
            mean_kernel<<<grd, blk, 0, st>>>(in, dst, w, h, kind == 3);
        elas_status s = launch_status(kind < 2 ? "gap_kernel" : "mean_kernel");
        if (s != ELAS_OK) return s;
        in = LineIn{nullptr, dst};
    }
    return ELAS_OK;
}

}  // namespace elas

extern "C" elas_status elas_lr_check(int16_t *dL, int16_t *dR, int32_t w, int32_t h, int32_t lr_threshold,
                                     uint8_t *maskL, uint8_t *maskR, elas_stream stream) {
    using namespace elas;
    if (w < 1 || h < 1 || w > 16383 || h > 16383) return fail(ELAS_ERR_INVALID_ARG, "image size %dx%d", w, h);
    if (!dL || !dR) return fail(ELAS_ERR_INVALID_ARG, "NULL disparity map");
    if (lr_threshold < 0) return fail(ELAS_ERR_INVALID_ARG, "lr_threshold %d", lr_threshold);
    return launch_lr_check(dL, dR, w, h, lr_threshold, maskL, maskR, to_stream(stream));
}

extern "C" size_t elas_postprocess_workspace_bytes(int32_t w, int32_t h) {
    if (w < 1 || h < 1) return 0;
    return elas::post_workspace(w, h);
}

extern "C" elas_status elas_postprocess(const int16_t *d, int32_t w, int32_t h, const elas_params *p, float *out,
                                        void *workspace, size_t workspace_bytes, elas_stream stream) {
    using namespace elas;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (!d || !out || !workspace) return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned(workspace, 256)) return fail(ELAS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (workspace_bytes < post_workspace(w, h))
        return fail(ELAS_ERR_CAPACITY, "workspace %zu < %zu bytes", workspace_bytes, post_workspace(w, h));
    return launch_post(d, w, h, p, out, workspace, to_stream(stream));
}
