// Left-right consistency check and post-processing (Sec. III.A, Fig. 1(i)).
//
// lr_check_kernel   one CTA per image row; both rows are staged in shared
//                   memory before any write, so the in-place update reads
//                   only unmodified values (rows are independent).
// post_pass_kernel  one pass per launch, one thread per pixel: gap
//                   interpolation along rows or columns (the maximal invalid
//                   run through a pixel is found by scanning at most
//                   ipol_gap_width steps each way), the adaptive mean along
//                   rows or columns (taps in ascending offset order, FP32
//                   without contraction), or the copy to float.
#include "launch.cuh"

namespace elas {

__device__ __forceinline__ void lr_check_body(const LrArgs &a, const VB &vb) {
    extern __shared__ int16_t s_rows[];
    const int w = a.w, thr = a.thr;
    int16_t *sL = s_rows, *sR = s_rows + w;
    int16_t *__restrict__ dL = a.dL;
    int16_t *__restrict__ dR = a.dR;
    uint8_t *maskL = a.maskL, *maskR = a.maskR;
    const size_t row = (size_t)vb.x * w;
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

__global__ void __launch_bounds__(256) lr_check_kernel(LrArgs a) { lr_check_body(a, vb_single()); }
__global__ void __launch_bounds__(256) lr_check_kernel_b(const LrArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    lr_check_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

// Gap interpolation along a row or a column at element k of a line of
// length len (stride es from base); In is LineIn (global maps, size_t
// indices) or SmemIn (a shared tile, int indices).
template <class In, class I>
__device__ __forceinline__ float gap_at(const In &in, I base, I es, int k, int len, int gap) {
    const float x = in.at(base + (I)k * es);
    float res = x;
    if (x < 0.0f) {
        // nearest valid element on each side within gap steps
        int l = -1, r = -1;
        for (int s = 1; s <= gap && k - s >= 0; ++s)
            if (in.at(base + (I)(k - s) * es) >= 0.0f) { l = k - s; break; }
        for (int s = 1; s <= gap && k + s < len; ++s)
            if (in.at(base + (I)(k + s) * es) >= 0.0f) { r = k + s; break; }
        if (l >= 0 && r >= 0 && r - l - 1 <= gap) {
            const float d1 = in.at(base + (I)l * es), d2 = in.at(base + (I)r * es);
            res = fabsf(__fsub_rn(d1, d2)) < 3.0f ? __fmul_rn(__fadd_rn(d1, d2), 0.5f) : fminf(d1, d2);
        }
    }
    return res;
}

constexpr int kMeanRadius = 3;

// Adaptive mean along a line: taps in ascending offset order, FP32 without
// contraction.
template <class In, class I>
__device__ __forceinline__ float mean_at(const In &in, I base, I es, int k, int len) {
    const float d0 = in.at(base + (I)k * es);
    float res = d0;
    if (d0 >= 0.0f) {
        float sw = 0.0f, swd = 0.0f;
#pragma unroll
        for (int o = -kMeanRadius; o <= kMeanRadius; ++o) {
            const int m = k + o;
            if (m < 0 || m >= len) continue;
            const float di = in.at(base + (I)m * es);
            if (di < 0.0f) continue;
            const float wgt = __fsub_rn(4.0f, fabsf(__fsub_rn(di, d0)));
            if (wgt > 0.0f) {
                sw = __fadd_rn(sw, wgt);
                swd = __fadd_rn(swd, __fmul_rn(wgt, di));
            }
        }
        res = __fdiv_rn(swd, sw);
    }
    return res;
}

// One pass of post-processing over a 32x8 pixel tile: gap interpolation or
// adaptive mean along rows or columns, or the int16 -> float copy.
__device__ __forceinline__ void post_pass_body(const PostArgs &a, const VB &vb) {
    const int w = a.w, h = a.h;
    const int u = vb.x * blockDim.x + threadIdx.x;
    const int v = vb.y * blockDim.y + threadIdx.y;
    if (u >= w || v >= h) return;
    const int kind = a.kind;
    float res;
    if (kind == kPostCopy) {
        res = a.in.at((size_t)v * w + u);
    } else {
        const int vertical = kind == kPostGapCols || kind == kPostMeanCols;
        const int len = vertical ? h : w;
        const int k = vertical ? v : u;
        const size_t base = vertical ? (size_t)u : (size_t)v * w;
        const size_t es = vertical ? (size_t)w : 1;
        res = kind <= kPostGapCols ? gap_at(a.in, base, es, k, len, a.gap) : mean_at(a.in, base, es, k, len);
    }
    a.out[(size_t)v * w + u] = res;
}

__global__ void __launch_bounds__(256) post_pass_kernel(PostArgs a) { post_pass_body(a, vb_single()); }
__global__ void __launch_bounds__(256) post_pass_kernel_b(const PostArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    post_pass_body(slot_entry(tab, vm.stride, vb.slot), vb);
}

// ---------------------------------------------------------------------------
// Fused post-processing: the four passes on one TX x TY tile in shared memory
// (32 x 16 for one map, 32 x 32 in batched launches).
//
// The output tile needs the vertical mean over rows +-3 (r), which needs the
// horizontal mean over columns +-3, which needs the column gap pass over
// rows +-g (g = ipol_gap_width), which needs the row gap pass over columns
// +-g: the tile is loaded with a halo H = r + g, pixels outside the image
// read -1.  That is the same as the per-pass kernels, whose searches stop at
// the image border, because a -1 is never taken as a valid neighbour or a
// tap.  Each pass runs over exactly the region the next one reads, with the
// same per-element functions as the per-pass kernels.  Each region is walked
// as one linear index split into row and column by a multiply-high.
// ---------------------------------------------------------------------------
constexpr int kFusedTX = 32;       // tile width (one warp across)
constexpr int kFusedTY = 32;       // batched launches (many tiles in any case)
constexpr int kFusedTYOne = 16;    // one-map launches: more CTAs for one map
constexpr int kFusedMaxGap = 16;
constexpr int kFusedHalo = kFusedMaxGap + kMeanRadius;

struct SmemIn {
    const float *s;
    __device__ __forceinline__ float at(int idx) const { return s[idx]; }
};

// Row of element i of a region w wide: floor(i / w) = umulhi(i, m) with
// m = floor((2^32 - 1) / w) + 1, exact for i < 2^32 / w (here i < 2^13).
struct RowSplit {
    unsigned w, m;
    __device__ __forceinline__ explicit RowSplit(int width) : w((unsigned)width), m(0xFFFFFFFFu / (unsigned)width + 1u) {}
    __device__ __forceinline__ void at(int i, int &row, int &col) const {
        const unsigned q = w == 1u ? (unsigned)i : __umulhi((unsigned)i, m);
        row = (int)q;
        col = i - (int)(q * w);
    }
};

template <int TY>
__device__ __forceinline__ void fused_post_body(const FusedPostArgs &a, const VB &vb) {
    constexpr int TX = kFusedTX;
    __shared__ float s_a[(TY + 2 * kFusedHalo) * (TX + 2 * kFusedHalo)];
    __shared__ float s_b[(TY + 2 * kFusedHalo) * (TX + 2 * kFusedHalo)];
    const int w = a.w, h = a.h;
    const int g = a.gap, r = a.mean ? kMeanRadius : 0, H = g + r;
    const int PX = TX + 2 * H, PY = TY + 2 * H;  // tile pitch and rows
    const int x0 = vb.x * TX - H, y0 = vb.y * TY - H;
    const int tid = threadIdx.x, nth = blockDim.x;
    const RowSplit full(PX), inner(PX - 2 * g);
    for (int i = tid; i < PX * PY; i += nth) {
        int yy, xx;
        full.at(i, yy, xx);
        const int gx = x0 + xx, gy = y0 + yy;
        s_a[i] = (gx >= 0 && gx < w && gy >= 0 && gy < h) ? (float)a.d[(size_t)gy * w + gx] : -1.0f;
    }
    __syncthreads();
    float *cur = s_a, *nxt = s_b;
    if (g > 0) {
        const int cw = PX - 2 * g;
        // rows: every row, the columns the later passes read
        for (int i = tid; i < cw * PY; i += nth) {
            int yy, c;
            inner.at(i, yy, c);
            nxt[yy * PX + g + c] = gap_at(SmemIn{cur}, yy * PX, 1, g + c, PX, g);
        }
        __syncthreads();
        // columns: those columns, the rows the means read
        for (int i = tid; i < cw * (PY - 2 * g); i += nth) {
            int rr, c;
            inner.at(i, rr, c);
            cur[(g + rr) * PX + g + c] = gap_at(SmemIn{nxt}, g + c, PX, g + rr, PY, g);
        }
        __syncthreads();
    }
    if (r > 0) {
        // horizontal mean: the output columns, rows +-r (TX = 32: lane = column)
        for (int i = tid; i < TX * (TY + 2 * r); i += nth) {
            const int yy = g + i / TX, xx = H + i % TX;
            nxt[yy * PX + xx] = mean_at(SmemIn{cur}, yy * PX, 1, xx, PX);
        }
        __syncthreads();
    }
    // vertical mean (or, without the means, the gap passes' result) to the output
    const float *src = r > 0 ? nxt : cur;
    for (int i = tid; i < TX * TY; i += nth) {
        const int yy = H + i / TX, xx = H + i % TX;
        const int gx = x0 + xx, gy = y0 + yy;
        if (gx >= w || gy >= h) continue;
        a.out[(size_t)gy * w + gx] = r > 0 ? mean_at(SmemIn{src}, xx, PX, yy, PY) : src[yy * PX + xx];
    }
}

__global__ void __launch_bounds__(256) fused_post_kernel(FusedPostArgs a) {
    fused_post_body<kFusedTYOne>(a, vb_single());
}
template <int TY>
__global__ void __launch_bounds__(256) fused_post_kernel_b(const FusedPostArgs *__restrict__ tab, VMap vm) {
    const VB vb = vb_batch(vm);
    fused_post_body<TY>(slot_entry(tab, vm.stride, vb.slot), vb);
}

bool post_fusable(const elas_params *p) { return p->ipol_gap_width <= kFusedMaxGap; }

FusedPostArgs fused_post_args(const int16_t *d, int w, int h, const elas_params *p, float *out) {
    return FusedPostArgs{d, out, w, h, p->ipol_gap_width > 0 ? p->ipol_gap_width : 0,
                         p->filter_adaptive_mean ? 1 : 0};
}

dim3 fused_post_grid(int w, int h, int tile_y) { return dim3((w + kFusedTX - 1) / kFusedTX, (h + tile_y - 1) / tile_y); }

size_t post_workspace(int w, int h) { return 2 * align_up((size_t)w * h * sizeof(float), 256); }

size_t lr_smem(int w) { return 2 * (size_t)w * sizeof(int16_t); }

static elas_status lr_smem_attr(const void *fn, size_t smem) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return launch_status("lr_check smem attribute");
    return ELAS_OK;
}

elas_status launch_lr_check(int16_t *dL, int16_t *dR, int w, int h, int thr, uint8_t *maskL, uint8_t *maskR,
                            cudaStream_t st) {
    const size_t smem = lr_smem(w);
    elas_status s = lr_smem_attr((const void *)lr_check_kernel, smem);
    if (s != ELAS_OK) return s;
    lr_check_kernel<<<h, 256, smem, st>>>(LrArgs{dL, dR, w, h, thr, maskL, maskR});
    return launch_status("lr_check_kernel");
}

// The ordered passes of post-processing for one map: gap interpolation
// (rows, then columns) and the adaptive mean (rows, then columns); the last
// pass writes `out`, the others alternate between the two scratch maps.  With
// no pass enabled the one pass is the copy to float.
int post_passes(const int16_t *d, int w, int h, const elas_params *p, float *out, void *ws, PostArgs *passes) {
    float *A = reinterpret_cast<float *>(ws);
    float *B = reinterpret_cast<float *>(reinterpret_cast<char *>(ws) + align_up((size_t)w * h * sizeof(float), 256));
    int kinds[4], np = 0;
    if (p->ipol_gap_width > 0) {
        kinds[np++] = kPostGapRows;
        kinds[np++] = kPostGapCols;
    }
    if (p->filter_adaptive_mean) {
        kinds[np++] = kPostMeanRows;
        kinds[np++] = kPostMeanCols;
    }
    if (np == 0) kinds[np++] = kPostCopy;
    LineIn in{d, nullptr};
    for (int i = 0; i < np; ++i) {
        float *dst = (i == np - 1) ? out : ((i & 1) ? B : A);
        passes[i] = PostArgs{in, dst, w, h, kinds[i], p->ipol_gap_width};
        in = LineIn{nullptr, dst};
    }
    return np;
}

dim3 post_grid(int w, int h) { return dim3((w + 31) / 32, (h + 7) / 8); }

elas_status launch_post(const int16_t *d, int w, int h, const elas_params *p, float *out, void *ws, cudaStream_t st) {
    if (post_fusable(p)) {
        fused_post_kernel<<<fused_post_grid(w, h, kFusedTYOne), 256, 0, st>>>(fused_post_args(d, w, h, p, out));
        return launch_status("fused_post_kernel");
    }
    PostArgs passes[4];
    const int np = post_passes(d, w, h, p, out, ws, passes);
    for (int i = 0; i < np; ++i) {
        post_pass_kernel<<<post_grid(w, h), dim3(32, 8), 0, st>>>(passes[i]);
        elas_status s = launch_status("post_pass_kernel");
        if (s != ELAS_OK) return s;
    }
    return ELAS_OK;
}

// Batched LR check and post-processing.  Pairs with fused[i] run the fused
// kernel (table fused_tab); the others run npass[i] separate passes, pass k
// from table post_tab[k] (npass 0 and not fused: no post-processing).
elas_status launch_lr_post_b(const LrArgs *lr_tab, const LrArgs *host_lr, const PostArgs *const *post_tab,
                             const int *npass, const FusedPostArgs *fused_tab, const int *fused, const VMap &pairs,
                             cudaStream_t st) {
    if (pairs.n == 0) return ELAS_OK;
    VMap m_lr;
    vmap_clear(m_lr, pairs.stride);
    int maxw = 1, maxp = 0;
    for (int i = 0; i < pairs.n; ++i) {
        const LrArgs &l = slot_entry(host_lr, pairs.stride, pairs.slot[i]);
        vmap_add(m_lr, pairs.slot[i], dim3(l.h));
        maxw = max(maxw, l.w);
        maxp = max(maxp, npass[i]);
    }
    const size_t smem = lr_smem(maxw);
    elas_status s = lr_smem_attr((const void *)lr_check_kernel_b, smem);
    if (s != ELAS_OK) return s;
    lr_check_kernel_b<<<vmap_total(m_lr), 256, smem, st>>>(lr_tab, m_lr);
    if ((s = launch_status("lr_check_kernel_b")) != ELAS_OK) return s;
    VMap m_f;
    vmap_clear(m_f, pairs.stride);
    const int tile = pairs.n == 1 ? kFusedTYOne : kFusedTY;  // one map: the one-map tiles
    for (int i = 0; i < pairs.n; ++i) {
        const LrArgs &l = slot_entry(host_lr, pairs.stride, pairs.slot[i]);
        vmap_add(m_f, pairs.slot[i], fused[i] ? fused_post_grid(l.w, l.h, tile) : dim3(0));
    }
    if (vmap_total(m_f) > 0) {
        if (tile == kFusedTYOne)
            fused_post_kernel_b<kFusedTYOne><<<vmap_total(m_f), 256, 0, st>>>(fused_tab, m_f);
        else
            fused_post_kernel_b<kFusedTY><<<vmap_total(m_f), 256, 0, st>>>(fused_tab, m_f);
        if ((s = launch_status("fused_post_kernel_b")) != ELAS_OK) return s;
    }
    for (int k = 0; k < maxp && k < 4; ++k) {
        VMap m;
        vmap_clear(m, pairs.stride);
        for (int i = 0; i < pairs.n; ++i) {
            const LrArgs &l = slot_entry(host_lr, pairs.stride, pairs.slot[i]);
            vmap_add(m, pairs.slot[i], k < npass[i] ? post_grid(l.w, l.h) : dim3(0));
        }
        if (vmap_total(m) == 0) continue;
        post_pass_kernel_b<<<vmap_total(m), dim3(32, 8), 0, st>>>(post_tab[k], m);
        if ((s = launch_status("post_pass_kernel_b")) != ELAS_OK) return s;
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

// ---------------------------------------------------------------------------
// Median filter (Sec. VII, the refinement applied for the comparison with
// CSM; the paper gives no size).  Every valid pixel takes the median of the
// valid disparities in its (2r+1) x (2r+1) window clipped to the image (the
// lower median, element (n-1)/2 in sorted order, for an even count n);
// invalid pixels stay -1.  A 32x8 tile with its halo in shared memory (cells
// outside the image read -1, so they drop out as invalid values).  For a
// 3x3 window the nine values are sorted in registers by odd-even
// transposition (invalid -1 first); for larger ones the window is loaded
// into registers and the median is selected bit by bit: disparities are
// below 1024, so from bit 9 down, the count of valid values that share the
// bits chosen so far and have a 0 at the current bit decides that bit of the
// k-th smallest value (k = (n-1)/2).
// ---------------------------------------------------------------------------
namespace elas {

constexpr int kMedTX = 32, kMedTY = 8, kMedMaxR = 3;

template <int R> __device__ __forceinline__ int median_select(const int16_t *c, int SW) {
    constexpr int N = (2 * R + 1) * (2 * R + 1);
    int v[N];
    int n = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        v[j] = c[(j / (2 * R + 1) - R) * SW + (j % (2 * R + 1) - R)];
        n += v[j] >= 0;
    }
    int k = (n - 1) / 2, val = 0;
#pragma unroll
    for (int b = 9; b >= 0; --b) {
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) cnt += (v[j] >= 0) & ((v[j] >> b) == (val >> b));
        if (k >= cnt) {
            k -= cnt;
            val |= 1 << b;
        }
    }
    return val;
}

__global__ void __launch_bounds__(kMedTX *kMedTY) median_kernel(const int16_t *__restrict__ d, int w, int h, int r,
                                                                int16_t *__restrict__ out) {
    __shared__ int16_t s[(kMedTY + 2 * kMedMaxR) * (kMedTX + 2 * kMedMaxR)];
    const int SW = kMedTX + 2 * r, SH = kMedTY + 2 * r;
    const int x0 = blockIdx.x * kMedTX - r, y0 = blockIdx.y * kMedTY - r;
    const int tid = threadIdx.y * kMedTX + threadIdx.x;
    for (int k = tid; k < SW * SH; k += kMedTX * kMedTY) {
        const int x = x0 + k % SW, y = y0 + k / SW;
        s[k] = (x >= 0 && x < w && y >= 0 && y < h) ? d[(size_t)y * w + x] : (int16_t)-1;
    }
    __syncthreads();
    const int x = blockIdx.x * kMedTX + threadIdx.x, y = blockIdx.y * kMedTY + threadIdx.y;
    if (x >= w || y >= h) return;
    const int16_t *c = s + (threadIdx.y + r) * SW + threadIdx.x + r;
    int res = -1;
    if (c[0] >= 0 && r == 1) {
        // 3x3: odd-even transposition sort of the nine values in registers
        // (invalid -1 sorts first), the median among the valid ones after
        int v[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) v[j] = c[(j / 3 - 1) * SW + (j % 3 - 1)];
#pragma unroll
        for (int round = 0; round < 9; ++round)
#pragma unroll
            for (int j = round & 1; j + 1 < 9; j += 2) {
                const int lo = min(v[j], v[j + 1]), hi = max(v[j], v[j + 1]);
                v[j] = lo;
                v[j + 1] = hi;
            }
        int ninv = 0;
#pragma unroll
        for (int j = 0; j < 9; ++j) ninv += v[j] < 0;
        const int m = ninv + (9 - ninv - 1) / 2;
#pragma unroll
        for (int j = 0; j < 9; ++j)
            if (j == m) res = v[j];
    } else if (c[0] >= 0) {
        res = r == 0 ? c[0] : (r == 2 ? median_select<2>(c, SW) : median_select<3>(c, SW));
    }
    out[(size_t)y * w + x] = (int16_t)res;
}

}  // namespace elas

extern "C" elas_status elas_median(const int16_t *d, int32_t w, int32_t h, int32_t radius, int16_t *out,
                                   elas_stream stream) {
    using namespace elas;
    if (w < 1 || h < 1 || w > 16383 || h > 16383) return fail(ELAS_ERR_INVALID_ARG, "image size %dx%d", w, h);
    if (radius < 0 || radius > kMedMaxR) return fail(ELAS_ERR_INVALID_ARG, "median radius %d (0..%d)", radius, kMedMaxR);
    if (!d || !out) return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (d == out) return fail(ELAS_ERR_INVALID_ARG, "median output must not alias its input");
    const dim3 grid((w + kMedTX - 1) / kMedTX, (h + kMedTY - 1) / kMedTY);
    median_kernel<<<grid, dim3(kMedTX, kMedTY), 0, to_stream(stream)>>>(d, w, h, radius, out);
    return launch_status("median_kernel");
}
