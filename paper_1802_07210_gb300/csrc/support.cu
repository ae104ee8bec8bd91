// Support points (Sec. III.A; ratio test of Eq. 1-2), consistency and
// redundancy filtering (Sec. III.A), grid vectors (Sec. III.A, Fig. 2;
// one-hot masks, Sec. VI.D) and raster-order compaction.
//
// Kernels, in launch order:
//   support_match_kernel   one warp per lattice candidate; lanes stride the
//                          disparity range, each lane keeps (best, second)
//                          and the warp merges them with two min-reductions;
//                          the right-to-left re-match runs in the same warp.
//   consistency_kernel     one thread per candidate, window count.
//   redundancy_kernel      one thread per candidate, four directional scans.
//   grid_vector_kernel     one thread per surviving point, atomicOr of the
//                          {d-1,d,d+1} bits into the 3x3 cells (OR is order
//                          free, so the masks are deterministic).
//   compact_kernel         one CTA, block-wide exclusive scan, raster order.
#include "launch.cuh"

namespace elas {

struct SupportArgs {
    int w, h, step, wc, hc;
    int dmin, dmax;
    float thr;
    int support_texture, lr_threshold;
};

// Best disparity of the window (a0..a3 at (u+-2, v+-2)) against `oth`,
// searching other position uo = u + dir*d with 4 <= uo <= w-5.  Warp
// collective; returns d1 or -1 (ambiguous / not enough disparities).
__device__ __forceinline__ int warp_best_disparity(const uint4 *__restrict__ oth, int w, const uint4 &a0,
                                                   const uint4 &a1, const uint4 &a2, const uint4 &a3, int u,
                                                   int v, int dir, int dmin, int dmax, float thr, int lane) {
    int lo, hi;
    if (dir < 0) {
        lo = max(dmin, u - w + 5);
        hi = min(dmax, u - 4);
    } else {
        lo = max(dmin, 4 - u);
        hi = min(dmax, w - 5 - u);
    }
    if (hi - lo + 1 < 2) return -1;
    const uint4 *rowT = oth + (size_t)(v - 2) * w;
    const uint4 *rowB = oth + (size_t)(v + 2) * w;
    uint32_t m1 = 0xFFFFFFFFu, m2 = 0xFFFFFFFFu;
    int d1 = -1;
    for (int d = lo + lane; d <= hi; d += 32) {
        const int uo = u + dir * d;
        uint32_t c = sad16(a0, __ldg(rowT + uo - 2));
        c += sad16(a1, __ldg(rowT + uo + 2));
        c += sad16(a2, __ldg(rowB + uo - 2));
        c += sad16(a3, __ldg(rowB + uo + 2));
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
    return (__uint2float_rn(gm1) <= __fmul_rn(thr, __uint2float_rn(gm2))) ? gd1 : -1;
}

__global__ void __launch_bounds__(256)
support_match_kernel(const uint4 *__restrict__ dL, const uint4 *__restrict__ dR, SupportArgs a,
                     int16_t *__restrict__ raw) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.wc * a.hc) return;
    const int ic = warp / a.wc, jc = warp - ic * a.wc;
    const int u = jc * a.step, v = ic * a.step;
    int out = -1;
    if (u >= 4 && u <= a.w - 5 && v >= 4 && v <= a.h - 5) {
        const size_t rt = (size_t)(v - 2) * a.w, rb = (size_t)(v + 2) * a.w;
        const uint4 l0 = __ldg(dL + rt + u - 2), l1 = __ldg(dL + rt + u + 2);
        const uint4 l2 = __ldg(dL + rb + u - 2), l3 = __ldg(dL + rb + u + 2);
        const uint32_t texL = texture16(l0) + texture16(l1) + texture16(l2) + texture16(l3);
        if ((int)texL >= a.support_texture) {
            const int d1 = warp_best_disparity(dR, a.w, l0, l1, l2, l3, u, v, -1, a.dmin, a.dmax, a.thr, lane);
            if (d1 >= 0) {
                const int ur = u - d1;
                const uint4 r0 = __ldg(dR + rt + ur - 2), r1 = __ldg(dR + rt + ur + 2);
                const uint4 r2 = __ldg(dR + rb + ur - 2), r3 = __ldg(dR + rb + ur + 2);
                const uint32_t texR = texture16(r0) + texture16(r1) + texture16(r2) + texture16(r3);
                if ((int)texR >= a.support_texture) {
                    const int d2 =
                        warp_best_disparity(dL, a.w, r0, r1, r2, r3, ur, v, +1, a.dmin, a.dmax, a.thr, lane);
                    if (d2 >= 0 && abs(d1 - d2) <= a.lr_threshold) out = d1;
                }
            }
        }
    }
    if (lane == 0) raw[warp] = (int16_t)out;
}

__global__ void consistency_kernel(const int16_t *__restrict__ in, int wc, int hc, int r, int thr, int min_support,
                                   int16_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= wc * hc) return;
    const int ic = i / wc, jc = i - ic * wc;
    const int d = in[i];
    int res = -1;
    if (d >= 0) {
        int cnt = 0;
        const int i0 = max(0, ic - r), i1 = min(hc - 1, ic + r);
        const int j0 = max(0, jc - r), j1 = min(wc - 1, jc + r);
        for (int i2 = i0; i2 <= i1; ++i2)
            for (int j2 = j0; j2 <= j1; ++j2) {
                const int d2 = in[i2 * wc + j2];
                cnt += (d2 >= 0) & (abs(d2 - d) <= thr) & !(i2 == ic && j2 == jc);
            }
        if (cnt >= min_support) res = d;
    }
    out[i] = (int16_t)res;
}

__global__ void redundancy_kernel(const int16_t *__restrict__ in, int wc, int hc, int maxd, int enabled,
                                  int16_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= wc * hc) return;
    const int ic = i / wc, jc = i - ic * wc;
    const int d = in[i];
    int res = d;
    if (d >= 0 && enabled) {
        const int di[4] = {0, 0, -1, 1}, dj[4] = {-1, 1, 0, 0};
        bool redundant = true;
        for (int k = 0; k < 4 && redundant; ++k) {
            bool found = false;
            for (int s = 1; s <= maxd; ++s) {
                const int i2 = ic + s * di[k], j2 = jc + s * dj[k];
                if (i2 < 0 || i2 >= hc || j2 < 0 || j2 >= wc) break;
                if (in[i2 * wc + j2] == d) {
                    found = true;
                    break;
                }
            }
            redundant = found;
        }
        if (redundant) res = -1;
    }
    out[i] = (int16_t)(d >= 0 ? res : -1);
}

__device__ __forceinline__ void or_bits(uint32_t *cell, int d, int dmin, int dmax) {
    for (int dd = d - 1; dd <= d + 1; ++dd)
        if (dd >= dmin && dd <= dmax) atomicOr(cell + (dd >> 5), 1u << (dd & 31));
}

__global__ void grid_vector_kernel(const int16_t *__restrict__ dcan, int wc, int hc, int step, int G, int gw,
                                   int gh, int nw, int dmin, int dmax, uint32_t *__restrict__ gridL,
                                   uint32_t *__restrict__ gridR) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= wc * hc) return;
    const int d = dcan[i];
    if (d < 0) return;
    const int ic = i / wc, jc = i - ic * wc;
    const int u = jc * step, v = ic * step;
    const int cy = v / G;
    for (int side = 0; side < 2; ++side) {
        uint32_t *grid = side ? gridR : gridL;
        if (!grid) continue;
        const int cx = (side ? u - d : u) / G;
        for (int y = cy - 1; y <= cy + 1; ++y) {
            if (y < 0 || y >= gh) continue;
            for (int x = cx - 1; x <= cx + 1; ++x) {
                if (x < 0 || x >= gw) continue;
                or_bits(grid + ((size_t)y * gw + x) * nw, d, dmin, dmax);
            }
        }
    }
}

constexpr int kCompactThreads = 1024;

__global__ void __launch_bounds__(kCompactThreads)
compact_kernel(const int16_t *__restrict__ dcan, int wc, int hc, int step, int16_t *__restrict__ list,
               int32_t *__restrict__ count) {
    __shared__ int s_warp[kCompactThreads / 32];
    const int nc = wc * hc;
    const int t = threadIdx.x;
    const int chunk = (nc + kCompactThreads - 1) / kCompactThreads;
    const int b0 = min(nc, t * chunk), b1 = min(nc, b0 + chunk);
    int mine = 0;
    for (int i = b0; i < b1; ++i) mine += dcan[i] >= 0;
    // block-wide exclusive scan of `mine`
    const int lane = t & 31, wid = t >> 5;
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int x = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        s_warp[lane] = x;  // inclusive totals per warp
    }
    __syncthreads();
    int pos = incl - mine + (wid ? s_warp[wid - 1] : 0);
    for (int i = b0; i < b1; ++i) {
        const int d = dcan[i];
        if (d < 0) continue;
        const int ic = i / wc, jc = i - ic * wc;
        list[3 * pos + 0] = (int16_t)(jc * step);
        list[3 * pos + 1] = (int16_t)(ic * step);
        list[3 * pos + 2] = (int16_t)d;
        ++pos;
    }
    if (t == kCompactThreads - 1) *count = pos;
}

size_t support_workspace(int w, int h, const elas_params *p) {
    const size_t nc = (size_t)(w / p->candidate_stepsize) * (h / p->candidate_stepsize);
    return 2 * align_up(nc * sizeof(int16_t) + 16, 256);
}

elas_status launch_support(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                           int16_t *d_can, int16_t *list, int32_t *count, uint32_t *grid_L, uint32_t *grid_R,
                           void *ws, cudaStream_t st) {
    SupportArgs a;
    a.w = w;
    a.h = h;
    a.step = p->candidate_stepsize;
    a.wc = w / a.step;
    a.hc = h / a.step;
    a.dmin = p->disp_min;
    a.dmax = p->disp_max;
    a.thr = p->support_threshold;
    a.support_texture = p->support_texture;
    a.lr_threshold = p->lr_threshold;
    const int nc = a.wc * a.hc;
    const GridGeom g = grid_geom(w, h, p);
    const size_t gbytes = (size_t)g.gw * g.gh * g.nw * sizeof(uint32_t);
    if (grid_L && cudaMemsetAsync(grid_L, 0, gbytes, st) != cudaSuccess) return launch_status("memset grid_L");
    if (grid_R && cudaMemsetAsync(grid_R, 0, gbytes, st) != cudaSuccess) return launch_status("memset grid_R");
    if (nc == 0) {
        if (cudaMemsetAsync(count, 0, sizeof(int32_t), st) != cudaSuccess) return launch_status("memset count");
        return ELAS_OK;
    }
    int16_t *raw = reinterpret_cast<int16_t *>(ws);
    int16_t *con = reinterpret_cast<int16_t *>(reinterpret_cast<char *>(ws) + align_up(nc * sizeof(int16_t) + 16, 256));
    const int warps_per_block = 8;
    support_match_kernel<<<(nc + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        reinterpret_cast<const uint4 *>(descL), reinterpret_cast<const uint4 *>(descR), a, raw);
    elas_status s = launch_status("support_match_kernel");
    if (s != ELAS_OK) return s;
    const int tb = 256, nb = (nc + tb - 1) / tb;
    consistency_kernel<<<nb, tb, 0, st>>>(raw, a.wc, a.hc, p->incon_window_size, p->incon_threshold,
                                          p->incon_min_support, con);
    if ((s = launch_status("consistency_kernel")) != ELAS_OK) return s;
    redundancy_kernel<<<nb, tb, 0, st>>>(con, a.wc, a.hc, p->redun_max_dist,
                                         (p->test_flags & ELAS_FLAG_REDUNDANCY_OFF) ? 0 : 1, d_can);
    if ((s = launch_status("redundancy_kernel")) != ELAS_OK) return s;
    if (grid_L || grid_R) {
        grid_vector_kernel<<<nb, tb, 0, st>>>(d_can, a.wc, a.hc, a.step, p->grid_size, g.gw, g.gh, g.nw, a.dmin,
                                              a.dmax, grid_L, grid_R);
        if ((s = launch_status("grid_vector_kernel")) != ELAS_OK) return s;
    }
    compact_kernel<<<1, kCompactThreads, 0, st>>>(d_can, a.wc, a.hc, a.step, list, count);
    return launch_status("compact_kernel");
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
