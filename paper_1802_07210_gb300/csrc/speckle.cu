// Small-segment (speckle) removal, ELAS post-processing: two 4-neighbouring
// valid pixels are linked iff their disparities differ by at most
// sim_threshold; segments (connected components of the links) with fewer
// than min_size pixels are invalidated.
//
// Connected components by union-find over pixel indices, every parent index
// below its child's, so a root is the least pixel index of its tree:
//   speckle_local_kernel   one CTA per 32x16 tile: union-find of the links
//                          inside the tile in shared memory, then each
//                          pixel's label = the global index of its tile-local
//                          root; clears the size counters.
//   speckle_border_kernel  links that cross a tile's right or bottom edge,
//                          united in global memory (atomicMin on roots).
//   speckle_count_kernel   label = root (path flattening), then segment sizes
//                          with one atomicAdd per distinct root per warp.
//   speckle_apply_kernel   out = d where the segment is large enough, else -1.
// The partition is unique, so the output is too.  Every loop is bounded by
// the pixel count (each step moves to a strictly smaller index); a loop that
// reaches its bound sets the status word instead of spinning on.
#include "launch.cuh"

namespace elas {

constexpr int kSpTX = 32, kSpTY = 16, kSpThreads = kSpTX * kSpTY;

struct SpeckleArgs {
    const int16_t *d;
    int16_t *out;
    int32_t *label;   // [h][w]: parent index, -1 for invalid pixels
    int32_t *size;    // [h][w]: pixel count of the segment rooted here
    int32_t *status;  // 0, or 1 if a loop bound was reached
    int w, h, thr, min_size;
};

__device__ __forceinline__ bool sp_linked(int a, int b, int thr) { return a >= 0 && b >= 0 && abs(a - b) <= thr; }

// Root of x in a forest whose parents are strictly smaller indices; reads
// through L2 (`ld.cg`) because other CTAs relink roots during the kernel.
__device__ __forceinline__ int sp_find_global(const int32_t *L, int x, int limit) {
    for (int it = 0; it < limit; ++it) {
        const int p = __ldcg(L + x);
        if (p == x) return x;
        x = p;
    }
    return -1;
}

// Joins the trees of a and b: the larger root is linked under the smaller
// one with atomicMin; if that root was relinked meanwhile, the returned old
// parent (a smaller index) is where the walk resumes.
__device__ void sp_unite_global(int32_t *L, int a, int b, int limit, int32_t *status) {
    for (int it = 0; it < limit; ++it) {
        a = sp_find_global(L, a, limit);
        b = sp_find_global(L, b, limit);
        if (a < 0 || b < 0) break;
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(L + b, a);
        if (old == b) return;
        b = old;
    }
    atomicExch(status, 1);
}

__device__ __forceinline__ int sp_find_shared(volatile int *L, int x) {
    for (int it = 0; it < kSpThreads; ++it) {
        const int p = L[x];
        if (p == x) return x;
        x = p;
    }
    return -1;
}

__device__ void sp_unite_shared(int *L, int a, int b, int32_t *status) {
    for (int it = 0; it < kSpThreads; ++it) {
        a = sp_find_shared(L, a);
        b = sp_find_shared(L, b);
        if (a < 0 || b < 0) break;
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(L + b, a);
        if (old == b) return;
        b = old;
    }
    atomicExch(status, 1);
}

__global__ void __launch_bounds__(kSpThreads) speckle_local_kernel(SpeckleArgs a) {
    __shared__ int sL[kSpThreads];
    __shared__ int16_t sD[kSpThreads];
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * kSpTX + tx;
    const int x0 = blockIdx.x * kSpTX, y0 = blockIdx.y * kSpTY;
    const int x = x0 + tx, y = y0 + ty;
    const bool in = x < a.w && y < a.h;
    const size_t i = (size_t)y * a.w + x;
    const int dv = in ? a.d[i] : -1;
    sD[t] = (int16_t)dv;
    sL[t] = dv >= 0 ? t : -1;
    if (in) a.size[i] = 0;
    __syncthreads();
    if (dv >= 0) {
        if (tx + 1 < kSpTX && sp_linked(dv, sD[t + 1], a.thr)) sp_unite_shared(sL, t, t + 1, a.status);
        if (ty + 1 < kSpTY && sp_linked(dv, sD[t + kSpTX], a.thr)) sp_unite_shared(sL, t, t + kSpTX, a.status);
    }
    __syncthreads();
    if (in) {
        int lab = -1;
        if (dv >= 0) {
            const int r = sp_find_shared(sL, t);
            // the tile-local root's global index: local order is raster order
            // inside the tile, so the label is still <= i
            lab = r < 0 ? (int)i : (y0 + r / kSpTX) * a.w + (x0 + r % kSpTX);
            if (r < 0) atomicExch(a.status, 1);
        }
        a.label[i] = lab;
    }
}

__global__ void __launch_bounds__(256) speckle_border_kernel(SpeckleArgs a) {
    const int n = a.w * a.h;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / a.w, x = i - y * a.w;
        const bool right = (x % kSpTX) == kSpTX - 1 && x + 1 < a.w;
        const bool down = (y % kSpTY) == kSpTY - 1 && y + 1 < a.h;
        if (!right && !down) continue;
        const int dv = a.d[i];
        if (dv < 0) continue;
        if (right && sp_linked(dv, a.d[i + 1], a.thr)) sp_unite_global(a.label, i, i + 1, n, a.status);
        if (down && sp_linked(dv, a.d[i + a.w], a.thr)) sp_unite_global(a.label, i, i + a.w, n, a.status);
    }
}

__global__ void __launch_bounds__(256) speckle_count_kernel(SpeckleArgs a) {
    const int n = a.w * a.h;
    const int lane = threadIdx.x & 31;
    // whole warps iterate together so that the match below sees every lane
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int i = base + threadIdx.x;
        int root = -1;
        if (i < n && __ldcg(a.label + i) >= 0) {
            root = sp_find_global(a.label, i, n);
            if (root < 0) atomicExch(a.status, 1);
            else a.label[i] = root;  // an ancestor: the forest stays valid
        }
        const unsigned same = __match_any_sync(0xFFFFFFFFu, root);
        if (root >= 0 && lane == __ffs(same) - 1) atomicAdd(a.size + root, __popc(same));
    }
}

__global__ void __launch_bounds__(256) speckle_apply_kernel(SpeckleArgs a) {
    const int n = a.w * a.h;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int lab = a.label[i];
        const int16_t dv = a.d[i];
        a.out[i] = (lab >= 0 && a.size[lab] >= a.min_size) ? dv : (int16_t)-1;
    }
}

size_t speckle_workspace(int w, int h) {
    return align_up(16, 256) + 2 * align_up((size_t)w * h * sizeof(int32_t), 256);
}

elas_status launch_speckle(const int16_t *d, int w, int h, int thr, int min_size, int16_t *out, void *ws,
                           cudaStream_t st) {
    SpeckleArgs a;
    char *b = reinterpret_cast<char *>(ws);
    a.status = reinterpret_cast<int32_t *>(b);
    a.label = reinterpret_cast<int32_t *>(b + align_up(16, 256));
    a.size = reinterpret_cast<int32_t *>(b + align_up(16, 256) + align_up((size_t)w * h * sizeof(int32_t), 256));
    a.d = d;
    a.out = out;
    a.w = w;
    a.h = h;
    a.thr = thr;
    a.min_size = min_size;
    if (cudaMemsetAsync(a.status, 0, sizeof(int32_t), st) != cudaSuccess) return launch_status("speckle status");
    const dim3 tiles((w + kSpTX - 1) / kSpTX, (h + kSpTY - 1) / kSpTY);
    speckle_local_kernel<<<tiles, dim3(kSpTX, kSpTY), 0, st>>>(a);
    elas_status s = launch_status("speckle_local_kernel");
    if (s != ELAS_OK) return s;
    const int n = w * h;
    int blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    speckle_border_kernel<<<blocks, 256, 0, st>>>(a);
    if ((s = launch_status("speckle_border_kernel")) != ELAS_OK) return s;
    speckle_count_kernel<<<blocks, 256, 0, st>>>(a);
    if ((s = launch_status("speckle_count_kernel")) != ELAS_OK) return s;
    speckle_apply_kernel<<<blocks, 256, 0, st>>>(a);
    return launch_status("speckle_apply_kernel");
}

}  // namespace elas

extern "C" size_t elas_speckle_workspace_bytes(int32_t w, int32_t h) {
    if (w < 1 || h < 1 || w > 16383 || h > 16383) return 0;
    return elas::speckle_workspace(w, h);
}

extern "C" elas_status elas_speckle(const int16_t *d, int32_t w, int32_t h, int32_t sim_threshold,
                                    int32_t min_size, int16_t *out, void *workspace, size_t workspace_bytes,
                                    elas_stream stream) {
    using namespace elas;
    if (w < 1 || h < 1 || w > 16383 || h > 16383) return fail(ELAS_ERR_INVALID_ARG, "map size %dx%d", w, h);
    if (sim_threshold < 0) return fail(ELAS_ERR_INVALID_ARG, "sim_threshold %d < 0", sim_threshold);
    if (!d || !out || !workspace) return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned(workspace, 256)) return fail(ELAS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (workspace_bytes < speckle_workspace(w, h))
        return fail(ELAS_ERR_CAPACITY, "workspace %zu < %zu bytes", workspace_bytes, speckle_workspace(w, h));
    return launch_speckle(d, w, h, sim_threshold, min_size, out, workspace, to_stream(stream));
}
