// Small-segment (speckle) removal, ELAS post-processing: two 4-neighbouring
// valid pixels are linked iff their disparities differ by at most
// sim_threshold; segments (connected components of the links) with fewer
// than min_size pixels are invalidated.
//
// Connected components by union-find over pixel indices, every parent index
// below its child's, so a root is the least pixel index of its tree:
//   speckle_local_kernel   one CTA per 32x16 tile: union-find of the links
//                          inside the tile in shared memory; each pixel's
//                          label = the global index of its tile-local root,
//                          and each tile-local root's size entry = its
//                          pixel count in the tile (0 for other pixels).
//   speckle_border_kernel  one thread per link across a tile's right or
//                          bottom edge: union in global memory (atomicMin on
//                          roots).
//   speckle_resolve_kernel each tile-local root finds its final root, points
//                          its label there and adds its count to the root's
//                          (one atomic per tile-local segment).
//   speckle_apply_kernel   two hops (pixel -> tile-local root -> final root)
//                          give the segment size: out = d if large enough,
//                          else -1.
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
// Path halving: a visited non-root is pointed at its grandparent (an
// ancestor, so the forest stays valid; roots are only changed by unions).
__device__ __forceinline__ int sp_find_global(int32_t *L, int x, int limit) {
    for (int it = 0; it < limit; ++it) {
        const int p = __ldcg(L + x);
        if (p == x) return x;
        const int g = __ldcg(L + p);
        if (g != p) __stcg(L + x, g);
        x = g;
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

// The same walk without writes: after the unions, each tile-local root's
// label is set to its final root by that root's own thread alone, which a
// halving write from another walk could overwrite with an intermediate root.
__device__ __forceinline__ int sp_find_readonly(const int32_t *L, int x, int limit) {
    for (int it = 0; it < limit; ++it) {
        const int p = __ldcg(L + x);
        if (p == x) return x;
        x = p;
    }
    return -1;
}

__device__ __forceinline__ int sp_find_shared(volatile int *L, int x) {
    for (int it = 0; it < kSpThreads; ++it) {
        const int p = L[x];
        if (p == x) return x;
        const int g = L[p];
        if (g != p) L[x] = g;
        x = g;
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

// A tile row is one warp: the horizontal links of a row become runs from one
// ballot (a pixel's run root is the nearest run start at or left of it), so
// union-find only joins runs through vertical links, and a vertical link is
// skipped where the link to its left, with the two horizontal links beside
// it, already connects the same pixels (those links are processed or
// skipped for the same reason further left, ending at a processed one).
__global__ void __launch_bounds__(kSpThreads) speckle_local_kernel(SpeckleArgs a) {
    __shared__ int sL[kSpThreads];
    __shared__ int sC[kSpThreads];
    __shared__ int16_t sD[kSpThreads];
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * kSpTX + tx;
    const int x0 = blockIdx.x * kSpTX, y0 = blockIdx.y * kSpTY;
    const int x = x0 + tx, y = y0 + ty;
    const bool in = x < a.w && y < a.h;
    const size_t i = (size_t)y * a.w + x;
    const int dv = in ? a.d[i] : -1;
    sD[t] = (int16_t)dv;
    sC[t] = 0;
    __syncthreads();
    const bool left = tx > 0 && sp_linked(sD[t - 1], dv, a.thr);
    const unsigned linked_left = __ballot_sync(0xFFFFFFFFu, left);
    // run starts at or left of this lane (lane 0 is never linked left)
    const unsigned starts = ~linked_left & (0xFFFFFFFFu >> (31 - tx));
    sL[t] = dv >= 0 ? ty * kSpTX + (31 - __clz(starts)) : -1;
    __syncthreads();
    if (dv >= 0 && ty + 1 < kSpTY && sp_linked(dv, sD[t + kSpTX], a.thr)) {
        const bool redundant = left && sp_linked(sD[t - 1], sD[t - 1 + kSpTX], a.thr) &&
                               sp_linked(sD[t - 1 + kSpTX], sD[t + kSpTX], a.thr);
        if (!redundant) sp_unite_shared(sL, t, t + kSpTX, a.status);
    }
    __syncthreads();
    int r = -1;
    if (dv >= 0) {
        r = sp_find_shared(sL, t);
        if (r < 0) {
            atomicExch(a.status, 1);
            r = t;
        }
        atomicAdd(sC + r, 1);
    }
    __syncthreads();
    if (in) {
        // the tile-local root's global index: local order is raster order
        // inside the tile, so the label is still <= i
        a.label[i] = r < 0 ? -1 : (y0 + r / kSpTX) * a.w + (x0 + r % kSpTX);
        a.size[i] = sC[t];  // the tile-local count at a tile-local root, else 0
    }
}

// Links across tile edges: first every right edge (x = 32k + 31, k =
// 0..ntx-2) of every row, then every bottom edge (y = 16k + 15) of every
// column.  A right-edge link is skipped where the link above it and the two
// vertical links beside it connect the same pixels and those vertical links
// lie inside a tile (not on a tile's first row); a bottom-edge link likewise
// with the link to its left and horizontal links inside a tile.  Each skip
// rests on a link one row up or one column left, so the chain ends at a
// processed link and no component loses a connection.
__global__ void __launch_bounds__(256) speckle_border_kernel(SpeckleArgs a) {
    const int ntx = (a.w + kSpTX - 1) / kSpTX, nty = (a.h + kSpTY - 1) / kSpTY;
    const int nr = (ntx - 1) * a.h, nb = (nty - 1) * a.w;
    const int n = a.w * a.h, w = a.w, thr = a.thr;
    const int16_t *d = a.d;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nr + nb; k += gridDim.x * blockDim.x) {
        int i, j;
        bool redundant;
        if (k < nr) {
            const int y = k / (ntx - 1), e = k - y * (ntx - 1);
            i = y * w + e * kSpTX + kSpTX - 1;
            j = i + 1;
            if (!sp_linked(d[i], d[j], thr)) continue;
            redundant = (y % kSpTY) != 0 && sp_linked(d[i - w], d[j - w], thr) && sp_linked(d[i - w], d[i], thr) &&
                        sp_linked(d[j - w], d[j], thr);
        } else {
            const int kb = k - nr, e = kb / w, x = kb - e * w;
            i = (e * kSpTY + kSpTY - 1) * w + x;
            j = i + w;
            if (!sp_linked(d[i], d[j], thr)) continue;
            redundant = (x % kSpTX) != 0 && sp_linked(d[i - 1], d[j - 1], thr) && sp_linked(d[i - 1], d[i], thr) &&
                        sp_linked(d[j - 1], d[j], thr);
        }
        if (!redundant) sp_unite_global(a.label, i, j, n, a.status);
    }
}

__global__ void __launch_bounds__(256) speckle_resolve_kernel(SpeckleArgs a) {
    const int n = a.w * a.h;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // tile-local roots hold their tile count (>= 1); adds only go to
        // final roots, which are tile-local roots too, so the test is stable
        const int c = __ldcg(a.size + i);
        if (c <= 0) continue;
        const int root = sp_find_readonly(a.label, i, n);
        if (root < 0) {
            atomicExch(a.status, 1);
            continue;
        }
        if (root != i) {
            __stcg(a.label + i, root);  // an ancestor: the forest stays valid
            atomicAdd(a.size + root, c);
        }
    }
}

__global__ void __launch_bounds__(256) speckle_apply_kernel(SpeckleArgs a) {
    const int n = a.w * a.h;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = a.label[i];
        const int16_t dv = a.d[i];
        bool keep = false;
        if (r >= 0) {
            const int root = a.label[r];  // r's final root (r itself if it is one)
            keep = a.size[root] >= a.min_size;
        }
        a.out[i] = keep ? dv : (int16_t)-1;
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
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    speckle_border_kernel<<<blocks, 256, 0, st>>>(a);
    if ((s = launch_status("speckle_border_kernel")) != ELAS_OK) return s;
    speckle_resolve_kernel<<<blocks, 256, 0, st>>>(a);
    if ((s = launch_status("speckle_resolve_kernel")) != ELAS_OK) return s;
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
