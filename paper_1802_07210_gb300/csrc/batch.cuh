// Batched launches: one grid covers the tiles of many stereo pairs.
//
// Every stage kernel is written once as a body over (its argument struct, a
// local block index).  The one-pair launch passes the struct by value and
// takes the local block from blockIdx/gridDim.  The batched launch passes a
// device table of structs (one entry per slot, i.e. per resident pair
// state) and a VMap: pair i of the launch owns the blocks
// [off[i], off[i+1]) of a 1-D grid and runs on the state of slot slot[i]
// with its own local grid (gx, gy, gz).  So pairs of different sizes and
// disparity ranges share one launch, each with exactly its own tiles, and
// the hardware block scheduler hands the tiles of all pairs to the SMs as
// they free up.  The VMap travels in the kernel parameters (about 4 KB):
// the block-to-pair search is a handful of uniform constant-bank loads.
#pragma once

#include "common.cuh"

namespace elas {

constexpr int kMaxBatch = 256;

struct VMap {
    int n;                    // pairs in the launch
    int stride;               // bytes between the table entries of consecutive slots
    int off[kMaxBatch + 1];   // first block of each pair, off[n] = total
    int gx[kMaxBatch];        // local grid width of each pair
    int gxy[kMaxBatch];       // local grid width * height
    int slot[kMaxBatch];      // table entry of each pair
};

struct VB {
    int slot;
    int x, y, z;     // local block index
    int gx, gy, gz;  // local grid
};

__device__ __forceinline__ VB vb_single() {
    VB v;
    v.slot = 0;
    v.x = blockIdx.x;
    v.y = blockIdx.y;
    v.z = blockIdx.z;
    v.gx = gridDim.x;
    v.gy = gridDim.y;
    v.gz = gridDim.z;
    return v;
}

// Pair and local block of block b of a batched grid.
__device__ __forceinline__ VB vb_at(const VMap &m, int b) {
    // last pair whose first block is <= b (pairs with no blocks are skipped
    // because a later pair starts at the same offset)
    int lo = 0, hi = m.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m.off[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    VB v;
    const int local = b - m.off[lo];
    v.slot = m.slot[lo];
    v.gx = m.gx[lo];
    const int gxy = m.gxy[lo];
    v.gy = gxy / v.gx;
    v.gz = (m.off[lo + 1] - m.off[lo]) / gxy;
    v.z = local / gxy;
    const int r = local - v.z * gxy;
    v.y = r / v.gx;
    v.x = r - v.y * v.gx;
    return v;
}

__device__ __forceinline__ VB vb_batch(const VMap &m) { return vb_at(m, blockIdx.x); }

// Entry of `slot` in a table whose entries are `stride` bytes apart (the
// tables are arrays of per-slot records; tab points at slot 0's entry).
template <class T> __host__ __device__ __forceinline__ const T &slot_entry(const T *tab, int stride, int slot) {
    return *reinterpret_cast<const T *>(reinterpret_cast<const char *>(tab) + (size_t)slot * stride);
}

// Host: appends pair `slot` with local grid g (a grid with no blocks adds
// nothing but keeps the slot listed).
inline void vmap_clear(VMap &m, int stride) {
    m.n = 0;
    m.stride = stride;
    m.off[0] = 0;
}
inline bool vmap_add(VMap &m, int slot, dim3 g) {
    if (m.n >= kMaxBatch) return false;
    const long long blocks = (long long)g.x * g.y * g.z;
    if ((long long)m.off[m.n] + blocks > 0x7FFFFFFFLL) return false;
    m.gx[m.n] = g.x > 0 ? (int)g.x : 1;
    m.gxy[m.n] = m.gx[m.n] * (g.y > 0 ? (int)g.y : 1);
    m.slot[m.n] = slot;
    m.off[m.n + 1] = m.off[m.n] + (int)blocks;
    ++m.n;
    return true;
}
__host__ __device__ inline int vmap_total(const VMap &m) { return m.off[m.n]; }

}  // namespace elas
