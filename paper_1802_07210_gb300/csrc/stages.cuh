// Argument blocks of the stage kernels.  A one-pair launch passes one block
// by value; a batched launch passes a device table with one block per slot
// (resident pair state) and a VMap (batch.cuh).
#pragma once

#include "batch.cuh"

namespace elas {

// ---- descriptors ----------------------------------------------------------
struct DescArgs {
    const uint8_t *imgL, *imgR;  // imgR may be NULL (local grid z = 1)
    int w, h, pitch;
    uint4 *descL, *descR;
};

// Census records of one pair (Sec. VI.A): window x window comparisons in
// 32-byte (support) or 16-byte (dense) records per pixel.
struct CensusArgs {
    const uint8_t *imgL, *imgR;
    int w, h, pitch;
    uint4 *outL, *outR;
    int window;
};

// ---- support points ---------------------------------------------------------
struct SupportArgs {
    int w, h, step, wc, hc;
    int dmin, dmax;
    float thr;
    int support_texture, lr_threshold;
    int shift_sum;  // Eq. 3 threshold instead of the ratio test
    int census;     // descriptors are 32-byte support census records (Sec. VI.A)
};

struct MatchArgs {
    const uint4 *dL, *dR;
    SupportArgs a;
    int16_t *raw;  // [hc][wc] unfiltered candidate disparities
};

struct ConsArgs {
    const int16_t *in;
    int wc, hc, r, thr, min_support;
    int16_t *out;
    uint32_t *gL, *gR;  // grid-vector masks cleared by this kernel
    int gwords;
};

struct GridArgs {
    int step, G, gw, gh, nw, dmin, dmax;
};

struct RedArgs {
    const int16_t *con;
    int wc, hc, maxd, enabled, past_only;
    GridArgs g;
    int16_t *dcan;
    uint32_t *gridL, *gridR;
    int32_t *rowcount;
    int defer_grid;  // down-sampling: the grid vectors come from the list instead
};

struct CompactArgs {
    int16_t *dcan;  // down-sampling clears the points it drops
    int wc, hc, step;
    const int32_t *rowcount;
    int16_t *list;
    int32_t *count;
    int keep_every;  // support down-sampling k (<= 1: every point)
};

// Grid vectors of a down-sampled support list.
struct ListGridArgs {
    const int16_t *list;
    const int32_t *count;
    int cap;
    GridArgs g;
    uint32_t *gridL, *gridR;
};

// The launches of the support stage for one pair, and their tables (the
// list-grid launch only with down-sampling).
struct SupportStage {
    MatchArgs match;
    ConsArgs cons;
    RedArgs red;
    CompactArgs compact;
    ListGridArgs lg;
};
struct SupportTables {
    const MatchArgs *match;
    const ConsArgs *cons;
    const RedArgs *red;
    const CompactArgs *compact;
    const ListGridArgs *lg;
};

// ---- triangulation ----------------------------------------------------------
struct DtSide {
    int right;
    int32_t *X, *Y;            // [cap] coordinates per list index
    int4 *pts;                 // [cap] (x, y, index, alive) sorted by grid cell
    int32_t *slot;             // [cap] position of each point in pts
    int32_t *cell_cnt;         // [ncell + 1]
    int32_t *cell_start;       // [ncell + 1]
    int32_t *cell_fill;        // [ncell + 1]
    int32_t *status;           // [cap] 0 pending, k: star done in pass k, -1 duplicate
    int32_t *owned;            // [cap] triangles owned (lowest-index vertex)
    int32_t *offset;           // [cap] exclusive scan of owned
    int32_t *slots;            // [cap][kDtSlots][2] owned triangles (the other two vertices)
    int32_t *pending;          // [cap] points queued for the CTA pass
    int32_t *npending;         // queue length
    int32_t *pending2;         // [cap] points queued again
    int32_t *npending2;        // its length (one pair: side 0's is the CTA pass's work counter)
    int32_t *npending3;        // batches: the third queue's length (its entries reuse `pending`)
    int32_t *rowmin, *rowmax;  // [h] extreme x of the points of each image row
    int32_t *tri;              // output [cap_tri][3]
    int32_t *ntri;             // output count
    int32_t *err;              // bit 0: a star failed, bit 1: capacity, bit 2: slots overflowed
};

struct DtArgs {
    const int16_t *list;
    const int32_t *count;  // number of support points (device)
    int cap;               // capacity in points
    int cap_tri;
    int w, h, gw, gh;
    DtSide s[2];
};

// ---- plane prior and dense matching ------------------------------------------
struct RasterSide {
    const int32_t *tri;
    int ntri, right;          // ntri: used when ntri_dev is NULL (else the capacity)
    int16_t *dplane;
    const int32_t *ntri_dev;  // device triangle count (negative = none)
    int4 *rec;                // [cap][4] rasteriser records (edge functions, plane, box)
    int32_t *ucnt;            // [cap] work units (box chunks) of each triangle
    int2 *ulist;              // [unit_cap] extra units: (triangle, chunk >= 1)
    unsigned long long *nunits;  // extra units of the mesh (the list is complete up to unit_cap)
    // the dense step's candidate lists, expanded here from the grid vectors
    // when lstride > 0 (the argmin runs after the prior)
    const uint32_t *grid;  // [gh][gw][nw] grid-vector masks
    uint16_t *clist;       // [gh * gw][lstride] ascending candidates, then 2047
    int32_t *ccount;       // [gh * gw] candidates per cell
};

struct RasterArgs {
    const int16_t *list;
    RasterSide s[2];
    int nsides;
    int w, h, dmin, dmax;
    int unit_cap;  // entries of each mesh's list of extra units
    int gw, gh, nw, lstride;  // grid-vector cells and the candidate lists' stride (0: none)
};

struct CellSide {
    const uint4 *ref, *oth;
    const uint32_t *grid;   // [gh][gw][nw]
    const int16_t *dplane;  // prior map (may be NULL with full range)
    int16_t *out;
    int dir;
    const uint16_t *clist;  // the cells' candidate lists (CellArgs::lstride > 0)
    const int32_t *ccount;
};

struct CellArgs {
    CellSide s[2];
    int w, h, G, gw, nw, dmin, dmax, sradius, match_texture, full, prior_off;
    int census;  // descriptors are 16-byte dense census records, Hamming cost (Sec. VI.A)
    int lstride;  // > 0: candidate lists ready in clist (else each CTA expands its cell's mask)
    int P[kMaxSradius + 1];
};

struct DenseStage {
    RasterArgs raster;
    CellArgs cell;
};
struct DenseTables {
    const RasterArgs *raster;
    const CellArgs *cell;
};

// ---- LR check and post-processing -------------------------------------------
struct LrArgs {
    int16_t *dL, *dR;
    int w, h, thr;
    uint8_t *maskL, *maskR;
};

// Value of element k along a line: from the int16 map or the float buffer.
struct LineIn {
    const int16_t *i16;
    const float *f32;
    __device__ __forceinline__ float at(size_t idx) const { return i16 ? (float)i16[idx] : f32[idx]; }
};

enum PostKind { kPostGapRows = 0, kPostGapCols = 1, kPostMeanRows = 2, kPostMeanCols = 3, kPostCopy = 4 };

struct PostArgs {
    LineIn in;
    float *out;
    int w, h, kind, gap;
};

// All four passes in one launch (gap widths up to 16).
struct FusedPostArgs {
    const int16_t *d;
    float *out;
    int w, h, gap, mean;
};

}  // namespace elas
