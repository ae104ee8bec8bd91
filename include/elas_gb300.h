/*
 * elas_gb300 -- C-ABI of the GB300 (sm_103a) implementation of the ELAS
 * data-parallel stereo path (Rahnama, Frost, Miksik, Torr, "Real-Time Dense
 * Stereo Matching with ELAS on FPGA Accelerated Embedded Devices",
 * arXiv 1802.07210, Sec. III.A).
 *
 * Pipeline per rectified 8-bit stereo pair (Sec. III.A, Fig. 1):
 *   elas_descriptors      gradient (Sobel) images -> 16-byte descriptors
 *   elas_support_points   sparse matches with ratio test (Eq. 1-2), texture
 *                         and left-right checks, consistency + redundancy
 *                         filters, grid vectors (Fig. 2), raster-order list
 *   elas_triangulate      Delaunay mesh of the support points (host)
 *   elas_plane_prior      per-triangle slanted plane -> image-sized prior
 *                         matrix (Sec. VI.D)
 *   elas_dense_argmin     per-pixel argmin of SAD + tabulated prior over the
 *   elas_dense_match      grid-vector and plane-neighbourhood candidates
 *   elas_lr_check         left-right consistency (occlusion invalidation)
 *   elas_postprocess      gap interpolation + adaptive mean (smoothing)
 *   elas_median           median filter of valid disparities (Sec. VII)
 *   elas_speckle          small-segment removal (ELAS post-processing)
 *
 * The paper's own variant (Sec. VI) as parameters: elas_census records with
 * Hamming costs in place of the descriptors and SAD (census_support_w,
 * census_dense_w), the shift-sum ambiguity test of Eq. 3 and the past-only
 * redundancy rule (ELAS_FLAG_SHIFT_SUM, ELAS_FLAG_PAST_REDUNDANCY), and the
 * support down-sampling of Sec. VII (support_downsample).
 *
 * Conventions shared by every call
 *   - All device pointers are owned by the caller.  Calls never allocate
 *     device memory: scratch comes from a caller-provided workspace whose
 *     size the matching *_workspace_bytes() call returns.  Only the handles
 *     own memory: the pipeline (elas_pipeline_*, created in
 *     elas_pipeline_create), the batch and the server.  The one exception
 *     to the workspace rule is elas_support_points_static, whose scratch is
 *     a static device array of the library shared by all its calls (its own
 *     comment gives the size limit and the race between overlapping calls).
 *   - Device calls are asynchronous on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream).  Argument errors are detected on the host and
 *     returned synchronously; a launch failure returns ELAS_ERR_CUDA;
 *     execution errors surface on the caller's next synchronisation.
 *   - No call aborts, traps or prints.  elas_last_error() returns a
 *     thread-local text for the last non-OK status of the calling thread.
 *   - Layouts: image uint8 [h][pitch]; descriptors uint8 [h][w][16] (16-byte
 *     aligned; census records [h][w][32] or [h][w][16]); candidate grid int16 [h/step][w/step] with candidate (jc,ic)
 *     at pixel (jc*step, ic*step), -1 = none; support list int16 triples
 *     (u, v, d) in raster order of the candidate grid; grid vectors uint32
 *     [ceil(h/G)][ceil(w/G)][ceil((disp_max+1)/32)], bit d set = candidate d;
 *     triangles int32 triples of support-list indices; disparity maps int16
 *     [h][w] with -1 = invalid; post-processed map float [h][w], -1 = invalid.
 *   - Integer outputs are bit-exact functions of the inputs (independent of
 *     launch shape and scheduling).  Float outputs use single IEEE-754 ops
 *     in a fixed order without contraction.
 */
#ifndef ELAS_GB300_H
#define ELAS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ELAS_OK = 0,
    ELAS_ERR_INVALID_ARG = 1, /* bad size, pointer, alignment or parameter    */
    ELAS_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed         */
    ELAS_ERR_CAPACITY = 3,    /* an output buffer is smaller than required    */
    ELAS_ERR_TIMEOUT = 4,     /* a bounded wait ran out                       */
    ELAS_ERR_NO_MEMORY = 5,   /* host or device allocation refused (handles)  */
    ELAS_ERR_INTERNAL = 6     /* internal invariant broken                    */
} elas_status;

/* Switches in elas_params.test_flags: PRIOR_OFF, FULL_RANGE and
 * REDUNDANCY_OFF are test modes; SHIFT_SUM and PAST_REDUNDANCY select the
 * paper's variant rules (Sec. VI.B, VI.C). */
#define ELAS_FLAG_PRIOR_OFF      1u /* dense: prior term forced to 0                  */
#define ELAS_FLAG_FULL_RANGE     2u /* dense: every in-range d is a candidate and no
                                       plane is required                             */
#define ELAS_FLAG_REDUNDANCY_OFF 4u /* support: skip the redundancy filter           */
#define ELAS_FLAG_SHIFT_SUM      8u /* support: the ambiguity test of Eq. 3 (Sec. VI.B):
                                       accept iff m1 <= (m2>>1)+(m2>>2)+(m2>>3)+(m2>>5),
                                       support_threshold unused                       */
#define ELAS_FLAG_PAST_REDUNDANCY 16u /* support: the past-only redundancy rule of
                                       Sec. VI.C: an identical d within redun_max_dist
                                       to the left and above removes a point          */

/* Method parameters.  Names follow the libelas "robotics" setting used to
 * quote the workloads; elas_params_default() fills disp_max = 255 and
 * support_threshold 0.85, support_texture 10, candidate_stepsize 5,
 * incon_window_size 5, incon_threshold 5, incon_min_support 5,
 * redun_max_dist 5, grid_size 20, beta 0.02, gamma 3, sigma 1, sradius 2,
 * match_texture 1, lr_threshold 2, ipol_gap_width 3, filter_adaptive_mean 1.
 * Limits: 0 <= disp_min <= disp_max <= 1023, candidate_stepsize >= 1,
 * grid_size >= 1, 0 <= sradius <= 15, 0 < support_threshold; census
 * windows 0 (Sobel descriptors, the default) or as stated below. */
typedef struct {
    int32_t disp_min, disp_max;
    float support_threshold;     /* Eq. 2: accept iff m1 <= t * m2                  */
    int32_t support_texture;     /* min 64-byte window texture (sum |b-128|)        */
    int32_t candidate_stepsize;  /* support candidate lattice spacing (pixels)      */
    int32_t incon_window_size;   /* consistency window, candidate units             */
    int32_t incon_threshold;     /* |dd| <= threshold counts as agreement           */
    int32_t incon_min_support;   /* agreeing neighbours needed to keep a point      */
    int32_t redun_max_dist;      /* redundancy search distance, candidate units     */
    int32_t grid_size;           /* grid-vector cell size G (pixels)                */
    float beta, gamma, sigma;    /* prior P[delta] parameters                       */
    int32_t sradius;             /* plane neighbourhood radius                      */
    int32_t match_texture;       /* min 16-byte descriptor texture for dense        */
    int32_t lr_threshold;        /* left-right tolerance (support and dense)        */
    int32_t ipol_gap_width;      /* max gap length filled by interpolation (0=off)  */
    int32_t filter_adaptive_mean;/* 1 = adaptive mean after interpolation           */
    uint32_t test_flags;         /* ELAS_FLAG_* (test modes, variant rules)         */
    /* The census variant of Sec. VI.A: census windows of the support and the
     * dense stage.  Both 0 (default): Sobel descriptors with SAD costs.
     * Otherwise both odd, 3 <= census_support_w <= 15, 3 <= census_dense_w
     * <= 11: the support stage takes 32-byte support census records
     * (elas_census with window census_support_w) in place of the
     * descriptors and costs a candidate by the Hamming distance of the two
     * pixels' records; the dense stage takes 16-byte dense census records
     * (window census_dense_w) and costs by Hamming distance too; neither
     * applies a texture test (support_texture and match_texture unused). */
    int32_t census_support_w, census_dense_w;
    /* Support down-sampling (Sec. VII sweeps 1/8, 1/14, 1/32 of the extracted
     * support points): 0 or 1 keeps every point; k >= 2 keeps the filtered
     * points numbered 0, k, 2k, ... in raster order of the candidate grid
     * (d_can shows -1 for the others), and the list, its count, the grid
     * vectors and so the triangulation and the dense prior see only those.
     * Every route takes it: per-pair calls, the pipeline, batches, server. */
    int32_t support_downsample;
} elas_params;

/* A cudaStream_t passed through the C ABI. */
typedef void *elas_stream;

/* One workspace size for every per-pair call that takes a workspace
 * (support points, device triangulation of one side, plane prior, dense
 * match, post-processing, speckle removal) when they run one after another
 * on the same buffer: the largest of their *_workspace_bytes at this size.
 * 0 if p is invalid for w x h.  Host only. */
size_t elas_workspace_bytes(int32_t w, int32_t h, const elas_params *p);

/* Fills `p` with the default parameter set listed above.  Host only. */
elas_status elas_params_default(elas_params *p);

/* Text of the calling thread's last error (never NULL). */
const char *elas_last_error(void);

/* Library version string. */
const char *elas_version(void);

/*
 * Descriptors (Sec. III.A: matching runs on the horizontal and vertical
 * gradient images, Fig. 1(b-d); Sec. VI.A: 16-byte descriptors).
 * du/dv: 3x3 Sobel responses (du weights -1 0 1 / -2 0 2 / -1 0 1 with +1 on
 * the right column; dv its transpose), 0 on the one-pixel frame;
 * q(s) = clamp(128 + trunc(s/4), 1, 255).  Byte k of pixel (u,v): q(du) at
 * offsets (-2,-2),(2,-2),(-1,0),(1,0),(-2,2),(2,2),(0,-1),(0,1) for k<8,
 * q(dv) at (0,-2),(0,2),(-2,0),(2,0),(-1,-1),(1,-1),(-1,1),(1,1) for k>=8;
 * samples outside the image read 128.
 * imgL/imgR: device uint8 [h][pitch] (pitch >= w); descL/descR: device
 * uint8 [h][w][16], 16-byte aligned.  imgR/descR may both be NULL.
 * Errors: ELAS_ERR_INVALID_ARG for w,h < 1, pitch < w, NULL or misaligned.
 */
elas_status elas_descriptors(const uint8_t *imgL, const uint8_t *imgR, int32_t w, int32_t h,
                             int32_t pitch, uint8_t *descL, uint8_t *descR, elas_stream stream);

/*
 * Census transform (Sec. VI.A: census descriptors compared by Hamming
 * distance replace the Sobel descriptors and SAD).  Bit k = (dy + W/2) * W +
 * (dx + W/2) of pixel p, for the neighbour q = p + (dx, dy) of the W x W
 * window, is 1 iff I(q) < I(p); neighbours outside the image take the value
 * of the nearest border pixel, so the centre bit is the only one that is
 * always 0 and every pixel has W*W bits.  Bits are packed from the least
 * significant bit of byte 0 (word k/32, bit k%32 of little-endian 32-bit
 * words) into nbytes bytes per pixel, the rest 0.  window odd; nbytes 32
 * (window 3..15: the support record) or 16 (window 3..11: the dense record).
 * imgL/imgR: device uint8 [h][pitch] (pitch >= w); outL/outR: device uint8
 * [h][w][nbytes], 16-byte aligned.  imgR/outR may both be NULL.
 * Errors: ELAS_ERR_INVALID_ARG for w,h < 1, pitch < w, a window that is even,
 * below 3 or too large for nbytes, other nbytes, NULL or misaligned buffers.
 */
elas_status elas_census(const uint8_t *imgL, const uint8_t *imgR, int32_t w, int32_t h, int32_t pitch,
                        int32_t window, int32_t nbytes, uint8_t *outL, uint8_t *outR, elas_stream stream);

/*
 * Support points (Sec. III.A; Eq. 1-2).  For every lattice candidate
 * (u,v) = (jc*step, ic*step) with 4 <= u <= w-5, 4 <= v <= h-5: the 64-byte
 * window = descriptors at (u+-2, v+-2); cost(d) = window SAD against the
 * right window at u-d (searched for d in [disp_min, disp_max] with
 * u-d >= 4).  d1 = smallest d of the minimum m1, m2 = minimum over d != d1;
 * accepted iff >= 2 disparities were searched, m2 > 0 and
 * (float)m1 <= support_threshold * (float)m2, the left window texture and
 * the right window texture at u-d1 are >= support_texture, and the
 * right-to-left re-match from u-d1 (searching u-d1+d <= w-5, same test)
 * returns d_rl with |d1 - d_rl| <= lr_threshold.  Then the consistency
 * filter (keep iff >= incon_min_support other valid points in the
 * +-incon_window_size candidate window differ by <= incon_threshold) and
 * the redundancy filter (drop iff the identical disparity occurs within
 * redun_max_dist candidates in each of the four axis directions) run, each
 * reading the previous grid as a whole.  Grid vectors: bits {d-1,d,d+1}
 * (clipped to the range) of every point are OR-ed into the 3x3 cells around
 * cell(u,v) (grid_L) and cell(u-d,v) (grid_R).
 * Outputs (device): d_can int16 [h/step][w/step]; list int16 [cap][3];
 * count int32 (true number of points); grid_L/grid_R (may be NULL).
 * cap must be >= (w/step)*(h/step), so the list can never overflow.
 * workspace: device, >= elas_support_workspace_bytes(w,h,p), 256-byte
 * aligned.
 * With census windows in p (Sec. VI.A), descL/descR are the 32-byte support
 * census records [h][w][32] of elas_census (window census_support_w), the
 * window of (u,v) is the record of (u,v) itself, cost(d) is the Hamming
 * distance of the two records, and no texture test applies; everything else
 * (bounds, search ranges, tests, filters) is unchanged.
 * With support_downsample k >= 2 in p, the filtered points numbered 0, k,
 * 2k, ... in raster order are kept: d_can holds -1 for the others, the list
 * holds the kept points in order, *count = ceil(n / k) for n filtered points,
 * and the grid vectors are those of the kept points (one more launch).
 */
size_t elas_support_workspace_bytes(int32_t w, int32_t h, const elas_params *p);
elas_status elas_support_points(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                                const elas_params *p, int16_t *d_can, int16_t *list, int32_t cap,
                                int32_t *count, uint32_t *grid_L, uint32_t *grid_R,
                                void *workspace, size_t workspace_bytes, elas_stream stream);

/*
 * Support points with no allocation at all.  The paper has no counterpart:
 * this is a deployment variant of elas_support_points for callers that are
 * not allowed to allocate device memory -- for example a robot's real-time
 * stereo loop that reserves all its memory at start-up and must not call
 * cudaMalloc per frame (an allocation can block and synchronise the device),
 * or a plug-in whose host application owns every device buffer.  The caller
 * still passes the descriptors and all outputs; the scratch that
 * elas_support_points takes as `workspace` comes instead from one static
 * device array of ELAS_STATIC_SUPPORT_SCRATCH_BYTES, which every GPU that
 * loads the library keeps until the process exits.
 *   - Same arguments, semantics and results as elas_support_points, minus
 *     the workspace.
 *   - Limit: elas_support_workspace_bytes(w, h, p) must not exceed
 *     ELAS_STATIC_SUPPORT_SCRATCH_BYTES (512 KiB: e.g. 1920x1080 or
 *     2048x1536 with candidate_stepsize 5); larger sizes return
 *     ELAS_ERR_CAPACITY with a message and launch nothing.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  No call allocates or frees memory.
 *   - All calls share the one array, and it keeps the previous call's
 *     contents.  Every scratch byte a call reads was written earlier in the
 *     same call, so nothing has to be cleared, but calls that overlap on the
 *     GPU (other streams, other threads) race on it: serialise them.
 */
#define ELAS_STATIC_SUPPORT_SCRATCH_BYTES (512u * 1024u)
elas_status elas_support_points_static(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                                       const elas_params *p, int16_t *d_can, int16_t *list, int32_t cap,
                                       int32_t *count, uint32_t *grid_L, uint32_t *grid_R,
                                       elas_stream stream);

/*
 * Delaunay triangulation of the support list (Sec. III.A), on the host,
 * synchronous.  right = 0: points (u, v); right = 1: points (u - d, v), where
 * coincident points keep only the lowest list index.  Cocircular ties are
 * broken by the symbolic perturbation |p_i|^2 + eps_i of the lifted heights
 * with eps_0 >> eps_1 >> ... (lower list index dominates), so the result is
 * unique.  tri: host int32 [cap][3], counter-clockwise in (u, v) with v
 * pointing down as the y axis; *ntri = triangle count (also on
 * ELAS_ERR_CAPACITY, when it exceeds cap).  cap >= 2n always suffices.
 */
elas_status elas_triangulate(const int16_t *list, int32_t n, int32_t right, int32_t *tri,
                             int32_t cap, int32_t *ntri);

/*
 * Delaunay triangulation of the support list on the GPU (Sec. III.A), the
 * same unique triangulation as elas_triangulate (symbolic tie-break on list
 * indices, coincident right-image points keep the lowest index).  Each point
 * builds its own star by exact gift-wrapping among its neighbours, certified
 * by the circumdisc test; uncertified stars are redone with a larger radius.
 * list: device int16 [cap][3] with 0 <= v < h (u - d may be negative);
 * count: device int32, number of points (<= cap); right: 0 = (u, v),
 * 1 = (u - d, v).  Outputs on the device: tri int32
 * [cap_tri][3] (counter-clockwise, each triangle once, deterministic order),
 * *ntri = triangle count, or -1 if the triangulation failed.  cap_tri must be
 * >= 2*cap + 8.  workspace: device, 256-byte aligned,
 * >= elas_triangulate_device_workspace_bytes(cap, w, h).  Asynchronous.
 */
size_t elas_triangulate_device_workspace_bytes(int32_t cap, int32_t w, int32_t h);
elas_status elas_triangulate_device(const int16_t *list, const int32_t *count, int32_t cap, int32_t w,
                                    int32_t h, int32_t right, int32_t *tri, int32_t cap_tri,
                                    int32_t *ntri, void *workspace, size_t workspace_bytes,
                                    elas_stream stream);

/*
 * Slanted-plane prior (Sec. III.A; image-sized prior matrix, Sec. VI.D).
 * For each triangle, with its vertices taken in ascending list index:
 * det = du1*dv2 - du2*dv1, a = (float)(dd1*dv2 - dd2*dv1) / (float)det,
 * b = (float)(du1*dd2 - du2*dd1) / (float)det, c = (d0 - a*u0) - b*v0 (FP32,
 * left to right, no fused multiply-add).  Pixels owned by the triangle under
 * integer edge functions with the top-left rule get
 * d_plane = clamp(floor((a*u + b*v) + c + 0.5), disp_min, disp_max); all
 * other pixels get -1.  right = 1: vertices at (u - d, v).
 * list/tri/d_plane: device; d_plane int16 [h][w].  workspace: device,
 * 256-byte aligned, >= elas_plane_prior_workspace_bytes(ntri) (a 64-byte
 * plane and edge record per triangle and the list of the work units of
 * large triangles; 0 for a negative count).
 */
size_t elas_plane_prior_workspace_bytes(int32_t ntri);
elas_status elas_plane_prior(const int16_t *list, int32_t n, const int32_t *tri, int32_t ntri,
                             int32_t right, int32_t w, int32_t h, const elas_params *p,
                             int16_t *d_plane, void *workspace, size_t workspace_bytes,
                             elas_stream stream);

/*
 * Dense argmin for one reference image (Sec. III.A, Fig. 1(h)).
 * right = 0: reference = left, other position u-d; right = 1: reference =
 * right, other position u+d.  Pixel (u,v) with 2 <= u <= w-3, 2 <= v <= h-3,
 * reference texture >= match_texture and d_plane >= 0 searches
 * S = ({d : |d - d_plane| <= sradius} U grid(cell(u,v))) within
 * [disp_min, disp_max] and 2 <= other position <= w-3, with
 * cost(d) = SAD16 + (|d - d_plane| <= sradius ? P[|d - d_plane|] : 0),
 * P[k] = trunc((ln gamma - ln(gamma + exp(-k^2/(2 sigma^2)))) / beta)
 * (computed on the host in double).  Output = smallest d of the minimum
 * cost, -1 if S is empty or the pixel is not matched.  d_plane and grid may
 * be NULL only with ELAS_FLAG_FULL_RANGE.  With census windows in p
 * (Sec. VI.A), descL/descR are the 16-byte dense census records of
 * elas_census (window census_dense_w), the cost is their Hamming distance in
 * place of the SAD, and no texture test applies.
 */
elas_status elas_dense_argmin(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                              const elas_params *p, const int16_t *d_plane, const uint32_t *grid,
                              int32_t right, int16_t *out, elas_stream stream);

/*
 * Plane prior + dense argmin for both reference images (elas_plane_prior
 * then elas_dense_argmin on each side, in two launches).  list (device) is
 * the support list of n points, triL/triR (device) the triangulations in
 * left and right coordinates, grid_L/grid_R the grid vectors.  Outputs dL,
 * dR int16 [h][w]; each mesh has at most 2*(w/step)*(h/step)+8 triangles.
 * workspace: device, 256-byte aligned, >= elas_dense_workspace_bytes() (it
 * holds the two prior maps).
 */
size_t elas_dense_workspace_bytes(int32_t w, int32_t h, const elas_params *p);
elas_status elas_dense_match(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                             const elas_params *p, const int16_t *list, int32_t n,
                             const int32_t *triL, int32_t ntriL, const int32_t *triR,
                             int32_t ntriR, const uint32_t *grid_L, const uint32_t *grid_R,
                             int16_t *dL, int16_t *dR, void *workspace, size_t workspace_bytes,
                             elas_stream stream);

/*
 * Left-right consistency check (Sec. III.A, Fig. 1(i)), in place.  Decisions
 * read the unmodified maps: dL(u) is kept iff d >= 0, u-d >= 0,
 * dR(u-d) >= 0 and |d - dR(u-d)| <= lr_threshold; dR(u) symmetrically with
 * u+d <= w-1 and dL(u+d).  Rejected pixels become -1; maskL/maskR (uint8,
 * may be NULL) get 1 = kept, 0 = invalid.  Requires w <= 16384.
 */
elas_status elas_lr_check(int16_t *dL, int16_t *dR, int32_t w, int32_t h, int32_t lr_threshold,
                          uint8_t *maskL, uint8_t *maskR, elas_stream stream);

/*
 * Post-processing (Sec. III.A, Fig. 1(i)).  If ipol_gap_width > 0: each
 * maximal run of invalid pixels in a row no longer than ipol_gap_width and
 * bounded by valid d1, d2 is filled with (d1+d2)/2 if |d1-d2| < 3 else
 * min(d1,d2); then the same along columns.  If filter_adaptive_mean: for
 * valid pixels, horizontal then vertical weighted mean over offsets -3..3
 * (ascending) of valid neighbours with weight max(0, 4 - |d_i - d_0|).
 * d: device int16 [h][w]; out: device float [h][w], -1 = invalid.
 * workspace >= elas_postprocess_workspace_bytes(w, h).
 */
size_t elas_postprocess_workspace_bytes(int32_t w, int32_t h);
elas_status elas_postprocess(const int16_t *d, int32_t w, int32_t h, const elas_params *p,
                             float *out, void *workspace, size_t workspace_bytes,
                             elas_stream stream);

/*
 * Median filter (Sec. VII: the refinement the paper applies for its
 * comparison with CSM; it gives no window size).  Every valid pixel of d
 * takes the median of the valid disparities in its (2*radius+1)^2 window,
 * clipped to the image (the lower median, element (n-1)/2 in sorted order,
 * when the count n is even); invalid pixels (< 0) are written as -1.
 * d, out: device int16 [h][w], distinct (out must not alias d);
 * radius 0..3 (0 copies).  No workspace.  Errors: ELAS_ERR_INVALID_ARG for a
 * size, radius or pointer out of range.
 */
elas_status elas_median(const int16_t *d, int32_t w, int32_t h, int32_t radius, int16_t *out,
                        elas_stream stream);

/*
 * Small-segment (speckle) removal, ELAS post-processing (the paper names
 * post-processing in Sec. III.A without describing it).  Two 4-neighbouring
 * valid pixels are linked iff their disparities differ by at most
 * sim_threshold; a segment is a connected component of the links (it may
 * drift by more than sim_threshold end to end); every pixel of a segment
 * with fewer than min_size pixels becomes -1, the others and the invalid
 * pixels are copied (invalid as -1).  The partition is unique, so the
 * output is.  d, out: device int16 [h][w]; out may equal d (in place).
 * workspace: device, 256-byte aligned, >= elas_speckle_workspace_bytes(w, h)
 * (two int32 maps); its first int32 is a status the caller may read after
 * the stream completes: 0, or 1 if a union-find loop reached its bound (the
 * pixel count), which the construction excludes.  Errors:
 * ELAS_ERR_INVALID_ARG for a size outside 1..16383, sim_threshold < 0, NULL
 * or misaligned buffers; ELAS_ERR_CAPACITY for a short workspace.
 */
size_t elas_speckle_workspace_bytes(int32_t w, int32_t h);
elas_status elas_speckle(const int16_t *d, int32_t w, int32_t h, int32_t sim_threshold, int32_t min_size,
                         int16_t *out, void *workspace, size_t workspace_bytes, elas_stream stream);

/*
 * Pipeline handle: owns device buffers, pinned staging and a host worker
 * thread for one image size, and runs the whole path per pair, one launch
 * per kernel for that pair (the plain per-pair path).
 * elas_pipeline_run: device images in, device maps out (dR, post may be
 * NULL); with triangulation on the GPU (the default) nothing in the step
 * waits for the host and the call returns with everything enqueued; with
 * host triangulation the stream is synchronised once in the middle (support
 * list to the host).
 * elas_pipeline_run_host: host buffers in and out, copies included; returns
 * when the outputs are on the host.
 */
typedef struct elas_pipeline elas_pipeline;
typedef struct {
    int32_t n_support;     /* support points of the last pair           */
    int32_t n_tri_left;    /* triangles, left coordinates                */
    int32_t n_tri_right;   /* triangles, right coordinates               */
    double  triangulate_ms;/* host wall time of both triangulations (host
                              triangulation only, else 0)               */
    float   stage_ms[6];   /* with profiling on and GPU triangulation:
                              device ms of descriptors, support points,
                              triangulation, plane prior, dense argmin,
                              LR check + post-processing; else 0        */
} elas_pipeline_stats;

elas_status elas_pipeline_create(int32_t w, int32_t h, const elas_params *p, elas_pipeline **out);
elas_status elas_pipeline_run(elas_pipeline *pl, const uint8_t *imgL, const uint8_t *imgR,
                              int32_t pitch, int16_t *dL, int16_t *dR, float *post,
                              elas_stream stream);
elas_status elas_pipeline_run_host(elas_pipeline *pl, const uint8_t *imgL, const uint8_t *imgR,
                                   int16_t *dL, int16_t *dR, float *post, elas_stream stream);
/* Where the pipeline triangulates: on_gpu = 1 (default) runs
 * elas_triangulate_device inside the step, with no host synchronisation;
 * on_gpu = 0 copies the support list to the host and runs elas_triangulate
 * (left and right meshes on two threads).  Both give identical meshes. */
elas_status elas_pipeline_set_triangulation(elas_pipeline *pl, int32_t on_gpu);
/* With GPU triangulation the step is captured into a CUDA graph on the
 * second run with the same buffers and replayed from then on (on = 1, the
 * default); one graph is kept per set of buffers (input and output pointers,
 * pitch, profiling), up to 8 sets, the least recently used replaced, so a
 * ring of camera buffers replays too.  on = 0 launches every kernel each
 * run. */
elas_status elas_pipeline_set_graph(elas_pipeline *pl, int32_t on);
/* on = 1: every run records events between its stages (GPU triangulation
 * only) and elas_pipeline_stats_get reports the stage times. */
elas_status elas_pipeline_set_profiling(elas_pipeline *pl, int32_t on);
/* Counts (and stage times) of the last pair; waits for the pipeline's last
 * stream. */
elas_status elas_pipeline_stats_get(const elas_pipeline *pl, elas_pipeline_stats *st);
void elas_pipeline_destroy(elas_pipeline *pl);

/*
 * Batch handle: many stereo pairs, of any mix of sizes and disparity
 * ranges, run through the whole path together.  Each pair keeps its own
 * resident state on the device (a "slot"); every kernel of the path is
 * launched once for the whole batch, its grid covering the tiles of every
 * pair (per-pair block ranges, so small and large pairs share one launch),
 * and the triangulation's CTA pass takes its work from one queue over all
 * pairs.  With use_graph the launch sequence is captured once into a CUDA
 * graph and replayed.  Results are identical to the per-pair path.
 * Pairs of the paper's variant (census windows, support down-sampling) mix
 * with the others: each stage whose kernel depends on the cost kind (the
 * descriptors or census records of each window size, support matching, the
 * dense argmin) is launched once per kind present in the batch.
 *
 * elas_batch_create: n pairs (1 <= n <= 256), pair i of w[i] x h[i] with
 *   params[i] (w, h >= candidate_stepsize).  Allocates every slot.
 * elas_batch_run: device pointers, arrays of n entries.  imgL/imgR [h][pitch]
 *   uint8 (pitch NULL = widths); dL int16 [h][w] (required); dR NULL or
 *   entries NULL = internal buffers; post NULL or entries NULL = no
 *   post-processing for that pair.  Asynchronous on `stream`; the handle
 *   must not be run on two streams at once.  Changing pointers between runs
 *   costs one small table upload.
 * elas_batch_run_host: host pointers (pinned for speed); copies in, runs,
 *   copies out and returns when the outputs are on the host.
 * elas_batch_stats: per-pair counts of the last run (waits for it).
 * elas_batch_tune: times each tile-shape knob on the given inputs (device
 *   pointers as in elas_batch_run, dL required) and keeps the fastest;
 *   *chosen (may be NULL) receives the result.  Results are cached per
 *   process by the batch's shape list.
 */
typedef struct elas_batch elas_batch;
typedef struct {
    int32_t desc_tile_rows;          /* descriptor rows per warp: 12, 24, 36  */
    int32_t support_warps;           /* candidates per support CTA: 4, 8, 16  */
    int32_t dense_threads_per_pixel; /* dense argmin threads per pixel: 1, 2, 4 */
    int32_t use_graph;               /* capture and replay a CUDA graph       */
    int32_t dense_pixels_per_thread; /* dense argmin pixels per thread: 1, 2, 4, 8, 16 */
    int32_t dense_fused;             /* 1: plane prior and dense argmin as one persistent
                                        cooperative launch (one warp per cell); 0: one
                                        launch per kernel */
} elas_batch_config;

elas_status elas_batch_create(int32_t n, const int32_t *w, const int32_t *h, const elas_params *params,
                              elas_batch **out);
elas_status elas_batch_get_config(const elas_batch *b, elas_batch_config *cfg);
elas_status elas_batch_set_config(elas_batch *b, const elas_batch_config *cfg);
elas_status elas_batch_run(elas_batch *b, const uint8_t *const *imgL, const uint8_t *const *imgR,
                           const int32_t *pitch, int16_t *const *dL, int16_t *const *dR, float *const *post,
                           elas_stream stream);
elas_status elas_batch_run_host(elas_batch *b, const uint8_t *const *imgL, const uint8_t *const *imgR,
                                int16_t *const *dL, int16_t *const *dR, float *const *post, elas_stream stream);
elas_status elas_batch_stats(elas_batch *b, int32_t *n_support, int32_t *n_tri_left, int32_t *n_tri_right);
elas_status elas_batch_tune(elas_batch *b, const uint8_t *const *imgL, const uint8_t *const *imgR,
                            const int32_t *pitch, int16_t *const *dL, elas_stream stream,
                            elas_batch_config *chosen);
/* One eager run (with the buffers of the last elas_batch_run) bracketed by
 * events: stage_ms[0..5] = descriptors, support points, triangulation,
 * plane prior, dense argmin, LR check + post-processing (device ms).
 * Returns when done. */
elas_status elas_batch_profile(elas_batch *b, elas_stream stream, float *stage_ms);
/* Device bytes the batch holds (slots, tables and scratch). */
size_t elas_batch_device_bytes(const elas_batch *b);
void elas_batch_destroy(elas_batch *b);

/*
 * Server: a request loop over resident pair state with continuous batching.
 * Requests (host images in, host maps out) are queued by elas_server_submit
 * and handled by a scheduler thread of the library:
 *  - admission: a request takes an idle slot of its shape (w, h, params) or
 *    a new one while the slots' device bytes stay within the HBM budget
 *    (idle slots of other shapes are released to make room); requests are
 *    admitted in arrival order;
 *  - waves: admitted requests are launched together as one wave of batched
 *    launches (images to the device, the whole path, maps to the host) on
 *    one of `lanes` streams; a new wave starts whenever a lane is free, so
 *    pairs that arrive while others are on the GPU join the next wave and
 *    overlap with the running ones;
 *  - out of device memory (an allocation refused although the budget
 *    allows it, e.g. memory taken by other users of the GPU): idle slots are
 *    released, least recently used first, and the allocation retried; with
 *    nothing idle to release the request waits for running waves, and with
 *    nothing running either its result is ELAS_ERR_NO_MEMORY;
 *  - plain = 1 instead runs one request at a time through the per-pair path
 *    (an elas_pipeline per shape), in arrival order: the comparison.
 * Results are bit-identical to the per-pair path.  Host buffers passed to
 * elas_server_submit must stay valid until the request's result has been
 * polled; pinned memory makes the copies faster.  Times are milliseconds on
 * the server's steady clock (elas_server_now_ms).
 */
typedef struct elas_server elas_server;
typedef struct {
    int32_t  lanes;              /* waves in flight at once, 1..8 (plain: 1)      */
    int32_t  max_wave;           /* requests per wave at most, 1..256             */
    int32_t  max_slots;          /* resident pair states at most, 1..1024         */
    int32_t  plain;              /* 1: per-pair path, one request at a time       */
    uint64_t hbm_budget_bytes;   /* device bytes for slots; 0 = free memory at
                                    creation minus hbm_reserve_bytes            */
    uint64_t hbm_reserve_bytes;  /* left free with hbm_budget_bytes = 0          */
} elas_server_config;

typedef struct {
    uint64_t id;          /* the id given to elas_server_submit              */
    int32_t  status;      /* elas_status of the request                      */
    int32_t  n_support;   /* support points of the pair                      */
    int32_t  wave_size;   /* requests in the wave it ran in (plain: 1)       */
    int32_t  pad;
    double   t_submit_ms; /* submitted                                        */
    double   t_start_ms;  /* its wave launched                                */
    double   t_done_ms;   /* its outputs on the host, seen by the scheduler   */
} elas_server_result;

typedef struct {
    int64_t  submitted, completed, waves, slots_created, slots_released;
    int32_t  slots_in_use, max_wave_seen;
    uint64_t slot_bytes, hbm_budget_bytes;
} elas_server_stats;

elas_status elas_server_config_default(elas_server_config *cfg);
/* Device bytes of one resident pair state (slot) of this shape; 0 if the
 * shape or parameters are invalid. */
size_t elas_slot_device_bytes(int32_t w, int32_t h, const elas_params *p);
elas_status elas_server_create(const elas_server_config *cfg, elas_server **out);
/* Queues one pair: imgL/imgR host uint8 [h][w]; dL host int16 [h][w];
 * post host float [h][w] or NULL (post-processing off). */
elas_status elas_server_submit(elas_server *s, uint64_t id, int32_t w, int32_t h, const elas_params *p,
                               const uint8_t *imgL, const uint8_t *imgR, int16_t *dL, float *post);
/* Up to max finished results (oldest first); waits up to timeout_ms for the
 * first one.  Returns the number written, or -1 on a NULL argument. */
int32_t elas_server_poll(elas_server *s, elas_server_result *out, int32_t max, int32_t timeout_ms);
double elas_server_now_ms(const elas_server *s);
elas_status elas_server_stats_get(elas_server *s, elas_server_stats *st);
/* Waits until every request submitted so far has its result (polled or
 * not), at most timeout_ms: ELAS_OK, or ELAS_ERR_TIMEOUT when the wait ran
 * out (the requests stay queued or in flight and complete later). */
elas_status elas_server_drain(elas_server *s, int32_t timeout_ms);
/* Fault injection for tests: the next n slot allocations of the scheduler
 * report out of memory, as a device whose memory other users took would. */
elas_status elas_server_inject_alloc_failures(elas_server *s, int32_t n);
/* Waits for every queued request, then stops the scheduler and frees all. */
void elas_server_destroy(elas_server *s);

#ifdef __cplusplus
}
#endif
#endif /* ELAS_GB300_H */
