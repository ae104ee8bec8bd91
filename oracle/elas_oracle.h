/*
 * ELAS oracle: plain, slow, obviously-correct CPU reference of the ELAS
 * data-parallel path (Rahnama et al., "Real-Time Dense Stereo Matching with
 * ELAS on FPGA Accelerated Embedded Devices", arXiv 1802.07210, Sec. III.A).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * path (the CUDA library and its Python binding) never calls it and shares
 * no code, header, table or constant with it.
 *
 * Every function follows the plain definition of its step: exhaustive loops,
 * no tiling, no fusion, no reordering.  Floating-point steps use single
 * IEEE-754 operations in the stated order and are compiled with
 * -ffp-contract=off so no multiply-add is ever fused.
 *
 * Conventions (shared meaning with the product, not shared code):
 *   images           uint8  [h][w], row-major, no padding
 *   descriptors      uint8  [h][w][16]
 *   candidate grid   int16  [h/step][w/step], candidate (jc,ic) at pixel
 *                    (u,v) = (jc*step, ic*step); -1 = no support point
 *   support list     int16  triples (u, v, d) in raster order of the grid
 *   grid vectors     uint32 [ceil(h/G)][ceil(w/G)][ceil((disp_max+1)/32)]
 *   triangles        int32  triples of support-list indices
 *   disparity maps   int16  [h][w], -1 = invalid
 *   postprocessed    float  [h][w], -1.0f = invalid
 */
#ifndef ELAS_ORACLE_H
#define ELAS_ORACLE_H
#include <stdint.h>

#define ORACLE_FLAG_PRIOR_OFF      1u  /* dense: prior term forced to 0      */
#define ORACLE_FLAG_FULL_RANGE     2u  /* dense: every in-range d is a candidate,
                                          d_plane is not required            */
#define ORACLE_FLAG_REDUNDANCY_OFF 4u  /* support: skip the redundancy filter */
#define ORACLE_FLAG_SHIFT_SUM      8u  /* support: Eq. 3 shift-sum threshold
                                          m1 <= (m2>>1)+(m2>>2)+(m2>>3)+(m2>>5) */
#define ORACLE_FLAG_PAST_REDUNDANCY 16u /* support: Sec. VI.C past-only rule:
                                          redundant iff the identical d lies
                                          within redun_max_dist to the left and
                                          above */

typedef struct {
    int32_t disp_min, disp_max;
    float   support_threshold;
    int32_t support_texture;
    int32_t candidate_stepsize;
    int32_t incon_window_size, incon_threshold, incon_min_support;
    int32_t redun_max_dist;
    int32_t grid_size;
    float   beta, gamma, sigma;
    int32_t sradius, match_texture, lr_threshold;
    int32_t ipol_gap_width, filter_adaptive_mean;
    uint32_t flags;
    /* Census variant (Sec. VI.A): window widths of the support and dense
     * census descriptors; both 0 = Sobel descriptors with SAD (Sec. III.A),
     * else both odd, 3 <= census_support_w <= 15, 3 <= census_dense_w <= 11. */
    int32_t census_support_w, census_dense_w;
    /* Support down-sampling (Sec. VII, the 1/8, 1/14, 1/32 of the extracted
     * support points the paper sweeps): 0 or 1 keeps every point; k >= 2
     * keeps the points numbered 0, k, 2k, ... in raster order of the
     * filtered candidate grid (the others become -1), so the list, the grid
     * vectors and the triangulation see 1/k of them. */
    int32_t support_downsample;
} oracle_params;

void oracle_params_default(oracle_params *p);

/* Sec. III.A / Fig. 1(b-d): Sobel responses (int32) and 16-byte descriptors. */
void oracle_sobel(const uint8_t *img, int w, int h, int32_t *du, int32_t *dv);
void oracle_descriptors(const uint8_t *img, int w, int h, uint8_t *desc);

/* Sec. VI.A: census transform over a W x W window (W odd).  Bit k of pixel p,
 * k = (dy + W/2) * W + (dx + W/2) for the neighbour q = p + (dx, dy), is 1 iff
 * I(q) < I(p); a neighbour outside the image takes the value of the nearest
 * border pixel (coordinates clamped).  The centre bit is always 0, so the
 * descriptor has W*W bits as the paper counts them.  Bits are packed from the
 * least significant bit of byte 0 into nbytes bytes per pixel (W*W <= 8*nbytes),
 * the rest zero: out is uint8 [h][w][nbytes].
 *
 * With census widths set in the parameters the support stage takes the
 * 32-byte support census (W = census_support_w) of each image in place of the
 * descriptors and costs a candidate by the Hamming distance between the two
 * pixels' census bits; the dense stage takes the 16-byte dense census
 * (W = census_dense_w) and costs by Hamming distance too.  Neither stage then
 * applies a texture test (the texture measure belongs to the Sobel
 * descriptors, which the census variant does not compute). */
void oracle_census(const uint8_t *img, int w, int h, int W, int nbytes, uint8_t *out);

/* Sec. III.A, Eq. 1-2: support matching on the candidate lattice with the
 * ratio test, the texture check and the left-right re-match. */
void oracle_support_match(const uint8_t *descL, const uint8_t *descR, int w, int h,
                          const oracle_params *p, int16_t *dcan);
/* Sec. III.A: consistency filter and redundancy filter on the candidate grid. */
void oracle_filter_consistency(const int16_t *in, int wc, int hc,
                               const oracle_params *p, int16_t *out);
void oracle_filter_redundancy(const int16_t *in, int wc, int hc,
                              const oracle_params *p, int16_t *out);
/* Whole support step: match, consistency, redundancy (unless disabled), then
 * the down-sampling of support_downsample. */
void oracle_support_points(const uint8_t *descL, const uint8_t *descR, int w, int h,
                           const oracle_params *p, int16_t *dcan);
/* Raster-order compaction of the candidate grid; returns the count. */
int  oracle_support_list(const int16_t *dcan, int wc, int hc, int step, int16_t *list);

/* Sec. III.A, Fig. 2, Sec. VI.D: grid vectors as one-hot masks. */
void oracle_grid_vectors(const int16_t *list, int n, int w, int h,
                         const oracle_params *p, int right, uint32_t *grid);

/* Sec. III.A: Delaunay triangulation (symbolic perturbation of the lifted
 * heights, lower support-list index = dominant perturbation). */
int  oracle_delaunay(const int32_t *x, const int32_t *y, int n, int32_t *tri, int cap);
/* Triangulates the support list in left (u,v) or right (u-d,v) coordinates;
 * coincident right-image points keep only the lowest list index.  Returns the
 * triangle count (or -1 if cap is too small). */
int  oracle_triangulate(const int16_t *list, int n, int right, int32_t *tri, int cap);
/* Exact integer predicates, exported for the tests. */
int64_t oracle_orient(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy);
int64_t oracle_incircle(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                        int64_t cx, int64_t cy, int64_t dx, int64_t dy);

/* Sec. III.A, Sec. VI.D: prior table and the image-sized prior matrix. */
void oracle_prior_table(const oracle_params *p, int32_t *P /* sradius+1 */);
void oracle_plane_prior(const int16_t *list, int n, const int32_t *tri, int ntri,
                        int right, int w, int h, const oracle_params *p,
                        int16_t *dplane, int32_t *owners /* may be NULL */);

/* Sec. III.A, Fig. 1(h): dense per-pixel argmin.  right=0 matches the left
 * image against the right one, right=1 the reverse. */
void oracle_dense(const uint8_t *descL, const uint8_t *descR, int w, int h,
                  const oracle_params *p, const int16_t *dplane,
                  const uint32_t *grid, int right, int16_t *out);

/* Sec. III.A, Fig. 1(i): left-right consistency check. */
void oracle_lr_check(const int16_t *dL, const int16_t *dR, int w, int h, int thr,
                     int16_t *outL, int16_t *outR, uint8_t *maskL, uint8_t *maskR);

/* Sec. III.A, Fig. 1(i): gap interpolation then adaptive mean. */
void oracle_postprocess(const int16_t *d, int w, int h, const oracle_params *p, float *out);

/* Sec. VII (the median filter applied for the comparison with CSM; the paper
 * gives no size).  Reading: every valid pixel takes the median of the valid
 * disparities in the (2r+1) x (2r+1) window around it, clipped to the image
 * (the lower median, element (n-1)/2 of the sorted values, when n is even);
 * invalid pixels stay -1.  out must not alias d. */
void oracle_median(const int16_t *d, int w, int h, int r, int16_t *out);

/* Small-segment (speckle) removal of ELAS's post-processing (not described
 * in the paper, whose Sec. III.A only names post-processing).  Reading: two
 * 4-neighbouring valid pixels are linked iff their disparities differ by at
 * most sim_threshold; a segment is a connected component of this relation
 * (so it can drift by more than sim_threshold end to end); every pixel of a
 * segment with fewer than min_size pixels becomes -1, the rest are copied.
 * The partition is unique, so the output is. */
void oracle_speckle(const int16_t *d, int w, int h, int sim_threshold, int min_size, int16_t *out);

#endif
