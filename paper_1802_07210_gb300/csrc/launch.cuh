// Internal launchers (no argument validation) used by the C-ABI entry points,
// the pipeline runtime and the batch runtime.
#pragma once

#include <vector>

#include "stages.cuh"

namespace elas {

// ---- one pair per launch ----------------------------------------------------
elas_status launch_descriptors(const uint8_t *imgL, const uint8_t *imgR, int w, int h, int pitch, uint8_t *descL,
                               uint8_t *descR, cudaStream_t st);
// Census records: window odd, 3..15 in 32 bytes per pixel or 3..11 in 16.
bool census_shape_ok(int window, int nbytes);
elas_status launch_census(const uint8_t *imgL, const uint8_t *imgR, int w, int h, int pitch, int window, int nbytes,
                          uint8_t *outL, uint8_t *outR, cudaStream_t st);
size_t support_workspace(int w, int h, const elas_params *p);
elas_status launch_support(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                           int16_t *d_can, int16_t *list, int32_t *count, uint32_t *grid_L, uint32_t *grid_R,
                           void *ws, cudaStream_t st);
int max_triangles(int w, int h, const elas_params *p);
size_t raster_scratch_bytes(int tri_cap, int nsides);
elas_status launch_plane_prior(const int16_t *list, const int32_t *tri, int ntri, int right, int w, int h,
                               const elas_params *p, int16_t *dplane, void *scratch, cudaStream_t st);
elas_status launch_dense(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                         const int16_t *dplane, const uint32_t *grid, int right, int16_t *out, cudaStream_t st);
size_t dense_workspace(int w, int h, const elas_params *p);
// With ntri_dev (two device counts) the triangle counts are read on the device
// and ntriL/ntriR are the capacities the launch is sized for; after_prior (may
// be NULL) is recorded between the prior and the argmin.
elas_status launch_dense_both(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                              const int16_t *list, const int32_t *triL, int ntriL, const int32_t *triR, int ntriR,
                              const uint32_t *gridL, const uint32_t *gridR, int16_t *dL, int16_t *dR, void *ws,
                              cudaStream_t st, const int32_t *ntri_dev, cudaEvent_t after_prior = nullptr);
size_t triangulate_device_workspace(int cap, int w, int h, int nsides);
elas_status launch_triangulate_device(const int16_t *list, const int32_t *count, int cap, int w, int h, int nsides,
                                      const int *rights, int32_t *const *tri, int32_t *const *ntri, int cap_tri,
                                      void *ws, cudaStream_t st);
elas_status launch_lr_check(int16_t *dL, int16_t *dR, int w, int h, int thr, uint8_t *maskL, uint8_t *maskR,
                            cudaStream_t st);
size_t post_workspace(int w, int h);
elas_status launch_post(const int16_t *d, int w, int h, const elas_params *p, float *out, void *ws,
                        cudaStream_t st);
int64_t delaunay_points(const int32_t *x, const int32_t *y, int n, std::vector<int32_t> &tri);

// ---- argument blocks (shared by one-pair and batched launches) --------------
dim3 descriptor_grid(int w, int h, int two, int rows);
elas_status support_args(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                         int16_t *d_can, int16_t *list, int32_t *count, uint32_t *grid_L, uint32_t *grid_R,
                         void *ws, SupportStage *o);
dim3 support_match_grid(const MatchArgs &m, int warps);
dim3 consistency_grid(const ConsArgs &c);
size_t consistency_smem(int r);
dim3 lattice_row_grid(int hc);
DtArgs triangulate_args(const int16_t *list, const int32_t *count, int cap, int w, int h, int32_t *const *tri,
                        int32_t *const *ntri, int cap_tri, void *ws);
elas_status dense_args(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                       const int16_t *list, const int32_t *triL, int ntriL, const int32_t *triR, int ntriR,
                       const uint32_t *gridL, const uint32_t *gridR, int16_t *dL, int16_t *dR, void *ws,
                       const int32_t *ntri_dev, DenseStage *o,
                       bool cell_lists);
int cell_threads(int G, int tpp, int ppt);
int post_passes(const int16_t *d, int w, int h, const elas_params *p, float *out, void *ws, PostArgs *passes);
bool post_fusable(const elas_params *p);
FusedPostArgs fused_post_args(const int16_t *d, int w, int h, const elas_params *p, float *out);
dim3 fused_post_grid(int w, int h, int tile_y);

// ---- many pairs per launch --------------------------------------------------
// Tables are arrays of per-slot records `pairs.stride` bytes apart: `tab`
// points at slot 0's entry on the device, `host` at the same entry of the
// host copy.  Pair i of `pairs` runs on slot pairs.slot[i].
elas_status launch_descriptors_b(const DescArgs *tab, const DescArgs *host, const VMap &pairs, int rows,
                                 cudaStream_t st);
// Census records (nbytes 32 or 16 per pixel) of the pairs, each with the
// window of its own table entry.
elas_status launch_census_b(const CensusArgs *tab, const CensusArgs *host, const VMap &pairs, int nbytes,
                            cudaStream_t st);
elas_status launch_support_b(const SupportTables &t, const SupportStage *host, const VMap &pairs, int match_warps,
                             cudaStream_t st);
// counter: one device int, the CTA pass's queue position.
elas_status launch_triangulate_b(const DtArgs *tab, const DtArgs *host, const VMap &pairs, int nsides,
                                 int32_t *counter, cudaStream_t st);
// after_prior (may be NULL) is recorded between the prior and the argmin.
// fused: the prior and the argmin as one persistent cooperative launch.
elas_status launch_dense_b(const DenseTables &t, const DenseStage *host, const VMap &pairs, int tpp, int ppt,
                           cudaStream_t st, cudaEvent_t after_prior = nullptr, bool fused = false);
// post_tab[k]: table of post-processing pass k (k < 4); npass[i]: passes of
// pair i of `pairs`; fused[i]: pair i uses the fused kernel (table fused_tab).
elas_status launch_lr_post_b(const LrArgs *lr_tab, const LrArgs *host_lr, const PostArgs *const *post_tab,
                             const int *npass, const FusedPostArgs *fused_tab, const int *fused, const VMap &pairs,
                             cudaStream_t st);

}  // namespace elas
