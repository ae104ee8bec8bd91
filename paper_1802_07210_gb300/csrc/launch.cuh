// Internal launchers (no argument validation) used by the C-ABI entry points
// and by the pipeline runtime.
#pragma once

#include <vector>

#include "common.cuh"

namespace elas {

elas_status launch_descriptors(const uint8_t *imgL, const uint8_t *imgR, int w, int h, int pitch, uint8_t *descL,
                               uint8_t *descR, cudaStream_t st);
size_t support_workspace(int w, int h, const elas_params *p);
elas_status launch_support(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                           int16_t *d_can, int16_t *list, int32_t *count, uint32_t *grid_L, uint32_t *grid_R,
                           void *ws, cudaStream_t st);
int max_triangles(int w, int h, const elas_params *p);
size_t raster_scratch_bytes(int ntri_total);
elas_status launch_plane_prior(const int16_t *list, const int32_t *tri, int ntri, int right, int w, int h,
                               const elas_params *p, int16_t *dplane, void *scratch, cudaStream_t st);
elas_status launch_dense(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                         const int16_t *dplane, const uint32_t *grid, int right, int16_t *out, cudaStream_t st);
size_t dense_workspace(int w, int h, const elas_params *p);
// With ntri_dev (two device counts) the triangle counts are read on the device
// and ntriL/ntriR are the capacities the launch is sized for.
elas_status launch_dense_both(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                              const int16_t *list, const int32_t *triL, int ntriL, const int32_t *triR, int ntriR,
                              const uint32_t *gridL, const uint32_t *gridR, int16_t *dL, int16_t *dR, void *ws,
                              cudaStream_t st, const int32_t *ntri_dev);
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

}  // namespace elas
