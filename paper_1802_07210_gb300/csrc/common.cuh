// Internal helpers shared by the CUDA translation units of libelas_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "elas_gb300.h"

namespace elas {

// Thread-local error text behind elas_last_error().
void set_error(const char *fmt, ...);
elas_status fail(elas_status st, const char *fmt, ...);
// Converts a pending launch error into ELAS_ERR_CUDA.
elas_status launch_status(const char *what);
// Validates the parameter block against the image size.
elas_status check_params(const elas_params *p, int32_t w, int32_t h);
// Streaming multiprocessors of the current device (queried once per device;
// launch grids are sized in multiples of it).
int sm_count();

inline cudaStream_t to_stream(elas_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// Records a timing mark on st; while st is being captured into a graph the
// record becomes an event-record node of the graph.
inline cudaError_t record_mark(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return cudaGetLastError();
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal)
                                               : cudaEventRecord(e, st);
}
inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int kMaxSradius = 15;
constexpr int kMaxDisp = 1023;

// Grid-vector geometry.
struct GridGeom {
    int gw, gh, nw;  // cells across, cells down, 32-bit words per cell
};
inline GridGeom grid_geom(int w, int h, const elas_params *p) {
    GridGeom g;
    g.gw = (w + p->grid_size - 1) / p->grid_size;
    g.gh = (h + p->grid_size - 1) / p->grid_size;
    g.nw = (p->disp_max + 1 + 31) / 32;
    return g;
}

// Prior table P[0..sradius] from the parameters (host, double precision).
void prior_table(const elas_params *p, int32_t *P);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Sum of |a_i - b_i| over the 4 bytes of a and b, added to acc.
__device__ __forceinline__ uint32_t sad4_acc(uint32_t a, uint32_t b, uint32_t acc) {
    return __dp4a(__vabsdiffu4(a, b), 0x01010101u, acc);
}

// The same sum with the byte-SIMD absolute difference and its accumulating
// merge (one instruction per 4 bytes): the matchers' form (measured faster
// than the dp4a form in both).
__device__ __forceinline__ uint32_t sad4_vacc(uint32_t a, uint32_t b, uint32_t acc) {
    uint32_t r = acc;
    asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(r) : "r"(a), "r"(b));
    return r;
}

__device__ __forceinline__ uint32_t sad16_vacc(const uint4 &a, const uint4 &b) {
    uint32_t s = sad4_vacc(a.x, b.x, 0u);
    s = sad4_vacc(a.y, b.y, s);
    s = sad4_vacc(a.z, b.z, s);
    return sad4_vacc(a.w, b.w, s);
}

// Texture of a descriptor: sum of |b - 128| over its 16 bytes.
__device__ __forceinline__ uint32_t texture16(const uint4 &a) {
    const uint32_t m = 0x80808080u;
    uint32_t s = sad4_acc(a.x, m, 0u);
    s = sad4_acc(a.y, m, s);
    s = sad4_acc(a.z, m, s);
    return sad4_acc(a.w, m, s);
}

// Hamming distance of two 128-bit census strings (Sec. VI.A).
__device__ __forceinline__ uint32_t ham16(const uint4 &a, const uint4 &b) {
    return __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
}

}  // namespace elas
