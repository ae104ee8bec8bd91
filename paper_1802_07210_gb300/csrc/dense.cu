// Slanted-plane prior (Sec. III.A; image-sized prior matrix, Sec. VI.D) and
// dense per-pixel argmin of descriptor SAD plus tabulated prior over the
// grid-vector and plane-neighbourhood candidates (Sec. III.A, Fig. 1(h)).
//
// plane_prior_kernel  one warp per triangle (grid-stride over triangles):
//                     every lane evaluates the FP32 plane in the fixed order,
//                     lanes stride the bounding box and write the pixels the
//                     triangle owns under the top-left rule.  Ownership is
//                     unique, so no two writes ever race.
// dense_kernel        one thread per pixel in 32x8 tiles; the reference
//                     descriptor stays in registers, the other image's
//                     descriptors are 16-byte read-only loads; the cell's
//                     grid vector is walked bit by bit, then the plane
//                     neighbourhood not already covered by the mask.
#include "launch.cuh"

namespace elas {

struct PriorArgs {
    int w, h, dmin, dmax, right;
};

__device__ __forceinline__ bool edge_owned(int px, int py, int qx, int qy) {
    return (qy == py && qx > px) || (qy < py);
}

__global__ void __launch_bounds__(256)
plane_prior_kernel(const int16_t *__restrict__ list, const int32_t *__restrict__ tri, int ntri, PriorArgs a,
                   int16_t *__restrict__ dplane) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int t = blockIdx.x * wpb + (threadIdx.x >> 5); t < ntri; t += gridDim.x * wpb) {
        int i0 = __ldg(tri + 3 * t), i1 = __ldg(tri + 3 * t + 1), i2 = __ldg(tri + 3 * t + 2);
        // canonical vertex order: ascending list index
        if (i1 < i0) { int s = i0; i0 = i1; i1 = s; }
        if (i2 < i1) { int s = i1; i1 = i2; i2 = s; }
        if (i1 < i0) { int s = i0; i0 = i1; i1 = s; }
        int X[3], Y[3], Z[3];
        const int id[3] = {i0, i1, i2};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int u = __ldg(list + 3 * id[k]), v = __ldg(list + 3 * id[k] + 1), d = __ldg(list + 3 * id[k] + 2);
            X[k] = a.right ? u - d : u;
            Y[k] = v;
            Z[k] = d;
        }
        const int det = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]);
        if (det == 0) continue;
        const int na = (Z[1] - Z[0]) * (Y[2] - Y[0]) - (Z[2] - Z[0]) * (Y[1] - Y[0]);
        const int nb = (X[1] - X[0]) * (Z[2] - Z[0]) - (X[2] - X[0]) * (Z[1] - Z[0]);
        const float fa = __fdiv_rn(__int2float_rn(na), __int2float_rn(det));
        const float fb = __fdiv_rn(__int2float_rn(nb), __int2float_rn(det));
        float fc = __fsub_rn(__int2float_rn(Z[0]), __fmul_rn(fa, __int2float_rn(X[0])));
        fc = __fsub_rn(fc, __fmul_rn(fb, __int2float_rn(Y[0])));
        // positively oriented order for the edge functions
        int ex[3], ey[3];
        ex[0] = X[0];
        ey[0] = Y[0];
        if (det > 0) {
            ex[1] = X[1]; ey[1] = Y[1]; ex[2] = X[2]; ey[2] = Y[2];
        } else {
            ex[1] = X[2]; ey[1] = Y[2]; ex[2] = X[1]; ey[2] = Y[1];
        }
        const int xmin = max(0, min(X[0], min(X[1], X[2]))), xmax = min(a.w - 1, max(X[0], max(X[1], X[2])));
        const int ymin = max(0, min(Y[0], min(Y[1], Y[2]))), ymax = min(a.h - 1, max(Y[0], max(Y[1], Y[2])));
        if (xmax < xmin || ymax < ymin) continue;
        const int bw = xmax - xmin + 1;
        const int npx = bw * (ymax - ymin + 1);
        const bool own0 = edge_owned(ex[0], ey[0], ex[1], ey[1]);
        const bool own1 = edge_owned(ex[1], ey[1], ex[2], ey[2]);
        const bool own2 = edge_owned(ex[2], ey[2], ex[0], ey[0]);
        for (int k = lane; k < npx; k += 32) {
            const int yy = ymin + k / bw, xx = xmin + k % bw;
            const int e0 = (ex[1] - ex[0]) * (yy - ey[0]) - (ey[1] - ey[0]) * (xx - ex[0]);
            const int e1 = (ex[2] - ex[1]) * (yy - ey[1]) - (ey[2] - ey[1]) * (xx - ex[1]);
            const int e2 = (ex[0] - ex[2]) * (yy - ey[2]) - (ey[0] - ey[2]) * (xx - ex[2]);
            const bool in = (e0 > 0 || (e0 == 0 && own0)) && (e1 > 0 || (e1 == 0 && own1)) &&
                            (e2 > 0 || (e2 == 0 && own2));
            if (!in) continue;
            const float t1 = __fmul_rn(fa, __int2float_rn(xx));
            const float t2 = __fmul_rn(fb, __int2float_rn(yy));
            const float mu = __fadd_rn(__fadd_rn(t1, t2), fc);
            int dp = __float2int_rz(floorf(__fadd_rn(mu, 0.5f)));
            dp = min(max(dp, a.dmin), a.dmax);
            dplane[(size_t)yy * a.w + xx] = (int16_t)dp;
        }
    }
}

struct DenseArgs {
    int w, h, dmin, dmax, sradius, match_texture, G, gw, nw, dir, full, prior_off;
    int P[kMaxSradius + 1];
};

__global__ void __launch_bounds__(256)
dense_kernel(const uint4 *__restrict__ ref, const uint4 *__restrict__ oth, const int16_t *__restrict__ dplane,
             const uint32_t *__restrict__ grid, DenseArgs a, int16_t *__restrict__ out) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= a.w || v >= a.h) return;
    int res = -1;
    const size_t row = (size_t)v * a.w;
    if (u >= 2 && u <= a.w - 3 && v >= 2 && v <= a.h - 3) {
        const uint4 r = __ldg(ref + row + u);
        const int dp = a.full ? -1 : __ldg(dplane + row + u);
        if ((int)texture16(r) >= a.match_texture && (a.full || dp >= 0)) {
            // admissible disparities: 2 <= u + dir*d <= w-3
            int lo, hi;
            if (a.dir < 0) {
                lo = max(a.dmin, u - (a.w - 3));
                hi = min(a.dmax, u - 2);
            } else {
                lo = max(a.dmin, 2 - u);
                hi = min(a.dmax, a.w - 3 - u);
            }
            int bc = 0x7FFFFFFF, bd = -1;
            const uint4 *orow = oth + row;
            if (a.full) {
                for (int d = lo; d <= hi; ++d) {  // no plane, so no prior term
                    const int c = (int)sad16(r, __ldg(orow + u + a.dir * d));
                    if (c < bc) { bc = c; bd = d; }
                }
            } else {
                const uint32_t *cell = grid + ((size_t)(v / a.G) * a.gw + (u / a.G)) * a.nw;
                for (int wd = 0; wd < a.nw; ++wd) {
                    uint32_t m = __ldg(cell + wd);
                    while (m) {
                        const int d = wd * 32 + __ffs(m) - 1;
                        m &= m - 1;
                        if (d < lo || d > hi) continue;
                        int c = (int)sad16(r, __ldg(orow + u + a.dir * d));
                        const int ad = abs(d - dp);
                        if (!a.prior_off && ad <= a.sradius) c += a.P[ad];
                        if (c < bc || (c == bc && d < bd)) { bc = c; bd = d; }
                    }
                }
                for (int d = max(lo, dp - a.sradius); d <= min(hi, dp + a.sradius); ++d) {
                    if ((__ldg(cell + (d >> 5)) >> (d & 31)) & 1u) continue;  // already evaluated
                    int c = (int)sad16(r, __ldg(orow + u + a.dir * d));
                    if (!a.prior_off) c += a.P[abs(d - dp)];
                    if (c < bc || (c == bc && d < bd)) { bc = c; bd = d; }
                }
            }
            res = bd;
        }
    }
    out[row + u] = (int16_t)res;
}

elas_status launch_plane_prior(const int16_t *list, const int32_t *tri, int ntri, int right, int w, int h,
                               const elas_params *p, int16_t *dplane, cudaStream_t st) {
    if (cudaMemsetAsync(dplane, 0xFF, (size_t)w * h * sizeof(int16_t), st) != cudaSuccess)
        return launch_status("memset d_plane");
    if (ntri <= 0) return ELAS_OK;
    PriorArgs a{w, h, p->disp_min, p->disp_max, right};
    const int wpb = 8;
    int blocks = (ntri + wpb - 1) / wpb;
    if (blocks > 152 * 16) blocks = 152 * 16;
    plane_prior_kernel<<<blocks, 32 * wpb, 0, st>>>(list, tri, ntri, a, dplane);
    return launch_status("plane_prior_kernel");
}

elas_status launch_dense(const uint8_t *descL, const uint8_t *descR, int w, int h, const elas_params *p,
                         const int16_t *dplane, const uint32_t *grid, int right, int16_t *out, cudaStream_t st) {
    DenseArgs a;
    a.w = w;
    a.h = h;
    a.dmin = p->disp_min;
    a.dmax = p->disp_max;
    a.sradius = p->sradius;
    a.match_texture = p->match_texture;
    a.G = p->grid_size;
    const GridGeom g = grid_geom(w, h, p);
    a.gw = g.gw;
    a.nw = g.nw;
    a.dir = right ? +1 : -1;
    a.full = (p->test_flags & ELAS_FLAG_FULL_RANGE) ? 1 : 0;
    a.prior_off = (p->test_flags & ELAS_FLAG_PRIOR_OFF) ? 1 : 0;
    for (int k = 0; k <= kMaxSradius; ++k) a.P[k] = 0;
    prior_table(p, a.P);
    const uint4 *ref = reinterpret_cast<const uint4 *>(right ? descR : descL);
    const uint4 *oth = reinterpret_cast<const uint4 *>(right ? descL : descR);
    dim3 block(32, 8);
    dim3 gridd((w + 31) / 32, (h + 7) / 8);
    dense_kernel<<<gridd, block, 0, st>>>(ref, oth, dplane, grid, a, out);
    return launch_status("dense_kernel");
}

size_t dense_workspace(int w, int h) { return 2 * align_up((size_t)w * h * sizeof(int16_t), 256); }

}  // namespace elas

extern "C" elas_status elas_plane_prior(const int16_t *list, int32_t n, const int32_t *tri, int32_t ntri,
                                        int32_t right, int32_t w, int32_t h, const elas_params *p,
                                        int16_t *d_plane, elas_stream stream) {
    using namespace elas;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (!d_plane || (ntri > 0 && (!list || !tri))) return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (n < 0 || ntri < 0) return fail(ELAS_ERR_INVALID_ARG, "negative count");
    return launch_plane_prior(list, tri, ntri, right, w, h, p, d_plane, to_stream(stream));
}

extern "C" elas_status elas_dense_argmin(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                                         const elas_params *p, const int16_t *d_plane, const uint32_t *grid,
                                         int32_t right, int16_t *out, elas_stream stream) {
    using namespace elas;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (!descL || !descR || !out) return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if (!(p->test_flags & ELAS_FLAG_FULL_RANGE) && (!d_plane || !grid))
        return fail(ELAS_ERR_INVALID_ARG, "d_plane and grid are required without ELAS_FLAG_FULL_RANGE");
    if (!aligned(descL, 16) || !aligned(descR, 16)) return fail(ELAS_ERR_INVALID_ARG, "descriptors not 16-byte aligned");
    return launch_dense(descL, descR, w, h, p, d_plane, grid, right, out, to_stream(stream));
}

extern "C" size_t elas_dense_workspace_bytes(int32_t w, int32_t h, const elas_params *p) {
    if (elas::check_params(p, w, h) != ELAS_OK) return 0;
    return elas::dense_workspace(w, h);
}

extern "C" elas_status elas_dense_match(const uint8_t *descL, const uint8_t *descR, int32_t w, int32_t h,
                                        const elas_params *p, const int16_t *list, int32_t n, const int32_t *triL,
                                        int32_t ntriL, const int32_t *triR, int32_t ntriR,
                                        const uint32_t *grid_L, const uint32_t *grid_R, int16_t *dL, int16_t *dR,
                                        void *workspace, size_t workspace_bytes, elas_stream stream) {
    using namespace elas;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (!descL || !descR || !grid_L || !grid_R || !dL || !dR || !workspace)
        return fail(ELAS_ERR_INVALID_ARG, "NULL buffer");
    if ((ntriL > 0 || ntriR > 0) && !list) return fail(ELAS_ERR_INVALID_ARG, "NULL support list");
    if ((ntriL > 0 && !triL) || (ntriR > 0 && !triR)) return fail(ELAS_ERR_INVALID_ARG, "NULL triangles");
    if (n < 0 || ntriL < 0 || ntriR < 0) return fail(ELAS_ERR_INVALID_ARG, "negative count");
    if (!aligned(descL, 16) || !aligned(descR, 16)) return fail(ELAS_ERR_INVALID_ARG, "descriptors not 16-byte aligned");
    if (!aligned(workspace, 256)) return fail(ELAS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (workspace_bytes < dense_workspace(w, h))
        return fail(ELAS_ERR_CAPACITY, "workspace %zu < %zu bytes", workspace_bytes, dense_workspace(w, h));
    cudaStream_t st = to_stream(stream);
    int16_t *dpL = reinterpret_cast<int16_t *>(workspace);
    int16_t *dpR = reinterpret_cast<int16_t *>(reinterpret_cast<char *>(workspace) +
                                               align_up((size_t)w * h * sizeof(int16_t), 256));
    if ((s = launch_plane_prior(list, triL, ntriL, 0, w, h, p, dpL, st)) != ELAS_OK) return s;
    if ((s = launch_plane_prior(list, triR, ntriR, 1, w, h, p, dpR, st)) != ELAS_OK) return s;
    if ((s = launch_dense(descL, descR, w, h, p, dpL, grid_L, 0, dL, st)) != ELAS_OK) return s;
    return launch_dense(descL, descR, w, h, p, dpR, grid_R, 1, dR, st);
}
