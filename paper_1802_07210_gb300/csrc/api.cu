// Library-wide host entry points: defaults, errors, validation, prior table.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace elas {

static thread_local char g_err[512] = "no error";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int sm_count() {
    static std::atomic<int> cached[64];  // 0 = not yet queried
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    int n = cached[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 152;
    }
    cached[dev].store(n, std::memory_order_relaxed);
    return n;
}

elas_status fail(elas_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

elas_status launch_status(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(ELAS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return ELAS_OK;
}

elas_status check_params(const elas_params *p, int32_t w, int32_t h) {
    if (!p) return fail(ELAS_ERR_INVALID_ARG, "params is NULL");
    if (w < 1 || h < 1) return fail(ELAS_ERR_INVALID_ARG, "image size %dx%d", w, h);
    if (w > 16383 || h > 16383) return fail(ELAS_ERR_INVALID_ARG, "image size %dx%d above 16383", w, h);
    if (p->disp_min < 0 || p->disp_max < p->disp_min || p->disp_max > kMaxDisp)
        return fail(ELAS_ERR_INVALID_ARG, "disparity range [%d,%d]", p->disp_min, p->disp_max);
    if (p->candidate_stepsize < 1) return fail(ELAS_ERR_INVALID_ARG, "candidate_stepsize %d", p->candidate_stepsize);
    if (p->grid_size < 1) return fail(ELAS_ERR_INVALID_ARG, "grid_size %d", p->grid_size);
    if (p->sradius < 0 || p->sradius > kMaxSradius) return fail(ELAS_ERR_INVALID_ARG, "sradius %d", p->sradius);
    if (!(p->support_threshold > 0.0f)) return fail(ELAS_ERR_INVALID_ARG, "support_threshold");
    if (p->incon_window_size < 0 || p->redun_max_dist < 0 || p->ipol_gap_width < 0 || p->lr_threshold < 0)
        return fail(ELAS_ERR_INVALID_ARG, "negative window parameter");
    if (!(p->beta > 0.0f) || !(p->gamma > 0.0f) || !(p->sigma > 0.0f))
        return fail(ELAS_ERR_INVALID_ARG, "beta, gamma, sigma must be > 0");
    if (p->support_downsample < 0) return fail(ELAS_ERR_INVALID_ARG, "support_downsample %d < 0", p->support_downsample);
    const int cs = p->census_support_w, cd = p->census_dense_w;
    if (cs != 0 || cd != 0) {
        if (cs < 3 || cs > 15 || cs % 2 == 0 || cd < 3 || cd > 11 || cd % 2 == 0)
            return fail(ELAS_ERR_INVALID_ARG,
                        "census windows %d / %d: both 0, or odd with support 3..15 and dense 3..11", cs, cd);
    }
    return ELAS_OK;
}

// P[k] = trunc((ln gamma - ln(gamma + exp(-k^2 / (2 sigma^2)))) / beta) in double.
void prior_table(const elas_params *p, int32_t *P) {
    const double g = p->gamma, s = p->sigma, b = p->beta;
    for (int k = 0; k <= p->sradius; ++k) {
        const double e = std::exp(-(double(k) * double(k)) / (2.0 * s * s));
        P[k] = static_cast<int32_t>((std::log(g) - std::log(g + e)) / b);
    }
}

}  // namespace elas

extern "C" {

// One workspace for the per-pair calls made one after another: the largest
// of their own requirements at this size (the device triangulation of one
// side with the full candidate count, the plane prior with the triangle
// bound of one mesh).
size_t elas_workspace_bytes(int32_t w, int32_t h, const elas_params *p) {
    if (elas::check_params(p, w, h) != ELAS_OK) return 0;
    const int32_t step = p->candidate_stepsize;
    const int32_t cap = (w / step) * (h / step);
    size_t m = elas_support_workspace_bytes(w, h, p);
    m = std::max(m, elas_triangulate_device_workspace_bytes(cap > 0 ? cap : 1, w, h));
    m = std::max(m, elas_plane_prior_workspace_bytes(2 * cap + 8));
    m = std::max(m, elas_dense_workspace_bytes(w, h, p));
    m = std::max(m, elas_postprocess_workspace_bytes(w, h));
    m = std::max(m, elas_speckle_workspace_bytes(w, h));
    return m;
}

elas_status elas_params_default(elas_params *p) {
    if (!p) return elas::fail(ELAS_ERR_INVALID_ARG, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->disp_min = 0;
    p->disp_max = 255;
    p->support_threshold = 0.85f;
    p->support_texture = 10;
    p->candidate_stepsize = 5;
    p->incon_window_size = 5;
    p->incon_threshold = 5;
    p->incon_min_support = 5;
    p->redun_max_dist = 5;
    p->grid_size = 20;
    p->beta = 0.02f;
    p->gamma = 3.0f;
    p->sigma = 1.0f;
    p->sradius = 2;
    p->match_texture = 1;
    p->lr_threshold = 2;
    p->ipol_gap_width = 3;
    p->filter_adaptive_mean = 1;
    p->test_flags = 0;
    p->census_support_w = 0;
    p->census_dense_w = 0;
    p->support_downsample = 0;
    return ELAS_OK;
}

const char *elas_last_error(void) { return elas::g_err; }

const char *elas_version(void) { return "elas_gb300 0.1 (sm_103a)"; }

}  // extern "C"
