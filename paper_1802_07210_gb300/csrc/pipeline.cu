// Pipeline handle: the per-pair runtime around the kernels.
//
// Owns, for one image size: device buffers for every intermediate, the
// workspaces, a pinned staging area for the support list (device -> host)
// and the triangles (host -> device), and one helper thread so that the
// left- and right-coordinate triangulations of the host route run
// concurrently.
//
// Per pair, GPU triangulation (the default): descriptors (or the two census
// records) -> support -> both triangulations -> plane prior -> dense -> LR
// check -> post-processing, all on the device and replayed as one CUDA graph
// per set of buffers; the support and triangle counts go to the host on a
// side stream for the statistics.  Host route: support (GPU) | count + list
// to host | two triangulations (host, in parallel) | triangles to device |
// plane prior -> dense -> LR check -> post-processing (GPU).
#include <chrono>
#include <condition_variable>
#include <functional>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "launch.cuh"

namespace {

// One persistent helper thread running one job at a time.
class Helper {
  public:
    Helper() : th_([this] { loop(); }) {}
    ~Helper() {
        {
            std::lock_guard<std::mutex> g(m_);
            stop_ = true;
        }
        cv_.notify_all();
        th_.join();
    }
    template <class F> void submit(F &&f) {
        std::lock_guard<std::mutex> g(m_);
        job_ = std::forward<F>(f);
        has_job_ = true;
        done_ = false;
        cv_.notify_all();
    }
    void wait() {
        std::unique_lock<std::mutex> g(m_);
        cv_.wait(g, [this] { return done_; });
    }

  private:
    void loop() {
        for (;;) {
            std::function<void()> job;
            {
                std::unique_lock<std::mutex> g(m_);
                cv_.wait(g, [this] { return stop_ || has_job_; });
                if (stop_) return;
                job = std::move(job_);
                has_job_ = false;
            }
            job();
            {
                std::lock_guard<std::mutex> g(m_);
                done_ = true;
            }
            cv_.notify_all();
        }
    }
    std::mutex m_;
    std::condition_variable cv_;
    std::function<void()> job_;
    bool has_job_ = false, done_ = true, stop_ = false;
    std::thread th_;
};

}  // namespace

struct elas_pipeline {
    int w = 0, h = 0, wc = 0, hc = 0, nc = 0;
    elas_params p{};
    elas::GridGeom g{};
    // device
    uint8_t *img = nullptr;  // L then R (host-input path)
    uint8_t *descL = nullptr, *descR = nullptr;  // Sobel descriptors, or dense census records
    uint8_t *sdescL = nullptr, *sdescR = nullptr;  // census variant: support census records
    int16_t *dcan = nullptr;
    char *countlist = nullptr;  // int32 count at offset 0, int16 list at offset 16
    uint32_t *gridL = nullptr, *gridR = nullptr;
    int32_t *tri = nullptr;  // left triangles then right triangles
    void *ws_support = nullptr, *ws_dense = nullptr, *ws_post = nullptr;
    int16_t *dL = nullptr, *dR = nullptr;  // host-output path
    float *post = nullptr;
    size_t ws_support_bytes = 0, ws_dense_bytes = 0, ws_post_bytes = 0;
    // pinned host
    char *h_countlist = nullptr;
    int32_t *h_tri = nullptr;
    size_t countlist_bytes = 0;
    int tri_cap = 0;  // per side
    // triangulation on the GPU (default) or on the host
    int gpu_tri = 1;
    void *ws_dt = nullptr;
    size_t ws_dt_bytes = 0;
    cudaStream_t last_stream = nullptr;
    // stage marks (profiling on): descriptors | support | triangulation |
    // plane prior | dense argmin | LR check + post-processing
    int profiling = 0;
    bool marked = false;
    cudaEvent_t marks[7] = {};
    // graph replay of the step (GPU triangulation): one executable graph per
    // argument signature (input/output pointers, pitch, profiling), up to
    // kGraphCache of them, least recently used replaced; a signature is run
    // eagerly the first time and captured the second
    struct GraphEntry {
        std::vector<const void *> sig;
        cudaGraphExec_t exec = nullptr;
        uint64_t last = 0;
    };
    static constexpr size_t kGraphCache = 8;
    int use_graph = 1;
    cudaStream_t work = nullptr;
    // the counts' read-back runs on a branch of its own, joined at the end
    // of the step, so the LR check does not wait for the copy
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<GraphEntry> graphs;
    uint64_t graph_clock = 0;
    // last run
    elas_pipeline_stats stats{};
    std::vector<int32_t> triL_v, triR_v;
    Helper *helper = nullptr;
};

namespace {

template <class T> cudaError_t dalloc(T **p, size_t bytes) {
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

void release(elas_pipeline *pl) {
    if (!pl) return;
    delete pl->helper;
    if (pl->work) cudaStreamSynchronize(pl->work);
    for (auto &g : pl->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (pl->side) cudaStreamSynchronize(pl->side);
    if (pl->work) cudaStreamDestroy(pl->work);
    if (pl->side) cudaStreamDestroy(pl->side);
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->ev_join) cudaEventDestroy(pl->ev_join);
    for (cudaEvent_t &e : pl->marks)
        if (e) cudaEventDestroy(e);
    void *dev[] = {pl->img, pl->descL, pl->descR, pl->sdescL, pl->sdescR, pl->dcan, pl->countlist, pl->gridL, pl->gridR, pl->tri,
                   pl->ws_support, pl->ws_dense, pl->ws_post, pl->dL, pl->dR, pl->post, pl->ws_dt};
    for (void *d : dev)
        if (d) cudaFree(d);
    if (pl->h_countlist) cudaFreeHost(pl->h_countlist);
    if (pl->h_tri) cudaFreeHost(pl->h_tri);
    delete pl;
}

// Host part of one pair: triangulations in left and right coordinates.
elas_status triangulate_both(elas_pipeline *pl, int n, const int16_t *list, int *ntL, int *ntR) {
    std::vector<int32_t> &tl = pl->triL_v, &tr = pl->triR_v;
    int32_t cntL = 0, cntR = 0;
    elas_status sR = ELAS_OK;
    tr.resize((size_t)3 * pl->tri_cap);
    tl.resize((size_t)3 * pl->tri_cap);
    pl->helper->submit([&] { sR = elas_triangulate(list, n, 1, tr.data(), pl->tri_cap, &cntR); });
    elas_status sL = elas_triangulate(list, n, 0, tl.data(), pl->tri_cap, &cntL);
    pl->helper->wait();
    if (sL != ELAS_OK) return sL;
    if (sR != ELAS_OK) return sR;
    *ntL = cntL;
    *ntR = cntR;
    std::memcpy(pl->h_tri, tl.data(), sizeof(int32_t) * 3 * (size_t)cntL);
    std::memcpy(pl->h_tri + 3 * (size_t)cntL, tr.data(), sizeof(int32_t) * 3 * (size_t)cntR);
    return ELAS_OK;
}

}  // namespace

extern "C" elas_status elas_pipeline_create(int32_t w, int32_t h, const elas_params *p, elas_pipeline **out) {
    using namespace elas;
    if (!out) return fail(ELAS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    elas_pipeline *pl = new (std::nothrow) elas_pipeline();
    if (!pl) return fail(ELAS_ERR_NO_MEMORY, "host allocation");
    pl->w = w;
    pl->h = h;
    pl->p = *p;
    pl->wc = w / p->candidate_stepsize;
    pl->hc = h / p->candidate_stepsize;
    pl->nc = pl->wc * pl->hc;
    pl->g = grid_geom(w, h, p);
    const size_t npx = (size_t)w * h;
    const size_t gbytes = (size_t)pl->g.gw * pl->g.gh * pl->g.nw * sizeof(uint32_t);
    pl->tri_cap = 2 * pl->nc + 8;
    pl->countlist_bytes = 16 + align_up((size_t)pl->nc * 3 * sizeof(int16_t) + 16, 16);
    pl->ws_support_bytes = support_workspace(w, h, p);
    pl->ws_dense_bytes = dense_workspace(w, h, p);
    pl->ws_post_bytes = post_workspace(w, h);
    pl->ws_dt_bytes = triangulate_device_workspace(pl->nc, w, h, 2);
    bool ok = dalloc(&pl->img, 2 * align_up(npx, 256)) == cudaSuccess &&
              dalloc(&pl->descL, npx * 16) == cudaSuccess && dalloc(&pl->descR, npx * 16) == cudaSuccess &&
              dalloc(&pl->dcan, (size_t)pl->nc * 2 + 16) == cudaSuccess &&
              dalloc(&pl->countlist, pl->countlist_bytes) == cudaSuccess &&
              dalloc(&pl->gridL, gbytes) == cudaSuccess && dalloc(&pl->gridR, gbytes) == cudaSuccess &&
              dalloc(&pl->tri, sizeof(int32_t) * 3 * 2 * (size_t)pl->tri_cap) == cudaSuccess &&
              dalloc(&pl->ws_support, pl->ws_support_bytes) == cudaSuccess &&
              dalloc(&pl->ws_dense, pl->ws_dense_bytes) == cudaSuccess &&
              dalloc(&pl->ws_post, pl->ws_post_bytes) == cudaSuccess &&
              dalloc(&pl->dL, npx * 2) == cudaSuccess && dalloc(&pl->dR, npx * 2) == cudaSuccess &&
              dalloc(&pl->post, npx * 4) == cudaSuccess && dalloc(&pl->ws_dt, pl->ws_dt_bytes) == cudaSuccess &&
              (p->census_support_w == 0 ||
               (dalloc(&pl->sdescL, npx * 32) == cudaSuccess && dalloc(&pl->sdescR, npx * 32) == cudaSuccess)) &&
              cudaMallocHost(reinterpret_cast<void **>(&pl->h_countlist), pl->countlist_bytes) == cudaSuccess &&
              cudaMallocHost(reinterpret_cast<void **>(&pl->h_tri), sizeof(int32_t) * 3 * 2 * (size_t)pl->tri_cap) ==
                  cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(pl);
        return fail(ELAS_ERR_NO_MEMORY, "pipeline allocation for %dx%d failed", w, h);
    }
    pl->helper = new (std::nothrow) Helper();
    if (!pl->helper) {
        release(pl);
        return fail(ELAS_ERR_NO_MEMORY, "helper thread");
    }
    if (cudaStreamCreateWithFlags(&pl->work, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        release(pl);
        return fail(ELAS_ERR_NO_MEMORY, "pipeline streams");
    }
    *out = pl;
    return ELAS_OK;
}

// The whole step for one pair on stream st (validated arguments).
static elas_status run_step(elas_pipeline *pl, const uint8_t *imgL, const uint8_t *imgR, int32_t pitch, int16_t *dL,
                            int16_t *dR, float *post, cudaStream_t st) {
    using namespace elas;
    const int w = pl->w, h = pl->h;
    const elas_params *p = &pl->p;
    int16_t *list = reinterpret_cast<int16_t *>(pl->countlist + 16);
    int32_t *count = reinterpret_cast<int32_t *>(pl->countlist);
    elas_status s;
    pl->last_stream = st;
    const bool prof = pl->profiling && pl->gpu_tri;
    auto mark = [&](int i) {
        if (prof) record_mark(pl->marks[i], st);
    };
    pl->marked = prof;
    mark(0);
    const bool census = p->census_support_w > 0;
    if (census) {
        // Sec. VI.A: support and dense census records in place of the descriptors
        if ((s = launch_census(imgL, imgR, w, h, pitch, p->census_support_w, 32, pl->sdescL, pl->sdescR, st)) !=
                ELAS_OK ||
            (s = launch_census(imgL, imgR, w, h, pitch, p->census_dense_w, 16, pl->descL, pl->descR, st)) != ELAS_OK)
            return s;
    } else if ((s = launch_descriptors(imgL, imgR, w, h, pitch, pl->descL, pl->descR, st)) != ELAS_OK) {
        return s;
    }
    mark(1);
    if ((s = launch_support(census ? pl->sdescL : pl->descL, census ? pl->sdescR : pl->descR, w, h, p, pl->dcan,
                            list, count, pl->gridL, pl->gridR, pl->ws_support, st)) != ELAS_OK)
        return s;
    mark(2);
    int16_t *outR = dR ? dR : pl->dR;
    if (pl->gpu_tri) {
        // everything stays on the device: no synchronisation in the step
        int32_t *ntri_dev = count + 1;  // [count, ntri left, ntri right, -] then the list
        const int rights[2] = {0, 1};
        int32_t *tris[2] = {pl->tri, pl->tri + 3 * (size_t)pl->tri_cap};
        int32_t *nts[2] = {ntri_dev, ntri_dev + 1};
        if ((s = launch_triangulate_device(list, count, pl->nc, w, h, 2, rights, tris, nts, pl->tri_cap, pl->ws_dt,
                                           st)) != ELAS_OK)
            return s;
        mark(3);
        if ((s = launch_dense_both(pl->descL, pl->descR, w, h, p, list, tris[0], pl->tri_cap, tris[1], pl->tri_cap,
                                   pl->gridL, pl->gridR, dL, outR, pl->ws_dense, st, ntri_dev,
                                   prof ? pl->marks[4] : nullptr)) != ELAS_OK)
            return s;
        mark(5);
        if (cudaEventRecord(pl->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(pl->side, pl->ev_fork, 0) != cudaSuccess ||
            cudaMemcpyAsync(pl->h_countlist, pl->countlist, 16, cudaMemcpyDeviceToHost, pl->side) != cudaSuccess ||
            cudaEventRecord(pl->ev_join, pl->side) != cudaSuccess)
            return launch_status("stats to host");
        pl->stats.triangulate_ms = 0.0;
    } else {
        if (cudaMemcpyAsync(pl->h_countlist, pl->countlist, pl->countlist_bytes, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return launch_status("support list to host");
        const int n = *reinterpret_cast<const int32_t *>(pl->h_countlist);
        if (n < 0 || n > pl->nc) return fail(ELAS_ERR_INTERNAL, "support count %d out of range", n);
        const auto t0 = std::chrono::steady_clock::now();
        int ntL = 0, ntR = 0;
        if ((s = triangulate_both(pl, n, reinterpret_cast<const int16_t *>(pl->h_countlist + 16), &ntL, &ntR)) !=
            ELAS_OK)
            return s;
        const auto t1 = std::chrono::steady_clock::now();
        pl->stats.n_support = n;
        pl->stats.n_tri_left = ntL;
        pl->stats.n_tri_right = ntR;
        pl->stats.triangulate_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        if (ntL + ntR > 0 && cudaMemcpyAsync(pl->tri, pl->h_tri, sizeof(int32_t) * 3 * (size_t)(ntL + ntR),
                                             cudaMemcpyHostToDevice, st) != cudaSuccess)
            return launch_status("triangles to device");
        if ((s = launch_dense_both(pl->descL, pl->descR, w, h, p, list, pl->tri, ntL, pl->tri + 3 * (size_t)ntL,
                                   ntR, pl->gridL, pl->gridR, dL, outR, pl->ws_dense, st, nullptr)) != ELAS_OK)
            return s;
    }
    if ((s = launch_lr_check(dL, outR, w, h, p->lr_threshold, nullptr, nullptr, st)) != ELAS_OK) return s;
    if (post && (s = launch_post(dL, w, h, p, post, pl->ws_post, st)) != ELAS_OK) return s;
    if (pl->gpu_tri && cudaStreamWaitEvent(st, pl->ev_join, 0) != cudaSuccess) return launch_status("stats join");
    mark(6);
    return ELAS_OK;
}

// With GPU triangulation nothing in the step depends on the host, so the
// step is captured once per set of buffers into a CUDA graph (recorded on an
// internal stream, which executes nothing while capturing) and replayed on
// the caller's stream: one launch instead of ~30 kernels and memsets.  The
// first run with new buffers goes eagerly.
static elas_status run_graph(elas_pipeline *pl, const uint8_t *imgL, const uint8_t *imgR, int32_t pitch, int16_t *dL,
                             int16_t *dR, float *post, cudaStream_t st) {
    using namespace elas;
    const std::vector<const void *> sig{imgL, imgR, reinterpret_cast<const void *>((intptr_t)pitch), dL, dR, post,
                                        reinterpret_cast<const void *>((intptr_t)pl->profiling)};
    elas_pipeline::GraphEntry *ge = nullptr;
    for (auto &g : pl->graphs)
        if (g.sig == sig) ge = &g;
    if (!ge) {  // first time: eager, remembered (replacing the least recently used)
        if (pl->graphs.size() < elas_pipeline::kGraphCache) {
            pl->graphs.emplace_back();
            ge = &pl->graphs.back();
        } else {
            ge = &pl->graphs[0];
            for (auto &g : pl->graphs)
                if (g.last < ge->last) ge = &g;
            if (ge->exec) cudaGraphExecDestroy(ge->exec);
            ge->exec = nullptr;
        }
        ge->sig = sig;
        ge->last = ++pl->graph_clock;
        return run_step(pl, imgL, imgR, pitch, dL, dR, post, st);
    }
    ge->last = ++pl->graph_clock;
    if (!ge->exec) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(pl->work, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return launch_status("begin pipeline capture");
        elas_status s = run_step(pl, imgL, imgR, pitch, dL, dR, post, pl->work);
        const cudaError_t e = cudaStreamEndCapture(pl->work, &g);
        if (s == ELAS_OK && e != cudaSuccess) s = fail(ELAS_ERR_CUDA, "pipeline capture: %s", cudaGetErrorString(e));
        if (s == ELAS_OK && cudaGraphInstantiate(&ge->exec, g, 0) != cudaSuccess) {
            ge->exec = nullptr;
            s = launch_status("pipeline graph instantiate");
        }
        if (g) cudaGraphDestroy(g);
        if (s != ELAS_OK) {
            ge->sig.clear();
            return s;
        }
    }
    if (cudaGraphLaunch(ge->exec, st) != cudaSuccess) return launch_status("pipeline graph launch");
    pl->last_stream = st;
    return ELAS_OK;
}

extern "C" elas_status elas_pipeline_run(elas_pipeline *pl, const uint8_t *imgL, const uint8_t *imgR, int32_t pitch,
                                         int16_t *dL, int16_t *dR, float *post, elas_stream stream) {
    using namespace elas;
    if (!pl || !imgL || !imgR || !dL) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    if (pitch < pl->w) return fail(ELAS_ERR_INVALID_ARG, "pitch %d < width %d", pitch, pl->w);
    cudaStream_t st = to_stream(stream);
    if (pl->gpu_tri && pl->use_graph) return run_graph(pl, imgL, imgR, pitch, dL, dR, post, st);
    return run_step(pl, imgL, imgR, pitch, dL, dR, post, st);
}

extern "C" elas_status elas_pipeline_run_host(elas_pipeline *pl, const uint8_t *imgL, const uint8_t *imgR,
                                              int16_t *dL, int16_t *dR, float *post, elas_stream stream) {
    using namespace elas;
    if (!pl || !imgL || !imgR || !dL) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = to_stream(stream);
    const size_t npx = (size_t)pl->w * pl->h;
    uint8_t *iL = pl->img, *iR = pl->img + align_up(npx, 256);
    if (cudaMemcpyAsync(iL, imgL, npx, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(iR, imgR, npx, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return launch_status("images to device");
    elas_status s = elas_pipeline_run(pl, iL, iR, pl->w, pl->dL, pl->dR, post ? pl->post : nullptr, stream);
    if (s != ELAS_OK) return s;
    if (cudaMemcpyAsync(dL, pl->dL, npx * 2, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return launch_status("left map to host");
    if (dR && cudaMemcpyAsync(dR, pl->dR, npx * 2, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return launch_status("right map to host");
    if (post && cudaMemcpyAsync(post, pl->post, npx * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return launch_status("post map to host");
    if (cudaStreamSynchronize(st) != cudaSuccess) return launch_status("pipeline sync");
    return ELAS_OK;
}

extern "C" elas_status elas_pipeline_set_triangulation(elas_pipeline *pl, int32_t on_gpu) {
    if (!pl) return elas::fail(ELAS_ERR_INVALID_ARG, "NULL pipeline");
    pl->gpu_tri = on_gpu ? 1 : 0;
    return ELAS_OK;
}

extern "C" elas_status elas_pipeline_set_graph(elas_pipeline *pl, int32_t on) {
    if (!pl) return elas::fail(ELAS_ERR_INVALID_ARG, "NULL pipeline");
    if ((on ? 1 : 0) != pl->use_graph) {
        pl->use_graph = on ? 1 : 0;
        if (pl->work) cudaStreamSynchronize(pl->work);
        for (auto &g : pl->graphs)  // the next graph runs start eagerly
            if (g.exec) cudaGraphExecDestroy(g.exec);
        pl->graphs.clear();
    }
    return ELAS_OK;
}

extern "C" elas_status elas_pipeline_set_profiling(elas_pipeline *pl, int32_t on) {
    if (!pl) return elas::fail(ELAS_ERR_INVALID_ARG, "NULL pipeline");
    if (on && !pl->marks[0])
        for (cudaEvent_t &e : pl->marks)
            if (cudaEventCreate(&e) != cudaSuccess) return elas::launch_status("profiling events");
    pl->profiling = on ? 1 : 0;
    return ELAS_OK;
}

extern "C" elas_status elas_pipeline_stats_get(const elas_pipeline *pl, elas_pipeline_stats *st) {
    if (!pl || !st) return elas::fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    *st = pl->stats;
    for (float &v : st->stage_ms) v = 0.0f;
    if (pl->marked) {
        if (cudaEventSynchronize(pl->marks[6]) != cudaSuccess) return elas::launch_status("stage marks");
        for (int i = 0; i < 6; ++i) cudaEventElapsedTime(&st->stage_ms[i], pl->marks[i], pl->marks[i + 1]);
    }
    if (pl->gpu_tri) {
        if (cudaStreamSynchronize(pl->last_stream) != cudaSuccess) return elas::launch_status("stats sync");
        const int32_t *c = reinterpret_cast<const int32_t *>(pl->h_countlist);
        st->n_support = c[0];
        st->n_tri_left = c[1];
        st->n_tri_right = c[2];
        if (c[1] < 0 || c[2] < 0) return elas::fail(ELAS_ERR_INTERNAL, "device triangulation failed");
    }
    return ELAS_OK;
}

extern "C" void elas_pipeline_destroy(elas_pipeline *pl) { release(pl); }
