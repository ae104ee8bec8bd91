// Batch handle (elas_batch_*): a fixed set of slots run as one wave of
// batched launches, optionally captured once into a CUDA graph, with a
// tuner for the tile-shape knobs.
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "slots.cuh"

namespace elas {
namespace {

// Tuned knobs per process, keyed by the batch's shape list.
std::mutex g_tune_mu;
std::map<std::vector<int>, Knobs> g_tuned;

std::vector<int> shape_key(const SlotPool &pool, const std::vector<int> &ids) {
    std::vector<int> k;
    for (int id : ids) {
        const Slot &s = pool[id];
        k.insert(k.end(), {s.w, s.h, s.p.disp_min, s.p.disp_max, s.p.grid_size, s.p.candidate_stepsize});
    }
    return k;
}

}  // namespace
}  // namespace elas

struct elas_batch {
    elas::SlotPool pool;
    std::vector<int> ids;
    elas::Knobs knobs;
    int use_graph = 1;
    cudaStream_t work = nullptr;  // internal stream the batch runs on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int32_t *counter = nullptr;   // device: the CTA pass's queue position
    cudaGraphExec_t exec = nullptr;
    std::vector<int> graph_sig;   // post passes and knobs the graph was captured with
    size_t extra_bytes = 0;
    bool ran = false;
};

namespace {

using namespace elas;

void drop_graph(elas_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_sig.clear();
}

void release(elas_batch *b) {
    if (!b) return;
    if (b->work) cudaStreamSynchronize(b->work);
    drop_graph(b);
    if (b->counter) cudaFree(b->counter);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->work) cudaStreamDestroy(b->work);
    delete b;
}

std::vector<int> signature(const elas_batch *b) {
    std::vector<int> sig{b->knobs.desc_rows, b->knobs.support_warps, b->knobs.dense_tpp, b->knobs.dense_ppt,
                         b->knobs.dense_fused};
    for (int id : b->ids) sig.push_back(b->pool[id].npass * 2 + b->pool[id].fused);
    return sig;
}

// The wave on the internal stream (eager launches).
elas_status wave(elas_batch *b, const StageMarks *marks) {
    elas_status s = b->pool.launch(b->ids.data(), (int)b->ids.size(), b->knobs, b->work, b->counter, marks);
    if (s != ELAS_OK) return s;
    return b->pool.fetch_counters(b->work);
}

elas_status capture(elas_batch *b) {
    drop_graph(b);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->work, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return launch_status("begin graph capture");
    const elas_status s = wave(b, nullptr);
    const cudaError_t e = cudaStreamEndCapture(b->work, &g);
    if (s != ELAS_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return fail(ELAS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        b->exec = nullptr;
        return fail(ELAS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e2));
    }
    b->graph_sig = signature(b);
    return ELAS_OK;
}

// Points every slot at the caller's buffers (NULL arrays/entries as documented).
elas_status bind_io(elas_batch *b, const uint8_t *const *imgL, const uint8_t *const *imgR, const int32_t *pitch,
                    int16_t *const *dL, int16_t *const *dR, float *const *post) {
    const int n = (int)b->ids.size();
    for (int i = 0; i < n; ++i) {
        const int id = b->ids[i];
        const Slot &sl = b->pool[id];
        if (!imgL[i] || !imgR[i] || !dL[i]) return fail(ELAS_ERR_INVALID_ARG, "pair %d: NULL image or dL", i);
        const int pt = pitch ? pitch[i] : sl.w;
        float *po = post ? post[i] : nullptr;
        elas_status s = b->pool.set_io(id, imgL[i], imgR[i], pt, dL[i], dR ? dR[i] : nullptr, po != nullptr, po);
        if (s != ELAS_OK) return s;
    }
    return ELAS_OK;
}

// Uploads changed records and runs the wave on the internal stream, joined
// to `st` on both sides.
elas_status run_bound(elas_batch *b, cudaStream_t st) {
    if (cudaEventRecord(b->ev_in, st) != cudaSuccess || cudaStreamWaitEvent(b->work, b->ev_in, 0) != cudaSuccess)
        return launch_status("batch fork");
    elas_status s = b->pool.upload(b->work);
    if (s != ELAS_OK) return s;
    if (b->use_graph && b->ran) {
        // the first run goes eagerly: it sets the kernels' attributes outside
        // a capture
        if (!b->exec || b->graph_sig != signature(b))
            if ((s = capture(b)) != ELAS_OK) return s;
        if (cudaGraphLaunch(b->exec, b->work) != cudaSuccess) return launch_status("graph launch");
    } else {
        if ((s = wave(b, nullptr)) != ELAS_OK) return s;
    }
    b->ran = true;
    if (cudaEventRecord(b->ev_out, b->work) != cudaSuccess || cudaStreamWaitEvent(st, b->ev_out, 0) != cudaSuccess)
        return launch_status("batch join");
    return ELAS_OK;
}

bool knob_ok(const Knobs &k) {
    return (k.desc_rows == 12 || k.desc_rows == 24 || k.desc_rows == 36) &&
           (k.support_warps == 4 || k.support_warps == 8 || k.support_warps == 16) &&
           (k.dense_tpp == 1 || k.dense_tpp == 2 || k.dense_tpp == 4) &&
           (k.dense_ppt == 1 || k.dense_ppt == 2 || k.dense_ppt == 4 || k.dense_ppt == 8 || k.dense_ppt == 16) &&
           (k.dense_fused == 0 || k.dense_fused == 1);
}

}  // namespace

extern "C" elas_status elas_batch_create(int32_t n, const int32_t *w, const int32_t *h, const elas_params *params,
                                         elas_batch **out) {
    if (!out) return fail(ELAS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxBatch) return fail(ELAS_ERR_INVALID_ARG, "batch of %d pairs (1..%d)", n, kMaxBatch);
    if (!w || !h || !params) return fail(ELAS_ERR_INVALID_ARG, "NULL shape or parameter array");
    elas_batch *b = new (std::nothrow) elas_batch();
    if (!b) return fail(ELAS_ERR_NO_MEMORY, "host allocation");
    elas_status s = b->pool.init(n);
    if (s != ELAS_OK) {
        release(b);
        return s;
    }
    for (int i = 0; i < n; ++i) {
        int id = -1;
        if ((s = b->pool.add(w[i], h[i], params + i, &id)) != ELAS_OK) {
            release(b);
            return s;
        }
        b->ids.push_back(id);
    }
    if (cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&b->counter), 256) != cudaSuccess) {
        cudaGetLastError();
        release(b);
        return fail(ELAS_ERR_NO_MEMORY, "batch stream, events or counter");
    }
    b->extra_bytes = 256 + sizeof(SlotTables) * (size_t)n + 16 * (size_t)n;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tuned.find(shape_key(b->pool, b->ids));
        if (it != g_tuned.end()) b->knobs = it->second;
    }
    *out = b;
    return ELAS_OK;
}

extern "C" elas_status elas_batch_get_config(const elas_batch *b, elas_batch_config *cfg) {
    if (!b || !cfg) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    cfg->desc_tile_rows = b->knobs.desc_rows;
    cfg->support_warps = b->knobs.support_warps;
    cfg->dense_threads_per_pixel = b->knobs.dense_tpp;
    cfg->dense_pixels_per_thread = b->knobs.dense_ppt;
    cfg->dense_fused = b->knobs.dense_fused;
    cfg->use_graph = b->use_graph;
    return ELAS_OK;
}

extern "C" elas_status elas_batch_set_config(elas_batch *b, const elas_batch_config *cfg) {
    if (!b || !cfg) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    Knobs k;
    k.desc_rows = cfg->desc_tile_rows;
    k.support_warps = cfg->support_warps;
    k.dense_tpp = cfg->dense_threads_per_pixel;
    k.dense_ppt = cfg->dense_pixels_per_thread;
    k.dense_fused = cfg->dense_fused;
    if (!knob_ok(k))
        return fail(ELAS_ERR_INVALID_ARG,
                    "config %d/%d/%d/%d/%d outside {12,24,36}/{4,8,16}/{1,2,4}/{1,2,4,8,16}/{0,1}", k.desc_rows,
                    k.support_warps, k.dense_tpp, k.dense_ppt, k.dense_fused);
    b->knobs = k;
    b->use_graph = cfg->use_graph ? 1 : 0;
    return ELAS_OK;
}

extern "C" elas_status elas_batch_run(elas_batch *b, const uint8_t *const *imgL, const uint8_t *const *imgR,
                                      const int32_t *pitch, int16_t *const *dL, int16_t *const *dR,
                                      float *const *post, elas_stream stream) {
    if (!b || !imgL || !imgR || !dL) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    elas_status s = bind_io(b, imgL, imgR, pitch, dL, dR, post);
    if (s != ELAS_OK) return s;
    return run_bound(b, to_stream(stream));
}

extern "C" elas_status elas_batch_run_host(elas_batch *b, const uint8_t *const *imgL, const uint8_t *const *imgR,
                                           int16_t *const *dL, int16_t *const *dR, float *const *post,
                                           elas_stream stream) {
    if (!b || !imgL || !imgR || !dL) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = to_stream(stream);
    const int n = (int)b->ids.size();
    elas_status s;
    for (int i = 0; i < n; ++i) {
        const int id = b->ids[i];
        const Slot &sl = b->pool[id];
        if (!imgL[i] || !imgR[i] || !dL[i]) return fail(ELAS_ERR_INVALID_ARG, "pair %d: NULL image or dL", i);
        const bool want_post = post && post[i];
        if ((s = b->pool.set_io(id, nullptr, nullptr, 0, nullptr, nullptr, want_post, nullptr)) != ELAS_OK) return s;
        const size_t npx = (size_t)sl.w * sl.h;
        if (cudaMemcpyAsync(sl.img, imgL[i], npx, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(sl.img + align_up(npx, 256), imgR[i], npx, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return launch_status("images to device");
    }
    if ((s = run_bound(b, st)) != ELAS_OK) return s;
    for (int i = 0; i < n; ++i) {
        const Slot &sl = b->pool[b->ids[i]];
        const size_t npx = (size_t)sl.w * sl.h;
        if (cudaMemcpyAsync(dL[i], sl.dL, npx * 2, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            (dR && dR[i] && cudaMemcpyAsync(dR[i], sl.dR, npx * 2, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
            (post && post[i] && cudaMemcpyAsync(post[i], sl.post, npx * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess))
            return launch_status("maps to host");
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return launch_status("batch run");
    return ELAS_OK;
}

extern "C" elas_status elas_batch_stats(elas_batch *b, int32_t *n_support, int32_t *n_tri_left,
                                        int32_t *n_tri_right) {
    if (!b) return fail(ELAS_ERR_INVALID_ARG, "NULL batch");
    if (b->work && cudaStreamSynchronize(b->work) != cudaSuccess) return launch_status("batch stats");
    for (size_t i = 0; i < b->ids.size(); ++i) {
        const int32_t *c = b->pool.host_counters(b->ids[i]);
        if (n_support) n_support[i] = c[0];
        if (n_tri_left) n_tri_left[i] = c[1];
        if (n_tri_right) n_tri_right[i] = c[2];
    }
    return ELAS_OK;
}

extern "C" elas_status elas_batch_tune(elas_batch *b, const uint8_t *const *imgL, const uint8_t *const *imgR,
                                       const int32_t *pitch, int16_t *const *dL, elas_stream stream,
                                       elas_batch_config *chosen) {
    if (!b || !imgL || !imgR || !dL) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = to_stream(stream);
    elas_status s = bind_io(b, imgL, imgR, pitch, dL, nullptr, nullptr);
    if (s != ELAS_OK) return s;
    if (cudaEventRecord(b->ev_in, st) != cudaSuccess || cudaStreamWaitEvent(b->work, b->ev_in, 0) != cudaSuccess)
        return launch_status("tune fork");
    if ((s = b->pool.upload(b->work)) != ELAS_OK) return s;
    StageMarks mk;
    for (int i = 0; i < kStageMarks; ++i)
        if (cudaEventCreate(&mk.ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(mk.ev[j]);
            return launch_status("tune events");
        }
    // the stages each knob is timed over (between marks first and last); the
    // persistent prior + argmin launch is weighed against the separate
    // launches over both stages, with the shapes found for the latter
    struct Axis {
        int *field;
        int first, last;
        int nv;
        int values[3];
    };
    Knobs k = b->knobs;
    k.dense_fused = 0;
    Axis axes[5] = {{&k.desc_rows, 0, 1, 3, {12, 24, 36}},
                    {&k.support_warps, 1, 2, 3, {4, 8, 16}},
                    {&k.dense_tpp, 4, 5, 3, {1, 2, 4}},
                    {&k.dense_ppt, 4, 5, 3, {4, 8, 16}},
                    {&k.dense_fused, 3, 5, 2, {0, 1, 0}}};
    const int reps = 3;
    for (Axis &ax : axes) {
        float best_ms = 1e30f;
        int best_v = *ax.field;
        for (int vi = 0; vi < ax.nv; ++vi) {
            const int v = ax.values[vi];
            *ax.field = v;
            float tot = 0.0f;
            for (int r = 0; r <= reps && s == ELAS_OK; ++r) {  // r = 0 warms up
                s = b->pool.launch(b->ids.data(), (int)b->ids.size(), k, b->work, b->counter, &mk);
                if (s != ELAS_OK) break;
                if (cudaEventSynchronize(mk.ev[kStageMarks - 1]) != cudaSuccess) {
                    s = launch_status("tune run");
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, mk.ev[ax.first], mk.ev[ax.last]);
                if (r > 0) tot += ms;
            }
            if (s != ELAS_OK) break;
            if (tot < best_ms) {
                best_ms = tot;
                best_v = v;
            }
        }
        *ax.field = best_v;
        if (s != ELAS_OK) break;
    }
    for (int i = 0; i < kStageMarks; ++i) cudaEventDestroy(mk.ev[i]);
    if (s != ELAS_OK) return s;
    if (cudaEventRecord(b->ev_out, b->work) != cudaSuccess || cudaStreamWaitEvent(st, b->ev_out, 0) != cudaSuccess)
        return launch_status("tune join");
    b->knobs = k;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tuned[shape_key(b->pool, b->ids)] = k;
    }
    if (chosen) elas_batch_get_config(b, chosen);
    return ELAS_OK;
}

extern "C" elas_status elas_batch_profile(elas_batch *b, elas_stream stream, float *stage_ms) {
    if (!b || !stage_ms) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    if (!b->ran) return fail(ELAS_ERR_INVALID_ARG, "run the batch once first");
    cudaStream_t st = to_stream(stream);
    StageMarks mk;
    elas_status s = ELAS_OK;
    int made = 0;
    for (; made < kStageMarks; ++made)
        if (cudaEventCreate(&mk.ev[made]) != cudaSuccess) {
            s = launch_status("profile events");
            break;
        }
    if (s == ELAS_OK && (cudaEventRecord(b->ev_in, st) != cudaSuccess ||
                         cudaStreamWaitEvent(b->work, b->ev_in, 0) != cudaSuccess))
        s = launch_status("profile fork");
    if (s == ELAS_OK) s = b->pool.upload(b->work);
    if (s == ELAS_OK) s = wave(b, &mk);
    if (s == ELAS_OK && cudaEventSynchronize(mk.ev[kStageMarks - 1]) != cudaSuccess) s = launch_status("profile run");
    if (s == ELAS_OK)
        for (int i = 0; i + 1 < kStageMarks; ++i) {
            stage_ms[i] = 0.0f;
            cudaEventElapsedTime(&stage_ms[i], mk.ev[i], mk.ev[i + 1]);
        }
    if (s == ELAS_OK && (cudaEventRecord(b->ev_out, b->work) != cudaSuccess ||
                         cudaStreamWaitEvent(st, b->ev_out, 0) != cudaSuccess))
        s = launch_status("profile join");
    for (int i = 0; i < made; ++i) cudaEventDestroy(mk.ev[i]);
    return s;
}

extern "C" size_t elas_batch_device_bytes(const elas_batch *b) {
    return b ? b->pool.bytes_in_use() + b->extra_bytes : 0;
}

extern "C" void elas_batch_destroy(elas_batch *b) { release(b); }
