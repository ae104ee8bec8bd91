// Server (elas_server_*): request loop with continuous batching over
// resident slots.
//
// One scheduler thread owns the slot pool and the lanes (streams).  Each
// pass of its loop (1) retires the waves whose completion event has fired,
// handing their results to the poll queue and their slots back as idle;
// (2) when a lane is free, admits queued requests in arrival order (idle
// slot of the same shape, else a new slot within the HBM budget, releasing
// idle slots of other shapes when needed) and launches them as one wave:
// host-to-device copies, the batched path, device-to-host copies, the
// counters, an event; (3) sleeps briefly while waves run, or waits for new
// requests.  A request that arrives while waves are running joins the next
// wave on a free lane, so waves overlap on the device.  The plain mode runs
// one request at a time through the per-pair pipeline instead.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "slots.cuh"

namespace {

using namespace elas;
using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    int w = 0, h = 0;
    elas_params p{};
    const uint8_t *L = nullptr, *R = nullptr;
    int16_t *dL = nullptr;
    float *post = nullptr;
    std::vector<int> key;
    double t_submit = 0, t_start = 0, t_done = 0;
    int slot = -1, wave = 0;
};

struct Lane {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    int32_t *h_counters = nullptr; // pinned, capacity * 4
    std::vector<Request *> reqs;
    bool busy = false;
};

std::vector<int> shape_key(int w, int h, const elas_params *p) {
    std::vector<int> k{w, h};
    const int *words = reinterpret_cast<const int *>(p);
    k.insert(k.end(), words, words + sizeof(elas_params) / sizeof(int));
    return k;
}

}  // namespace

struct elas_server {
    elas_server_config cfg{};
    int device = 0;
    Clock::time_point t0;
    SlotPool pool;
    std::vector<std::vector<int>> slot_key;
    std::vector<char> slot_busy;
    std::vector<double> slot_used_at;
    std::vector<Lane> lanes;
    uint64_t budget = 0, slot_bytes = 0;
    // shared with the callers
    std::mutex mu;
    std::condition_variable cv_sched, cv_poll;
    std::deque<Request *> queue;
    std::deque<elas_server_result> results;
    bool stop = false;
    elas_server_stats stats{};
    // captured waves, by composition (slot, generation, post passes per slot);
    // a composition is captured the second time it is launched
    cudaStream_t cap_st = nullptr;
    std::map<std::vector<uint32_t>, cudaGraphExec_t> graphs;
    std::map<std::vector<uint32_t>, int> seen;
    // plain mode
    std::map<std::vector<int>, elas_pipeline *> pipelines;
    std::thread th;
    std::atomic<int> fail_allocs{0};  // injected slot-allocation refusals still to come

    double now() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

void push_result(elas_server *s, const Request *r, int status, int n_support) {
    elas_server_result res{};
    res.id = r->id;
    res.status = status;
    res.n_support = n_support;
    res.wave_size = r->wave;
    res.t_submit_ms = r->t_submit;
    res.t_start_ms = r->t_start;
    res.t_done_ms = r->t_done;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->results.push_back(res);
        s->stats.completed++;
    }
    s->cv_poll.notify_all();
}

void retire(elas_server *s, Lane &ln, int status) {
    const double t = s->now();
    for (Request *r : ln.reqs) {
        r->t_done = t;
        const int ns = status == ELAS_OK ? ln.h_counters[4 * r->slot] : 0;
        s->slot_busy[r->slot] = 0;
        s->slot_used_at[r->slot] = t;
        push_result(s, r, status, ns);
        delete r;
    }
    ln.reqs.clear();
    ln.busy = false;
}

// An idle slot for r (existing, or new within the budget); -1 if none now.
int admit(elas_server *s, Request *r, cudaStream_t st, int *error) {
    *error = ELAS_OK;
    const int cap = s->pool.capacity();
    for (int i = 0; i < cap; ++i)
        if (s->pool[i].used && !s->slot_busy[i] && s->slot_key[i] == r->key) return i;
    const size_t need = SlotPool::slot_bytes(r->w, r->h, &r->p);
    if (need > s->budget) {
        *error = ELAS_ERR_NO_MEMORY;
        return -1;
    }
    auto free_slot = [&] {
        for (int i = 0; i < cap; ++i)
            if (!s->pool[i].used) return true;
        return false;
    };
    // release idle slots of other shapes, least recently used first
    while (s->pool.bytes_in_use() + need > s->budget || !free_slot()) {
        int victim = -1;
        for (int i = 0; i < cap; ++i)
            if (s->pool[i].used && !s->slot_busy[i] && (victim < 0 || s->slot_used_at[i] < s->slot_used_at[victim]))
                victim = i;
        if (victim < 0) return -1;  // everything is busy: wait for a wave
        s->pool.remove(victim, st);
        s->slot_key[victim].clear();
        std::lock_guard<std::mutex> g(s->mu);
        s->stats.slots_released++;
        s->stats.slots_in_use--;
        s->stats.slot_bytes = s->pool.bytes_in_use();
    }
    int id = -1;
    for (;;) {
        elas_status e;
        int inj = s->fail_allocs.load();
        while (inj > 0 && !s->fail_allocs.compare_exchange_weak(inj, inj - 1)) {
        }
        if (inj > 0) {  // injected refusal (tests)
            e = fail(ELAS_ERR_NO_MEMORY, "slot allocation refused (injected)");
        } else {
            e = s->pool.add(r->w, r->h, &r->p, &id, st);
        }
        if (e == ELAS_OK) break;
        if (e != ELAS_ERR_NO_MEMORY) {
            *error = e;
            return -1;
        }
        // the device refused although the budget allows it (memory taken by
        // others): release an idle slot, least recently used first, and retry
        int victim = -1;
        bool busy = false;
        for (int i = 0; i < cap; ++i) {
            if (!s->pool[i].used) continue;
            if (s->slot_busy[i]) {
                busy = true;
            } else if (victim < 0 || s->slot_used_at[i] < s->slot_used_at[victim]) {
                victim = i;
            }
        }
        if (victim < 0) {
            if (busy) return -1;  // running waves hold memory: try again once they retire
            *error = ELAS_ERR_NO_MEMORY;  // nothing to release and nothing running
            return -1;
        }
        s->pool.remove(victim, st);
        s->slot_key[victim].clear();
        std::lock_guard<std::mutex> g(s->mu);
        s->stats.slots_released++;
        s->stats.slots_in_use--;
        s->stats.slot_bytes = s->pool.bytes_in_use();
    }
    s->slot_key[id] = r->key;
    s->slot_used_at[id] = s->now();
    std::lock_guard<std::mutex> g(s->mu);
    s->stats.slots_created++;
    s->stats.slots_in_use++;
    s->stats.slot_bytes = s->pool.bytes_in_use();
    return id;
}

void drop_graphs(elas_server *s) {
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
    s->seen.clear();
}

// The kernels of a wave: replayed from a graph when this composition was
// launched before, else eagerly (captured on its second launch).
elas_status launch_kernels(elas_server *s, const std::vector<int> &ids, const Knobs &knobs, cudaStream_t st) {
    std::vector<uint32_t> key;
    for (int id : ids) {
        const Slot &sl = s->pool[id];
        key.insert(key.end(), {(uint32_t)id, sl.generation, (uint32_t)sl.npass, (uint32_t)sl.fused});
    }
    auto it = s->graphs.find(key);
    if (it != s->graphs.end()) {
        if (cudaGraphLaunch(it->second, st) != cudaSuccess) return launch_status("wave graph launch");
        return ELAS_OK;
    }
    if (s->seen.size() > 8192) s->seen.clear();
    if (s->seen[key]++ == 0 || s->graphs.size() >= 512)
        return s->pool.launch(ids.data(), (int)ids.size(), knobs, st, nullptr);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(s->cap_st, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return launch_status("begin wave capture");
    elas_status e = s->pool.launch(ids.data(), (int)ids.size(), knobs, s->cap_st, nullptr);
    const cudaError_t ce = cudaStreamEndCapture(s->cap_st, &g);
    if (e == ELAS_OK && ce != cudaSuccess) e = fail(ELAS_ERR_CUDA, "wave capture: %s", cudaGetErrorString(ce));
    if (e == ELAS_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) e = launch_status("wave graph instantiate");
    if (g) cudaGraphDestroy(g);
    if (e != ELAS_OK) return e;
    s->graphs[key] = exec;
    if (cudaGraphLaunch(exec, st) != cudaSuccess) return launch_status("wave graph launch");
    return ELAS_OK;
}

elas_status launch_wave(elas_server *s, Lane &ln) {
    Knobs knobs;
    if (ln.reqs.size() == 1) knobs.dense_ppt = 1;  // a lone pair: one pixel per thread, as the per-pair path
    std::vector<int> ids;
    elas_status e = ELAS_OK;
    for (Request *r : ln.reqs) {
        const Slot &sl = s->pool[r->slot];
        ids.push_back(r->slot);
        if ((e = s->pool.set_io(r->slot, nullptr, nullptr, 0, nullptr, nullptr, r->post != nullptr, nullptr)) !=
            ELAS_OK)
            return e;
        const size_t npx = (size_t)sl.w * sl.h;
        if (cudaMemcpyAsync(sl.img, r->L, npx, cudaMemcpyHostToDevice, ln.st) != cudaSuccess ||
            cudaMemcpyAsync(sl.img + align_up(npx, 256), r->R, npx, cudaMemcpyHostToDevice, ln.st) != cudaSuccess)
            return launch_status("request images to device");
    }
    if ((e = s->pool.upload(ln.st)) != ELAS_OK) return e;
    if ((e = launch_kernels(s, ids, knobs, ln.st)) != ELAS_OK) return e;
    for (Request *r : ln.reqs) {
        const Slot &sl = s->pool[r->slot];
        const size_t npx = (size_t)sl.w * sl.h;
        if (cudaMemcpyAsync(r->dL, sl.dL, npx * 2, cudaMemcpyDeviceToHost, ln.st) != cudaSuccess ||
            (r->post && cudaMemcpyAsync(r->post, sl.post, npx * 4, cudaMemcpyDeviceToHost, ln.st) != cudaSuccess))
            return launch_status("request maps to host");
    }
    if ((e = s->pool.fetch_counters(ln.st, ln.h_counters)) != ELAS_OK) return e;
    if (cudaEventRecord(ln.done, ln.st) != cudaSuccess) return launch_status("wave event");
    return ELAS_OK;
}

void run_batched(elas_server *s) {
    for (;;) {
        // 1. retire finished waves
        bool busy = false;
        for (Lane &ln : s->lanes) {
            if (!ln.busy) continue;
            const cudaError_t q = cudaEventQuery(ln.done);
            if (q == cudaSuccess) {
                retire(s, ln, ELAS_OK);
            } else if (q == cudaErrorNotReady) {
                busy = true;
            } else {
                set_error("wave failed: %s", cudaGetErrorString(q));
                retire(s, ln, ELAS_ERR_CUDA);
            }
        }
        // 2. admit and launch on a free lane
        Lane *free_lane = nullptr;
        for (Lane &ln : s->lanes)
            if (!ln.busy) {
                free_lane = &ln;
                break;
            }
        bool launched = false;
        if (free_lane) {
            std::vector<Request *> wave, failed;
            std::vector<int> failed_status;
            {
                std::unique_lock<std::mutex> g(s->mu);
                while (!s->queue.empty() && (int)wave.size() < s->cfg.max_wave) {
                    Request *r = s->queue.front();
                    g.unlock();
                    int err = ELAS_OK;
                    const int slot = admit(s, r, free_lane->st, &err);
                    g.lock();
                    if (slot < 0 && err == ELAS_OK) break;  // in arrival order: wait for room
                    s->queue.pop_front();
                    if (slot < 0) {
                        failed.push_back(r);
                        failed_status.push_back(err);
                        continue;
                    }
                    s->slot_busy[slot] = 1;
                    r->slot = slot;
                    wave.push_back(r);
                }
            }
            for (size_t i = 0; i < failed.size(); ++i) {
                failed[i]->t_start = failed[i]->t_done = s->now();
                push_result(s, failed[i], failed_status[i], 0);
                delete failed[i];
            }
            if (!wave.empty()) {
                const double t = s->now();
                for (Request *r : wave) {
                    r->t_start = t;
                    r->wave = (int)wave.size();
                }
                free_lane->reqs = wave;
                free_lane->busy = true;
                const elas_status e = launch_wave(s, *free_lane);
                {
                    std::lock_guard<std::mutex> g(s->mu);
                    s->stats.waves++;
                    s->stats.max_wave_seen = std::max(s->stats.max_wave_seen, (int32_t)wave.size());
                }
                if (e != ELAS_OK) {
                    cudaStreamSynchronize(free_lane->st);
                    retire(s, *free_lane, e);
                } else {
                    launched = true;
                    busy = true;
                }
            }
        }
        // 3. wait
        std::unique_lock<std::mutex> g(s->mu);
        if (s->stop && s->queue.empty() && !busy) return;
        if (launched) continue;
        if (busy) {
            // waves in flight: poll their events again right away
            g.unlock();
            std::this_thread::yield();
        } else if (s->queue.empty()) {
            s->cv_sched.wait_for(g, std::chrono::milliseconds(2));
        } else {
            // queued requests but no room and nothing running: retry shortly
            g.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    }
}

void run_plain(elas_server *s) {
    Lane &ln = s->lanes[0];
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> g(s->mu);
            s->cv_sched.wait(g, [s] { return s->stop || !s->queue.empty(); });
            if (s->queue.empty()) return;  // stop requested and drained
            r = s->queue.front();
            s->queue.pop_front();
        }
        r->t_start = s->now();
        r->wave = 1;
        elas_pipeline *pl = nullptr;
        auto it = s->pipelines.find(r->key);
        elas_status e = ELAS_OK;
        if (it != s->pipelines.end()) {
            pl = it->second;
        } else if ((e = elas_pipeline_create(r->w, r->h, &r->p, &pl)) == ELAS_OK) {
            s->pipelines[r->key] = pl;
            std::lock_guard<std::mutex> g(s->mu);
            s->stats.slots_created++;
            s->stats.slots_in_use++;
        }
        int ns = 0;
        if (e == ELAS_OK) e = elas_pipeline_run_host(pl, r->L, r->R, r->dL, nullptr, r->post, ln.st);
        if (e == ELAS_OK) {
            elas_pipeline_stats st{};
            e = elas_pipeline_stats_get(pl, &st);
            ns = st.n_support;
        }
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->stats.waves++;
            s->stats.max_wave_seen = 1;
        }
        r->t_done = s->now();
        push_result(s, r, e, ns);
        delete r;
    }
}

void scheduler(elas_server *s) {
    cudaSetDevice(s->device);
    if (s->cfg.plain)
        run_plain(s);
    else
        run_batched(s);
}

void release(elas_server *s) {
    if (!s) return;
    for (Lane &ln : s->lanes) {
        if (ln.st) cudaStreamSynchronize(ln.st);
        if (ln.done) cudaEventDestroy(ln.done);
        if (ln.h_counters) cudaFreeHost(ln.h_counters);
        if (ln.st) cudaStreamDestroy(ln.st);
    }
    drop_graphs(s);
    if (s->cap_st) cudaStreamDestroy(s->cap_st);
    for (auto &kv : s->pipelines) elas_pipeline_destroy(kv.second);
    for (Request *r : s->queue) delete r;
    delete s;
}

}  // namespace

extern "C" elas_status elas_server_config_default(elas_server_config *cfg) {
    if (!cfg) return fail(ELAS_ERR_INVALID_ARG, "NULL config");
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->lanes = 3;
    cfg->max_wave = 64;
    cfg->max_slots = 256;
    cfg->plain = 0;
    cfg->hbm_budget_bytes = 0;
    cfg->hbm_reserve_bytes = 4ull << 30;
    return ELAS_OK;
}

extern "C" size_t elas_slot_device_bytes(int32_t w, int32_t h, const elas_params *p) {
    if (!p || check_params(p, w, h) != ELAS_OK || w < p->candidate_stepsize || h < p->candidate_stepsize) return 0;
    return SlotPool::slot_bytes(w, h, p);
}

extern "C" elas_status elas_server_create(const elas_server_config *cfg, elas_server **out) {
    if (!cfg || !out) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (cfg->lanes < 1 || cfg->lanes > 8) return fail(ELAS_ERR_INVALID_ARG, "lanes %d (1..8)", cfg->lanes);
    if (cfg->max_wave < 1 || cfg->max_wave > kMaxBatch)
        return fail(ELAS_ERR_INVALID_ARG, "max_wave %d (1..%d)", cfg->max_wave, kMaxBatch);
    if (cfg->max_slots < 1 || cfg->max_slots > 1024)
        return fail(ELAS_ERR_INVALID_ARG, "max_slots %d (1..1024)", cfg->max_slots);
    elas_server *s = new (std::nothrow) elas_server();
    if (!s) return fail(ELAS_ERR_NO_MEMORY, "host allocation");
    s->cfg = *cfg;
    if (s->cfg.plain) s->cfg.lanes = 1;
    s->t0 = Clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        release(s);
        return launch_status("server device");
    }
    elas_status e = ELAS_OK;
    if (!s->cfg.plain) {
        if ((e = s->pool.init(s->cfg.max_slots)) != ELAS_OK) {
            release(s);
            return e;
        }
        s->slot_key.assign(s->cfg.max_slots, {});
        s->slot_busy.assign(s->cfg.max_slots, 0);
        s->slot_used_at.assign(s->cfg.max_slots, 0.0);
    }
    s->budget = s->cfg.hbm_budget_bytes;
    if (s->budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            release(s);
            return launch_status("device memory info");
        }
        s->budget = fr > s->cfg.hbm_reserve_bytes ? fr - s->cfg.hbm_reserve_bytes : 0;
    }
    if (!s->cfg.plain) {  // slots of every shape stay mapped up to the budget once allocated
        elas_status e = s->pool.use_own_pool(s->budget);
        if (e != ELAS_OK) {
            release(s);
            return e;
        }
    }
    s->lanes.resize(s->cfg.lanes);
    for (Lane &ln : s->lanes) {
        const size_t cb = sizeof(int32_t) * 4 * (size_t)std::max(1, s->cfg.max_slots);
        if (cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void **>(&ln.h_counters), cb) != cudaSuccess) {
            cudaGetLastError();
            release(s);
            return fail(ELAS_ERR_NO_MEMORY, "server lanes");
        }
    }
    if (cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        release(s);
        return fail(ELAS_ERR_NO_MEMORY, "server capture stream");
    }
    s->stats.hbm_budget_bytes = s->budget;
    try {
        s->th = std::thread(scheduler, s);
    } catch (...) {
        release(s);
        return fail(ELAS_ERR_INTERNAL, "scheduler thread");
    }
    *out = s;
    return ELAS_OK;
}

extern "C" elas_status elas_server_submit(elas_server *s, uint64_t id, int32_t w, int32_t h, const elas_params *p,
                                          const uint8_t *imgL, const uint8_t *imgR, int16_t *dL, float *post) {
    if (!s || !p || !imgL || !imgR || !dL) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    elas_status e = check_params(p, w, h);
    if (e != ELAS_OK) return e;
    if (w < p->candidate_stepsize || h < p->candidate_stepsize)
        return fail(ELAS_ERR_INVALID_ARG, "%dx%d has no lattice candidate at step %d", w, h, p->candidate_stepsize);
    Request *r = new (std::nothrow) Request();
    if (!r) return fail(ELAS_ERR_NO_MEMORY, "request");
    r->id = id;
    r->w = w;
    r->h = h;
    r->p = *p;
    r->L = imgL;
    r->R = imgR;
    r->dL = dL;
    r->post = post;
    r->key = shape_key(w, h, p);
    r->t_submit = s->now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) {
            delete r;
            return fail(ELAS_ERR_INVALID_ARG, "server is stopping");
        }
        s->queue.push_back(r);
        s->stats.submitted++;
    }
    s->cv_sched.notify_all();
    return ELAS_OK;
}

extern "C" int32_t elas_server_poll(elas_server *s, elas_server_result *out, int32_t max, int32_t timeout_ms) {
    if (!s || !out || max < 1) return -1;
    std::unique_lock<std::mutex> g(s->mu);
    if (s->results.empty() && timeout_ms > 0)
        s->cv_poll.wait_for(g, std::chrono::milliseconds(timeout_ms), [s] { return !s->results.empty(); });
    int32_t k = 0;
    while (k < max && !s->results.empty()) {
        out[k++] = s->results.front();
        s->results.pop_front();
    }
    return k;
}

extern "C" double elas_server_now_ms(const elas_server *s) { return s ? s->now() : 0.0; }

extern "C" elas_status elas_server_stats_get(elas_server *s, elas_server_stats *st) {
    if (!s || !st) return fail(ELAS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    *st = s->stats;
    return ELAS_OK;
}

extern "C" elas_status elas_server_drain(elas_server *s, int32_t timeout_ms) {
    if (!s) return fail(ELAS_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> g(s->mu);
    const bool done = s->cv_poll.wait_for(g, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                          [s] { return s->stats.completed >= s->stats.submitted; });
    if (!done)
        return fail(ELAS_ERR_TIMEOUT, "%lld of %lld requests done after %d ms", (long long)s->stats.completed,
                    (long long)s->stats.submitted, timeout_ms);
    return ELAS_OK;
}

extern "C" elas_status elas_server_inject_alloc_failures(elas_server *s, int32_t n) {
    if (!s || n < 0) return fail(ELAS_ERR_INVALID_ARG, "NULL server or negative count");
    s->fail_allocs.store(n);
    return ELAS_OK;
}

extern "C" void elas_server_destroy(elas_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->th.joinable()) s->th.join();
    release(s);
}
