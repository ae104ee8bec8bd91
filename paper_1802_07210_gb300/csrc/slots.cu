// Slot pool: resident pair state and batched waves (see slots.cuh).
#include <algorithm>
#include <cstring>

#include "slots.cuh"

namespace elas {

namespace {

struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(char *b) : base(b) {}
    template <class T> T *take(size_t bytes) {
        T *r = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += align_up(bytes > 0 ? bytes : 1, 256);
        return r;
    }
};

struct Layout {
    uint8_t *img;
    uint8_t *descL, *descR, *sdescL, *sdescR;
    int16_t *dcan, *list;
    uint32_t *gridL, *gridR;
    int32_t *tri;
    void *ws_support, *ws_dense, *ws_dt, *ws_post;
    int16_t *dL, *dR;
    float *post;
    size_t bytes;
};

Layout layout(char *base, int w, int h, const elas_params *p) {
    const size_t npx = (size_t)w * h;
    const int nc = (w / p->candidate_stepsize) * (h / p->candidate_stepsize);
    const GridGeom g = grid_geom(w, h, p);
    const size_t gbytes = (size_t)g.gw * g.gh * g.nw * sizeof(uint32_t);
    const int tri_cap = 2 * nc + 8;
    Carve c(base);
    Layout l;
    l.img = c.take<uint8_t>(2 * align_up(npx, 256));
    l.descL = c.take<uint8_t>(npx * 16);
    l.descR = c.take<uint8_t>(npx * 16);
    const bool census = p->census_support_w > 0;  // 32-byte support census records
    l.sdescL = census ? c.take<uint8_t>(npx * 32) : nullptr;
    l.sdescR = census ? c.take<uint8_t>(npx * 32) : nullptr;
    l.dcan = c.take<int16_t>((size_t)nc * 2 + 16);
    l.list = c.take<int16_t>((size_t)nc * 6 + 16);
    l.gridL = c.take<uint32_t>(gbytes);
    l.gridR = c.take<uint32_t>(gbytes);
    l.tri = c.take<int32_t>(sizeof(int32_t) * 3 * 2 * (size_t)tri_cap);
    l.ws_support = c.take<void>(support_workspace(w, h, p));
    l.ws_dense = c.take<void>(dense_workspace(w, h, p));
    l.ws_dt = c.take<void>(triangulate_device_workspace(nc, w, h, 2));
    l.ws_post = c.take<void>(post_workspace(w, h));
    l.dL = c.take<int16_t>(npx * 2);
    l.dR = c.take<int16_t>(npx * 2);
    l.post = c.take<float>(npx * 4);
    l.bytes = c.off;
    return l;
}

}  // namespace

SlotPool::~SlotPool() {
    if (upload_in_flight_ && mirror_free_) cudaEventSynchronize(mirror_free_);
    for (Slot &s : slots_)
        if (s.mem) cudaFree(s.mem);
    if (dev_tab_) cudaFree(dev_tab_);
    if (dev_counters_) cudaFree(dev_counters_);
    if (host_tab_) cudaFreeHost(host_tab_);
    if (h_counters_) cudaFreeHost(h_counters_);
    if (mirror_free_) cudaEventDestroy(mirror_free_);
    if (mem_pool_) cudaMemPoolDestroy(mem_pool_);
}

elas_status SlotPool::use_own_pool(size_t keep_bytes) {
    if (mem_pool_) return ELAS_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return launch_status("current device");
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&mem_pool_, &props) != cudaSuccess) {
        mem_pool_ = nullptr;
        return launch_status("slot memory pool");
    }
    uint64_t keep = keep_bytes;
    if (cudaMemPoolSetAttribute(mem_pool_, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
        return launch_status("slot memory pool threshold");
    return ELAS_OK;
}

elas_status SlotPool::init(int max_slots) {
    if (max_slots < 1 || max_slots > 4096) return fail(ELAS_ERR_INVALID_ARG, "slot capacity %d", max_slots);
    slots_.assign(max_slots, Slot());
    const size_t tb = sizeof(SlotTables) * (size_t)max_slots;
    if (cudaMalloc(reinterpret_cast<void **>(&dev_tab_), tb) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&dev_counters_), sizeof(int32_t) * 4 * (size_t)max_slots) !=
            cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&host_tab_), tb) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&h_counters_), sizeof(int32_t) * 4 * (size_t)max_slots) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&mirror_free_, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(ELAS_ERR_NO_MEMORY, "slot pool of %d slots", max_slots);
    }
    std::memset(host_tab_, 0, tb);
    std::memset(h_counters_, 0, sizeof(int32_t) * 4 * (size_t)max_slots);
    return ELAS_OK;
}

size_t SlotPool::slot_bytes(int w, int h, const elas_params *p) { return layout(nullptr, w, h, p).bytes; }

elas_status SlotPool::wait_mirror() {
    if (upload_in_flight_) {
        if (cudaEventSynchronize(mirror_free_) != cudaSuccess) return launch_status("slot table upload");
        upload_in_flight_ = false;
    }
    return ELAS_OK;
}

elas_status SlotPool::add(int w, int h, const elas_params *p, int *id, cudaStream_t alloc_stream) {
    elas_status s = check_params(p, w, h);
    if (s != ELAS_OK) return s;
    if (w < p->candidate_stepsize || h < p->candidate_stepsize)
        return fail(ELAS_ERR_INVALID_ARG, "%dx%d has no lattice candidate at step %d", w, h, p->candidate_stepsize);
    int k = -1;
    for (int i = 0; i < (int)slots_.size(); ++i)
        if (!slots_[i].used) {
            k = i;
            break;
        }
    if (k < 0) return fail(ELAS_ERR_CAPACITY, "all %d slots in use", (int)slots_.size());
    if ((s = wait_mirror()) != ELAS_OK) return s;
    Slot &sl = slots_[k];
    const uint32_t gen = sl.generation + 1;
    sl = Slot();
    sl.generation = gen;
    sl.w = w;
    sl.h = h;
    sl.p = *p;
    sl.nc = (w / p->candidate_stepsize) * (h / p->candidate_stepsize);
    sl.tri_cap = 2 * sl.nc + 8;
    const Layout need = layout(nullptr, w, h, p);
    sl.async_mem = alloc_stream != nullptr;
    const cudaError_t ae =
        !alloc_stream ? cudaMalloc(reinterpret_cast<void **>(&sl.mem), need.bytes)
        : mem_pool_   ? cudaMallocFromPoolAsync(reinterpret_cast<void **>(&sl.mem), need.bytes, mem_pool_, alloc_stream)
                      : cudaMallocAsync(reinterpret_cast<void **>(&sl.mem), need.bytes, alloc_stream);
    if (ae != cudaSuccess) {
        cudaGetLastError();
        sl.mem = nullptr;
        return fail(ELAS_ERR_NO_MEMORY, "slot of %zu bytes for %dx%d", need.bytes, w, h);
    }
    const Layout l = layout(sl.mem, w, h, p);
    sl.bytes = l.bytes;
    sl.img = l.img;
    sl.descL = l.descL;
    sl.descR = l.descR;
    sl.sdescL = l.sdescL;
    sl.sdescR = l.sdescR;
    sl.dcan = l.dcan;
    sl.list = l.list;
    sl.gridL = l.gridL;
    sl.gridR = l.gridR;
    sl.tri = l.tri;
    sl.ws_support = l.ws_support;
    sl.ws_dense = l.ws_dense;
    sl.ws_dt = l.ws_dt;
    sl.ws_post = l.ws_post;
    sl.dL = l.dL;
    sl.dR = l.dR;
    sl.post = l.post;
    sl.counters = dev_counters_ + 4 * k;
    sl.used = true;
    bytes_in_use_ += sl.bytes;
    sl.io_imgL = sl.img;
    sl.io_imgR = sl.img + align_up((size_t)w * h, 256);
    sl.io_pitch = w;
    sl.io_dL = sl.dL;
    sl.io_dR = sl.dR;
    sl.io_post = nullptr;
    sl.post_on = false;
    if ((s = write_records(k)) != ELAS_OK) {
        remove(k);
        return s;
    }
    *id = k;
    return ELAS_OK;
}

void SlotPool::remove(int id, cudaStream_t free_stream) {
    if (id < 0 || id >= (int)slots_.size() || !slots_[id].used) return;
    Slot &sl = slots_[id];
    // the caller guarantees that no launch on this slot is still running
    if (sl.async_mem && free_stream)
        cudaFreeAsync(sl.mem, free_stream);
    else
        cudaFree(sl.mem);
    bytes_in_use_ -= sl.bytes;
    const uint32_t gen = sl.generation;
    sl = Slot();
    sl.generation = gen;
}

elas_status SlotPool::write_records(int id) {
    Slot &sl = slots_[id];
    SlotTables &t = host_tab_[id];
    std::memset(&t, 0, sizeof(t));
    const int w = sl.w, h = sl.h;
    const elas_params *p = &sl.p;
    t.desc = DescArgs{sl.io_imgL, sl.io_imgR, w, h, sl.io_pitch, reinterpret_cast<uint4 *>(sl.descL),
                      reinterpret_cast<uint4 *>(sl.descR)};
    const bool census = p->census_support_w > 0;
    if (census) {
        t.cs = CensusArgs{sl.io_imgL, sl.io_imgR, w, h, sl.io_pitch, reinterpret_cast<uint4 *>(sl.sdescL),
                          reinterpret_cast<uint4 *>(sl.sdescR), p->census_support_w};
        t.cd = CensusArgs{sl.io_imgL, sl.io_imgR, w, h, sl.io_pitch, reinterpret_cast<uint4 *>(sl.descL),
                          reinterpret_cast<uint4 *>(sl.descR), p->census_dense_w};
    }
    elas_status s0 = support_args(census ? sl.sdescL : sl.descL, census ? sl.sdescR : sl.descR, w, h, p, sl.dcan,
                                  sl.list, sl.counters, sl.gridL, sl.gridR, sl.ws_support, &t.sup);
    if (s0 != ELAS_OK) return s0;
    int32_t *tris[2] = {sl.tri, sl.tri + 3 * (size_t)sl.tri_cap};
    int32_t *nts[2] = {sl.counters + 1, sl.counters + 2};
    t.dt = triangulate_args(sl.list, sl.counters, sl.nc, w, h, tris, nts, sl.tri_cap, sl.ws_dt);
    elas_status s = dense_args(sl.descL, sl.descR, w, h, p, sl.list, tris[0], sl.tri_cap, tris[1], sl.tri_cap,
                               sl.gridL, sl.gridR, sl.io_dL, sl.io_dR, sl.ws_dense, sl.counters + 1, &t.dense, false);
    if (s != ELAS_OK) return s;
    t.lr = LrArgs{sl.io_dL, sl.io_dR, w, h, p->lr_threshold, nullptr, nullptr};
    sl.fused = sl.post_on && post_fusable(p) ? 1 : 0;
    sl.npass = sl.post_on && !sl.fused ? post_passes(sl.io_dL, w, h, p, sl.io_post, sl.ws_post, t.post) : 0;
    if (sl.fused) t.fpost = fused_post_args(sl.io_dL, w, h, p, sl.io_post);
    dirty_lo_ = std::min(dirty_lo_, id);
    dirty_hi_ = std::max(dirty_hi_, id);
    return ELAS_OK;
}

elas_status SlotPool::set_io(int id, const uint8_t *imgL, const uint8_t *imgR, int pitch, int16_t *dL, int16_t *dR,
                             bool post_on, float *post) {
    if (id < 0 || id >= (int)slots_.size() || !slots_[id].used) return fail(ELAS_ERR_INVALID_ARG, "slot %d", id);
    Slot &sl = slots_[id];
    const uint8_t *iL = imgL ? imgL : sl.img;
    const uint8_t *iR = imgL ? imgR : sl.img + align_up((size_t)sl.w * sl.h, 256);
    const int pt = imgL ? pitch : sl.w;
    if (!iR) return fail(ELAS_ERR_INVALID_ARG, "slot %d: right image is NULL", id);
    if (pt < sl.w) return fail(ELAS_ERR_INVALID_ARG, "slot %d: pitch %d < width %d", id, pt, sl.w);
    int16_t *oL = dL ? dL : sl.dL;
    int16_t *oR = dR ? dR : sl.dR;
    float *po = post_on ? (post ? post : sl.post) : nullptr;
    if (iL == sl.io_imgL && iR == sl.io_imgR && pt == sl.io_pitch && oL == sl.io_dL && oR == sl.io_dR &&
        post_on == sl.post_on && po == sl.io_post)
        return ELAS_OK;
    elas_status s = wait_mirror();
    if (s != ELAS_OK) return s;
    sl.io_imgL = iL;
    sl.io_imgR = iR;
    sl.io_pitch = pt;
    sl.io_dL = oL;
    sl.io_dR = oR;
    sl.io_post = po;
    sl.post_on = post_on;
    return write_records(id);
}

elas_status SlotPool::upload(cudaStream_t st) {
    if (dirty_hi_ < dirty_lo_) return ELAS_OK;
    const size_t off = sizeof(SlotTables) * (size_t)dirty_lo_;
    const size_t bytes = sizeof(SlotTables) * (size_t)(dirty_hi_ - dirty_lo_ + 1);
    if (cudaMemcpyAsync(reinterpret_cast<char *>(dev_tab_) + off, reinterpret_cast<char *>(host_tab_) + off, bytes,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaEventRecord(mirror_free_, st) != cudaSuccess)
        return launch_status("slot table upload");
    upload_in_flight_ = true;
    dirty_lo_ = 1 << 30;
    dirty_hi_ = -1;
    return ELAS_OK;
}

elas_status SlotPool::launch(const int *ids, int n, const Knobs &k, cudaStream_t st, int32_t *counter,
                             const StageMarks *marks) {
    if (n < 1) return ELAS_OK;
    if (n > kMaxBatch) return fail(ELAS_ERR_CAPACITY, "%d pairs in one wave (at most %d)", n, kMaxBatch);
    if (dirty_hi_ >= dirty_lo_) return fail(ELAS_ERR_INTERNAL, "slot records changed without an upload");
    if (!counter) counter = dev_counters_ + 4 * ids[0] + 3;
    VMap pairs, sobel, census;
    vmap_clear(pairs, (int)sizeof(SlotTables));
    vmap_clear(sobel, (int)sizeof(SlotTables));
    vmap_clear(census, (int)sizeof(SlotTables));
    int npass[kMaxBatch], fused[kMaxBatch];
    for (int i = 0; i < n; ++i) {
        const int id = ids[i];
        if (id < 0 || id >= (int)slots_.size() || !slots_[id].used) return fail(ELAS_ERR_INVALID_ARG, "slot %d", id);
        vmap_add(pairs, id, dim3(0));
        vmap_add(slots_[id].p.census_support_w > 0 ? census : sobel, id, dim3(0));
        npass[i] = slots_[id].npass;
        fused[i] = slots_[id].fused;
    }
    auto mark = [&](int i) {
        if (marks && marks->ev[i]) record_mark(marks->ev[i], st);
    };
    const SlotTables *D = dev_tab_;
    const SlotTables *H = host_tab_;
    elas_status s;
    mark(0);
    if (sobel.n > 0 && (s = launch_descriptors_b(&D->desc, &H->desc, sobel, k.desc_rows, st)) != ELAS_OK) return s;
    if (census.n > 0 && ((s = launch_census_b(&D->cs, &H->cs, census, 32, st)) != ELAS_OK ||
                         (s = launch_census_b(&D->cd, &H->cd, census, 16, st)) != ELAS_OK))
        return s;
    mark(1);
    const SupportTables sup{&D->sup.match, &D->sup.cons, &D->sup.red, &D->sup.compact, &D->sup.lg};
    if ((s = launch_support_b(sup, &H->sup, pairs, k.support_warps, st)) != ELAS_OK) return s;
    mark(2);
    if ((s = launch_triangulate_b(&D->dt, &H->dt, pairs, 2, counter, st)) != ELAS_OK) return s;
    mark(3);
    const DenseTables dn{&D->dense.raster, &D->dense.cell};
    if ((s = launch_dense_b(dn, &H->dense, pairs, k.dense_tpp, k.dense_ppt, st, marks ? marks->ev[4] : nullptr,
                            k.dense_fused != 0)) != ELAS_OK)
        return s;
    mark(5);
    const PostArgs *post_tabs[4] = {&D->post[0], &D->post[1], &D->post[2], &D->post[3]};
    if ((s = launch_lr_post_b(&D->lr, &H->lr, post_tabs, npass, &D->fpost, fused, pairs, st)) != ELAS_OK) return s;
    mark(6);
    return ELAS_OK;
}

elas_status SlotPool::fetch_counters(cudaStream_t st, int32_t *dst) {
    if (cudaMemcpyAsync(dst ? dst : h_counters_, dev_counters_, sizeof(int32_t) * 4 * slots_.size(),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return launch_status("counters to host");
    return ELAS_OK;
}

}  // namespace elas
