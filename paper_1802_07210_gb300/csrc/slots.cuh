// Resident pair state ("slots") and waves of batched launches over them.
//
// A slot holds everything one stereo pair needs on the device: its
// descriptors, candidate grids, support list, triangles, prior maps and
// workspaces, internal input/output buffers, and one record of stage
// arguments in the pool's table.  A wave runs the whole path for any set of
// slots with one launch per kernel (batch.cuh): pairs of different sizes and
// disparity ranges share every launch.  The batch handle is a fixed set of
// slots; the server creates and retires slots as requests come and go.
#pragma once

#include <vector>

#include "launch.cuh"

namespace elas {

// Tile shapes of the batched kernels (picked by the tuner).
struct Knobs {
    int desc_rows = 24;     // image rows a descriptor warp walks: 12, 24, 36
    int support_warps = 8;  // lattice candidates (warps) per support CTA: 4, 8, 16
    int dense_tpp = 1;      // threads per pixel in the dense argmin: 1, 2, 4
    int dense_ppt = 4;      // pixels per thread (per pixel group) in the dense argmin: 1, 2, 4, 8
    int dense_fused = 0;    // 1: prior and argmin in one persistent cooperative launch
};

// The stage arguments of one slot, one record per slot in the tables.
struct SlotTables {
    DescArgs desc;
    CensusArgs cs, cd;  // the paper's variant: support and dense census records
    SupportStage sup;
    DtArgs dt;
    DenseStage dense;
    LrArgs lr;
    PostArgs post[4];      // post-processing as separate passes (wide gaps)
    FusedPostArgs fpost;   // or as one fused launch
};

struct Slot {
    bool used = false;
    int w = 0, h = 0, nc = 0, tri_cap = 0, npass = 0;
    int fused = 0;  // post-processing by the fused kernel (npass = 0 then)
    elas_params p{};
    char *mem = nullptr;  // one device allocation holding every buffer below
    size_t bytes = 0;
    uint8_t *img = nullptr;  // internal inputs: left then right plane
    uint8_t *descL = nullptr, *descR = nullptr;  // descriptors, or the dense census records
    uint8_t *sdescL = nullptr, *sdescR = nullptr;  // support census records (census slots only)
    int16_t *dcan = nullptr, *list = nullptr;
    uint32_t *gridL = nullptr, *gridR = nullptr;
    int32_t *tri = nullptr;
    void *ws_support = nullptr, *ws_dense = nullptr, *ws_dt = nullptr, *ws_post = nullptr;
    int16_t *dL = nullptr, *dR = nullptr;  // internal outputs
    float *post = nullptr;
    int32_t *counters = nullptr;  // [support count, triangles left, triangles right, spare]
    // inputs and outputs the slot's records point at
    const uint8_t *io_imgL = nullptr, *io_imgR = nullptr;
    int io_pitch = 0;
    int16_t *io_dL = nullptr, *io_dR = nullptr;
    float *io_post = nullptr;
    bool post_on = false;
    bool async_mem = false;  // memory from the stream-ordered allocator
    uint32_t generation = 0;  // changes whenever the slot's buffers do
};

// Event marks of a wave (tuner, profiling); NULL entries are skipped.  The
// intervals are: descriptors, support points, triangulation, plane prior,
// dense argmin, LR check + post-processing.
constexpr int kStageMarks = 7;
struct StageMarks {
    cudaEvent_t ev[kStageMarks] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

class SlotPool {
  public:
    SlotPool() = default;
    SlotPool(const SlotPool &) = delete;
    SlotPool &operator=(const SlotPool &) = delete;
    ~SlotPool();

    elas_status init(int max_slots);
    // Stream-ordered slot memory from a pool of this pool's own that keeps
    // up to keep_bytes of freed memory mapped (no remapping when slots of
    // other shapes come and go); without it the device's default pool.
    elas_status use_own_pool(size_t keep_bytes);
    // Device bytes a slot of this shape takes.
    static size_t slot_bytes(int w, int h, const elas_params *p);
    // alloc_stream != NULL: the slot's memory comes from the stream-ordered
    // allocator on that stream (no device-wide synchronisation), and remove
    // returns it on free_stream the same way.
    elas_status add(int w, int h, const elas_params *p, int *id, cudaStream_t alloc_stream = nullptr);
    void remove(int id, cudaStream_t free_stream = nullptr);
    // Points the slot's records at these inputs and outputs; NULL images or
    // dL select the internal buffers, NULL dR the internal right map;
    // post_on with a NULL post selects the internal float map.
    elas_status set_io(int id, const uint8_t *imgL, const uint8_t *imgR, int pitch, int16_t *dL, int16_t *dR,
                       bool post_on, float *post);
    // Copies changed records to the device, on `st`.
    elas_status upload(cudaStream_t st);
    // The whole path for the slots ids[0..n-1]; counter = one device int for
    // the triangulation's queue, or NULL for the first slot's spare counter
    // (a slot is in one wave at a time, so waves on different streams and
    // graphs captured from them never share it).
    elas_status launch(const int *ids, int n, const Knobs &k, cudaStream_t st, int32_t *counter,
                       const StageMarks *marks = nullptr);
    // Counters of every slot to pinned host memory (after launch, same
    // stream): to the pool's array, or to dst (capacity() * 4 ints, pinned).
    elas_status fetch_counters(cudaStream_t st, int32_t *dst = nullptr);
    const int32_t *host_counters(int id) const { return h_counters_ + 4 * id; }

    Slot &operator[](int id) { return slots_[id]; }
    const Slot &operator[](int id) const { return slots_[id]; }
    int capacity() const { return (int)slots_.size(); }
    size_t bytes_in_use() const { return bytes_in_use_; }

  private:
    elas_status write_records(int id);
    elas_status wait_mirror();

    std::vector<Slot> slots_;
    SlotTables *dev_tab_ = nullptr;
    SlotTables *host_tab_ = nullptr;  // pinned mirror of the device table
    int32_t *dev_counters_ = nullptr;
    int32_t *h_counters_ = nullptr;   // pinned
    int dirty_lo_ = 1 << 30, dirty_hi_ = -1;
    cudaEvent_t mirror_free_ = nullptr;  // recorded after each upload
    bool upload_in_flight_ = false;
    size_t bytes_in_use_ = 0;
    cudaMemPool_t mem_pool_ = nullptr;
};

}  // namespace elas
