// runtime.cu -- host runtime behind the C ABI (include/vol.h).
//
// Owns one volume: the brick atlas (a cache of fixed-size slots, Sec. III-C's VRAM store
// specialised to equally sized bricks), one page table per LOD level laid end to end
// (Sec. III-E), host mirrors of the page tables and of slot ownership, the least-recently-
// used eviction policy driven by per-slot usage stamps written by the render kernel
// (Sec. III-C/III-E: garbage collection frees down to a 10% target), the brick-request loop
// (Sec. III-H), and the buffers of the last render needed by the adjoint.
#include <sched.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

using namespace volrc;

namespace {

thread_local std::string g_create_error;

// Cores this process may run on (its affinity mask), at least 1.
int host_cores() {
    cpu_set_t set;
    if (sched_getaffinity(0, sizeof(set), &set) == 0) return std::max(1, CPU_COUNT(&set));
    return (int)std::max(1u, std::thread::hardware_concurrency());
}

int64_t now_us() {
    return std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

int bpv_of(int dtype) {
    switch (dtype) {
    case VOL_U8: return 1;
    case VOL_U16: return 2;
    case VOL_F16: return 2;
    case VOL_F32: return 4;
    }
    return 0;
}

bool conversion_ok(int src, int dst) {
    if (src == dst) return true;
    return (src == VOL_U16 && dst == VOL_F16) || (src == VOL_U8 && dst == VOL_F32) || (src == VOL_U16 && dst == VOL_F32);
}

int plan(const int64_t dims[3], int dtype, int brick, int levels, uint64_t cache_bytes, uint32_t flags, vol_layout* o,
         std::string& err) {
    if (!dims || !o) { err = "null argument"; return VOL_ERR_INVALID_ARG; }
    memset(o, 0, sizeof(*o));
    const int bpv = bpv_of(dtype);
    if (!bpv) { err = "unknown dtype"; return VOL_ERR_INVALID_ARG; }
    if (brick < 4 || brick > 128 || (brick & (brick - 1))) { err = "brick must be a power of two in 4..128"; return VOL_ERR_INVALID_ARG; }
    if (levels < 1 || levels > VOL_MAX_LEVELS) { err = "levels must be 1..16"; return VOL_ERR_INVALID_ARG; }
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (1 << 24)) { err = "dims must be 1..2^24"; return VOL_ERR_INVALID_ARG; }
    o->dtype = dtype;
    o->brick = brick;
    o->levels = levels;
    o->bytes_per_voxel = bpv;
    if (flags & ~(VOL_LAYOUT_COMPACT | VOL_LAYOUT_SPARSE_PT)) { err = "unknown flags"; return VOL_ERR_INVALID_ARG; }
    o->layout = (flags & VOL_LAYOUT_COMPACT) ? 1 : 0;
    const bool sparse = (flags & VOL_LAYOUT_SPARSE_PT) != 0;
    o->sparse_pt = sparse ? 1 : 0;
    o->entry_voxels = o->layout ? 1 : 4;
    int64_t off = 0;
    for (int l = 0; l < levels; ++l) {
        for (int a = 0; a < 3; ++a) {
            o->dims[a] = dims[a];
            o->level_dims[l][a] = l == 0 ? dims[a] : (o->level_dims[l - 1][a] + 1) / 2;
            o->level_bricks[l][a] = (o->level_dims[l][a] + brick - 1) / brick;
        }
        if (!sparse) o->level_pt_offset[l] = off;
        off += o->level_bricks[l][0] * o->level_bricks[l][1] * o->level_bricks[l][2];
    }
    o->total_bricks = off;
    if (sparse) {
        // top grids, one entry per 256^3 bricks, laid end to end
        const int64_t span = int64_t(1) << (2 * kPageShift);
        int64_t top = 0;
        for (int l = 0; l < levels; ++l) {
            int64_t n = 1;
            for (int a = 0; a < 3; ++a) {
                if (o->level_bricks[l][a] > (int64_t(1) << 20)) {
                    err = "sparse page table: at most 2^20 bricks per axis";
                    return VOL_ERR_UNSUPPORTED;
                }
                n *= (o->level_bricks[l][a] + span - 1) / span;
            }
            o->level_pt_offset[l] = top;
            top += n;
        }
        if (top >= (int64_t(1) << 30)) { err = "sparse page table: top grids too large"; return VOL_ERR_UNSUPPORTED; }
        o->pt_top_entries = top;
        if (cache_bytes == 0) { err = "a sparse page table needs cache_bytes > 0"; return VOL_ERR_INVALID_ARG; }
    } else if (off >= (int64_t)0xFFFFFFF0ll) {
        err = "too many bricks for 32-bit page-table indices (VOL_LAYOUT_SPARSE_PT takes more)";
        return VOL_ERR_UNSUPPORTED;
    }
    const int64_t B1 = brick + 1;
    const int64_t slot_voxels = o->layout ? B1 * B1 * B1 : 4 * (int64_t)brick * brick * B1;
    o->slot_bytes = ((slot_voxels * bpv + 255) / 256) * 256;
    int64_t ns = cache_bytes == 0 ? off : (int64_t)(cache_bytes / (uint64_t)o->slot_bytes);
    if (ns > off) ns = off;
    if (ns < 1) { err = "cache smaller than one brick"; return VOL_ERR_INVALID_ARG; }
    if (ns >= (int64_t)0xFFFFFFF0ll) { err = "too many slots"; return VOL_ERR_UNSUPPORTED; }
    o->nslots = ns;
    o->atlas_bytes = ns * o->slot_bytes;
    return VOL_OK;
}

}  // namespace

struct vol_s {
    int device = 0;
    int nsm = 1;
    cudaStream_t stream = nullptr;
    vol_layout lay{};
    int dtype = 0, B = 0, bshift = 0, L = 1;
    std::string err;

    void* atlas = nullptr;
    uint32_t* pt = nullptr;
    unsigned* last_used = nullptr;
    unsigned* counters = nullptr;     // kNumCounters words
    unsigned* aux = nullptr;          // [0] downsample error word

    std::vector<uint32_t> pt_host;    // page tables (mirror)
    std::vector<uint32_t> owner;      // slot -> page-table index or invalid
    std::vector<uint32_t> protect;    // slot -> operation epoch that must not evict it
    std::vector<uint8_t> reserved;    // slot -> 1 while a brick is being generated into it
    // sparse page table: bricks get handles (the index the flat table would use) on first use;
    // `pt` is then the pool (top grids, then 16^3-entry pages) and pool_host its mirror
    bool sparse = false;
    std::unordered_map<uint64_t, uint32_t> handle_of;  // (level, brick) key -> handle
    std::vector<uint64_t> key_of;                      // handle -> key
    std::vector<uint32_t> pool_host;
    size_t pool_used = 0, pool_cap = 0;                // entries in use / allocated on the device
    unsigned long long* req_table64 = nullptr;
    unsigned long long* req_list64 = nullptr;
    std::vector<uint8_t> queued;      // page-table index -> 1 while waiting for or in generation
    std::vector<uint32_t> free_slots; // stack
    uint32_t op_epoch = 1;
    int64_t resident = 0;
    std::vector<int64_t> level_resident;

    // pending page-table updates
    std::vector<uint32_t> upd_idx, upd_val;
    uint32_t* upd_dev = nullptr;
    size_t upd_cap = 0;

    // render state
    ViewDev* views_dev = nullptr;
    int views_cap = 0;
    std::vector<ViewDev> views_host;
    // the view table the device copy holds, and the page-locked staging buffer it was copied from
    // (reused once the event says the last copy out of it is done)
    std::vector<ViewDev> views_sent;
    ViewDev* views_pinned = nullptr;
    int views_pinned_cap = 0;
    cudaEvent_t ev_views = nullptr;
    int nviews = 0;
    int ntiles = 0;
    int64_t nrays = 0;
    vol_params params{};
    const float* tf = nullptr;
    float* out = nullptr;
    int32_t* nsamp = nullptr;
    bool grad = false;
    bool have_forward = false;
    uint32_t frame = 0;

    // misses
    unsigned* req_table = nullptr;
    uint32_t req_cap = 0;
    unsigned* req_list = nullptr;
    uint32_t req_list_cap = 0;
    SuspRec* susp[2] = {nullptr, nullptr};
    int64_t susp_cap = 0;
    int susp_cur = 0;          // buffer holding the rays still suspended
    int64_t nsusp = 0;         // rays still suspended
    std::vector<uint32_t> last_requests;

    // gradient state
    float* ckpt = nullptr;
    size_t ckpt_cap = 0;
    int ckpt_shift = kCkptShift;  // checkpoints every 2^ckpt_shift samples (0: VOL_RENDER_CKPT_ALL)
    float* tape = nullptr;        // sample values of the last gradient render (RenderDev::tape layout)
    size_t tape_cap = 0;
    bool taped = false;           // the last gradient render wrote the tape
    int* ray_n = nullptr;
    size_t ray_n_cap = 0;
    float* dlev_buf = nullptr;  // adjoint with LOD: gradients of levels 1..L-1
    size_t dlev_cap = 0;

    // provider
    vol_provider_fn prov = nullptr;
    vol_provider_batch_fn prov_batch = nullptr;
    void* prov_user = nullptr;
    int prov_dtype = 0;
    void* stage_host = nullptr;
    void* stage_dev = nullptr;
    uint32_t* stage_slots_dev = nullptr;
    int stage_bricks = 0;
    // overlapped loading: a pinned host ring the batch provider fills and the upload kernels
    // read directly, a stream for reading the request list while a pass runs, and one worker
    // thread that runs the provider
    struct Ring {
        char* host = nullptr;        // cap bricks of `brick_bytes` (source type), pinned, mapped
        uint32_t* slots = nullptr;   // cap: slot of each ring entry (pinned, mapped)
        uint32_t* ptis = nullptr;    // cap: page-table index of each ring entry (pinned, mapped)
        char* host_dev = nullptr;    // device-side addresses of the three arrays
        uint32_t* slots_dev = nullptr;
        uint32_t* ptis_dev = nullptr;
        int cap = 0;
        size_t brick_bytes = 0;
        int head = 0, used = 0;      // next free entry; entries in use (gaps at the wrap included)
        struct Region {
            int start, n, gap;
            cudaEvent_t ev;          // recorded after the region's upload kernels
        };
        std::deque<Region> inflight;
        std::vector<cudaEvent_t> spare;
    } ring;
    struct LoadJob {
        int start = 0, nalloc = 0, gap = 0, n = 0;  // ring region, bricks in it
        std::vector<int32_t> coords;                 // [n][4] level, bx, by, bz
    };
    struct Ovl {
        std::deque<uint32_t> pending;  // requested bricks (page-table indices) not yet in generation
        LoadJob job;
        bool running = false;          // job is in the loader thread
    } ovl;
    cudaStream_t poll_stream = nullptr;
    uint32_t* poll_host = nullptr;   // pinned: request count, then request keys
    cudaEvent_t ev_pass_start = nullptr, ev_pass_end = nullptr;  // around each pass's launch
    struct Loader {
        std::thread th;
        std::mutex m;
        std::condition_variable cv;
        bool quit = false, job = false, done = true;
        int n = 0, rc = 0;
        const int32_t* coords = nullptr;
        void* dst = nullptr;
    } loader;

    // longest-ray-first scheduling from the previous frame's per-tile longest ray
    int* tile_cost = nullptr;
    size_t tile_cost_cap = 0;
    int* tile_order = nullptr;
    size_t tile_order_cap = 0;
    std::vector<unsigned char> order_key;  // tile partition the order was built for
    bool order_ready = false;
    int* order_buckets = nullptr;          // 64 ints: bucket counts and fill cursors
    float2* range = nullptr;               // per slot: min and max stored value
    uint16_t* cells = nullptr;             // per slot: TF-entry span of each macro-cell
    int cbits = 0, cshift = 0;             // log2 cells per brick axis, log2 cell edge

    vol_stats stats{};
    int64_t allocations = 0;  // device and pinned-host allocations since vol_create
    bool counters_collected = true;  // the counter words hold a pass collect_pass already read
    unsigned* last_counters = nullptr;  // the counter words of the last pass (NULL: counters)
    int occ_cache[4][2] = {{0}};
    ViewDev noalloc_views[VOL_NOALLOC_MAX_VIEWS];  // vol_render_noalloc's host staging of its view table
};

namespace {

// Every device and pinned-host allocation of a volume goes through these two, which count it
// (vol_stats.allocations).
cudaError_t dev_alloc(vol_t v, void** p, size_t bytes) {
    ++v->allocations;
    return cudaMalloc(p, bytes);
}
cudaError_t host_alloc(vol_t v, void** p, size_t bytes, unsigned flags) {
    ++v->allocations;
    return cudaHostAlloc(p, bytes, flags);
}

int fail(vol_t v, int code, const std::string& msg) {
    if (v) v->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(vol_t v, cudaError_t e, const char* what) {
    return fail(v, e == cudaErrorMemoryAllocation ? VOL_ERR_OOM : VOL_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(v, call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail((v), e_, #call);      \
    } while (0)

VolDev vol_dev(const vol_t v) {
    VolDev d{};
    d.atlas = v->atlas;
    d.slot_elems = (unsigned long long)(v->lay.slot_bytes / v->lay.bytes_per_voxel);
    d.quad = v->lay.layout == 0 ? 1 : 0;
    d.slot_entries = d.slot_elems / 4;
    d.bshift = v->bshift;
    d.bmask = v->B - 1;
    d.B1 = v->B + 1;
    d.nlevels = v->L;
    d.pt = v->pt;
    d.range = v->range;
    d.cells = v->cells;
    d.cbits = v->cbits;
    d.cshift = v->cshift;
    for (int l = 0; l < v->L; ++l) {
        for (int a = 0; a < 3; ++a) {
            d.lv[l].D[a] = (int)v->lay.level_dims[l][a];
            d.lv[l].nb[a] = (int)v->lay.level_bricks[l][a];
            d.lv[l].r[a] = (float)v->lay.level_dims[l][a] / (float)v->lay.level_dims[0][a];
            d.lv[l].ir[a] = (float)((double)v->lay.level_dims[0][a] / (double)v->lay.level_dims[l][a]);
        }
        d.lv[l].pt_off = (uint32_t)v->lay.level_pt_offset[l];
        for (int a = 0; a < 3; ++a) {
            const int64_t span = int64_t(1) << (2 * kPageShift);
            d.lv[l].tn[a] = (int)((v->lay.level_bricks[l][a] + span - 1) / span);
        }
    }
    for (int a = 0; a < 3; ++a) d.D0f[a] = (float)v->lay.dims[a];
    d.sparse = v->sparse ? 1 : 0;
    return d;
}

// ---- sparse page table: brick keys and handles, pages ------------------------------------

uint64_t brick_key(int l, int64_t bx, int64_t by, int64_t bz) {
    return ((uint64_t)l << 60) | ((uint64_t)bz << 40) | ((uint64_t)by << 20) | (uint64_t)bx;
}

// Handle of brick key `key`, assigned on first use.
uint32_t handle_for(vol_t v, uint64_t key) {
    auto it = v->handle_of.find(key);
    if (it != v->handle_of.end()) return it->second;
    const uint32_t h = (uint32_t)v->key_of.size();
    v->handle_of.emplace(key, h);
    v->key_of.push_back(key);
    v->pt_host.push_back(kInvalidSlot);
    v->queued.push_back(0);
    return h;
}

// A zeroed (all kInvalidSlot) page of the pool, growing the device pool when it is full.  Only
// between passes: growing synchronises the stream.
int pool_page(vol_t v, uint32_t* base) {
    if (v->pool_used + kPageEntries > v->pool_cap) {
        const size_t cap = std::max(v->pool_cap * 2, v->pool_used + kPageEntries);
        if (cap >= (size_t(1) << 32) - 16) return fail(v, VOL_ERR_OOM, "sparse page table: pool full");
        uint32_t* np = nullptr;
        CK(v, cudaStreamSynchronize(v->stream));
        CK(v, dev_alloc(v, (void**)&np, sizeof(uint32_t) * cap));
        CK(v, cudaMemcpyAsync(np, v->pt, sizeof(uint32_t) * v->pool_used, cudaMemcpyDeviceToDevice, v->stream));
        CK(v, cudaMemsetAsync(np + v->pool_used, 0xFF, sizeof(uint32_t) * (cap - v->pool_used), v->stream));
        CK(v, cudaStreamSynchronize(v->stream));
        cudaFree(v->pt);
        v->pt = np;
        v->pool_cap = cap;
        v->pool_host.resize(cap, kInvalidSlot);
    }
    *base = (uint32_t)v->pool_used;
    v->pool_used += kPageEntries;
    return VOL_OK;
}

// Pool index of the leaf entry of brick handle h; with create, allocates the missing middle
// and leaf pages (their parent entries are queued as page-table updates).  kInvalidSlot when
// absent and not created.
int sparse_leaf(vol_t v, uint32_t h, bool create, uint32_t* out) {
    const uint64_t key = v->key_of[h];
    const int l = (int)(key >> 60);
    const int64_t b[3] = {(int64_t)(key & 0xFFFFF), (int64_t)((key >> 20) & 0xFFFFF), (int64_t)((key >> 40) & 0xFFFFF)};
    const int64_t span = int64_t(1) << (2 * kPageShift), pm = (int64_t(1) << kPageShift) - 1;
    int64_t tn[3];
    for (int a = 0; a < 3; ++a) tn[a] = (v->lay.level_bricks[l][a] + span - 1) / span;
    const size_t top = (size_t)(v->lay.level_pt_offset[l] + ((b[2] / span) * tn[1] + b[1] / span) * tn[0] + b[0] / span);
    auto local = [&](int shift) {
        return (uint32_t)((((b[2] >> shift) & pm) << (2 * kPageShift)) | (((b[1] >> shift) & pm) << kPageShift) |
                          ((b[0] >> shift) & pm));
    };
    *out = kInvalidSlot;
    size_t at = top;
    for (int shift : {kPageShift, 0}) {
        uint32_t child = v->pool_host[at];
        if (child == kInvalidSlot) {
            if (!create) return VOL_OK;
            if (int rc = pool_page(v, &child)) return rc;
            v->pool_host[at] = child;
            v->upd_idx.push_back((uint32_t)at);
            v->upd_val.push_back(child);
        }
        at = (size_t)child + local(shift);
    }
    *out = (uint32_t)at;
    return VOL_OK;
}

int64_t level_nbricks(const vol_t v, int l) {
    return v->lay.level_bricks[l][0] * v->lay.level_bricks[l][1] * v->lay.level_bricks[l][2];
}

int level_of_pti(const vol_t v, uint32_t pti) {
    if (v->sparse) return (int)(v->key_of[pti] >> 60);
    int l = 0;
    while (l + 1 < v->L && (int64_t)pti >= v->lay.level_pt_offset[l + 1]) ++l;
    return l;
}

template <class T>
int ensure(vol_t v, T*& ptr, size_t& cap, size_t n, const char* what) {
    if (n <= cap && ptr) return VOL_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    cudaError_t e = dev_alloc(v, (void**)&ptr, sizeof(T) * std::max<size_t>(n, 1));
    if (e != cudaSuccess) return cuda_fail(v, e, what);
    cap = std::max<size_t>(n, 1);
    return VOL_OK;
}

// Publishes the queued page-table writes.  The update kernel writes them in parallel, so an
// entry written twice since the last flush (assigned, then given back) keeps only its last value.
int flush_pt_updates(vol_t v) {
    if (v->upd_idx.empty()) return VOL_OK;
    std::unordered_map<uint32_t, uint32_t> last;
    last.reserve(v->upd_idx.size());
    std::vector<uint32_t> order;
    for (size_t i = 0; i < v->upd_idx.size(); ++i) {
        auto it = last.find(v->upd_idx[i]);
        if (it == last.end()) {
            last.emplace(v->upd_idx[i], v->upd_val[i]);
            order.push_back(v->upd_idx[i]);
        } else {
            it->second = v->upd_val[i];
        }
    }
    const size_t n = order.size();
    if (int rc = ensure(v, v->upd_dev, v->upd_cap, 2 * n, "page-table update buffer")) return rc;
    std::vector<uint32_t> packed(2 * n);
    for (size_t i = 0; i < n; ++i) {
        packed[i] = order[i];
        packed[n + i] = last[order[i]];
    }
    CK(v, cudaMemcpyAsync(v->upd_dev, packed.data(), sizeof(uint32_t) * 2 * n, cudaMemcpyHostToDevice, v->stream));
    CK(v, launch_pt_update(v->pt, v->upd_dev, v->upd_dev + n, (int)n, v->stream));
    v->stats.launches += 1;
    v->upd_idx.clear();
    v->upd_val.clear();
    return VOL_OK;
}

void set_entry(vol_t v, uint32_t pti, uint32_t slot) {
    const uint32_t old = v->pt_host[pti];
    const int l = level_of_pti(v, pti);
    if (old == kInvalidSlot && slot != kInvalidSlot) { ++v->resident; ++v->level_resident[l]; }
    if (old != kInvalidSlot && slot == kInvalidSlot) { --v->resident; --v->level_resident[l]; }
    v->pt_host[pti] = slot;
    uint32_t idx = pti;
    if (v->sparse) {
        sparse_leaf(v, pti, false, &idx);  // the pages exist: slot_for created them
        if (idx == kInvalidSlot) return;
    }
    v->upd_idx.push_back(idx);
    v->upd_val.push_back(slot);
}

// Level and brick coordinates of page-table index (flat) or handle (sparse) pti.
void pti_brick(const vol_t v, uint32_t pti, int* l, int32_t b[3]) {
    if (v->sparse) {
        const uint64_t key = v->key_of[pti];
        *l = (int)(key >> 60);
        b[0] = (int32_t)(key & 0xFFFFF);
        b[1] = (int32_t)((key >> 20) & 0xFFFFF);
        b[2] = (int32_t)((key >> 40) & 0xFFFFF);
        return;
    }
    *l = level_of_pti(v, pti);
    const int64_t id = (int64_t)pti - v->lay.level_pt_offset[*l];
    const int64_t nbx = v->lay.level_bricks[*l][0], nby = v->lay.level_bricks[*l][1];
    b[0] = (int32_t)(id % nbx);
    b[1] = (int32_t)((id / nbx) % nby);
    b[2] = (int32_t)(id / (nbx * nby));
}

// Least-recently-used eviction (usage stamps written by the render kernel).  Frees slots
// until `need` are free and at least 10% of the atlas is free (the collection target),
// never a slot protected by the current operation; slots used in the current frame only
// when nothing older is left.
int evict_lru(vol_t v, size_t need) {
    const int64_t ns = v->lay.nslots;
    std::vector<uint32_t> stamp(ns);
    CK(v, cudaMemcpyAsync(stamp.data(), v->last_used, sizeof(uint32_t) * ns, cudaMemcpyDeviceToHost, v->stream));
    CK(v, cudaStreamSynchronize(v->stream));
    std::vector<uint32_t> cand;
    cand.reserve(ns);
    for (int64_t s = 0; s < ns; ++s)
        if (v->owner[s] != kInvalidSlot && v->protect[s] != v->op_epoch && !v->reserved[s]) cand.push_back((uint32_t)s);
    // age order: older frames first; the current frame last
    std::stable_sort(cand.begin(), cand.end(), [&](uint32_t a, uint32_t b) {
        const uint32_t fa = stamp[a] == v->frame ? 0xFFFFFFFFu : stamp[a];
        const uint32_t fb = stamp[b] == v->frame ? 0xFFFFFFFFu : stamp[b];
        return fa < fb;
    });
    const size_t target = std::max<size_t>(need, (size_t)(ns / 10));
    size_t i = 0;
    while (v->free_slots.size() < target && i < cand.size()) {
        const uint32_t s = cand[i++];
        set_entry(v, v->owner[s], kInvalidSlot);
        v->owner[s] = kInvalidSlot;
        v->free_slots.push_back(s);
        v->stats.evicted++;
    }
    if (v->free_slots.size() < need) return fail(v, VOL_ERR_CACHE_FULL, "brick cache full: nothing evictable");
    return flush_pt_updates(v);
}

// Slot for page-table entry pti (existing one if resident), protected for this operation.
int slot_for(vol_t v, uint32_t pti, uint32_t* out) {
    uint32_t s = v->pt_host[pti];
    if (s == kInvalidSlot) {
        if (v->sparse) {
            uint32_t leaf;
            if (int rc = sparse_leaf(v, pti, true, &leaf)) return rc;
        }
        if (v->free_slots.empty())
            if (int rc = evict_lru(v, 1)) return rc;
        s = v->free_slots.back();
        v->free_slots.pop_back();
        v->owner[s] = pti;
        set_entry(v, pti, s);
    }
    v->protect[s] = v->op_epoch;
    *out = s;
    return VOL_OK;
}

int brick_pti(vol_t v, int level, const int32_t b[3], uint32_t* pti) {
    if (level < 0 || level >= v->L || !b) return VOL_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (b[a] < 0 || b[a] >= v->lay.level_bricks[level][a]) return VOL_ERR_INVALID_ARG;
    if (v->sparse) {
        *pti = handle_for(v, brick_key(level, b[0], b[1], b[2]));
        return VOL_OK;
    }
    *pti = (uint32_t)(v->lay.level_pt_offset[level] + b[0] +
                      v->lay.level_bricks[level][0] * (b[1] + v->lay.level_bricks[level][1] * (int64_t)b[2]));
    return VOL_OK;
}

bool all_resident(const vol_t v, bool lod) {
    const int n = lod ? v->L : 1;
    for (int l = 0; l < n; ++l)
        if (v->level_resident[l] != level_nbricks(v, l)) return false;
    return true;
}

int grid_for(vol_t v, int dtype, bool grad, int ctas_per_sm) {
    int& occ = v->occ_cache[dtype][grad ? 1 : 0];
    if (!occ) occ = render_blocks_per_sm(dtype, grad);
    int per = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
    return std::max(1, per * v->nsm);
}

int ensure_miss_buffers(vol_t v) {
    if (!v->req_table) {
        v->req_cap = 1u << 16;
        v->req_list_cap = 1u << 16;
        CK(v, dev_alloc(v, (void**)&v->req_table, sizeof(unsigned) * v->req_cap));
        CK(v, dev_alloc(v, (void**)&v->req_list, sizeof(unsigned) * v->req_list_cap));
    }
    if (v->sparse && !v->req_table64) {
        CK(v, dev_alloc(v, (void**)&v->req_table64, sizeof(unsigned long long) * v->req_cap));
        CK(v, dev_alloc(v, (void**)&v->req_list64, sizeof(unsigned long long) * v->req_list_cap));
    }
    if (v->susp_cap < v->nrays) {
        for (int i = 0; i < 2; ++i) {
            if (v->susp[i]) cudaFree(v->susp[i]);
            v->susp[i] = nullptr;
        }
        v->susp_cap = 0;
        for (int i = 0; i < 2; ++i) CK(v, dev_alloc(v, (void**)&v->susp[i], sizeof(SuspRec) * (size_t)v->nrays));
        v->susp_cap = v->nrays;
    }
    return VOL_OK;
}

int render_mode(const vol_params& p, bool grad) {
    if (grad) return kDvrGrad;
    if (p.composite == VOL_COMPOSITE_MOP) return kMop;
    if (p.composite == VOL_COMPOSITE_MIP) return kMip;
    return kDvr;
}

RenderDev render_args(vol_t v) {
    RenderDev p{};
    p.vol = vol_dev(v);
    p.views = v->views_dev;
    p.nviews = v->nviews;
    p.tile_w = v->params.tile_w;
    p.tile_h = v->params.tile_h;
    p.refill_thresh = v->params.refill;
    p.tf = (const float4*)v->tf;
    p.step = v->params.step;
    p.et = v->params.et_threshold;
    p.bg = make_float4(v->params.bg[0], v->params.bg[1], v->params.bg[2], v->params.bg[3]);
    p.lod_mode = v->params.lod_mode;
    p.lod_bias = v->params.lod_bias;
    p.skip_empty = (v->params.flags & VOL_RENDER_SKIP_EMPTY) ? 1 : 0;
    p.preview = (v->params.flags & VOL_RENDER_PREVIEW) ? 1 : 0;
    p.level_step = (v->params.flags & VOL_RENDER_LEVEL_STEP) ? 1 : 0;
    p.out = (float4*)v->out;
    p.nsamp = v->nsamp;
    p.counters = v->counters;
    p.last_used = v->last_used;
    p.frame = v->frame;
    p.nrays = v->nrays;
    if (v->grad) {
        p.ckpt = v->ckpt;
        p.ckpt_shift = v->ckpt_shift;
        p.ray_n = v->ray_n;
        p.tape = v->taped ? v->tape : nullptr;
    }
    return p;
}

// Pixel box outside of which no ray of view c meets the volume [0, D0): the 8 corners of the box
// are expressed in the camera basis (fwd, right, up; any non-singular basis, solved in double),
// projected to pixel-centre coordinates, and their bounding box widened by 2 pixels.  A ray's
// direction is rounded to binary32 only, so a pixel 2 pixels outside that box cannot reach the
// volume.  When a corner is not in front of the eye (the eye near or inside the volume) or the
// basis is singular, the box is the whole image.
void view_cull_box(const vol_camera& c, const float D0f[3], ViewDev& V) {
    V.cx0 = 0;
    V.cx1 = c.w - 1;
    V.cy0 = 0;
    V.cy1 = c.h - 1;
    const double F[3] = {c.fwd[0], c.fwd[1], c.fwd[2]}, R[3] = {c.right[0], c.right[1], c.right[2]},
                 U[3] = {c.up[0], c.up[1], c.up[2]};
    // inverse of the matrix with columns F, R, U (rows of the inverse: cross products / det)
    const double cRU[3] = {R[1] * U[2] - R[2] * U[1], R[2] * U[0] - R[0] * U[2], R[0] * U[1] - R[1] * U[0]};
    const double cUF[3] = {U[1] * F[2] - U[2] * F[1], U[2] * F[0] - U[0] * F[2], U[0] * F[1] - U[1] * F[0]};
    const double cFR[3] = {F[1] * R[2] - F[2] * R[1], F[2] * R[0] - F[0] * R[2], F[0] * R[1] - F[1] * R[0]};
    const double det = F[0] * cRU[0] + F[1] * cRU[1] + F[2] * cRU[2];
    const double ta = (double)c.tan_half_fov * (double)c.aspect, tv = (double)c.tan_half_fov;
    if (!(std::fabs(det) > 1e-12) || !(ta > 0.0) || !(tv > 0.0)) return;
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int k = 0; k < 8; ++k) {
        const double p[3] = {(k & 1) ? (double)D0f[0] : 0.0, (k & 2) ? (double)D0f[1] : 0.0,
                             (k & 4) ? (double)D0f[2] : 0.0};
        const double r[3] = {p[0] - c.eye[0], p[1] - c.eye[1], p[2] - c.eye[2]};
        const double len = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        // r = lam (F + a R + b U): lam, lam a, lam b
        const double lam = (r[0] * cRU[0] + r[1] * cRU[1] + r[2] * cRU[2]) / det;
        const double la = (r[0] * cUF[0] + r[1] * cUF[1] + r[2] * cUF[2]) / det;
        const double lb = (r[0] * cFR[0] + r[1] * cFR[1] + r[2] * cFR[2]) / det;
        if (!(lam > 1e-6 * (len + 1.0))) return;  // not clearly in front of the eye
        const double u = la / lam / ta, vv = lb / lam / tv;
        const double px = (u + 1.0) * 0.5 * c.w - 0.5, py = (1.0 - vv) * 0.5 * c.h - 0.5;
        if (!std::isfinite(px) || !std::isfinite(py)) return;
        x0 = std::min(x0, px);
        x1 = std::max(x1, px);
        y0 = std::min(y0, py);
        y1 = std::max(y1, py);
    }
    const double m = 2.0;
    V.cx0 = (int)std::max(0.0, std::min((double)c.w, std::floor(x0 - m)));
    V.cx1 = (int)std::max(-1.0, std::min((double)c.w - 1.0, std::ceil(x1 + m)));
    V.cy0 = (int)std::max(0.0, std::min((double)c.h, std::floor(y0 - m)));
    V.cy1 = (int)std::max(-1.0, std::min((double)c.h - 1.0, std::ceil(y1 + m)));
}

// Default lane-refill threshold: projections keep every ray to its exit, and fetch new rays later
// (measured on the 1024^3 frame: MOP 3.62 -> 3.38 ms, MIP 3.17 -> 2.95 ms at 28 instead of 20;
// emission/absorption is fastest at 20).
int default_refill(int composite) { return composite == VOL_COMPOSITE_DVR ? 20 : 28; }

// One kernel pass.  resume = false: all tiles; true: the rays suspended in susp[susp_cur].
int run_pass(vol_t v, bool resume, bool may_miss) {
    RenderDev p = render_args(v);
    if (may_miss) {
        p.req_table = v->req_table;
        p.req_cap_mask = v->req_cap - 1;
        p.req_list = v->req_list;
        p.req_list_cap = v->req_list_cap;
        CK(v, cudaMemsetAsync(v->req_table, 0, sizeof(unsigned) * v->req_cap, v->stream));
        CK(v, cudaMemsetAsync(v->req_list, 0, sizeof(unsigned) * v->req_list_cap, v->stream));
        // look-ahead of a few bricks for rays that wait: only when a provider will load them
        p.prefetch = (v->prov || v->prov_batch) && !(v->params.flags & VOL_RENDER_NO_PREFETCH) ? kPrefetchBricks : 0;
        if (v->sparse) {
            p.req_table64 = v->req_table64;
            p.req_list64 = v->req_list64;
            CK(v, cudaMemsetAsync(v->req_table64, 0, sizeof(unsigned long long) * v->req_cap, v->stream));
        }
    }
    if (resume) {
        p.resume = 1;
        p.susp_in = v->susp[v->susp_cur];
        p.nsusp_in = (int)v->nsusp;
        p.susp_out = v->susp[v->susp_cur ^ 1];
        p.nwork = (int)((v->nsusp + 31) / 32);
    } else {
        p.resume = 0;
        p.susp_out = v->susp[v->susp_cur];
        p.nwork = v->ntiles;
        p.tile_order = v->order_ready ? v->tile_order : nullptr;
    }
    p.tile_cost = v->tile_cost;
    CK(v, cudaMemsetAsync(v->counters, 0, sizeof(unsigned) * kNumCounters, v->stream));
    v->counters_collected = false;
    v->last_counters = v->counters;
    const int grid = grid_for(v, v->dtype, v->grad, v->params.ctas_per_sm);
    if (v->ev_pass_start) CK(v, cudaEventRecord(v->ev_pass_start, v->stream));
    CK(v, launch_render(v->dtype, render_mode(v->params, v->grad), p, grid, v->stream));
    if (v->ev_pass_end) CK(v, cudaEventRecord(v->ev_pass_end, v->stream));
    v->stats.launches += 1;
    v->stats.passes++;
    return VOL_OK;
}

// After a pass that may have missed: read counters, keep the request list, and switch the
// suspended-ray buffer.  Synchronises.
int collect_pass(vol_t v, bool resumed) {
    unsigned c[kNumCounters];
    CK(v, cudaMemcpyAsync(c, v->counters, sizeof(c), cudaMemcpyDeviceToHost, v->stream));
    CK(v, cudaStreamSynchronize(v->stream));
    v->stats.device_error += c[kDevError];
    v->stats.preview_samples += c[kPreview];
    v->stats.skipped_samples += (int64_t)(((uint64_t)c[kSkipped + 1] << 32) | c[kSkipped]);
    v->counters_collected = true;
    v->stats.request_overflow += c[kReqOverflow];
    const uint32_t nreq = std::min<uint32_t>(c[kReqCount], v->req_list_cap);
    v->stats.requests += nreq;
    v->stats.suspended += c[kSuspCount];
    v->last_requests.resize(nreq);
    if (nreq && v->sparse) {
        std::vector<unsigned long long> keys(nreq);
        CK(v, cudaMemcpy(keys.data(), v->req_list64, sizeof(unsigned long long) * nreq, cudaMemcpyDeviceToHost));
        for (uint32_t i = 0; i < nreq; ++i) {
            const uint64_t key = keys[i] - 1ull;
            const int l = (int)(key >> 60);
            const int64_t b[3] = {(int64_t)(key & 0xFFFFF), (int64_t)((key >> 20) & 0xFFFFF), (int64_t)((key >> 40) & 0xFFFFF)};
            bool ok = keys[i] != 0ull && l < v->L;
            for (int a = 0; a < 3 && ok; ++a) ok = b[a] < v->lay.level_bricks[l][a];
            if (!ok) return fail(v, VOL_ERR_DEVICE, "corrupt brick request");
            v->last_requests[i] = handle_for(v, key) + 1u;
        }
    } else if (nreq) {
        CK(v, cudaMemcpy(v->last_requests.data(), v->req_list, sizeof(uint32_t) * nreq, cudaMemcpyDeviceToHost));
    }
    v->nsusp = c[kSuspCount];
    if (resumed) v->susp_cur ^= 1;
    if (c[kDevError]) return fail(v, VOL_ERR_DEVICE, "device-side check failed during render");
    return VOL_OK;
}

int ensure_stage(vol_t v) {
    if (v->stage_host) return VOL_OK;
    const int64_t B1 = v->B + 1;
    const size_t brick_bytes = (size_t)(B1 * B1 * B1) * 4;  // room for the widest source type
    v->stage_bricks = (int)std::max<int64_t>(1, std::min<int64_t>(256, (64ll << 20) / (int64_t)brick_bytes));
    CK(v, host_alloc(v, &v->stage_host, brick_bytes * v->stage_bricks, cudaHostAllocDefault));
    CK(v, dev_alloc(v, (void**)&v->stage_dev, brick_bytes * v->stage_bricks));
    CK(v, dev_alloc(v, (void**)&v->stage_slots_dev, sizeof(uint32_t) * v->stage_bricks));
    return VOL_OK;
}

// Loads the requested bricks through the provider in batches and publishes them.
int load_requests(vol_t v) {
    if (int rc = ensure_stage(v)) return rc;
    const int64_t B1 = v->B + 1;
    const size_t nvox = (size_t)(B1 * B1 * B1);
    const size_t src_bytes = nvox * bpv_of(v->prov_dtype);
    ++v->op_epoch;
    const std::vector<uint32_t> reqs = v->last_requests;
    std::vector<uint32_t> slots, ptis;
    std::vector<int32_t> batch;  // [n][4] level, bx, by, bz of the bricks to load
    const int64_t loaded0 = v->stats.bricks_loaded;
    bool full = false;
    size_t next = 0;
    while (next < reqs.size() && !full) {
        // collect up to stage_bricks bricks that need a slot
        slots.clear();
        ptis.clear();
        batch.clear();
        while (next < reqs.size() && slots.size() < (size_t)v->stage_bricks) {
            const uint32_t pti = reqs[next] - 1u;
            if (pti >= v->pt_host.size()) return fail(v, VOL_ERR_DEVICE, "corrupt brick request");
            if (v->pt_host[pti] != kInvalidSlot) {  // already resident (e.g. a duplicate)
                v->protect[v->pt_host[pti]] = v->op_epoch;
                ++next;
                continue;
            }
            uint32_t s;
            if (int rc = slot_for(v, pti, &s)) {
                // the cache cannot take more bricks in this pass: load what fits, the rest is
                // requested again by the rays that still wait for it
                if (rc == VOL_ERR_CACHE_FULL && (v->stats.bricks_loaded > loaded0 || !slots.empty())) {
                    full = true;
                    break;
                }
                return rc;
            }
            ++next;
            int l;
            int32_t b[3];
            pti_brick(v, pti, &l, b);
            slots.push_back(s);
            ptis.push_back(pti);
            batch.insert(batch.end(), {(int32_t)l, b[0], b[1], b[2]});
        }
        const size_t n = slots.size();
        if (!n) break;
        // fill the pinned stage from the source
        const int64_t t_prov = now_us();
        bool ok = true;
        if (v->prov_batch) {
            ok = v->prov_batch(v->prov_user, (int)n, batch.data(), v->stage_host) == 0;
        } else {
            for (size_t j = 0; j < n && ok; ++j)
                ok = v->prov(v->prov_user, batch[4 * j], &batch[4 * j + 1], (char*)v->stage_host + j * src_bytes) == 0;
        }
        if (!ok) {
            // the batch's slots were assigned but never filled: give them back, so that the bricks
            // count as absent (and are requested again) rather than resident with stale data
            for (size_t j = 0; j < n; ++j) {
                set_entry(v, ptis[j], kInvalidSlot);
                v->owner[slots[j]] = kInvalidSlot;
                v->free_slots.push_back(slots[j]);
            }
            // an eviction may already have published some of these entries: unpublish them now
            if (int rc = flush_pt_updates(v)) return rc;
            return fail(v, VOL_ERR_PROVIDER, "brick provider failed");
        }
        v->stats.load_wait_us += now_us() - t_prov;
        v->stats.bricks_loaded += (int64_t)n;
        v->stats.bytes_loaded += (int64_t)(n * src_bytes);
        CK(v, cudaMemcpyAsync(v->stage_dev, v->stage_host, src_bytes * n, cudaMemcpyHostToDevice, v->stream));
        CK(v, cudaMemcpyAsync(v->stage_slots_dev, slots.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, v->stream));
        CK(v, launch_upload_bricks(v->dtype, v->prov_dtype, v->stage_dev, vol_dev(v), v->stage_slots_dev, (long long)n,
                                   v->stream));
        CK(v, launch_slot_range(v->dtype, vol_dev(v), v->range, v->cells, v->stage_slots_dev, (long long)n, v->stream));
        v->stats.launches += 2;
        if (int rc = flush_pt_updates(v)) return rc;
        CK(v, cudaStreamSynchronize(v->stream));  // the pinned stage is reused by the next batch
    }
    return VOL_OK;
}

// ---- overlapped loading (batch provider) ----------------------------------------------
//
// The paper interleaves brick loading with rendering (Sec. III-H; Sec. V-A: raycaster tasks
// keep running while chunks load).  Here:
//  * while a pass runs, the host reads the brick requests the kernel appends (a copy on a
//    separate non-blocking stream) and hands them to one library thread that runs the batch
//    provider into a pinned, device-mapped host ring;
//  * a finished chunk is published without a blocking copy: its upload, value-range and
//    page-table kernels read the ring directly and are queued on the volume's stream behind
//    the pass in flight;
//  * the next pass starts once at least half of the bricks known to be missing are published.
// A page-table entry is inserted by a kernel queued after its brick's upload, so no pass ever
// samples a slot that is being filled.

void loader_main(vol_t v) {
    auto& L = v->loader;
    std::unique_lock<std::mutex> lk(L.m);
    for (;;) {
        L.cv.wait(lk, [&] { return L.quit || L.job; });
        if (L.quit) return;
        L.job = false;
        const int n = L.n;
        const int32_t* coords = L.coords;
        void* dst = L.dst;
        lk.unlock();
        const int rc = v->prov_batch(v->prov_user, n, coords, dst);
        lk.lock();
        L.rc = rc;
        L.done = true;
        L.cv.notify_all();
    }
}

int loader_submit(vol_t v, int n, const int32_t* coords, void* dst) {
    auto& L = v->loader;
    if (!L.th.joinable()) {
        try {
            L.th = std::thread(loader_main, v);
        } catch (...) {
            return fail(v, VOL_ERR_UNSUPPORTED, "cannot start the brick loader thread");
        }
    }
    {
        std::lock_guard<std::mutex> lk(L.m);
        L.n = n;
        L.coords = coords;
        L.dst = dst;
        L.done = false;
        L.job = true;
    }
    L.cv.notify_all();
    return VOL_OK;
}

bool loader_done(vol_t v) {
    std::lock_guard<std::mutex> lk(v->loader.m);
    return v->loader.done;
}

int loader_wait(vol_t v) {
    auto& L = v->loader;
    const int64_t t = now_us();
    std::unique_lock<std::mutex> lk(L.m);
    L.cv.wait(lk, [&] { return L.done; });
    v->stats.load_wait_us += now_us() - t;
    return L.rc;
}

void ring_reclaim(vol_t v) {
    auto& R = v->ring;
    while (!R.inflight.empty() && cudaEventQuery(R.inflight.front().ev) == cudaSuccess) {
        R.used -= R.inflight.front().n + R.inflight.front().gap;
        R.spare.push_back(R.inflight.front().ev);
        R.inflight.pop_front();
    }
}

// Ring buffers, the polling stream and the pass events; called before the first pass of a
// render whose misses will load through the overlapped path.
int ensure_overlap(vol_t v) {
    auto& R = v->ring;
    const int64_t B1 = v->B + 1;
    const size_t bb = (size_t)(B1 * B1 * B1) * bpv_of(v->prov_dtype);
    if (!v->poll_stream) CK(v, cudaStreamCreateWithFlags(&v->poll_stream, cudaStreamNonBlocking));
    if (!v->poll_host)
        CK(v, host_alloc(v, (void**)&v->poll_host, sizeof(uint32_t) * ((size_t)v->req_list_cap + 1), cudaHostAllocDefault));
    for (cudaEvent_t* e : {&v->ev_pass_start, &v->ev_pass_end})
        if (!*e) CK(v, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    if (R.host && R.brick_bytes == bb) return VOL_OK;
    // (re)size for this provider's source type: nothing of the old ring may be in flight
    CK(v, cudaStreamSynchronize(v->stream));
    ring_reclaim(v);
    for (void* b : {(void*)R.host, (void*)R.slots, (void*)R.ptis})
        if (b) cudaFreeHost(b);
    R.host = nullptr;
    R.slots = R.ptis = nullptr;
    R.brick_bytes = bb;
    R.cap = (int)std::max<size_t>(64, std::min<size_t>(65536, (size_t(1) << 30) / bb));
    const unsigned fl = cudaHostAllocMapped | cudaHostAllocPortable;
    CK(v, host_alloc(v, (void**)&R.host, bb * R.cap, fl));
    CK(v, host_alloc(v, (void**)&R.slots, sizeof(uint32_t) * R.cap, fl));
    CK(v, host_alloc(v, (void**)&R.ptis, sizeof(uint32_t) * R.cap, fl));
    CK(v, cudaHostGetDevicePointer((void**)&R.host_dev, R.host, 0));
    CK(v, cudaHostGetDevicePointer((void**)&R.slots_dev, R.slots, 0));
    CK(v, cudaHostGetDevicePointer((void**)&R.ptis_dev, R.ptis, 0));
    R.head = R.used = 0;
    return VOL_OK;
}

// n contiguous ring entries (wrapping to the start when the tail is too short), or -1 when
// the ring has no room until earlier uploads complete.
int ring_alloc(vol_t v, int n, int* gap) {
    auto& R = v->ring;
    ring_reclaim(v);
    const int g = R.head + n > R.cap ? R.cap - R.head : 0;
    if (n > R.cap || R.used + g + n > R.cap) return -1;
    const int start = g ? 0 : R.head;
    R.head = start + n == R.cap ? 0 : start + n;
    R.used += g + n;
    *gap = g;
    return start;
}

void ring_unalloc(vol_t v, int start, int n, int gap) {  // undo the newest allocation
    auto& R = v->ring;
    R.head = gap ? R.cap - gap : start;
    R.used -= n + gap;
}

// Mirror-only page-table insert (the device entry is written by a queued kernel).
void mirror_entry(vol_t v, uint32_t pti, uint32_t slot) {
    const uint32_t old = v->pt_host[pti];
    const int l = level_of_pti(v, pti);
    if (old == kInvalidSlot && slot != kInvalidSlot) { ++v->resident; ++v->level_resident[l]; }
    if (old != kInvalidSlot && slot == kInvalidSlot) { --v->resident; --v->level_resident[l]; }
    v->pt_host[pti] = slot;
}

// New request keys of the pass in flight: its count word, then the keys past `seen` that the
// kernel has stored (keys are non-zero; a zero is a reserved place not yet written, read again
// at the next poll).
int poll_live(vol_t v, uint32_t& seen, std::vector<uint32_t>& out) {
    CK(v, cudaMemcpyAsync(v->poll_host, v->counters + kReqCount, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                          v->poll_stream));
    CK(v, cudaStreamSynchronize(v->poll_stream));
    const uint32_t cnt = std::min<uint32_t>(v->poll_host[0], v->req_list_cap);
    if (cnt <= seen) return VOL_OK;
    CK(v, cudaMemcpyAsync(v->poll_host + 1, v->req_list + seen, sizeof(uint32_t) * (cnt - seen),
                          cudaMemcpyDeviceToHost, v->poll_stream));
    CK(v, cudaStreamSynchronize(v->poll_stream));
    uint32_t i = 0;
    for (; i < cnt - seen && v->poll_host[1 + i] != 0u; ++i) out.push_back(v->poll_host[1 + i]);
    seen += i;
    return VOL_OK;
}

size_t ovl_min_chunk() { return std::min<size_t>(64, 2 * (size_t)host_cores()); }  // bricks for every host core
size_t ovl_max_chunk(vol_t v) { return std::max<size_t>(ovl_min_chunk(), std::min<size_t>(512, (size_t)v->ring.cap / 4)); }

// Queue requested bricks (keys = page-table index + 1) that are neither resident nor queued;
// coarse levels first, since one coarse brick serves the rays of many fine ones.
int ovl_take(vol_t v, const std::vector<uint32_t>& keys) {
    std::vector<uint32_t> fresh;
    for (const uint32_t key : keys) {
        const uint32_t pti = key - 1u;
        if (pti >= v->pt_host.size()) return fail(v, VOL_ERR_DEVICE, "corrupt brick request");
        if (v->pt_host[pti] != kInvalidSlot) {
            v->protect[v->pt_host[pti]] = v->op_epoch;
            continue;
        }
        if (v->queued[pti]) continue;
        v->queued[pti] = 1;
        fresh.push_back(pti);
    }
    std::stable_sort(fresh.begin(), fresh.end(),
                     [&](uint32_t a, uint32_t b) { return level_of_pti(v, a) > level_of_pti(v, b); });
    v->ovl.pending.insert(v->ovl.pending.end(), fresh.begin(), fresh.end());
    return VOL_OK;
}

// Hand the next chunk of the queue to the loader thread when it is idle and at least min_n
// bricks wait: ring entries, then slots (evicting only when no pass is in flight).
int ovl_start(vol_t v, bool may_evict, size_t min_n) {
    auto& O = v->ovl;
    auto& R = v->ring;
    auto& J = O.job;
    if (O.running || O.pending.empty() || O.pending.size() < min_n) return VOL_OK;
    const int want = (int)std::min(O.pending.size(), ovl_max_chunk(v));
    int gap = 0;
    const int start = ring_alloc(v, want, &gap);
    if (start < 0) return VOL_OK;  // the ring drains as queued uploads run
    J.start = start;
    J.nalloc = want;
    J.gap = gap;
    J.n = 0;
    J.coords.clear();
    while (J.n < want) {
        const uint32_t pti = O.pending.front();
        if (v->free_slots.empty()) {
            if (!may_evict) break;
            const int rc = evict_lru(v, 1);
            if (rc == VOL_ERR_CACHE_FULL) break;  // retried after the next pass releases slots
            if (rc) return rc;
        }
        const uint32_t s = v->free_slots.back();
        v->free_slots.pop_back();
        v->owner[s] = pti;
        v->reserved[s] = 1;
        v->protect[s] = v->op_epoch;
        O.pending.pop_front();
        R.slots[start + J.n] = s;
        R.ptis[start + J.n] = pti;
        const int l = level_of_pti(v, pti);
        const int64_t id = (int64_t)pti - v->lay.level_pt_offset[l];
        const int64_t nbx = v->lay.level_bricks[l][0], nby = v->lay.level_bricks[l][1];
        J.coords.insert(J.coords.end(), {(int32_t)l, (int32_t)(id % nbx), (int32_t)((id / nbx) % nby),
                                         (int32_t)(id / (nbx * nby))});
        ++J.n;
    }
    if (J.n == 0) {
        ring_unalloc(v, start, want, gap);
        return VOL_OK;
    }
    if (int rc = loader_submit(v, J.n, J.coords.data(), R.host + (size_t)start * R.brick_bytes)) return rc;
    O.running = true;
    return VOL_OK;
}

void ovl_drop(vol_t v) {  // free the chunk's reservations
    auto& J = v->ovl.job;
    auto& R = v->ring;
    for (int j = 0; j < J.n; ++j) {
        const uint32_t s = R.slots[J.start + j];
        v->reserved[s] = 0;
        v->owner[s] = kInvalidSlot;
        v->free_slots.push_back(s);
        v->queued[R.ptis[J.start + j]] = 0;
    }
    ring_unalloc(v, J.start, J.nalloc, J.gap);
    J.n = 0;
}

// Queue the chunk's upload, value ranges and page-table inserts (all reading the ring) on the
// volume's stream.
int ovl_publish(vol_t v, int* published) {
    auto& J = v->ovl.job;
    auto& R = v->ring;
    const int n = J.n, st = J.start;
    const size_t bb = R.brick_bytes;
    CK(v, launch_upload_bricks(v->dtype, v->prov_dtype, R.host_dev + (size_t)st * bb, vol_dev(v), R.slots_dev + st,
                               (long long)n, v->stream));
    CK(v, launch_slot_range(v->dtype, vol_dev(v), v->range, v->cells, R.slots_dev + st, (long long)n, v->stream));
    CK(v, launch_pt_update(v->pt, R.ptis_dev + st, R.slots_dev + st, n, v->stream));
    v->stats.launches += 3;
    cudaEvent_t ev = nullptr;
    if (!R.spare.empty()) {
        ev = R.spare.back();
        R.spare.pop_back();
    } else {
        CK(v, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    CK(v, cudaEventRecord(ev, v->stream));
    R.inflight.push_back({st, J.nalloc, J.gap, ev});
    for (int j = 0; j < n; ++j) {
        const uint32_t s = R.slots[st + j], pti = R.ptis[st + j];
        v->reserved[s] = 0;
        v->protect[s] = v->op_epoch;
        v->queued[pti] = 0;
        mirror_entry(v, pti, s);
    }
    v->stats.bricks_loaded += n;
    v->stats.bytes_loaded += (int64_t)n * (int64_t)bb;
    if (published) *published += n;
    J.n = 0;
    return VOL_OK;
}

// Wait for the chunk in the loader thread; publish it (keep) or free it.
int ovl_finish(vol_t v, bool keep, int* published) {
    auto& O = v->ovl;
    if (!O.running) return VOL_OK;
    O.running = false;
    const int prc = loader_wait(v);
    if (prc != 0 || !keep) {
        ovl_drop(v);
        return prc != 0 ? fail(v, VOL_ERR_PROVIDER, "brick provider failed") : VOL_OK;
    }
    return ovl_publish(v, published);
}

// Before anything else changes the cache: publish the chunk still in generation (a preview
// render leaves it running) and forget the queue.
int ovl_settle(vol_t v) {
    int rc = ovl_finish(v, true, nullptr);
    for (const uint32_t pti : v->ovl.pending) v->queued[pti] = 0;
    v->ovl.pending.clear();
    return rc;
}

// While the pass in flight runs: read its requests, publish finished chunks, start new ones.
int ovl_poll_pass(vol_t v, int* published) {
    uint32_t seen = 0;
    std::vector<uint32_t> keys;
    for (;;) {
        bool progress = false;
        if (cudaEventQuery(v->ev_pass_start) == cudaSuccess) {  // the pass's counters are reset
            keys.clear();
            if (int rc = poll_live(v, seen, keys)) return rc;
            if (int rc = ovl_take(v, keys)) return rc;
        }
        if (v->ovl.running && loader_done(v)) {
            if (int rc = ovl_finish(v, true, published)) return rc;
            progress = true;
        }
        if (!v->ovl.running) {
            if (int rc = ovl_start(v, false, ovl_min_chunk())) return rc;
            progress = progress || v->ovl.running;
        }
        const cudaError_t q = cudaEventQuery(v->ev_pass_end);
        if (q == cudaSuccess) return VOL_OK;
        if (q != cudaErrorNotReady) return cuda_fail(v, q, "render pass");
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
}

// Miss loop of the overlapped path for the pass the caller launched.  preview: that pass took
// absent bricks from coarser levels, so no ray waits; its requests start loading and the
// chunk in generation is left running for the next render to publish.
int miss_loop_overlapped(vol_t v, bool preview) {
    auto& O = v->ovl;
    const int max_passes = v->params.max_passes > 0 ? v->params.max_passes : 256;
    ++v->op_epoch;
    int rc = VOL_OK;
    bool resumed = false;  // the pass in flight is the fresh one (launched by the caller)
    int published = 0;     // bricks published since the pass in flight was launched
    for (;;) {
        // (1) while the pass runs
        if ((rc = ovl_poll_pass(v, &published))) break;
        // (2) the pass is over: all of its requests
        if ((rc = collect_pass(v, resumed)) || (rc = ovl_take(v, v->last_requests))) break;
        if (preview) {
            rc = ovl_start(v, true, 1);
            return rc;
        }
        if (v->nsusp == 0) break;
        if (v->stats.passes >= max_passes) {
            rc = fail(v, VOL_ERR_INCOMPLETE, "max_passes reached");
            break;
        }
        // (3) load until at least half of what is known to be missing is published
        for (;;) {
            if ((rc = ovl_start(v, true, 1))) break;
            const size_t known = (size_t)published + (O.running ? (size_t)O.job.n : 0) + O.pending.size();
            if (published > 0 && 2 * (size_t)published >= known) break;
            if (!O.running) break;  // nothing loadable now: resume anyway (the rays ask again)
            if ((rc = ovl_finish(v, true, &published))) break;
        }
        if (rc) break;
        // (4) the next pass; the chunk in generation keeps going meanwhile
        ++v->op_epoch;
        published = 0;
        if ((rc = run_pass(v, true, true))) break;
        resumed = true;
    }
    const int frc = ovl_finish(v, rc == VOL_OK, nullptr);
    for (const uint32_t pti : O.pending) v->queued[pti] = 0;
    O.pending.clear();
    return rc ? rc : frc;
}

// Miss loop: load and resume until no ray is suspended or passes run out.
int miss_loop(vol_t v, bool first_resumed) {
    if (int rc = collect_pass(v, first_resumed)) return rc;
    const int max_passes = v->params.max_passes > 0 ? v->params.max_passes : 256;
    while (v->nsusp > 0) {
        if (!v->prov && !v->prov_batch)
            return fail(v, VOL_ERR_INCOMPLETE, "rays wait for non-resident bricks (no provider)");
        if (v->stats.passes >= max_passes) return fail(v, VOL_ERR_INCOMPLETE, "max_passes reached");
        if (int rc = load_requests(v)) return rc;
        if (int rc = run_pass(v, true, true)) return rc;
        if (int rc = collect_pass(v, true)) return rc;
    }
    return VOL_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

int vol_plan(const int64_t dims[3], int dtype, int brick, int levels, uint64_t cache_bytes, uint32_t flags,
             vol_layout* out) {
    std::string err;
    return plan(dims, dtype, brick, levels, cache_bytes, flags, out, err);
}

int vol_create(const int64_t dims[3], int dtype, int brick, int levels, uint64_t cache_bytes, uint32_t flags,
               void* stream, vol_t* out) {
    if (!out) return fail(nullptr, VOL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    vol_layout lay;
    std::string err;
    if (int rc = plan(dims, dtype, brick, levels, cache_bytes, flags, &lay, err)) return fail(nullptr, rc, err);
    vol_t v = new vol_s();
    v->lay = lay;
    v->dtype = dtype;
    v->B = brick;
    v->bshift = 0;
    while ((1 << v->bshift) < brick) ++v->bshift;
    v->L = levels;
    v->stream = (cudaStream_t)stream;
    v->sparse = lay.sparse_pt != 0;
    // flat: one entry per brick; sparse: the top grids plus room for 256 pages to start with
    const size_t pt_entries = v->sparse ? (size_t)lay.pt_top_entries + 256 * (size_t)kPageEntries : (size_t)lay.total_bricks;
    cudaError_t e = cudaGetDevice(&v->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v->nsm, cudaDevAttrMultiProcessorCount, v->device);
    if (e == cudaSuccess) e = dev_alloc(v, (void**)&v->atlas, (size_t)lay.atlas_bytes);
    if (e == cudaSuccess) e = dev_alloc(v, (void**)&v->pt, sizeof(uint32_t) * pt_entries);
    if (e == cudaSuccess) e = dev_alloc(v, (void**)&v->last_used, sizeof(unsigned) * (size_t)lay.nslots);
    if (e == cudaSuccess) e = dev_alloc(v, (void**)&v->counters, sizeof(unsigned) * kNumCounters);
    if (e == cudaSuccess) e = dev_alloc(v, (void**)&v->aux, sizeof(unsigned) * 4);
    if (e == cudaSuccess) e = dev_alloc(v, (void**)&v->order_buckets, sizeof(int) * 64);
    if (e == cudaSuccess) e = dev_alloc(v, (void**)&v->range, sizeof(float2) * (size_t)lay.nslots);
    // macro-cells for empty-space skipping: 8 per brick axis (B per axis for B < 8), 2 bytes each
    v->cbits = cell_bits_for(v->bshift);
    v->cshift = v->bshift - v->cbits;
    if (e == cudaSuccess)
        e = dev_alloc(v, (void**)&v->cells, sizeof(uint16_t) * ((size_t)1 << (3 * v->cbits)) * (size_t)lay.nslots);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->pt, 0xFF, sizeof(uint32_t) * pt_entries, v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->last_used, 0, sizeof(unsigned) * (size_t)lay.nslots, v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->aux, 0, sizeof(unsigned) * 4, v->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
    if (e != cudaSuccess) {
        const int code = e == cudaErrorMemoryAllocation ? VOL_ERR_OOM : VOL_ERR_CUDA;
        std::string msg = std::string("vol_create: ") + cudaGetErrorString(e);
        vol_destroy(v);
        return fail(nullptr, code, msg);
    }
    if (v->sparse) {  // per-brick vectors grow with the handles
        v->pool_host.assign(pt_entries, kInvalidSlot);
        v->pool_cap = pt_entries;
        v->pool_used = (size_t)lay.pt_top_entries;
    } else {
        v->pt_host.assign((size_t)lay.total_bricks, kInvalidSlot);
        v->queued.assign((size_t)lay.total_bricks, 0);
    }
    v->owner.assign((size_t)lay.nslots, kInvalidSlot);
    v->protect.assign((size_t)lay.nslots, 0);
    v->reserved.assign((size_t)lay.nslots, 0);
    v->free_slots.resize((size_t)lay.nslots);
    for (int64_t s = 0; s < lay.nslots; ++s) v->free_slots[(size_t)s] = (uint32_t)(lay.nslots - 1 - s);
    v->level_resident.assign(levels, 0);
    *out = v;
    return VOL_OK;
}

void vol_destroy(vol_t v) {
    if (!v) return;
    if (v->loader.th.joinable()) {
        {
            std::lock_guard<std::mutex> lk(v->loader.m);
            v->loader.quit = true;
        }
        v->loader.cv.notify_all();
        v->loader.th.join();
    }
    if (v->stream) cudaStreamSynchronize(v->stream);
    else cudaDeviceSynchronize();
    void* bufs[] = {v->atlas, v->pt, v->last_used, v->counters, v->aux, v->upd_dev, v->views_dev, v->req_table,
                    v->req_list, v->susp[0], v->susp[1], v->ckpt, v->tape, v->ray_n, v->stage_dev, v->stage_slots_dev,
                    v->tile_cost, v->tile_order, v->order_buckets, v->range, v->cells, v->dlev_buf, v->req_table64,
                    v->req_list64};
    for (void* b : bufs)
        if (b) cudaFree(b);
    void* hbufs[] = {v->stage_host, v->ring.host, v->ring.slots, v->ring.ptis, v->poll_host, v->views_pinned};
    if (v->ev_views) cudaEventDestroy(v->ev_views);
    for (void* b : hbufs)
        if (b) cudaFreeHost(b);
    for (auto& r : v->ring.inflight) cudaEventDestroy(r.ev);
    for (cudaEvent_t e : v->ring.spare) cudaEventDestroy(e);
    if (v->poll_stream) cudaStreamDestroy(v->poll_stream);
    for (cudaEvent_t e : {v->ev_pass_start, v->ev_pass_end})
        if (e) cudaEventDestroy(e);
    delete v;
}

const char* vol_last_error(vol_t v) { return v ? v->err.c_str() : g_create_error.c_str(); }

int vol_set_stream(vol_t v, void* stream) {
    if (!v) return VOL_ERR_INVALID_ARG;
    v->stream = (cudaStream_t)stream;
    return VOL_OK;
}

int vol_get_layout(vol_t v, vol_layout* out) {
    if (!v || !out) return VOL_ERR_INVALID_ARG;
    *out = v->lay;
    return VOL_OK;
}

int vol_get_stats(vol_t v, vol_stats* out) {
    if (!v || !out) return VOL_ERR_INVALID_ARG;
    unsigned c[kNumCounters], aux[4];
    CK(v, cudaMemcpyAsync(c, v->last_counters ? v->last_counters : v->counters, sizeof(c), cudaMemcpyDeviceToHost,
                          v->stream));
    CK(v, cudaMemcpyAsync(aux, v->aux, sizeof(aux), cudaMemcpyDeviceToHost, v->stream));
    CK(v, cudaStreamSynchronize(v->stream));
    std::vector<uint32_t> stamp((size_t)v->lay.nslots);
    CK(v, cudaMemcpy(stamp.data(), v->last_used, sizeof(uint32_t) * stamp.size(), cudaMemcpyDeviceToHost));
    *out = v->stats;
    out->touched = 0;
    for (size_t s = 0; s < stamp.size(); ++s)
        if (v->owner[s] != kInvalidSlot && stamp[s] == v->frame && v->frame) out->touched++;
    out->resident = v->resident;
    out->frame = v->frame;
    // the counters of a pass that collect_pass has not read yet (a render that missed nothing)
    if (!v->counters_collected) {
        out->device_error += c[kDevError];
        out->skipped_samples += (int64_t)(((uint64_t)c[kSkipped + 1] << 32) | c[kSkipped]);
    }
    out->device_error += aux[0];
    out->allocations = v->allocations;
    return VOL_OK;
}

int vol_upload_level(vol_t v, int level, const void* src, int src_dtype, int src_on_device) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    if (v->sparse) return fail(v, VOL_ERR_UNSUPPORTED, "sparse page table: load bricks one by one or by a provider");
    if (level < 0 || level >= v->L || !src) return fail(v, VOL_ERR_INVALID_ARG, "bad level or src");
    if (!bpv_of(src_dtype)) return fail(v, VOL_ERR_INVALID_ARG, "bad src dtype");
    if (!conversion_ok(src_dtype, v->dtype)) return fail(v, VOL_ERR_UNSUPPORTED, "unsupported conversion");
    const int64_t nb = level_nbricks(v, level);
    if (nb > v->lay.nslots) return fail(v, VOL_ERR_CACHE_FULL, "level does not fit the brick cache");
    ++v->op_epoch;
    std::vector<uint32_t> slots((size_t)nb);
    for (int64_t b = 0; b < nb; ++b)
        if (int rc = slot_for(v, (uint32_t)(v->lay.level_pt_offset[level] + b), &slots[(size_t)b])) return rc;
    const int64_t nvox = v->lay.level_dims[level][0] * v->lay.level_dims[level][1] * v->lay.level_dims[level][2];
    const size_t sbytes = (size_t)nvox * bpv_of(src_dtype);
    const void* dsrc = src;
    void* tmp = nullptr;
    uint32_t* dslots = nullptr;
    CK(v, dev_alloc(v, (void**)&dslots, sizeof(uint32_t) * (size_t)nb));
    if (!src_on_device) {
        cudaError_t e = dev_alloc(v, (void**)&tmp, sbytes);
        if (e != cudaSuccess) { cudaFree(dslots); return cuda_fail(v, e, "upload staging"); }
        e = cudaMemcpyAsync(tmp, src, sbytes, cudaMemcpyHostToDevice, v->stream);
        if (e != cudaSuccess) { cudaFree(dslots); cudaFree(tmp); return cuda_fail(v, e, "upload copy"); }
        dsrc = tmp;
    }
    cudaError_t e = cudaMemcpyAsync(dslots, slots.data(), sizeof(uint32_t) * (size_t)nb, cudaMemcpyHostToDevice, v->stream);
    if (e == cudaSuccess) e = launch_upload_level(v->dtype, src_dtype, dsrc, vol_dev(v), level, dslots, nb, v->stream);
    if (e == cudaSuccess) e = launch_slot_range(v->dtype, vol_dev(v), v->range, v->cells, dslots, nb, v->stream);
    int rc = e == cudaSuccess ? flush_pt_updates(v) : cuda_fail(v, e, "upload_level kernel");
    cudaError_t e2 = cudaStreamSynchronize(v->stream);
    cudaFree(dslots);
    if (tmp) cudaFree(tmp);
    if (rc) return rc;
    if (e2 != cudaSuccess) return cuda_fail(v, e2, "upload_level");
    return VOL_OK;
}

int vol_upload_brick(vol_t v, int level, const int32_t brick[3], const void* src, int src_dtype, int src_on_device) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    uint32_t pti;
    if (!src || brick_pti(v, level, brick, &pti)) return fail(v, VOL_ERR_INVALID_ARG, "bad level, brick or src");
    if (!conversion_ok(src_dtype, v->dtype)) return fail(v, VOL_ERR_UNSUPPORTED, "unsupported conversion");
    if (int rc = ensure_stage(v)) return rc;
    ++v->op_epoch;
    uint32_t s;
    if (int rc = slot_for(v, pti, &s)) return rc;
    const int64_t B1 = v->B + 1;
    const size_t bytes = (size_t)(B1 * B1 * B1) * bpv_of(src_dtype);
    const void* dsrc = src;
    if (!src_on_device) {
        CK(v, cudaMemcpyAsync(v->stage_dev, src, bytes, cudaMemcpyHostToDevice, v->stream));
        dsrc = v->stage_dev;
    }
    CK(v, cudaMemcpyAsync(v->stage_slots_dev, &s, sizeof(uint32_t), cudaMemcpyHostToDevice, v->stream));
    CK(v, launch_upload_bricks(v->dtype, src_dtype, dsrc, vol_dev(v), v->stage_slots_dev, 1, v->stream));
    CK(v, launch_slot_range(v->dtype, vol_dev(v), v->range, v->cells, v->stage_slots_dev, 1, v->stream));
    v->stats.launches += 2;
    if (int rc = flush_pt_updates(v)) return rc;
    CK(v, cudaStreamSynchronize(v->stream));
    return VOL_OK;
}

int vol_build_lod(vol_t v, int from_level) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    if (v->sparse) return fail(v, VOL_ERR_UNSUPPORTED, "sparse page table: coarser levels come from the provider");
    if (from_level < 0 || from_level >= v->L) return fail(v, VOL_ERR_INVALID_ARG, "bad from_level");
    for (int l = from_level + 1; l < v->L; ++l) {
        if (v->level_resident[l - 1] != level_nbricks(v, l - 1))
            return fail(v, VOL_ERR_INVALID_ARG, "source level not fully resident");
        const int64_t nb = level_nbricks(v, l);
        if (nb + level_nbricks(v, l - 1) > v->lay.nslots)
            return fail(v, VOL_ERR_CACHE_FULL, "levels do not fit the brick cache");
        ++v->op_epoch;
        // keep the source level while allocating the coarse one
        for (int64_t b = 0; b < level_nbricks(v, l - 1); ++b)
            v->protect[v->pt_host[(size_t)(v->lay.level_pt_offset[l - 1] + b)]] = v->op_epoch;
        std::vector<uint32_t> slots((size_t)nb);
        for (int64_t b = 0; b < nb; ++b)
            if (int rc = slot_for(v, (uint32_t)(v->lay.level_pt_offset[l] + b), &slots[(size_t)b])) return rc;
        uint32_t* dslots = nullptr;
        CK(v, dev_alloc(v, (void**)&dslots, sizeof(uint32_t) * (size_t)nb));
        cudaError_t e = cudaMemcpyAsync(dslots, slots.data(), sizeof(uint32_t) * (size_t)nb, cudaMemcpyHostToDevice, v->stream);
        int rc = VOL_OK;
        if (e == cudaSuccess) rc = flush_pt_updates(v);  // the source level's entries must be live
        if (e == cudaSuccess && !rc) e = launch_downsample(v->dtype, vol_dev(v), l, dslots, nb, v->aux, v->stream);
        if (e == cudaSuccess && !rc) e = launch_slot_range(v->dtype, vol_dev(v), v->range, v->cells, dslots, nb, v->stream);
        cudaError_t e2 = cudaStreamSynchronize(v->stream);
        cudaFree(dslots);
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_fail(v, e, "downsample");
        if (e2 != cudaSuccess) return cuda_fail(v, e2, "downsample");
    }
    unsigned aux0 = 0;
    CK(v, cudaMemcpy(&aux0, v->aux, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (aux0) return fail(v, VOL_ERR_DEVICE, "downsample met a non-resident brick");
    return VOL_OK;
}

int vol_download_brick(vol_t v, int level, const int32_t brick[3], void* dst) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    uint32_t pti;
    if (!dst || brick_pti(v, level, brick, &pti)) return fail(v, VOL_ERR_INVALID_ARG, "bad level, brick or dst");
    const uint32_t s = v->pt_host[pti];
    if (s == kInvalidSlot) return fail(v, VOL_ERR_INVALID_ARG, "brick not resident");
    const int64_t B = v->B, B1 = B + 1;
    const int bpv = v->lay.bytes_per_voxel;
    const char* src = (const char*)v->atlas + (size_t)s * v->lay.slot_bytes;
    if (v->lay.layout == 1) {
        CK(v, cudaMemcpyAsync(dst, src, (size_t)(B1 * B1 * B1) * bpv, cudaMemcpyDeviceToHost, v->stream));
        CK(v, cudaStreamSynchronize(v->stream));
        return VOL_OK;
    }
    // quad layout: voxel (x, y, z) of the (B+1)^3 region is component (x == B) + 2 (y == B) of
    // entry (min(x, B-1), min(y, B-1), z)
    std::vector<char> raw((size_t)v->lay.slot_bytes);
    CK(v, cudaMemcpyAsync(raw.data(), src, raw.size(), cudaMemcpyDeviceToHost, v->stream));
    CK(v, cudaStreamSynchronize(v->stream));
    char* out = (char*)dst;
    for (int64_t z = 0; z < B1; ++z)
        for (int64_t y = 0; y < B1; ++y)
            for (int64_t x = 0; x < B1; ++x) {
                const int64_t ex = x < B ? x : B - 1, ey = y < B ? y : B - 1;
                const int comp = (x == B ? 1 : 0) + (y == B ? 2 : 0);
                const int64_t e = (z * B + ey) * B + ex;
                memcpy(out + ((z * B1 + y) * B1 + x) * bpv, raw.data() + (e * 4 + comp) * bpv, bpv);
            }
    return VOL_OK;
}

int vol_evict_all(vol_t v) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    for (int64_t s = 0; s < v->lay.nslots; ++s)
        if (v->owner[(size_t)s] != kInvalidSlot) {
            v->owner[(size_t)s] = kInvalidSlot;
            v->free_slots.push_back((uint32_t)s);
        }
    std::fill(v->pt_host.begin(), v->pt_host.end(), kInvalidSlot);
    std::fill(v->level_resident.begin(), v->level_resident.end(), 0);
    v->resident = 0;
    v->upd_idx.clear();
    v->upd_val.clear();
    if (v->sparse) {  // every page back to the pool
        std::fill(v->pool_host.begin(), v->pool_host.end(), kInvalidSlot);
        v->pool_used = (size_t)v->lay.pt_top_entries;
        CK(v, cudaMemsetAsync(v->pt, 0xFF, sizeof(uint32_t) * v->pool_cap, v->stream));
    } else {
        CK(v, cudaMemsetAsync(v->pt, 0xFF, sizeof(uint32_t) * (size_t)v->lay.total_bricks, v->stream));
    }
    v->have_forward = false;
    return VOL_OK;
}

int vol_set_provider(vol_t v, vol_provider_fn fn, void* user, int src_dtype) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    if (fn && !conversion_ok(src_dtype, v->dtype)) return fail(v, VOL_ERR_UNSUPPORTED, "unsupported provider dtype");
    v->prov = fn;
    v->prov_batch = nullptr;
    v->prov_user = user;
    v->prov_dtype = src_dtype;
    return VOL_OK;
}

int vol_set_provider_batch(vol_t v, vol_provider_batch_fn fn, void* user, int src_dtype) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    if (fn && !conversion_ok(src_dtype, v->dtype)) return fail(v, VOL_ERR_UNSUPPORTED, "unsupported provider dtype");
    v->prov_batch = fn;
    v->prov = nullptr;
    v->prov_user = user;
    v->prov_dtype = src_dtype;
    return VOL_OK;
}

// The address the kernels write an output through: memory of the volume's GPU (or managed memory)
// as it is, page-locked host memory through its device mapping -- the kernels then write the
// image across the host link and the caller needs no copy -- and anything else is refused
// before any launch.
static int device_address(vol_t v, void* p, void** out, const char* what) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(v, VOL_ERR_INVALID_ARG, what);
    }
    if ((a.type == cudaMemoryTypeDevice && a.device == v->device) || a.type == cudaMemoryTypeManaged) {
        *out = p;
        return VOL_OK;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *out = a.devicePointer;
        return VOL_OK;
    }
    return fail(v, VOL_ERR_INVALID_ARG, what);
}

static int output_addresses(vol_t v, float*& rgba, int32_t*& nsamples) {
    void* p = nullptr;
    if (int rc = device_address(v, rgba, &p, "rgba must be memory of the volume's GPU or page-locked host memory"))
        return rc;
    rgba = (float*)p;
    if (nsamples) {
        if (int rc = device_address(v, nsamples, &p,
                                    "nsamples must be memory of the volume's GPU or page-locked host memory"))
            return rc;
        nsamples = (int32_t*)p;
    }
    return VOL_OK;
}

// The longest segment of a ray inside [0, D0) is the box diagonal: its sample count (plus the
// samples a batch computes past the exit) must stay within kMaxSamplesPerRay.
static bool samples_fit(const vol_s* v, float step) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) d2 += (double)v->lay.dims[a] * (double)v->lay.dims[a];
    return std::sqrt(d2) / (double)step + 2.0 < kMaxSamplesPerRay;
}

int vol_render(vol_t v, const vol_camera* cams, int nviews, const float* tf_dev, const vol_params* params,
               float* rgba_dev, int32_t* nsamples_dev) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (!cams || !tf_dev || !params || !rgba_dev) return fail(v, VOL_ERR_INVALID_ARG, "null argument");
    if (nviews < 1 || nviews > VOL_MAX_VIEWS) return fail(v, VOL_ERR_INVALID_ARG, "nviews out of range");
    if (int rc = output_addresses(v, rgba_dev, nsamples_dev)) return rc;
    vol_params p = *params;
    if (!(p.step > 0.0f) || !std::isfinite(p.step)) return fail(v, VOL_ERR_INVALID_ARG, "step must be > 0");
    if (!samples_fit(v, p.step))
        return fail(v, VOL_ERR_INVALID_ARG, "step too small: more than 2^24 samples along the volume diagonal");
    if (p.tile_w <= 0) p.tile_w = 4;
    if (p.tile_h <= 0) p.tile_h = 8;
    if (p.tile_w > 4096 || p.tile_h > 4096 || p.tile_w * p.tile_h > 4096)
        return fail(v, VOL_ERR_INVALID_ARG, "tile_w * tile_h must be at most 4096");
    if (p.refill <= 0 || p.refill > 32) p.refill = default_refill(p.composite);
    if (p.lod_mode != 0 && p.lod_mode != 1) return fail(v, VOL_ERR_INVALID_ARG, "lod_mode must be 0 or 1");
    if (p.composite < VOL_COMPOSITE_DVR || p.composite > VOL_COMPOSITE_MIP)
        return fail(v, VOL_ERR_INVALID_ARG, "composite must be VOL_COMPOSITE_DVR, _MOP or _MIP");
    const bool grad = (p.flags & VOL_RENDER_GRAD) != 0;
    if (grad && p.composite != VOL_COMPOSITE_DVR)
        return fail(v, VOL_ERR_UNSUPPORTED, "gradients need emission/absorption compositing");
    if ((p.flags & VOL_RENDER_CKPT_ALL) && !grad)
        return fail(v, VOL_ERR_INVALID_ARG, "VOL_RENDER_CKPT_ALL needs VOL_RENDER_GRAD");
    const bool preview = (p.flags & VOL_RENDER_PREVIEW) != 0;
    if (grad && preview) return fail(v, VOL_ERR_UNSUPPORTED, "a preview keeps no gradient state");
    if ((p.flags & VOL_RENDER_LEVEL_STEP) && (grad || p.composite != VOL_COMPOSITE_DVR))
        return fail(v, VOL_ERR_UNSUPPORTED, "level-scaled sampling is for emission/absorption without gradients");
    if (v->sparse && (grad || p.composite != VOL_COMPOSITE_DVR || (p.flags & VOL_RENDER_LEVEL_STEP)))
        return fail(v, VOL_ERR_UNSUPPORTED, "the sparse page table renders emission/absorption without gradients "
                                            "or level-scaled sampling");

    // view table
    v->views_host.resize(nviews);
    int64_t rays = 0;
    int64_t tiles = 0;
    for (int i = 0; i < nviews; ++i) {
        const vol_camera& c = cams[i];
        if (c.w < 1 || c.h < 1 || c.w > 65536 || c.h > 65536) return fail(v, VOL_ERR_INVALID_ARG, "bad image size");
        if (!(c.tan_half_fov > 0.0f) || !std::isfinite(c.tan_half_fov))
            return fail(v, VOL_ERR_INVALID_ARG, "tan_half_fov must be > 0");
        ViewDev& V = v->views_host[i];
        V = ViewDev{};  // (padding too: tables are compared bytewise)
        for (int a = 0; a < 3; ++a) {
            V.eye[a] = c.eye[a];
            V.right[a] = c.right[a];
            V.up[a] = c.up[a];
            V.fwd[a] = c.fwd[a];
        }
        V.tan = c.tan_half_fov;
        V.tan_aspect = c.tan_half_fov * c.aspect;
        V.lodscale = (2.0f * c.tan_half_fov) / (float)c.h;
        V.w = c.w;
        V.h = c.h;
        V.tiles_x = (c.w + p.tile_w - 1) / p.tile_w;
        V.tile_off = (int)tiles;
        V.ray_off = rays;
        const float D0f[3] = {(float)v->lay.dims[0], (float)v->lay.dims[1], (float)v->lay.dims[2]};
        view_cull_box(c, D0f, V);
        tiles += (int64_t)V.tiles_x * ((c.h + p.tile_h - 1) / p.tile_h);
        rays += (int64_t)c.w * c.h;
    }
    if (tiles >= (1ll << 31)) return fail(v, VOL_ERR_INVALID_ARG, "too many tiles");
    if (v->views_cap < nviews) {
        if (v->views_dev) cudaFree(v->views_dev);
        v->views_dev = nullptr;
        v->views_cap = 0;
        v->views_sent.clear();
        CK(v, dev_alloc(v, (void**)&v->views_dev, sizeof(ViewDev) * nviews));
        v->views_cap = nviews;
    }
    // the device table is copied only when the views changed, from page-locked memory (an
    // asynchronous copy; a copy from pageable memory would wait for the staging)
    if (v->views_sent.size() != (size_t)nviews ||
        memcmp(v->views_sent.data(), v->views_host.data(), sizeof(ViewDev) * nviews) != 0) {
        if (v->views_pinned_cap < nviews) {
            if (v->views_pinned) {
                CK(v, cudaEventSynchronize(v->ev_views));
                cudaFreeHost(v->views_pinned);
            }
            v->views_pinned = nullptr;
            v->views_pinned_cap = 0;
            CK(v, host_alloc(v, (void**)&v->views_pinned, sizeof(ViewDev) * nviews, cudaHostAllocDefault));
            v->views_pinned_cap = nviews;
        }
        if (!v->ev_views) CK(v, cudaEventCreateWithFlags(&v->ev_views, cudaEventDisableTiming));
        else CK(v, cudaEventSynchronize(v->ev_views));  // the last copy out of the buffer is done
        memcpy(v->views_pinned, v->views_host.data(), sizeof(ViewDev) * nviews);
        CK(v, cudaMemcpyAsync(v->views_dev, v->views_pinned, sizeof(ViewDev) * nviews, cudaMemcpyHostToDevice, v->stream));
        CK(v, cudaEventRecord(v->ev_views, v->stream));
        v->views_sent = v->views_host;
    }
    v->nviews = nviews;
    v->ntiles = (int)tiles;
    v->nrays = rays;
    v->params = p;
    v->tf = tf_dev;
    v->out = rgba_dev;
    v->nsamp = nsamples_dev;
    v->grad = grad;
    v->have_forward = false;
    v->nsusp = 0;
    v->susp_cur = 0;
    ++v->frame;
    v->stats = vol_stats{};
    v->stats.rays = rays;

    if (grad) {
        double diag = 0.0;
        for (int a = 0; a < 3; ++a) diag += (double)v->lay.dims[a] * (double)v->lay.dims[a];
        const int64_t max_n = (int64_t)std::ceil(std::sqrt(diag) / (double)p.step) + 2;
        v->ckpt_shift = (p.flags & VOL_RENDER_CKPT_ALL) ? 0 : kCkptShift;
        const int64_t every = int64_t(1) << v->ckpt_shift;
        const int64_t segs = (max_n + every - 1) / every;
        if (int rc = ensure(v, v->ckpt, v->ckpt_cap, (size_t)std::max<int64_t>(1, segs - 1) * (size_t)rays, "checkpoints")) return rc;
        if (int rc = ensure(v, v->ray_n, v->ray_n_cap, (size_t)rays, "ray sample counts")) return rc;
        // value tape: 32 values per checkpoint segment of every ray; when it cannot be had the
        // adjoint interpolates the values again from the bricks
        v->taped = false;
        if (v->ckpt_shift == kCkptShift && !(p.flags & VOL_RENDER_GRAD_RECOMPUTE)) {
            const size_t need = (size_t)((max_n + kCkptEvery - 1) / kCkptEvery) * (size_t)rays * kCkptEvery;
            if (ensure(v, v->tape, v->tape_cap, need, "value tape") == VOL_OK) {
                v->taped = true;
            } else {
                cudaGetLastError();  // (the failed allocation; gradients are still exact)
                v->err.clear();
            }
        }
    }
    // scheduling state: the previous frame's longest-ray-first order is reused while the tile
    // partition (tile shape, number of views, image sizes) is unchanged; cameras may move.
    // The order is only a schedule: the image never depends on it.
    {
        std::vector<int> key;
        key.reserve(3 + 2 * (size_t)nviews);
        key.push_back(p.tile_w);
        key.push_back(p.tile_h);
        key.push_back(nviews);
        for (int i = 0; i < nviews; ++i) {
            key.push_back(cams[i].w);
            key.push_back(cams[i].h);
        }
        std::vector<unsigned char> kb((const unsigned char*)key.data(), (const unsigned char*)(key.data() + key.size()));
        if (kb != v->order_key || !v->tile_cost || !v->tile_order) {
            if (int rc = ensure(v, v->tile_cost, v->tile_cost_cap, (size_t)tiles, "tile costs")) return rc;
            if (int rc = ensure(v, v->tile_order, v->tile_order_cap, (size_t)tiles, "tile order")) return rc;
            CK(v, cudaMemsetAsync(v->tile_cost, 0, sizeof(int) * (size_t)tiles, v->stream));
            v->order_ready = false;
            v->order_key = kb;
        }
    }
    const bool may_miss = !all_resident(v, p.lod_mode != 0);
    const bool overlap = may_miss && v->prov_batch && !(p.flags & VOL_RENDER_SERIAL_LOADS) && !v->sparse;
    if (!overlap)
        if (int rc = ovl_settle(v)) return rc;  // a chunk a preview left in generation
    if (may_miss)
        if (int rc = ensure_miss_buffers(v)) return rc;
    if (overlap)
        if (int rc = ensure_overlap(v)) return rc;
    if (int rc = run_pass(v, false, may_miss)) return rc;
    int rc = VOL_OK;
    if (may_miss) {
        if (overlap) {
            rc = miss_loop_overlapped(v, preview);
        } else if (preview) {
            // one pass (no ray waited); load what it requested for the next render
            rc = collect_pass(v, false);
            if (!rc && (v->prov || v->prov_batch) && !v->last_requests.empty()) rc = load_requests(v);
        } else {
            rc = miss_loop(v, false);
        }
    }
    if (rc == VOL_OK && !preview) v->have_forward = true;
    if (rc == VOL_OK || rc == VOL_ERR_INCOMPLETE) {
        CK(v, launch_tile_order(v->tile_cost, v->tile_order, (int)tiles, v->order_buckets, v->stream));
        v->stats.launches += 2;
        v->order_ready = true;
    }
    return rc;
}

int vol_render_resume(vol_t v) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    if (!v->out) return fail(v, VOL_ERR_NO_FORWARD_STATE, "no render to resume");
    if (v->nsusp == 0) return VOL_OK;
    if (int rc = run_pass(v, true, true)) return rc;
    int rc = miss_loop(v, true);
    if (rc == VOL_OK) v->have_forward = true;
    return rc;
}

int vol_poll_requests(vol_t v, int32_t* out, int cap, int* n) {
    if (!v || !n || (cap > 0 && !out)) return VOL_ERR_INVALID_ARG;
    *n = (int)v->last_requests.size();
    for (int i = 0; i < cap && i < *n; ++i) {
        const uint32_t pti = v->last_requests[i] - 1u;
        int l;
        int32_t b[3];
        pti_brick(v, pti, &l, b);
        out[4 * i + 0] = l;
        out[4 * i + 1] = b[0];
        out[4 * i + 2] = b[1];
        out[4 * i + 3] = b[2];
    }
    return VOL_OK;
}

int vol_render_backward(vol_t v, const float* drgba_dev, float* dtf_dev, float* dvoxel_dev) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    if (!drgba_dev) return fail(v, VOL_ERR_INVALID_ARG, "drgba is NULL");
    if (!v->have_forward || !v->grad) return fail(v, VOL_ERR_NO_FORWARD_STATE, "no gradient-mode render to differentiate");
    if (v->nsusp) return fail(v, VOL_ERR_NO_FORWARD_STATE, "last render is incomplete");
    const bool lod = v->params.lod_mode != 0;
    if (!all_resident(v, lod))
        return fail(v, VOL_ERR_NO_FORWARD_STATE, lod ? "a level is no longer fully resident" : "level 0 changed since the render");
    if (!dtf_dev && !dvoxel_dev) return VOL_OK;
    BackwardDev b{};
    b.vol = vol_dev(v);
    b.views = v->views_dev;
    b.nviews = v->nviews;
    b.nwork = v->ntiles * ((v->params.tile_w * v->params.tile_h + 31) / 32);  // 32 rays per work item
    b.tile_w = v->params.tile_w;
    b.tile_h = v->params.tile_h;
    b.tf = (const float4*)v->tf;
    b.step = v->params.step;
    b.bg = make_float4(v->params.bg[0], v->params.bg[1], v->params.bg[2], v->params.bg[3]);
    b.drgba = (const float4*)drgba_dev;
    b.dtf = dtf_dev;
    b.dvox = dvoxel_dev;
    b.lod_mode = v->params.lod_mode;
    b.lod_bias = v->params.lod_bias;
    b.dlev[0] = dvoxel_dev;
    if (lod && dvoxel_dev) {
        // gradient buffers for levels 1..L-1, zeroed; carried down to level 0 after the kernel
        size_t tot = 0;
        for (int l = 1; l < v->L; ++l)
            tot += (size_t)(v->lay.level_dims[l][0] * v->lay.level_dims[l][1] * v->lay.level_dims[l][2]);
        if (int rc = ensure(v, v->dlev_buf, v->dlev_cap, tot, "level gradient buffers")) return rc;
        CK(v, cudaMemsetAsync(v->dlev_buf, 0, sizeof(float) * tot, v->stream));
        size_t off = 0;
        for (int l = 1; l < v->L; ++l) {
            b.dlev[l] = v->dlev_buf + off;
            off += (size_t)(v->lay.level_dims[l][0] * v->lay.level_dims[l][1] * v->lay.level_dims[l][2]);
        }
    }
    b.counters = v->counters;
    b.ckpt = v->ckpt;
    b.ckpt_shift = v->ckpt_shift;
    b.tape = v->taped ? v->tape : nullptr;
    b.nrays = v->nrays;
    b.ray_n = v->ray_n;
    // the order built from this forward's per-tile longest rays: those tiles first
    b.tile_order = v->order_ready ? v->tile_order : nullptr;
    CK(v, cudaMemsetAsync(v->counters, 0, sizeof(unsigned) * kNumCounters, v->stream));
    v->counters_collected = false;  // vol_get_stats adds the adjoint's device-side check count
    v->last_counters = v->counters;
    const int grid = backward_blocks_per_sm(v->dtype, lod, b.tape != nullptr) * v->nsm;
    CK(v, launch_backward(v->dtype, b, grid, v->stream));
    v->stats.launches += 1;
    if (lod && dvoxel_dev) {
        // each level's gradient onto the level it was filtered from, coarsest first (Sec. III-D)
        for (int l = v->L - 1; l >= 1; --l) {
            const int Df[3] = {(int)v->lay.level_dims[l - 1][0], (int)v->lay.level_dims[l - 1][1],
                               (int)v->lay.level_dims[l - 1][2]};
            CK(v, launch_downsample_transpose(b.dlev[l], b.dlev[l - 1], Df, v->stream));
            v->stats.launches += 1;
        }
    }
    return VOL_OK;
}

int vol_trace(vol_t v, const vol_camera* cam, const vol_params* params, const int32_t* pixels_host, int npix,
              int max_samples, vol_trace_rec* out_host, int32_t* counts_host) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    if (!cam || !params || !pixels_host || !out_host || !counts_host || npix < 0 || max_samples < 0)
        return fail(v, VOL_ERR_INVALID_ARG, "bad trace arguments");
    if (npix == 0) return VOL_OK;
    if (cam->w < 1 || cam->h < 1) return fail(v, VOL_ERR_INVALID_ARG, "bad image size");
    if (!(cam->tan_half_fov > 0.0f) || !std::isfinite(cam->tan_half_fov))
        return fail(v, VOL_ERR_INVALID_ARG, "tan_half_fov must be > 0");
    for (int i = 0; i < npix; ++i)
        if (pixels_host[2 * i] < 0 || pixels_host[2 * i] >= cam->w || pixels_host[2 * i + 1] < 0 ||
            pixels_host[2 * i + 1] >= cam->h)
            return fail(v, VOL_ERR_INVALID_ARG, "pixel outside the image");
    TraceDev t{};
    t.vol = vol_dev(v);
    for (int a = 0; a < 3; ++a) {
        t.view.eye[a] = cam->eye[a];
        t.view.right[a] = cam->right[a];
        t.view.up[a] = cam->up[a];
        t.view.fwd[a] = cam->fwd[a];
    }
    t.view.tan = cam->tan_half_fov;
    t.view.tan_aspect = cam->tan_half_fov * cam->aspect;
    t.view.lodscale = (2.0f * cam->tan_half_fov) / (float)cam->h;
    t.view.w = cam->w;
    t.view.h = cam->h;
    t.step = params->step;
    t.lod_mode = params->lod_mode;
    t.level_step = (params->flags & VOL_RENDER_LEVEL_STEP) ? 1 : 0;
    t.lod_bias = params->lod_bias;
    t.npix = npix;
    t.max_samples = max_samples;
    int* dpix = nullptr;
    int* dcnt = nullptr;
    vol_trace_rec* drec = nullptr;
    const size_t nrec = (size_t)npix * (size_t)std::max(1, max_samples);
    cudaError_t e = dev_alloc(v, (void**)&dpix, sizeof(int) * 2 * npix);
    if (e == cudaSuccess) e = dev_alloc(v, (void**)&dcnt, sizeof(int) * npix);
    if (e == cudaSuccess) e = dev_alloc(v, (void**)&drec, sizeof(vol_trace_rec) * nrec);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dpix, pixels_host, sizeof(int) * 2 * npix, cudaMemcpyHostToDevice, v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(drec, 0, sizeof(vol_trace_rec) * nrec, v->stream);
    if (e == cudaSuccess) {
        t.pixels = dpix;
        t.out = drec;
        t.counts = dcnt;
        e = launch_trace(t, v->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, drec, sizeof(vol_trace_rec) * (size_t)npix * max_samples, cudaMemcpyDeviceToHost, v->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts_host, dcnt, sizeof(int) * npix, cudaMemcpyDeviceToHost, v->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->stream);
    cudaFree(dpix);
    cudaFree(dcnt);
    cudaFree(drec);
    if (e != cudaSuccess) return cuda_fail(v, e, "trace");
    return VOL_OK;
}

}  // extern "C"

// =====================================================================================
// Rendering without allocation (vol_render_noalloc).
//
// For callers that must not allocate device memory after set-up (a host application that
// hands out a fixed device-memory budget once, a render loop that must not stall in the
// allocator).  The per-call scratch of the render kernel -- its work counters and the view
// table -- lives in this file-scope device array instead of buffers the volume allocates on
// demand.  Every GPU that loads the library holds the array until the process exits.
// Host code must not use the array's name as an address (it names a host-side stand-in);
// the device address is looked up once per device with cudaGetSymbolAddress.
namespace {

constexpr size_t kNoallocCounterBytes = 256;  // kNumCounters words, padded
static_assert(sizeof(unsigned) * kNumCounters <= kNoallocCounterBytes, "counter area");
static_assert(kNoallocCounterBytes + sizeof(ViewDev) * VOL_NOALLOC_MAX_VIEWS <= VOL_NOALLOC_SCRATCH_BYTES,
              "scratch array too small for VOL_NOALLOC_MAX_VIEWS views");

static __device__ __align__(256) unsigned char g_noalloc_scratch[VOL_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 256;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoallocMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (set up on first use).
int noalloc_scratch(vol_t v, unsigned char** out) {
    int dev = 0;
    CK(v, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(v, VOL_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(v, e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        g_noalloc_addr[dev] = p;
    }
    *out = (unsigned char*)g_noalloc_addr[dev];
    return VOL_OK;
}

}  // namespace

extern "C" int vol_render_noalloc(vol_t v, const vol_camera* cams, int nviews, const float* tf_dev,
                                  const vol_params* params, float* rgba_dev, int32_t* nsamples_dev) {
    if (!v) return VOL_ERR_INVALID_ARG;
    if (int rc = ovl_settle(v)) return rc;  // no chunk of a preview still in generation
    if (!cams || !tf_dev || !params || !rgba_dev) return fail(v, VOL_ERR_INVALID_ARG, "null argument");
    if (nviews < 1 || nviews > VOL_NOALLOC_MAX_VIEWS)
        return fail(v, VOL_ERR_INVALID_ARG, "nviews must be 1..VOL_NOALLOC_MAX_VIEWS (64) for vol_render_noalloc");
    if (int rc = output_addresses(v, rgba_dev, nsamples_dev)) return rc;
    vol_params p = *params;
    if (!(p.step > 0.0f) || !std::isfinite(p.step)) return fail(v, VOL_ERR_INVALID_ARG, "step must be > 0");
    if (!samples_fit(v, p.step))
        return fail(v, VOL_ERR_INVALID_ARG, "step too small: more than 2^24 samples along the volume diagonal");
    if (p.tile_w <= 0) p.tile_w = 4;
    if (p.tile_h <= 0) p.tile_h = 8;
    if (p.tile_w > 4096 || p.tile_h > 4096 || p.tile_w * p.tile_h > 4096)
        return fail(v, VOL_ERR_INVALID_ARG, "tile_w * tile_h must be at most 4096");
    if (p.refill <= 0 || p.refill > 32) p.refill = default_refill(p.composite);
    if (p.lod_mode != 0 && p.lod_mode != 1) return fail(v, VOL_ERR_INVALID_ARG, "lod_mode must be 0 or 1");
    if (p.composite < VOL_COMPOSITE_DVR || p.composite > VOL_COMPOSITE_MIP)
        return fail(v, VOL_ERR_INVALID_ARG, "composite must be VOL_COMPOSITE_DVR, _MOP or _MIP");
    if (p.flags & VOL_RENDER_GRAD)
        return fail(v, VOL_ERR_UNSUPPORTED, "vol_render_noalloc keeps no gradient state; use vol_render");
    if ((p.flags & VOL_RENDER_LEVEL_STEP) && p.composite != VOL_COMPOSITE_DVR)
        return fail(v, VOL_ERR_UNSUPPORTED, "level-scaled sampling is for emission/absorption");
    if (v->sparse && (p.composite != VOL_COMPOSITE_DVR || (p.flags & VOL_RENDER_LEVEL_STEP)))
        return fail(v, VOL_ERR_UNSUPPORTED, "the sparse page table renders emission/absorption without "
                                            "level-scaled sampling");
    if (!all_resident(v, p.lod_mode != 0))
        return fail(v, VOL_ERR_UNSUPPORTED, "vol_render_noalloc needs every brick of the used levels resident");

    // the view table is staged in host memory the volume owns (not a local array), so the
    // source of the copy below outlives the call
    ViewDev* views = v->noalloc_views;
    int64_t rays = 0, tiles = 0;
    for (int i = 0; i < nviews; ++i) {
        const vol_camera& c = cams[i];
        if (c.w < 1 || c.h < 1 || c.w > 65536 || c.h > 65536) return fail(v, VOL_ERR_INVALID_ARG, "bad image size");
        if (!(c.tan_half_fov > 0.0f) || !std::isfinite(c.tan_half_fov))
            return fail(v, VOL_ERR_INVALID_ARG, "tan_half_fov must be > 0");
        ViewDev& V = views[i];
        V = ViewDev{};
        for (int a = 0; a < 3; ++a) {
            V.eye[a] = c.eye[a];
            V.right[a] = c.right[a];
            V.up[a] = c.up[a];
            V.fwd[a] = c.fwd[a];
        }
        V.tan = c.tan_half_fov;
        V.tan_aspect = c.tan_half_fov * c.aspect;
        V.lodscale = (2.0f * c.tan_half_fov) / (float)c.h;
        V.w = c.w;
        V.h = c.h;
        V.tiles_x = (c.w + p.tile_w - 1) / p.tile_w;
        V.tile_off = (int)tiles;
        V.ray_off = rays;
        const float D0f[3] = {(float)v->lay.dims[0], (float)v->lay.dims[1], (float)v->lay.dims[2]};
        view_cull_box(c, D0f, V);
        tiles += (int64_t)V.tiles_x * ((c.h + p.tile_h - 1) / p.tile_h);
        rays += (int64_t)c.w * c.h;
    }
    if (tiles >= (1ll << 31)) return fail(v, VOL_ERR_INVALID_ARG, "too many tiles");

    unsigned char* scratch = nullptr;
    if (int rc = noalloc_scratch(v, &scratch)) return rc;
    unsigned* counters = (unsigned*)scratch;
    ViewDev* views_dev = (ViewDev*)(scratch + kNoallocCounterBytes);
    // the array keeps the previous call's contents: the counters must start at zero
    CK(v, cudaMemcpyAsync(views_dev, views, sizeof(ViewDev) * nviews, cudaMemcpyHostToDevice, v->stream));
    CK(v, cudaMemsetAsync(counters, 0, sizeof(unsigned) * kNumCounters, v->stream));

    RenderDev r{};
    r.vol = vol_dev(v);
    r.views = views_dev;
    r.nviews = nviews;
    r.nwork = (int)tiles;
    r.resume = 0;
    r.tile_w = p.tile_w;
    r.tile_h = p.tile_h;
    r.refill_thresh = p.refill;
    r.tf = (const float4*)tf_dev;
    r.step = p.step;
    r.et = p.et_threshold;
    r.bg = make_float4(p.bg[0], p.bg[1], p.bg[2], p.bg[3]);
    r.lod_mode = p.lod_mode;
    r.lod_bias = p.lod_bias;
    r.skip_empty = (p.flags & VOL_RENDER_SKIP_EMPTY) ? 1 : 0;
    r.level_step = (p.flags & VOL_RENDER_LEVEL_STEP) ? 1 : 0;
    r.out = (float4*)rgba_dev;
    r.nsamp = nsamples_dev;
    r.counters = counters;
    r.nrays = rays;  // no request table, no suspension buffers, no usage stamps, no checkpoints
    const int grid = grid_for(v, v->dtype, false, p.ctas_per_sm);
    // the per-render counters describe this call, as they do after vol_render (the state a
    // gradient render left for vol_render_backward is not touched)
    v->stats = vol_stats{};
    v->stats.rays = rays;
    v->counters_collected = false;
    v->last_counters = counters;  // vol_get_stats reads this call's counters from the shared array
    CK(v, launch_render(v->dtype, render_mode(p, false), r, grid, v->stream));
    v->stats.launches = 1;
    v->stats.passes = 1;
    return VOL_OK;
}
