// Host side of the C ABI declared in include/tsdf.h: argument validation,
// device memory ownership, the tiered global chunk store (device memory,
// then pinned host memory, then optionally a file) and the launch sequence of
// each call. No float arithmetic of the method runs here
// beyond the per-map constants 1/voxel, QMAX/tau and K, derived once in
// binary64 and rounded to binary32.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "chunk_file.h"
#include "chunk_store.h"
#include "tsdf_internal.cuh"
#include "../../include/tsdf.h"

using namespace tsdf;

namespace {

thread_local int g_last_cuda_error = 0;

int cuda_fail(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return e == cudaErrorMemoryAllocation ? TSDF_ERR_OOM : TSDF_ERR_CUDA;
}

#define TSDF_CU(call)                          \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// Makes the map's device current for the scope of one call.
struct DeviceScope {
    int prev = -1;
    bool changed = false;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceScope() {
        if (changed) cudaSetDevice(prev);
    }
};

constexpr uint32_t kChunkBytes = 8 * 8 * 8 * 4;
constexpr uint32_t kSegChunks = 4096;   // 8 MiB store segments

bool is_pow2(int32_t v) { return v > 0 && (v & (v - 1)) == 0; }
int log2u(uint32_t v) {
    int s = 0;
    while ((1u << s) < v) ++s;
    return s;
}
long long floordiv8(long long v) { return v >= 0 ? v / 8 : -((-v + 7) / 8); }

const long long kOriginLimit = 1LL << 23;   // window voxels stay below 2^24: exact as float

enum KernelId { kRays = 0, kContrib = 1, kApply = 2, kShift = 3, kEmit = 4, kSort = 5, kNumKernels = 6 };
const char* const kKernelNames[kNumKernels] = {"rays", "contrib", "apply", "shift", "emit", "sort"};

struct Pending {
    int kernel;
    cudaEvent_t start, stop;
};

}  // namespace

struct tsdf_map {
    tsdf_params p;
    int device = 0;
    int num_sms = 1;
    float inv_vs = 0.f, qs = 0.f;
    int K = 0;
    WindowGeom geom{};
    long long origin[3] = {0, 0, 0};
    size_t voxels = 0;
    size_t bricks = 0;
    size_t ray_cap = 0;
    MapDev dev{};
    // global store of the 8^3 chunks outside the window that hold data: slots
    // in device memory (tier 0) and in pinned, device-mapped host memory
    // (tier 1), 4096 slots (8 MiB) per segment
    ChunkStore store;
    std::vector<char*> store_seg[2];     // device-visible address of each segment
    std::vector<char*> store_allocs[2];  // the allocations behind them (host tier: host pointers)
    std::vector<char*> store_seg_host;   // host tier: host address of each segment
    size_t store_dev_cap = 0;            // most device-tier slots (TSDF_OPT_STORE_DEVICE_CHUNKS; 0 = the window's bricks)
    uint32_t spill_age = 0;              // shifts after which a stored chunk moves to host memory (0: only when short)
    uint64_t shift_serial = 0;           // shifts done so far
    uint64_t chunks_spilled = 0;         // chunks moved from the device tier to the host tier
    uint64_t chunks_dropped = 0;         // leaving chunks found empty (not stored)
    // optional third tier (tsdf_map_set_store_file): at the start of a shift
    // the host tier keeps at most store_host_cap chunks, the older ones go to
    // the file, and entering file-tier chunks are read into host slots
    std::unique_ptr<ChunkFile> store_file;
    size_t store_host_cap = 0;
    uint64_t chunks_to_file = 0;         // chunks moved from the host tier to the file
    uint64_t chunks_from_file = 0;       // file-tier chunks read back on re-entry
    // per shift item: the candidate the kernel claimed for the leaving brick,
    // or -1 (pinned host memory written by the kernel in place)
    int* claim_host = nullptr;
    int* claim_dev = nullptr;            // its device-visible address
    size_t flags_cap = 0;
    cudaEvent_t flags_event = nullptr;   // the last shift's claims have reached claim_host
    std::vector<ChunkKey> leave_keys;    // the shift's leaving chunks, in item order
    std::vector<uint32_t> cand_locs;     // their candidate slots
    ChunkCopy* spill_dev = nullptr;      // copies device slot -> host slot of one shift
    ChunkCopy* spill_host = nullptr;
    size_t spill_cap = 0;
    cudaEvent_t spill_event = nullptr;   // the copy list of the last spill has been read
    bool spill_pending = false;
    ShiftItem* items_dev = nullptr;
    size_t items_dev_cap = 0;
    ShiftItem* items_host = nullptr;
    size_t items_host_cap = 0;
    cudaEvent_t items_event = nullptr;
    bool items_event_pending = false;
    // staging for host-resident points
    float4* stage_dev = nullptr;
    size_t stage_cap = 0;
    // tuning options
    bool merge = false;             // warp match-merge before the accumulator atomics
    int kpt = 4;                    // march steps per contribution item (1, 2 or 4)
    bool pdl = true;                // programmatic dependent launch between the scan's kernels
    int reduction = TSDF_REDUCTION_ATOMIC;   // per-scan reduction: accumulator atomics or sort
    bool zero_copy = true;          // tsdf_integrate_host reads device-mapped pinned points in place
    // The plain path's four launches as one CUDA graph (TSDF_OPT_LAUNCH_GRAPH):
    // captured on first use, then per scan the ray and contribution nodes get
    // the scan's arguments and the graph is launched once. Off by default: it
    // cuts the host's time per scan from about 9 to 3.5 us, but back-to-back
    // scans took 28.8 instead of 26.1 us on the device (the programmatic
    // overlap of one scan's last kernel with the next scan's first is lost).
    bool use_graph = false;
    bool graph_broken = false;      // capture or instantiation failed: plain launches from then on
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t chain_graph = nullptr;
    cudaGraphExec_t chain_exec = nullptr;
    cudaGraphNode_t node_rays = nullptr;
    cudaGraphNode_t node_contrib = nullptr;
    cudaKernelNodeParams kp_rays{};
    cudaKernelNodeParams kp_contrib{};
    MapDev chain_dev{};             // the buffers and options the graph was captured with
    int chain_kpt = 0;
    bool chain_merge = false;
    bool chain_pdl = false;
    long long* host_last = nullptr; // mapped pinned copy of the published counters (host address)
    double* reg_dev = nullptr;      // registration: the 29 sums of the normal equations
    size_t pair_cap_req = 0;        // sort reduction: requested pair capacity, 0 = from the scan size
    size_t pool_req = 0;            // pool reduction: requested slots, 0 = default
    // TSDF_REDUCTION_AUTO: the atomic, sort and pool reductions are timed on
    // the first calls (one untimed call each, then kAutoTrials timed) and the
    // fastest is kept
    static constexpr int kAutoCandidates = 3;
    static constexpr int kAutoTrials = 3;
    static constexpr int kAutoReduction[kAutoCandidates] = {TSDF_REDUCTION_ATOMIC, TSDF_REDUCTION_SORT,
                                                            TSDF_REDUCTION_POOL};
    struct AutoTrial {
        int candidate;
        cudaEvent_t start, stop;
    };
    std::vector<AutoTrial> auto_trials;
    int auto_started[kAutoCandidates] = {};
    int auto_timed[kAutoCandidates] = {};
    float auto_best[kAutoCandidates] = {};
    int auto_choice = -1;           // decided reduction, -1 while tuning
    size_t ray_slot_cap = 0;        // entries of dev.ray_slot
    // optional per-kernel event timing
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<Pending> pending;
    int64_t prof_launches[kNumKernels] = {};
    double prof_ms[kNumKernels] = {};
};

namespace {

int validate_params(const tsdf_params* p) {
    if (!p) return TSDF_ERR_INVALID;
    unsigned long long prod = 1;
    for (int a = 0; a < 3; ++a) {
        if (!is_pow2(p->dims[a]) || p->dims[a] < 8 || p->dims[a] > 32768) return TSDF_ERR_INVALID;
        prod *= (unsigned long long)p->dims[a];
        if (p->origin[a] % 8 != 0 || p->origin[a] > kOriginLimit || p->origin[a] < -kOriginLimit)
            return TSDF_ERR_INVALID;
    }
    if (prod > (1ull << 31)) return TSDF_ERR_INVALID;
    if (!std::isfinite(p->voxel_size) || !(p->voxel_size > 0.f)) return TSDF_ERR_INVALID;
    if (!std::isfinite(p->tau) || !(p->tau >= p->voxel_size) || (double)p->tau / p->voxel_size > 1024.0)
        return TSDF_ERR_INVALID;
    if (p->w_max < 1 || p->w_max > 32767) return TSDF_ERR_INVALID;
    if (!std::isfinite(p->delta_z) || p->delta_z < 0.f || p->delta_z > 1.f) return TSDF_ERR_INVALID;
    if (!std::isfinite(p->r_min) || !std::isfinite(p->r_max) || p->r_min < 0.f || p->r_max < p->r_min ||
        p->r_max > 1e5f)
        return TSDF_ERR_INVALID;
    if ((double)p->delta_z * ((double)p->r_max + p->tau) / p->voxel_size > 1e6) return TSDF_ERR_INVALID;
    if (p->reduce != TSDF_REDUCE_WSUM && p->reduce != TSDF_REDUCE_MIN_ABS) return TSDF_ERR_INVALID;
    if ((p->flags & ~(TSDF_FLAG_STEP_VALUE | TSDF_FLAG_SCAN_WEIGHT)) != 0) return TSDF_ERR_INVALID;
    return TSDF_OK;
}

cudaEvent_t take_event(tsdf_map* m) {
    if (!m->ev_pool.empty()) {
        cudaEvent_t e = m->ev_pool.back();
        m->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records an event on `s` when profiling; returns nullptr otherwise.
cudaEvent_t prof_mark(tsdf_map* m, cudaStream_t s) {
    if (!m->prof) return nullptr;
    cudaEvent_t e = take_event(m);
    if (e && cudaEventRecord(e, s) != cudaSuccess) {
        m->ev_pool.push_back(e);
        return nullptr;
    }
    return e;
}

void prof_push(tsdf_map* m, int kernel, cudaEvent_t a, cudaEvent_t b) {
    if (a && b) {
        m->pending.push_back(Pending{kernel, a, b});
        return;
    }
    if (a) m->ev_pool.push_back(a);
    if (b) m->ev_pool.push_back(b);
}

int prof_drain(tsdf_map* m) {
    for (const Pending& p : m->pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(p.stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.start, p.stop);
        if (e != cudaSuccess) return cuda_fail(e);
        m->prof_launches[p.kernel] += 1;
        m->prof_ms[p.kernel] += ms;
        m->ev_pool.push_back(p.start);
        m->ev_pool.push_back(p.stop);
    }
    m->pending.clear();
    return TSDF_OK;
}

static void chain_graph_reset(tsdf_map* m) {
    if (m->chain_exec) cudaGraphExecDestroy(m->chain_exec);
    if (m->chain_graph) cudaGraphDestroy(m->chain_graph);
    m->chain_exec = nullptr;
    m->chain_graph = nullptr;
    m->node_rays = m->node_contrib = nullptr;
}

void free_map(tsdf_map* m) {
    if (!m) return;
    chain_graph_reset(m);
    if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
    for (const Pending& p : m->pending) {
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
    }
    for (cudaEvent_t e : m->ev_pool) cudaEventDestroy(e);
    for (auto& t : m->auto_trials) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    cudaFree(m->dev.grid);
    cudaFree(m->dev.acc);
    cudaFree(m->dev.brick_flag);
    cudaFree(m->dev.brick_list);
    cudaFree(m->dev.ray_a);
    cudaFree(m->dev.ray_b);
    cudaFree(m->dev.ctr);
    if (m->host_last) cudaFreeHost(m->host_last);
    cudaFree(m->reg_dev);
    cudaFree(m->dev.pool_table);
    cudaFree(m->dev.pool_brick);
    cudaFree(m->dev.pool_acc);
    cudaFree(m->dev.brick_slot);
    cudaFree(m->dev.seg_count);
    cudaFree(m->dev.seg_start);
    cudaFree(m->dev.ray_slot);
    cudaFree(m->dev.pairs);
    cudaFree(m->dev.sorted);
    for (char* a : m->store_allocs[0]) cudaFree(a);
    for (char* a : m->store_allocs[1]) cudaFreeHost(a);
    if (m->claim_host) cudaFreeHost(m->claim_host);
    if (m->flags_event) cudaEventDestroy(m->flags_event);
    cudaFree(m->spill_dev);
    if (m->spill_host) cudaFreeHost(m->spill_host);
    if (m->spill_event) cudaEventDestroy(m->spill_event);
    cudaFree(m->items_dev);
    if (m->items_host) cudaFreeHost(m->items_host);
    if (m->items_event) cudaEventDestroy(m->items_event);
    cudaFree(m->stage_dev);
    delete m;
}

bool box_inside(const tsdf_map* m, const int64_t lo[3], const int64_t hi[3], uint32_t box[3]) {
    for (int a = 0; a < 3; ++a) {
        if (lo[a] < m->origin[a] || hi[a] > m->origin[a] + m->p.dims[a] || hi[a] < lo[a]) return false;
        box[a] = (uint32_t)(hi[a] - lo[a]);
    }
    return true;
}

// Most device-tier slots of the map's store.
size_t store_dev_limit(const tsdf_map* m) { return m->store_dev_cap ? m->store_dev_cap : m->bricks; }

// Device-visible address of a store location.
unsigned long long store_addr(const tsdf_map* m, uint32_t loc) {
    const int t = ChunkStore::is_host(loc) ? 1 : 0;
    const uint32_t slot = ChunkStore::slot_of(loc);
    return (unsigned long long)(m->store_seg[t][slot / kSegChunks] + (size_t)(slot % kSegChunks) * kChunkBytes);
}

// Host address of a host-tier location.
char* store_host_ptr(const tsdf_map* m, uint32_t loc) {
    const uint32_t slot = ChunkStore::slot_of(loc);
    return m->store_seg_host[slot / kSegChunks] + (size_t)(slot % kSegChunks) * kChunkBytes;
}

// Adds `segs` segments to a tier: device memory, or pinned host memory mapped
// into the device's address space. Returns false when the allocation fails.
bool store_grow(tsdf_map* m, int tier, size_t segs) {
    const size_t bytes = segs * (size_t)kSegChunks * kChunkBytes;
    char* base = nullptr;
    char* dev = nullptr;
    if (tier == 0) {
        if (cudaMalloc(&base, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        dev = base;
    } else {
        if (cudaHostAlloc(&base, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        void* dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, base, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(base);
            return false;
        }
        dev = static_cast<char*>(dp);
    }
    const uint32_t first = (uint32_t)(m->store_seg[tier].size() * kSegChunks);
    m->store_allocs[tier].push_back(base);
    for (size_t i = 0; i < segs; ++i) {
        m->store_seg[tier].push_back(dev + i * (size_t)kSegChunks * kChunkBytes);
        if (tier == 1) m->store_seg_host.push_back(base + i * (size_t)kSegChunks * kChunkBytes);
    }
    m->store.add_slots(tier, first, (uint32_t)(segs * kSegChunks));
    return true;
}


// Takes the previous shift's claims (waiting for them if needed): the leaving
// chunks that held data are recorded, the other candidate slots freed.
int store_resolve(tsdf_map* m) {
    if (!m->store.pending()) return TSDF_OK;
    TSDF_CU(cudaEventSynchronize(m->flags_event));
    const size_t n = m->leave_keys.size();
    m->chunks_dropped += n - m->store.commit(m->claim_host);
    return TSDF_OK;
}

// File tier, at the start of a shift (after store_resolve): the host tier's
// chunks beyond its limit move to the file, oldest first. Host slots are
// written by the device (shift kernel, tier copies), so the last shift's work
// is waited for before any is read here.
int store_trim_host(tsdf_map* m) {
    if (!m->store_file || m->store.used(1) <= m->store_host_cap) return TSDF_OK;
    TSDF_CU(cudaEventSynchronize(m->flags_event));
    while (m->store.used(1) > m->store_host_cap) {
        if (m->store.free_count(2) == 0) {
            if (m->store.capacity(2) + kSegChunks > ((size_t)1 << 30)) return TSDF_ERR_OOM;
            m->store.add_slots(2, (uint32_t)m->store.capacity(2), (uint32_t)kSegChunks);   // the file grows
        }
        uint32_t from = 0, to = 0;
        if (!m->store.spill_oldest_host(&from, &to)) break;
        if (!m->store_file->put(ChunkStore::slot_of(to), store_host_ptr(m, from))) return TSDF_ERR_IO;
        ++m->chunks_to_file;
    }
    return TSDF_OK;
}

// Bookkeeping buffers of a shift moving `cnt` bricks: the item list (pinned
// and device), the per-item flags (device and pinned) and the list of
// device -> host chunk copies (as many as the device tier has slots).
int ensure_shift_buffers(tsdf_map* m, size_t cnt) {
    if (m->items_event_pending && cnt > m->items_host_cap) {
        TSDF_CU(cudaEventSynchronize(m->items_event));
        m->items_event_pending = false;
    }
    // items: entry 0 is a header whose first word is the kernel's claim
    // counter (zero in every copy), entries 1..cnt the moved bricks
    if (cnt > m->items_host_cap) {
        if (m->items_host) cudaFreeHost(m->items_host);
        m->items_host = nullptr;
        m->items_host_cap = 0;
        TSDF_CU(cudaMallocHost(&m->items_host, (cnt + 1) * sizeof(ShiftItem)));
        m->items_host_cap = cnt;
    }
    if (cnt > m->items_dev_cap || cnt > m->flags_cap) {
        int rc = store_resolve(m);   // the claims still to be read live in these buffers
        if (rc != TSDF_OK) return rc;
        cudaFree(m->items_dev);   // waits for the device
        if (m->claim_host) cudaFreeHost(m->claim_host);
        m->items_dev = nullptr;
        m->claim_host = nullptr;
        m->claim_dev = nullptr;
        m->items_dev_cap = 0;
        m->flags_cap = 0;
        TSDF_CU(cudaMalloc(&m->items_dev, (cnt + 1) * sizeof(ShiftItem)));
        m->items_dev_cap = cnt;
        TSDF_CU(cudaHostAlloc(&m->claim_host, cnt * sizeof(int), cudaHostAllocMapped));
        void* dp = nullptr;
        TSDF_CU(cudaHostGetDevicePointer(&dp, m->claim_host, 0));
        m->claim_dev = static_cast<int*>(dp);
        m->flags_cap = cnt;
    }
    // (the copy list exists once chunks can move: the device tier is at its
    // limit, or chunks move by age)
    const size_t limit = store_dev_limit(m);
    const size_t moves = (m->store.capacity(0) >= limit || m->spill_age > 0) ? std::max(limit, m->store.capacity(0)) : 0;
    if (moves > m->spill_cap) {
        if (m->spill_pending) TSDF_CU(cudaEventSynchronize(m->spill_event));   // the old list has been read
        m->spill_pending = false;
        cudaFree(m->spill_dev);   // waits for the device
        if (m->spill_host) cudaFreeHost(m->spill_host);
        m->spill_dev = nullptr;
        m->spill_host = nullptr;
        m->spill_cap = 0;
        TSDF_CU(cudaMalloc(&m->spill_dev, moves * sizeof(ChunkCopy)));
        TSDF_CU(cudaMallocHost(&m->spill_host, moves * sizeof(ChunkCopy)));
        m->spill_cap = moves;
    }
    return TSDF_OK;
}

// Makes room for `need` leaving chunks before a shift: the device tier grows
// up to its limit, then its oldest chunks move to the host tier (as do chunks
// stored more than spill_age shifts ago), and the host tier takes whatever
// the device tier cannot. The moves are copies on `s`, issued before the
// shift kernel, so the device slots they free can be reused by this shift.
int store_make_room(tsdf_map* m, size_t need, cudaStream_t s) {
    const size_t limit = store_dev_limit(m);
    while (m->store.free_count(0) < need && m->store.capacity(0) < limit) {
        const size_t room = (limit - m->store.capacity(0) + kSegChunks - 1) / kSegChunks;
        size_t segs = (size_t)1 << std::min<size_t>(5, m->store_allocs[0].size());   // 1, 2, 4 ... 32 at a time
        segs = std::min(segs, room);
        if (!store_grow(m, 0, segs) && !(segs > 1 && store_grow(m, 0, 1))) break;   // short of memory: spill
    }
    int rc = ensure_shift_buffers(m, 0);   // the copy list, once chunks can move
    if (rc != TSDF_OK) return rc;
    std::vector<ChunkCopy> moves;
    auto host_slot = [&]() -> bool {
        return m->store.free_count(1) > 0 || store_grow(m, 1, 1);
    };
    // (a move is recorded in the index as it is planned, so every planned move
    // is launched below, also when the host tier cannot grow further)
    rc = TSDF_OK;
    // chunks stored too long ago
    if (m->spill_age > 0) {
        ChunkKey k;
        uint32_t loc;
        uint64_t stamp;
        while (m->store.oldest_device(&k, &loc, &stamp) && stamp + m->spill_age <= m->shift_serial) {
            if (!host_slot()) {
                rc = TSDF_ERR_OOM;
                break;
            }
            uint32_t from = 0, to = 0;
            if (!m->store.spill_oldest(&from, &to)) break;
            moves.push_back(ChunkCopy{store_addr(m, to), store_addr(m, from)});
        }
    }
    // room on the device tier for this shift's chunks
    while (rc == TSDF_OK && m->store.free_count(0) < need) {
        if (!host_slot()) {
            rc = TSDF_ERR_OOM;
            break;
        }
        uint32_t from = 0, to = 0;
        if (!m->store.spill_oldest(&from, &to)) break;
        moves.push_back(ChunkCopy{store_addr(m, to), store_addr(m, from)});
    }
    // whatever the device tier cannot take goes to the host tier
    const size_t dev_free = m->store.free_count(0);
    while (rc == TSDF_OK && dev_free + m->store.free_count(1) < need) {
        if (!store_grow(m, 1, (need - dev_free - m->store.free_count(1) + kSegChunks - 1) / kSegChunks))
            rc = TSDF_ERR_OOM;
    }
    if (!moves.empty()) {
        if (moves.size() > m->spill_cap) return TSDF_ERR_OOM;   // not reached: moves <= device-tier chunks
        if (m->spill_pending) TSDF_CU(cudaEventSynchronize(m->spill_event));   // the last copy list is read
        std::memcpy(m->spill_host, moves.data(), moves.size() * sizeof(ChunkCopy));
        TSDF_CU(cudaMemcpyAsync(m->spill_dev, m->spill_host, moves.size() * sizeof(ChunkCopy), cudaMemcpyHostToDevice, s));
        TSDF_CU(cudaEventRecord(m->spill_event, s));
        m->spill_pending = true;
        TSDF_CU(launch_copy_chunks(m->spill_dev, (int)moves.size(), s));
        m->chunks_spilled += moves.size();
    }
    return rc;
}

}  // namespace

extern "C" {

int tsdf_map_create(const tsdf_params* params, tsdf_map** out) {
    if (!out) return TSDF_ERR_INVALID;
    *out = nullptr;
    int rc = validate_params(params);
    if (rc != TSDF_OK) return rc;
    tsdf_map* m = new tsdf_map();
    m->p = *params;
    TSDF_CU(cudaGetDevice(&m->device));
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
    if (m->num_sms < 1) m->num_sms = 1;
    m->inv_vs = (float)(1.0 / (double)params->voxel_size);
    m->qs = (float)((double)kQMax / (double)params->tau);
    m->K = (int)std::floor((double)params->tau / (double)params->voxel_size + 1e-9);
    for (int a = 0; a < 3; ++a) {
        m->geom.dims[a] = (uint32_t)params->dims[a];
        m->geom.cmask[a] = (uint32_t)params->dims[a] / 8u - 1u;
        m->origin[a] = params->origin[a];
    }
    m->geom.lcx = (uint32_t)log2u((uint32_t)params->dims[0] / 8u);
    m->geom.lcxy = m->geom.lcx + (uint32_t)log2u((uint32_t)params->dims[1] / 8u);
    m->voxels = (size_t)params->dims[0] * params->dims[1] * params->dims[2];
    m->bricks = m->voxels / kBrickVoxels;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&m->dev.grid, m->voxels * sizeof(uint32_t));
    const size_t flag_bytes = (m->bricks + 3) / 4 * 4;
    if (e == cudaSuccess) e = cudaMalloc(&m->dev.brick_flag, flag_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&m->dev.brick_list, m->bricks * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&m->dev.ctr, sizeof(MapCounters));
    if (e == cudaSuccess) e = cudaMemset(m->dev.grid, 0, m->voxels * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(m->dev.brick_flag, 0, flag_bytes);
    if (e == cudaSuccess) e = cudaMemset(m->dev.ctr, 0, sizeof(MapCounters));
    // published counters mirrored into mapped pinned memory (falls back to a
    // device-to-host copy in tsdf_stats when the mapping is unavailable)
    if (e == cudaSuccess && cudaHostAlloc(&m->host_last, 4 * sizeof(long long), cudaHostAllocMapped) == cudaSuccess) {
        std::memset(m->host_last, 0, 4 * sizeof(long long));
        void* dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, m->host_last, 0) == cudaSuccess) {
            m->dev.host_last = static_cast<long long*>(dp);
        } else {
            cudaFreeHost(m->host_last);
            m->host_last = nullptr;
        }
    } else {
        m->host_last = nullptr;
        cudaGetLastError();   // clear a failed mapping request
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->items_event, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->flags_event, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->spill_event, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_map(m);
        return cuda_fail(e);
    }
    *out = m;
    return TSDF_OK;
}

int tsdf_map_destroy(tsdf_map* map) {
    if (!map) return TSDF_OK;
    DeviceScope ds(map->device);
    cudaDeviceSynchronize();
    free_map(map);
    return TSDF_OK;
}

// The dense per-scan accumulator (8 B per voxel, all zero between scans) is
// allocated on the first call that needs it: the atomic and sort reductions,
// batches and sessions. A map used only with the pool reduction never holds it.
static int ensure_acc(tsdf_map* map) {
    if (map->dev.acc) return TSDF_OK;
    unsigned long long* a = nullptr;
    TSDF_CU(cudaMalloc(&a, map->voxels * sizeof(unsigned long long)));
    cudaError_t e = cudaMemset(a, 0, map->voxels * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(a);
        return cuda_fail(e);
    }
    map->dev.acc = a;
    return TSDF_OK;
}

// Pool reduction: the brick -> slot table (all empty), the per-slot brick ids
// and the slot accumulators (all zero). Default capacity: an eighth of the
// window's bricks, at least 16384 and at most all of them.
static int ensure_pool(tsdf_map* map) {
    size_t want = map->pool_req;
    if (want == 0) {
        want = map->bricks / 8;
        if (want < 16384) want = 16384;
    }
    if (want > map->bricks) want = map->bricks;
    if (map->dev.pool_table && want == map->dev.pool_cap) return TSDF_OK;
    TSDF_CU(cudaDeviceSynchronize());   // an earlier scan may still use the old pool
    cudaFree(map->dev.pool_table);
    cudaFree(map->dev.pool_brick);
    cudaFree(map->dev.pool_acc);
    map->dev.pool_table = nullptr;
    map->dev.pool_brick = nullptr;
    map->dev.pool_acc = nullptr;
    map->dev.pool_cap = 0;
    TSDF_CU(cudaMalloc(&map->dev.pool_table, map->bricks * sizeof(uint32_t)));
    TSDF_CU(cudaMemset(map->dev.pool_table, 0xFF, map->bricks * sizeof(uint32_t)));
    TSDF_CU(cudaMalloc(&map->dev.pool_brick, want * sizeof(uint32_t)));
    TSDF_CU(cudaMalloc(&map->dev.pool_acc, want * kBrickVoxels * sizeof(unsigned long long)));
    TSDF_CU(cudaMemset(map->dev.pool_acc, 0, want * kBrickVoxels * sizeof(unsigned long long)));
    map->dev.pool_cap = (uint32_t)want;
    return TSDF_OK;
}

static int ensure_rays(tsdf_map* map, int64_t n) {
    if ((size_t)n <= map->ray_cap) return TSDF_OK;
    // a previous scan may still read the old buffers: cudaFree waits for the device
    cudaFree(map->dev.ray_a);
    cudaFree(map->dev.ray_b);
    map->dev.ray_a = map->dev.ray_b = nullptr;
    map->ray_cap = 0;
    map->dev.ray_cap = 0;
    size_t cap = 1024;
    while (cap < (size_t)n) cap *= 2;
    TSDF_CU(cudaMalloc(&map->dev.ray_a, cap * sizeof(float4)));
    TSDF_CU(cudaMalloc(&map->dev.ray_b, cap * sizeof(float4)));
    map->ray_cap = cap;
    map->dev.ray_cap = (uint32_t)cap;
    return TSDF_OK;
}

// Sort-reduction buffers: per-brick arrays once, per-ray slots with the ray
// buffers, pairs for `n` points (32 slots per point, at least 2^20, at most
// kPairCapMax, unless a capacity was requested). Growing waits for the device.
static int ensure_sort(tsdf_map* map, int64_t n) {
    if (!map->dev.brick_slot) {
        TSDF_CU(cudaMalloc(&map->dev.brick_slot, map->bricks * sizeof(uint32_t)));
        TSDF_CU(cudaMalloc(&map->dev.seg_count, map->bricks * sizeof(uint32_t)));
        TSDF_CU(cudaMalloc(&map->dev.seg_start, map->bricks * sizeof(uint32_t)));
        TSDF_CU(cudaMemset(map->dev.seg_count, 0, map->bricks * sizeof(uint32_t)));
    }
    if (map->ray_slot_cap < map->ray_cap) {
        cudaFree(map->dev.ray_slot);
        map->dev.ray_slot = nullptr;
        map->ray_slot_cap = 0;
        TSDF_CU(cudaMalloc(&map->dev.ray_slot, map->ray_cap * sizeof(uint32_t)));
        map->ray_slot_cap = map->ray_cap;
    }
    size_t want = map->pair_cap_req;
    if (want == 0) {
        want = (size_t)1 << 20;
        while (want < 32 * (size_t)n && want < kPairCapMax) want *= 2;
    }
    if (want != map->dev.pair_cap && (map->pair_cap_req != 0 || want > map->dev.pair_cap)) {
        cudaFree(map->dev.pairs);
        cudaFree(map->dev.sorted);
        map->dev.pairs = nullptr;
        map->dev.sorted = nullptr;
        map->dev.pair_cap = 0;
        TSDF_CU(cudaMalloc(&map->dev.pairs, want * sizeof(uint2)));
        TSDF_CU(cudaMalloc(&map->dev.sorted, want * sizeof(uint32_t)));
        map->dev.pair_cap = (uint32_t)want;
    }
    return TSDF_OK;
}

static void fill_scan_args(const tsdf_map* map, const float* points_dev, int64_t n, const float pose[12], ScanArgs& a) {
    a = ScanArgs{};
    a.pts = reinterpret_cast<const float4*>(points_dev);
    a.n = (int32_t)n;
    a.K = map->K;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) a.R[r * 3 + c] = pose[r * 4 + c];
        a.t[r] = pose[r * 4 + 3];
    }
    a.vs = map->p.voxel_size;
    a.inv_vs = map->inv_vs;
    a.tau = map->p.tau;
    a.qs = map->qs;
    a.dz = map->p.delta_z;
    a.rmin = map->p.r_min;
    a.rmax = map->p.r_max;
    a.fill = map->p.delta_z > 0.f ? 1 : 0;
    for (int ax = 0; ax < 3; ++ax) {
        const double lo = (double)map->origin[ax] * (double)map->p.voxel_size;
        const double hi = (double)(map->origin[ax] + map->p.dims[ax]) * (double)map->p.voxel_size;
        a.win_lo[ax] = std::nextafter((float)lo, -INFINITY);
        a.win_hi[ax] = std::nextafter((float)hi, INFINITY);
        a.fo[ax] = (float)map->origin[ax];
        a.fe[ax] = (float)(map->origin[ax] + map->p.dims[ax]);
        a.cmask[ax] = map->geom.cmask[ax];
        a.dmask[ax] = (uint32_t)map->p.dims[ax] - 1u;
        a.omod[ax] = (uint32_t)((unsigned long long)map->origin[ax] & (unsigned long long)(map->p.dims[ax] - 1));
    }
    a.lcx = map->geom.lcx;
    a.lcxy = map->geom.lcxy;
    a.flags = map->p.flags;
    fill_lean_args(a);
}

static_assert(sizeof(MapDev) == 160, "same_dev compares every field of MapDev");
static bool same_dev(const MapDev& x, const MapDev& y) {
    return x.grid == y.grid && x.acc == y.acc && x.brick_flag == y.brick_flag && x.brick_list == y.brick_list &&
           x.ray_a == y.ray_a && x.ray_b == y.ray_b && x.ray_cap == y.ray_cap && x.ctr == y.ctr &&
           x.host_last == y.host_last && x.brick_slot == y.brick_slot && x.seg_count == y.seg_count &&
           x.seg_start == y.seg_start && x.ray_slot == y.ray_slot && x.pairs == y.pairs && x.sorted == y.sorted &&
           x.pair_cap == y.pair_cap && x.pool_table == y.pool_table && x.pool_brick == y.pool_brick &&
           x.pool_acc == y.pool_acc && x.pool_cap == y.pool_cap;
}

// Capture the plain atomic path (rays, contribution, compaction, apply with
// the map's options) into chain_graph and instantiate it; false when any step
// fails (nothing is left half built).
static bool chain_graph_build(tsdf_map* map, const ScanArgs& a) {
    chain_graph_reset(map);
    if (!map->capture_stream &&
        cudaStreamCreateWithFlags(&map->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        map->capture_stream = nullptr;
        cudaGetLastError();
        return false;
    }
    cudaStream_t cs = map->capture_stream;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const MapDev& d = map->dev;
    cudaError_t e = launch_rays(a, d, false, true, map->pdl, cs);
    if (e == cudaSuccess) e = launch_contrib(a, d, map->p.reduce, map->merge, map->kpt, map->pdl, cs);
    if (e == cudaSuccess) e = launch_compact(d, (uint32_t)map->bricks, map->pdl, cs);
    if (e == cudaSuccess) e = launch_apply(d, map->p.reduce, map->p.w_max, map->p.flags, map->pdl, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess || ee != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    // the two kernel nodes whose arguments change from scan to scan
    const void* fr = rays_kernel_fn(false, true);
    const void* fc = contrib_kernel_fn(map->p.reduce, map->merge, map->kpt);
    size_t nn = 0;
    std::vector<cudaGraphNode_t> nodes;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        nodes.resize(nn);
        if (cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) nodes.clear();
    }
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType t;
        cudaKernelNodeParams kp{};
        if (cudaGraphNodeGetType(node, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        if (cudaGraphKernelNodeGetParams(node, &kp) != cudaSuccess) continue;
        if (kp.func == fr) {
            map->node_rays = node;
            map->kp_rays = kp;
        } else if (kp.func == fc) {
            map->node_contrib = node;
            map->kp_contrib = kp;
        }
    }
    cudaGraphExec_t x = nullptr;
    if (!map->node_rays || !map->node_contrib || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
        map->node_rays = map->node_contrib = nullptr;
        cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    map->chain_graph = g;
    map->chain_exec = x;
    map->chain_dev = map->dev;
    map->chain_kpt = map->kpt;
    map->chain_merge = map->merge;
    map->chain_pdl = map->pdl;
    return true;
}

// The plain atomic path through the captured graph: *launched tells whether
// the scan went to the stream (else the caller launches the kernels itself:
// the stream is being captured by the caller, or the graph could not be built
// or updated, which turns the graph off for this map).
static int chain_graph_launch(tsdf_map* map, const ScanArgs& a, cudaStream_t s, bool* launched) {
    *launched = false;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return TSDF_OK;
    }
    if (cap != cudaStreamCaptureStatusNone) return TSDF_OK;
    if (map->chain_exec && (!same_dev(map->chain_dev, map->dev) ||
                            map->chain_kpt != map->kpt || map->chain_merge != map->merge ||
                            map->chain_pdl != map->pdl))
        chain_graph_reset(map);
    if (!map->chain_exec && !chain_graph_build(map, a)) {
        map->graph_broken = true;
        return TSDF_OK;
    }
    void* args[2] = {const_cast<ScanArgs*>(&a), &map->dev};
    cudaKernelNodeParams kr = map->kp_rays;
    kr.gridDim = dim3(rays_grid(a.n, false));
    kr.kernelParams = args;
    kr.extra = nullptr;
    cudaKernelNodeParams kc = map->kp_contrib;
    kc.kernelParams = args;
    kc.extra = nullptr;
    if (cudaGraphExecKernelNodeSetParams(map->chain_exec, map->node_rays, &kr) != cudaSuccess ||
        cudaGraphExecKernelNodeSetParams(map->chain_exec, map->node_contrib, &kc) != cudaSuccess) {
        cudaGetLastError();
        chain_graph_reset(map);
        map->graph_broken = true;
        return TSDF_OK;
    }
    *launched = true;
    TSDF_CU(cudaGraphLaunch(map->chain_exec, s));
    return TSDF_OK;
}

static int integrate_with(tsdf_map* map, const float* points_dev, int64_t n, const float pose[12], cudaStream_t s,
                          int reduction) {
    int rc = ensure_rays(map, n);
    if (rc != TSDF_OK) return rc;
    ScanArgs a;
    fill_scan_args(map, points_dev, n, pose, a);
    const bool pdl = map->pdl;
    if (reduction == TSDF_REDUCTION_POOL) {
        rc = ensure_pool(map);
        if (rc != TSDF_OK) return rc;
        const MapDev& d = map->dev;
        cudaEvent_t e0 = n > 0 ? prof_mark(map, s) : nullptr;
        TSDF_CU(launch_rays(a, d, false, false, pdl, s));
        cudaEvent_t e1 = n > 0 ? prof_mark(map, s) : nullptr;
        cudaEvent_t e2 = n > 0 ? prof_mark(map, s) : nullptr;
        TSDF_CU(launch_pool_contrib(a, d, map->p.reduce, map->kpt, pdl, s));
        cudaEvent_t e3 = n > 0 ? prof_mark(map, s) : nullptr;
        cudaEvent_t e4 = prof_mark(map, s);
        TSDF_CU(launch_pool_apply(d, map->p.reduce, map->p.w_max, map->p.flags, pdl, s));   // + counters
        cudaEvent_t e5 = prof_mark(map, s);
        prof_push(map, kRays, e0, e1);
        prof_push(map, kContrib, e2, e3);
        prof_push(map, kApply, e4, e5);
        return TSDF_OK;
    }
    rc = ensure_acc(map);
    if (rc != TSDF_OK) return rc;
    if (reduction == TSDF_REDUCTION_SORT) {
        rc = ensure_sort(map, n);
        if (rc != TSDF_OK) return rc;
        const MapDev& d = map->dev;
        cudaEvent_t e0 = n > 0 ? prof_mark(map, s) : nullptr;
        TSDF_CU(launch_rays(a, d, true, false, pdl, s));
        cudaEvent_t e1 = n > 0 ? prof_mark(map, s) : nullptr;
        cudaEvent_t e2 = n > 0 ? prof_mark(map, s) : nullptr;
        TSDF_CU(launch_emit(a, d, map->p.reduce, map->kpt, pdl, s));
        cudaEvent_t e3 = n > 0 ? prof_mark(map, s) : nullptr;
        cudaEvent_t e4 = prof_mark(map, s);
        TSDF_CU(launch_compact(d, (uint32_t)map->bricks, pdl, s));
        TSDF_CU(launch_sort_count(d, pdl, s));
        TSDF_CU(launch_sort_scan(d, pdl, s));
        TSDF_CU(launch_sort_scatter(d, pdl, s));
        cudaEvent_t e5 = prof_mark(map, s);
        cudaEvent_t e6 = prof_mark(map, s);
        TSDF_CU(launch_sort_apply(d, map->p.reduce, map->p.w_max, map->p.flags, pdl, s));   // + counters
        cudaEvent_t e7 = prof_mark(map, s);
        prof_push(map, kRays, e0, e1);
        prof_push(map, kEmit, e2, e3);
        prof_push(map, kSort, e4, e5);
        prof_push(map, kApply, e6, e7);
        return TSDF_OK;
    }
    if (n > 0 && map->use_graph && !map->graph_broken && !map->prof) {
        bool launched = false;
        rc = chain_graph_launch(map, a, s, &launched);
        if (launched || rc != TSDF_OK) return rc;
    }
    cudaEvent_t e0 = n > 0 ? prof_mark(map, s) : nullptr;
    TSDF_CU(launch_rays(a, map->dev, false, true, pdl, s));
    cudaEvent_t e1 = n > 0 ? prof_mark(map, s) : nullptr;
    cudaEvent_t e2 = n > 0 ? prof_mark(map, s) : nullptr;
    TSDF_CU(launch_contrib(a, map->dev, map->p.reduce, map->merge, map->kpt, pdl, s));
    cudaEvent_t e3 = n > 0 ? prof_mark(map, s) : nullptr;
    cudaEvent_t e4 = prof_mark(map, s);
    TSDF_CU(launch_compact(map->dev, (uint32_t)map->bricks, pdl, s));
    TSDF_CU(launch_apply(map->dev, map->p.reduce, map->p.w_max, map->p.flags, pdl, s));   // + counters
    cudaEvent_t e5 = prof_mark(map, s);
    prof_push(map, kRays, e0, e1);
    prof_push(map, kContrib, e2, e3);
    prof_push(map, kApply, e4, e5);
    return TSDF_OK;
}

// TSDF_REDUCTION_AUTO: collect finished trials without waiting and decide
// once every candidate has enough of them (the fastest by its best time).
static void auto_harvest(tsdf_map* map) {
    std::vector<tsdf_map::AutoTrial> keep;
    for (auto& t : map->auto_trials) {
        if (cudaEventQuery(t.stop) != cudaSuccess) {
            keep.push_back(t);
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
            if (map->auto_timed[t.candidate] == 0 || ms < map->auto_best[t.candidate]) map->auto_best[t.candidate] = ms;
            map->auto_timed[t.candidate]++;
        }
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    map->auto_trials.swap(keep);
    cudaGetLastError();
    bool all = true;
    for (int c = 0; c < tsdf_map::kAutoCandidates; ++c) all = all && map->auto_timed[c] >= tsdf_map::kAutoTrials;
    if (all && map->auto_choice < 0) {
        int best = 0;
        for (int c = 1; c < tsdf_map::kAutoCandidates; ++c)
            if (map->auto_best[c] < map->auto_best[best]) best = c;
        map->auto_choice = tsdf_map::kAutoReduction[best];
    }
}

static int integrate_dev(tsdf_map* map, const float* points_dev, int64_t n, const float pose[12],
                         cudaStream_t s) {
    if (map->reduction != TSDF_REDUCTION_AUTO) return integrate_with(map, points_dev, n, pose, s, map->reduction);
    auto_harvest(map);
    if (map->auto_choice >= 0) return integrate_with(map, points_dev, n, pose, s, map->auto_choice);
    // still tuning: one untimed first call per candidate (buffer set-up), then timed calls
    int cand = -1;
    for (int c = 0; c < tsdf_map::kAutoCandidates && cand < 0; ++c)
        if (map->auto_started[c] < tsdf_map::kAutoTrials + 1) cand = c;
    if (cand < 0) return integrate_with(map, points_dev, n, pose, s, tsdf_map::kAutoReduction[0]);
    const int red = tsdf_map::kAutoReduction[cand];
    if (map->auto_started[cand]++ == 0) return integrate_with(map, points_dev, n, pose, s, red);
    tsdf_map::AutoTrial t{cand, nullptr, nullptr};
    if (cudaEventCreate(&t.start) != cudaSuccess || cudaEventCreate(&t.stop) != cudaSuccess) {
        if (t.start) cudaEventDestroy(t.start);
        cudaGetLastError();
        return integrate_with(map, points_dev, n, pose, s, red);
    }
    cudaEventRecord(t.start, s);
    const int rc = integrate_with(map, points_dev, n, pose, s, red);
    cudaEventRecord(t.stop, s);
    map->auto_trials.push_back(t);
    return rc;
}

static int check_scan_args(tsdf_map* map, const float* pts, int64_t n, const float pose[12]) {
    if (!map || !pose || n < 0 || n > TSDF_MAX_POINTS) return TSDF_ERR_INVALID;
    if (n > 0 && !pts) return TSDF_ERR_INVALID;
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(pose[i])) return TSDF_ERR_INVALID;
    return TSDF_OK;
}

int tsdf_integrate(tsdf_map* map, const float* points_dev, int64_t n, const float pose[12], void* stream) {
    int rc = check_scan_args(map, points_dev, n, pose);
    if (rc != TSDF_OK) return rc;
    if (((uintptr_t)points_dev & 15u) != 0) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    return integrate_dev(map, points_dev, n, pose, (cudaStream_t)stream);
}

int tsdf_integrate_host(tsdf_map* map, const float* points_host, int64_t n, const float pose[12], void* stream) {
    int rc = check_scan_args(map, points_host, n, pose);
    if (rc != TSDF_OK) return rc;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (map->zero_copy && n > 0 && ((uintptr_t)points_host & 15u) == 0) {
        // pinned host memory mapped into the device's address space: the rays
        // kernel reads the points in place (over the host link), no staging copy
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, points_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer != nullptr && ((uintptr_t)at.devicePointer & 15u) == 0)
            return integrate_dev(map, static_cast<const float*>(at.devicePointer), n, pose, s);
        cudaGetLastError();
    }
    if ((size_t)n > map->stage_cap) {
        // a previous call may still read the old buffer: cudaFree waits for the device
        cudaFree(map->stage_dev);
        map->stage_dev = nullptr;
        map->stage_cap = 0;
        size_t cap = (size_t)n < 4096 ? 4096 : (size_t)n;
        TSDF_CU(cudaMalloc(&map->stage_dev, cap * sizeof(float4)));
        map->stage_cap = cap;
    }
    if (n > 0) TSDF_CU(cudaMemcpyAsync(map->stage_dev, points_host, (size_t)n * sizeof(float4), cudaMemcpyHostToDevice, s));
    return integrate_dev(map, reinterpret_cast<const float*>(map->stage_dev), n, pose, s);
}

int tsdf_shift(tsdf_map* map, const int64_t new_origin[3], void* stream) {
    if (!map || !new_origin) return TSDF_ERR_INVALID;
    for (int a = 0; a < 3; ++a)
        if (new_origin[a] % 8 != 0 || new_origin[a] > kOriginLimit || new_origin[a] < -kOriginLimit)
            return TSDF_ERR_INVALID;
    if (new_origin[0] == map->origin[0] && new_origin[1] == map->origin[1] && new_origin[2] == map->origin[2])
        return TSDF_OK;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    const long long C[3] = {map->p.dims[0] / 8, map->p.dims[1] / 8, map->p.dims[2] / 8};
    std::vector<long long> oldc[3], newc[3];
    std::vector<char> chg[3];
    for (int a = 0; a < 3; ++a) {
        const long long co = floordiv8(map->origin[a]), cn = floordiv8(new_origin[a]);
        oldc[a].resize(C[a]);
        newc[a].resize(C[a]);
        chg[a].resize(C[a]);
        for (long long sl = 0; sl < C[a]; ++sl) {
            // the chunk of each window that occupies ring slot sl
            oldc[a][sl] = co + (((sl - co) % C[a]) + C[a]) % C[a];
            newc[a][sl] = cn + (((sl - cn) % C[a]) + C[a]) % C[a];
            chg[a][sl] = oldc[a][sl] != newc[a][sl];
        }
    }
    // ring slots whose chunk changes: every slot of a changed x, y or z layer
    std::vector<long long> chx;
    for (long long sx = 0; sx < C[0]; ++sx)
        if (chg[0][sx]) chx.push_back(sx);
    size_t cnt = 0;
    for (long long sz = 0; sz < C[2]; ++sz)
        for (long long sy = 0; sy < C[1]; ++sy)
            cnt += (chg[2][sz] || chg[1][sy]) ? (size_t)C[0] : chx.size();
    if (cnt > 0) {
        // the pinned item buffer may still be read by the previous shift's copy
        if (map->items_event_pending) {
            TSDF_CU(cudaEventSynchronize(map->items_event));
            map->items_event_pending = false;
        }
        int rc = store_resolve(map);   // the previous shift's empty chunks are dropped
        if (rc == TSDF_OK) rc = store_trim_host(map);
        if (rc == TSDF_OK) rc = ensure_shift_buffers(map, cnt);
        if (rc == TSDF_OK) rc = store_make_room(map, cnt, s);
        if (rc != TSDF_OK) return rc;
        // every leaving chunk gets a candidate slot (device tier first); the
        // kernel claims candidates in order for the chunks that hold data, and
        // the next shift records those. Then the entering chunks are looked up
        // and leave the store: their slots are freed after the candidates are
        // taken, so no slot is both read and written by this shift.
        const uint64_t stamp = ++map->shift_serial;
        map->leave_keys.clear();
        ShiftItem* items = map->items_host + 1;   // entry 0: the header (claim counter)
        map->items_host[0] = ShiftItem{};
        auto add_out = [&](long long sx, long long sy, long long sz) {
            ShiftItem& it = items[map->leave_keys.size()];
            it = ShiftItem{};
            it.brick = (uint32_t)((sz * C[1] + sy) * C[0] + sx);
            map->leave_keys.push_back(ChunkKey{oldc[0][sx], oldc[1][sy], oldc[2][sz]});
        };
        for (long long sz = 0; sz < C[2]; ++sz) {
            for (long long sy = 0; sy < C[1]; ++sy) {
                if (chg[2][sz] || chg[1][sy]) {
                    for (long long sx = 0; sx < C[0]; ++sx) add_out(sx, sy, sz);
                } else {
                    for (size_t q = 0; q < chx.size(); ++q) add_out(chx[q], sy, sz);
                }
            }
        }
        if (!map->store.candidates(map->leave_keys, stamp, &map->cand_locs)) return TSDF_ERR_OOM;
        int io = TSDF_OK;
        bool waited = false;
        for (size_t i = 0; i < cnt; ++i) {
            ShiftItem& it = items[i];
            it.out_ptr = store_addr(map, map->cand_locs[i]);   // candidate i, claimed in order by the kernel
            const long long b = it.brick;
            const long long sx = b % C[0], sy = (b / C[0]) % C[1], sz = b / (C[0] * C[1]);
            long long loc = map->store.take(ChunkKey{newc[0][sx], newc[1][sy], newc[2][sz]});
            if (loc >= 0 && ChunkStore::is_file((uint32_t)loc)) {
                // read into a free host slot (not one of this shift's
                // candidates, which are out of the free list), after the last
                // shift's kernel has finished reading the slots it freed
                if (!waited) {
                    const cudaError_t e = cudaEventSynchronize(map->flags_event);
                    if (e != cudaSuccess) io = cuda_fail(e);
                    waited = true;
                }
                long long h = map->store.take_slot(1);
                if (h < 0 && store_grow(map, 1, 1)) h = map->store.take_slot(1);
                if (io == TSDF_OK && h < 0) io = TSDF_ERR_OOM;
                if (h < 0 || !map->store_file->get(ChunkStore::slot_of((uint32_t)loc), store_host_ptr(map, (uint32_t)h))) {
                    if (io == TSDF_OK) io = TSDF_ERR_IO;
                    loc = -1;   // the chunk is lost: it enters as (0, 0)
                } else {
                    ++map->chunks_from_file;
                    loc = h;
                }
            }
            it.in_ptr = loc >= 0 ? store_addr(map, (uint32_t)loc) : 0ull;
        }
        map->store.end_shift();
        TSDF_CU(cudaMemcpyAsync(map->items_dev, map->items_host, (cnt + 1) * sizeof(ShiftItem), cudaMemcpyHostToDevice,
                                s));
        TSDF_CU(cudaEventRecord(map->items_event, s));
        map->items_event_pending = true;
        cudaEvent_t e0 = prof_mark(map, s);
        TSDF_CU(launch_shift(map->dev.grid, map->items_dev + 1, (int)cnt, reinterpret_cast<unsigned*>(map->items_dev),
                             map->claim_dev, s));
        prof_push(map, kShift, e0, prof_mark(map, s));
        TSDF_CU(cudaEventRecord(map->flags_event, s));   // the claims have reached claim_host
        for (int a = 0; a < 3; ++a) map->origin[a] = new_origin[a];
        return io;
    }
    for (int a = 0; a < 3; ++a) map->origin[a] = new_origin[a];
    return TSDF_OK;
}

int tsdf_read(tsdf_map* map, const int64_t lo[3], const int64_t hi[3], int16_t* value_host, int16_t* weight_host,
              void* stream) {
    if (!map || !lo || !hi) return TSDF_ERR_INVALID;
    uint32_t box[3];
    if (!box_inside(map, lo, hi, box)) return TSDF_ERR_INVALID;
    const size_t total = (size_t)box[0] * box[1] * box[2];
    if (total == 0 || (!value_host && !weight_host)) return TSDF_OK;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    int16_t* tmp = nullptr;
    TSDF_CU(cudaMallocAsync(&tmp, 2 * total * sizeof(int16_t), s));
    const long long l[3] = {lo[0], lo[1], lo[2]};
    cudaError_t e = launch_read_box(map->dev.grid, l, box, map->geom, tmp, tmp + total, s);
    if (e == cudaSuccess && value_host)
        e = cudaMemcpyAsync(value_host, tmp, total * sizeof(int16_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && weight_host)
        e = cudaMemcpyAsync(weight_host, tmp + total, total * sizeof(int16_t), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(tmp, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    return TSDF_OK;
}

int tsdf_write(tsdf_map* map, const int64_t lo[3], const int64_t hi[3], const int16_t* value_host,
               const int16_t* weight_host, void* stream) {
    if (!map || !lo || !hi || !value_host || !weight_host) return TSDF_ERR_INVALID;
    uint32_t box[3];
    if (!box_inside(map, lo, hi, box)) return TSDF_ERR_INVALID;
    const size_t total = (size_t)box[0] * box[1] * box[2];
    for (size_t i = 0; i < total; ++i)
        if (weight_host[i] < 0 || weight_host[i] > map->p.w_max) return TSDF_ERR_INVALID;
    if (total == 0) return TSDF_OK;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    int16_t* tmp = nullptr;
    TSDF_CU(cudaMallocAsync(&tmp, 2 * total * sizeof(int16_t), s));
    cudaError_t e = cudaMemcpyAsync(tmp, value_host, total * sizeof(int16_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tmp + total, weight_host, total * sizeof(int16_t), cudaMemcpyHostToDevice, s);
    const long long l[3] = {lo[0], lo[1], lo[2]};
    if (e == cudaSuccess)
        e = launch_write_box(map->dev.grid, l, box, map->geom, tmp, tmp + total, s);
    cudaFreeAsync(tmp, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    return TSDF_OK;
}

int tsdf_stats(tsdf_map* map, tsdf_scan_stats* out, void* stream) {
    if (!map || !out) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    long long last[3] = {0, 0, 0};   // last_valid, last_hits, last_touched are contiguous
    static_assert(offsetof(MapCounters, last_touched) == offsetof(MapCounters, last_valid) + 16, "layout");
    long long status = 0;
    static_assert(offsetof(MapCounters, last_status) == offsetof(MapCounters, last_valid) + 24, "layout");
    static_assert(kStatusCapacity == TSDF_ERR_CAPACITY, "status code");
    if (map->host_last) {
        // the last apply CTA of each scan also wrote them to mapped host memory
        TSDF_CU(cudaStreamSynchronize(s));
        std::memcpy(last, (const void*)map->host_last, sizeof(last));
        status = ((volatile long long*)map->host_last)[3];
    } else {
        long long buf[4] = {0, 0, 0, 0};
        TSDF_CU(cudaMemcpyAsync(buf, &map->dev.ctr->last_valid, sizeof(buf), cudaMemcpyDeviceToHost, s));
        TSDF_CU(cudaStreamSynchronize(s));
        std::memcpy(last, buf, sizeof(last));
        status = buf[3];
    }
    out->valid_rays = last[0];
    out->hits = last[1];
    out->touched = last[2];
    return status != 0 ? (int)status : TSDF_OK;
}

int tsdf_profile_enable(tsdf_map* map, int32_t enable) {
    if (!map) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    prof_drain(map);
    map->prof = enable != 0;
    for (int k = 0; k < kNumKernels; ++k) {
        map->prof_launches[k] = 0;
        map->prof_ms[k] = 0.0;
    }
    return TSDF_OK;
}

int tsdf_profile_read(tsdf_map* map, tsdf_kernel_time* out, int32_t capacity, int32_t* count) {
    if (!map || !count || capacity < 0 || (capacity > 0 && !out)) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    int rc = prof_drain(map);
    if (rc != TSDF_OK) return rc;
    int32_t c = 0;
    for (int k = 0; k < kNumKernels; ++k) {
        if (map->prof_launches[k] == 0) continue;
        if (c < capacity) {
            std::memset(out[c].name, 0, sizeof(out[c].name));
            std::strncpy(out[c].name, kKernelNames[k], sizeof(out[c].name) - 1);
            out[c].launches = map->prof_launches[k];
            out[c].total_ms = map->prof_ms[k];
        }
        ++c;
    }
    *count = c;
    return TSDF_OK;
}

int tsdf_set_option(tsdf_map* map, int32_t option, int64_t value) {
    if (!map) return TSDF_ERR_INVALID;
    switch (option) {
        case TSDF_OPT_WARP_MERGE:
            if (value != 0 && value != 1) return TSDF_ERR_INVALID;
            map->merge = value != 0;
            return TSDF_OK;
        case TSDF_OPT_STEPS_PER_THREAD:
            if (value != 1 && value != 2 && value != 4) return TSDF_ERR_INVALID;
            map->kpt = (int)value;
            return TSDF_OK;
        case TSDF_OPT_PDL:
            if (value != 0 && value != 1) return TSDF_ERR_INVALID;
            map->pdl = value != 0;
            return TSDF_OK;
        case TSDF_OPT_POOL_BRICKS:
            if (value != 0 && (value < 64 || value > (int64_t)map->bricks)) return TSDF_ERR_INVALID;
            map->pool_req = (size_t)value;
            return TSDF_OK;
        case TSDF_OPT_REDUCTION:
            if (value != TSDF_REDUCTION_ATOMIC && value != TSDF_REDUCTION_SORT && value != TSDF_REDUCTION_POOL &&
                value != TSDF_REDUCTION_AUTO)
                return TSDF_ERR_INVALID;
            map->reduction = (int)value;
            return TSDF_OK;
        case TSDF_OPT_HOST_ZERO_COPY:
            if (value != 0 && value != 1) return TSDF_ERR_INVALID;
            map->zero_copy = value != 0;
            return TSDF_OK;
        case TSDF_OPT_LAUNCH_GRAPH:
            if (value != 0 && value != 1) return TSDF_ERR_INVALID;
            map->use_graph = value != 0;
            if (map->use_graph) map->graph_broken = false;   // try again
            return TSDF_OK;
        case TSDF_OPT_SORT_CAPACITY:
            if (value != 0 && (value < 1024 || value > (int64_t)kPairCapMax)) return TSDF_ERR_INVALID;
            map->pair_cap_req = (size_t)value;
            return TSDF_OK;
        case TSDF_OPT_STORE_DEVICE_CHUNKS:
            if (value < 0 || value > (1LL << 30)) return TSDF_ERR_INVALID;
            map->store_dev_cap = (size_t)value;
            return TSDF_OK;
        case TSDF_OPT_STORE_SPILL_AGE:
            if (value < 0 || value > (1LL << 30)) return TSDF_ERR_INVALID;
            map->spill_age = (uint32_t)value;
            return TSDF_OK;
        default: return TSDF_ERR_INVALID;
    }
}

int tsdf_map_reserve_store(tsdf_map* map, int64_t device_chunks) {
    if (!map || device_chunks < 1 || device_chunks > (1LL << 30)) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    const size_t want = ((size_t)device_chunks + kSegChunks - 1) / kSegChunks * kSegChunks;
    map->store_dev_cap = std::max(want, map->store.capacity(0));
    while (map->store.capacity(0) < want) {
        const size_t segs = (want - map->store.capacity(0)) / kSegChunks;
        if (!store_grow(map, 0, segs) && !store_grow(map, 0, 1)) return TSDF_ERR_OOM;
    }
    // and the bookkeeping of a shift that moves every brick of the window
    return ensure_shift_buffers(map, map->bricks);
}

int tsdf_get_store_stats(tsdf_map* map, tsdf_store_stats* out) {
    if (!map || !out) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    int rc = store_resolve(map);
    if (rc != TSDF_OK) return rc;
    out->device_chunks = (int64_t)map->store.used(0);
    out->device_capacity = (int64_t)map->store.capacity(0);
    out->host_chunks = (int64_t)map->store.used(1);
    out->host_capacity = (int64_t)map->store.capacity(1);
    out->spilled = (int64_t)map->chunks_spilled;
    out->dropped = (int64_t)map->chunks_dropped;
    out->file_chunks = (int64_t)map->store.used(2);
    out->to_file = (int64_t)map->chunks_to_file;
    out->from_file = (int64_t)map->chunks_from_file;
    return TSDF_OK;
}

int tsdf_map_set_store_file(tsdf_map* map, const char* path, int64_t host_chunks) {
    if (!map || !path || host_chunks < 0 || map->store_file) return TSDF_ERR_INVALID;
    std::unique_ptr<ChunkFile> f(new ChunkFile());
    if (!f->open(path, kSegChunks)) return TSDF_ERR_IO;
    map->store_file = std::move(f);
    map->store_host_cap = (size_t)host_chunks;
    return TSDF_OK;
}

// ---- persistence ------------------------------------------------------------

namespace {

constexpr char kFileMagic[8] = {'T', 'S', 'D', 'F', 'M', 'A', 'P', '1'};

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    tsdf_params params;
    int64_t chunk_count;
    unsigned char zero[32];
};
static_assert(sizeof(tsdf_params) == 72, "tsdf_params layout");
static_assert(sizeof(FileHeader) == TSDF_FILE_HEADER_BYTES, "file header layout");

struct FileRecord {
    int64_t chunk[3];
    uint32_t word[512];
};
static_assert(sizeof(FileRecord) == TSDF_FILE_RECORD_BYTES, "file record layout");

struct FileCloser {
    FILE* f = nullptr;
    ~FileCloser() {
        if (f) fclose(f);
    }
};

struct PinnedBuffer {
    void* p = nullptr;
    ~PinnedBuffer() {
        if (p) cudaFreeHost(p);
    }
};

bool all_zero(const uint32_t* w) {
    for (int i = 0; i < 512; ++i)
        if (w[i] != 0u) return false;
    return true;
}

// Chunk coordinate of window ring slot s along one axis (C chunks per axis).
long long slot_chunk(long long origin, long long C, long long s) {
    const long long co = floordiv8(origin);
    return co + (((s - co) % C) + C) % C;
}

}  // namespace

int tsdf_map_save(tsdf_map* map, const char* path, void* stream) {
    if (!map || !path) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    TSDF_CU(cudaStreamSynchronize(s));
    FileCloser fc;
    fc.f = std::fopen(path, "wb");
    if (!fc.f) return TSDF_ERR_IO;
    FileHeader h{};
    std::memcpy(h.magic, kFileMagic, 8);
    h.version = 1;
    h.header_bytes = TSDF_FILE_HEADER_BYTES;
    h.params = map->p;
    for (int a = 0; a < 3; ++a) h.params.origin[a] = map->origin[a];
    h.chunk_count = 0;
    if (std::fwrite(&h, sizeof(h), 1, fc.f) != 1) return TSDF_ERR_IO;

    // staging: up to 4096 chunks (8 MiB) at a time
    const size_t kStage = kSegChunks;
    PinnedBuffer stage;
    TSDF_CU(cudaMallocHost(&stage.p, kStage * kChunkBytes));
    const uint32_t* sw = static_cast<const uint32_t*>(stage.p);
    FileRecord rec;
    int64_t count = 0;
    const long long C[3] = {map->p.dims[0] / 8, map->p.dims[1] / 8, map->p.dims[2] / 8};
    // 1. the window, brick by brick (ring slot order)
    for (size_t b0 = 0; b0 < map->bricks; b0 += kStage) {
        const size_t nb = map->bricks - b0 < kStage ? map->bricks - b0 : kStage;
        TSDF_CU(cudaMemcpyAsync(stage.p, map->dev.grid + b0 * kBrickVoxels, nb * kChunkBytes, cudaMemcpyDeviceToHost, s));
        TSDF_CU(cudaStreamSynchronize(s));
        for (size_t k = 0; k < nb; ++k) {
            const uint32_t* w = sw + k * kBrickVoxels;
            if (all_zero(w)) continue;
            const long long b = (long long)(b0 + k);
            rec.chunk[0] = slot_chunk(map->origin[0], C[0], b % C[0]);
            rec.chunk[1] = slot_chunk(map->origin[1], C[1], (b / C[0]) % C[1]);
            rec.chunk[2] = slot_chunk(map->origin[2], C[2], b / (C[0] * C[1]));
            std::memcpy(rec.word, w, kChunkBytes);
            if (std::fwrite(&rec, sizeof(rec), 1, fc.f) != 1) return TSDF_ERR_IO;
            ++count;
        }
    }
    // 2. stored chunks (all outside the window): device-tier chunks segment by
    //    segment through the staging buffer, host-tier chunks in place
    int rc = store_resolve(map);
    if (rc != TSDF_OK) return rc;
    std::vector<std::vector<std::pair<uint32_t, ChunkKey>>> by_seg(map->store_seg[0].size());
    std::vector<std::pair<uint32_t, ChunkKey>> on_host, on_file;
    map->store.for_each([&](const ChunkKey& k, uint32_t loc) {
        if (ChunkStore::is_host(loc)) on_host.push_back({ChunkStore::slot_of(loc), k});
        else if (ChunkStore::is_file(loc)) on_file.push_back({ChunkStore::slot_of(loc), k});
        else by_seg[loc / kSegChunks].push_back({loc % kSegChunks, k});
    });
    auto put = [&](const uint32_t* w, const ChunkKey& k) -> bool {
        if (all_zero(w)) return true;
        rec.chunk[0] = k.x;
        rec.chunk[1] = k.y;
        rec.chunk[2] = k.z;
        std::memcpy(rec.word, w, kChunkBytes);
        if (std::fwrite(&rec, sizeof(rec), 1, fc.f) != 1) return false;
        ++count;
        return true;
    };
    for (size_t sg = 0; sg < by_seg.size(); ++sg) {
        if (by_seg[sg].empty()) continue;
        TSDF_CU(cudaMemcpyAsync(stage.p, map->store_seg[0][sg], (size_t)kSegChunks * kChunkBytes,
                                cudaMemcpyDeviceToHost, s));
        TSDF_CU(cudaStreamSynchronize(s));
        for (const auto& e : by_seg[sg])
            if (!put(sw + (size_t)e.first * kBrickVoxels, e.second)) return TSDF_ERR_IO;
    }
    for (const auto& e : on_host) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(map->store_seg_host[e.first / kSegChunks] +
                                                              (size_t)(e.first % kSegChunks) * kChunkBytes);
        if (!put(w, e.second)) return TSDF_ERR_IO;
    }
    for (const auto& e : on_file) {
        if (!map->store_file->get(e.first, stage.p)) return TSDF_ERR_IO;
        if (!put(sw, e.second)) return TSDF_ERR_IO;
    }
    h.chunk_count = count;
    if (std::fseek(fc.f, 0, SEEK_SET) != 0 || std::fwrite(&h, sizeof(h), 1, fc.f) != 1) return TSDF_ERR_IO;
    if (std::fclose(fc.f) != 0) {
        fc.f = nullptr;
        return TSDF_ERR_IO;
    }
    fc.f = nullptr;
    return TSDF_OK;
}

int tsdf_map_load(const char* path, tsdf_map** out, void* stream) {
    if (!path || !out) return TSDF_ERR_INVALID;
    *out = nullptr;
    FileCloser fc;
    fc.f = std::fopen(path, "rb");
    if (!fc.f) return TSDF_ERR_IO;
    FileHeader h{};
    if (std::fread(&h, sizeof(h), 1, fc.f) != 1) return TSDF_ERR_IO;
    if (std::memcmp(h.magic, kFileMagic, 8) != 0 || h.version != 1 || h.header_bytes != TSDF_FILE_HEADER_BYTES ||
        h.chunk_count < 0)
        return TSDF_ERR_IO;
    if (std::fseek(fc.f, 0, SEEK_END) != 0) return TSDF_ERR_IO;
    const long long size = std::ftell(fc.f);
    if (size != (long long)TSDF_FILE_HEADER_BYTES + h.chunk_count * (long long)TSDF_FILE_RECORD_BYTES)
        return TSDF_ERR_IO;
    if (std::fseek(fc.f, TSDF_FILE_HEADER_BYTES, SEEK_SET) != 0) return TSDF_ERR_IO;
    if (validate_params(&h.params) != TSDF_OK) return TSDF_ERR_IO;

    tsdf_map* map = nullptr;
    int rc = tsdf_map_create(&h.params, &map);
    if (rc != TSDF_OK) return rc;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t kStage = kSegChunks;
    PinnedBuffer stage, items_h;
    void* stage_d = nullptr;
    ChunkCopy* items_d = nullptr;
    auto fail = [&](int code) {
        cudaFree(stage_d);
        cudaFree(items_d);
        tsdf_map_destroy(map);
        return code;
    };
    cudaError_t e = cudaMallocHost(&stage.p, kStage * kChunkBytes);
    if (e == cudaSuccess) e = cudaMallocHost(&items_h.p, kStage * sizeof(ChunkCopy));
    if (e == cudaSuccess) e = cudaMalloc(&stage_d, kStage * kChunkBytes);
    if (e == cudaSuccess) e = cudaMalloc(&items_d, kStage * sizeof(ChunkCopy));
    if (e != cudaSuccess) return fail(cuda_fail(e));
    const long long C[3] = {map->p.dims[0] / 8, map->p.dims[1] / 8, map->p.dims[2] / 8};
    ChunkCopy* items = static_cast<ChunkCopy*>(items_h.p);
    FileRecord rec;
    for (int64_t done = 0; done < h.chunk_count;) {
        const int64_t nb = h.chunk_count - done < (int64_t)kStage ? h.chunk_count - done : (int64_t)kStage;
        for (int64_t k = 0; k < nb; ++k) {
            if (std::fread(&rec, sizeof(rec), 1, fc.f) != 1) return fail(TSDF_ERR_IO);
            std::memcpy(static_cast<char*>(stage.p) + k * kChunkBytes, rec.word, kChunkBytes);
            bool inside = true;
            long long slot[3];
            for (int a = 0; a < 3; ++a) {
                const long long co = floordiv8(map->origin[a]);
                inside = inside && rec.chunk[a] >= co && rec.chunk[a] < co + C[a];
                slot[a] = ((rec.chunk[a] % C[a]) + C[a]) % C[a];
            }
            unsigned long long dst = 0;
            if (inside) {
                const size_t brick = (size_t)((slot[2] * C[1] + slot[1]) * C[0] + slot[0]);
                dst = (unsigned long long)(map->dev.grid + brick * kBrickVoxels);
            } else {
                if (map->store.free_count(0) == 0 && map->store.free_count(1) == 0) {
                    const bool dev = map->store.capacity(0) < store_dev_limit(map);
                    if (!store_grow(map, dev ? 0 : 1, 1) && !(dev && store_grow(map, 1, 1))) return fail(TSDF_ERR_OOM);
                }
                const long long loc = map->store.insert_stored(ChunkKey{rec.chunk[0], rec.chunk[1], rec.chunk[2]},
                                                               map->shift_serial);
                if (loc < 0) return fail(TSDF_ERR_OOM);
                dst = store_addr(map, (uint32_t)loc);
            }
            items[k].dst = dst;
            items[k].src = (unsigned long long)(static_cast<char*>(stage_d) + k * kChunkBytes);
        }
        e = cudaMemcpyAsync(stage_d, stage.p, (size_t)nb * kChunkBytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(items_d, items, (size_t)nb * sizeof(ChunkCopy), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_copy_chunks(items_d, (int)nb, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the staging buffers are reused
        if (e != cudaSuccess) return fail(cuda_fail(e));
        done += nb;
    }
    cudaFree(stage_d);
    cudaFree(items_d);
    *out = map;
    return TSDF_OK;
}

int tsdf_extract_mesh(tsdf_map* map, int32_t min_weight, float* out_dev, int64_t capacity, int64_t* count,
                      void* stream) {
    if (!map || !count || min_weight < 1 || min_weight > 32767 || capacity < 0) return TSDF_ERR_INVALID;
    if (capacity > 0 && (!out_dev || ((uintptr_t)out_dev & 3u) != 0)) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* cnt = &map->dev.ctr->surface_count;
    TSDF_CU(cudaMemsetAsync(cnt, 0, sizeof(*cnt), s));
    const long long o[3] = {map->origin[0], map->origin[1], map->origin[2]};
    TSDF_CU(launch_mesh(map->dev.grid, map->geom, o, min_weight, map->p.voxel_size, out_dev,
                        (unsigned long long)capacity, cnt, s));
    unsigned long long n = 0;
    TSDF_CU(cudaMemcpyAsync(&n, cnt, sizeof(n), cudaMemcpyDeviceToHost, s));
    TSDF_CU(cudaStreamSynchronize(s));
    *count = (int64_t)n;
    return TSDF_OK;
}

int tsdf_register_system(tsdf_map* map, const float* points_dev, int64_t n, const float pose[12],
                         int32_t min_weight, double* out_host, void* stream) {
    if (!map || !pose || !out_host || n < 0 || n > TSDF_MAX_POINTS || min_weight < 1 || min_weight > 32767)
        return TSDF_ERR_INVALID;
    if (n > 0 && (!points_dev || ((uintptr_t)points_dev & 15u) != 0)) return TSDF_ERR_INVALID;
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(pose[i])) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!map->reg_dev) TSDF_CU(cudaMalloc(&map->reg_dev, 29 * sizeof(double)));
    const long long o[3] = {map->origin[0], map->origin[1], map->origin[2]};
    TSDF_CU(launch_register(points_dev, (int)n, pose, map->dev.grid, map->geom, o, map->p.voxel_size, map->inv_vs,
                            map->p.tau, min_weight, map->reg_dev, s));
    TSDF_CU(cudaMemcpyAsync(out_host, map->reg_dev, 29 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TSDF_CU(cudaStreamSynchronize(s));
    return TSDF_OK;
}

int tsdf_register(tsdf_map* map, const float* points_dev, int64_t n, float pose_inout[12], int32_t iterations,
                  int32_t min_weight, tsdf_register_result* result, void* stream) {
    if (!pose_inout || iterations < 1 || iterations > 1000) return TSDF_ERR_INVALID;
    float pose[12];
    std::memcpy(pose, pose_inout, sizeof(pose));
    double sys[29];
    tsdf_register_result res{};
    int it = 0;
    for (; it < iterations; ++it) {
        int rc = tsdf_register_system(map, points_dev, n, pose, min_weight, sys, stream);
        if (rc != TSDF_OK) return rc;
        res.used_points = (int64_t)sys[28];
        res.rms = sys[28] > 0 ? std::sqrt(sys[27] / sys[28]) : 0.0;
        double step = 0.0;
        if (sys[28] < 6 || !register_step(sys, pose, &step)) {
            res.iterations = it;
            if (result) *result = res;
            return TSDF_ERR_DEGENERATE;   // too few points or no curvature in some direction: pose unchanged
        }
        res.step = step;
        std::memcpy(pose_inout, pose, sizeof(pose));
        if (step < 1e-7) {
            ++it;
            break;
        }
    }
    res.iterations = it;
    if (result) *result = res;
    return TSDF_OK;
}

int tsdf_extract_surface(tsdf_map* map, int32_t min_weight, float* out_dev, int64_t capacity, int64_t* count,
                         void* stream) {
    if (!map || !count || min_weight < 1 || min_weight > 32767 || capacity < 0) return TSDF_ERR_INVALID;
    if (capacity > 0 && (!out_dev || ((uintptr_t)out_dev & 15u) != 0)) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* cnt = &map->dev.ctr->surface_count;
    TSDF_CU(cudaMemsetAsync(cnt, 0, sizeof(*cnt), s));
    const long long o[3] = {map->origin[0], map->origin[1], map->origin[2]};
    TSDF_CU(launch_surface(map->dev.grid, map->geom, o, min_weight, map->p.voxel_size,
                           reinterpret_cast<float4*>(out_dev), (unsigned long long)capacity, cnt, s));
    unsigned long long n = 0;
    TSDF_CU(cudaMemcpyAsync(&n, cnt, sizeof(n), cudaMemcpyDeviceToHost, s));
    TSDF_CU(cudaStreamSynchronize(s));
    *count = (int64_t)n;
    return TSDF_OK;
}

int tsdf_map_device_bytes(const tsdf_map* map, int64_t* out) {
    if (!map || !out) return TSDF_ERR_INVALID;
    const size_t flag_bytes = (map->bricks + 3) / 4 * 4;
    size_t b = map->voxels * sizeof(uint32_t) + flag_bytes + map->bricks * sizeof(uint32_t) + sizeof(MapCounters);
    if (map->dev.acc) b += map->voxels * sizeof(unsigned long long);
    b += map->ray_cap * 2 * sizeof(float4);
    if (map->dev.brick_slot) b += 3 * map->bricks * sizeof(uint32_t);
    b += map->ray_slot_cap * sizeof(uint32_t);
    b += (size_t)map->dev.pair_cap * (sizeof(uint2) + sizeof(uint32_t));
    if (map->dev.pool_table)
        b += map->bricks * sizeof(uint32_t) +
             (size_t)map->dev.pool_cap * (sizeof(uint32_t) + kBrickVoxels * sizeof(unsigned long long));
    b += map->store_seg[0].size() * (size_t)kSegChunks * kChunkBytes;   // the host tier is host memory
    b += map->stage_cap * sizeof(float4) + (map->items_dev ? (map->items_dev_cap + 1) * sizeof(ShiftItem) : 0) +
         map->spill_cap * sizeof(ChunkCopy);
    *out = (int64_t)b;
    return TSDF_OK;
}

int tsdf_get_reduction(tsdf_map* map, int32_t* reduction) {
    if (!map || !reduction) return TSDF_ERR_INVALID;
    if (map->reduction == TSDF_REDUCTION_AUTO) {
        DeviceScope ds(map->device);
        auto_harvest(map);
        *reduction = map->auto_choice >= 0 ? map->auto_choice : TSDF_REDUCTION_AUTO;
    } else {
        *reduction = map->reduction;
    }
    return TSDF_OK;
}

int tsdf_get_origin(const tsdf_map* map, int64_t out[3]) {
    if (!map || !out) return TSDF_ERR_INVALID;
    for (int a = 0; a < 3; ++a) out[a] = map->origin[a];
    return TSDF_OK;
}

int tsdf_grid_device_ptr(const tsdf_map* map, void** out) {
    if (!map || !out) return TSDF_ERR_INVALID;
    *out = map->dev.grid;
    return TSDF_OK;
}

const char* tsdf_error_string(int code) {
    switch (code) {
        case TSDF_OK: return "ok";
        case TSDF_ERR_INVALID: return "invalid argument";
        case TSDF_ERR_OOM: return "out of memory";
        case TSDF_ERR_CUDA: return "CUDA error";
        case TSDF_ERR_TIMEOUT: return "device wait timed out";
        case TSDF_ERR_ADMISSION: return "device-memory budget exceeded";
        case TSDF_ERR_BUSY: return "resource busy";
        case TSDF_ERR_IO: return "file error or not a map file";
        case TSDF_ERR_CAPACITY: return "scan dropped: the accumulator pool is full";
        case TSDF_ERR_DEGENERATE: return "registration is degenerate (too few observed points)";
        default: return "unknown error";
    }
}

int tsdf_last_cuda_error(void) { return g_last_cuda_error; }

}  // extern "C"

namespace tsdf {

int prepare_batch_item(::tsdf_map* map, const float* points_dev, int64_t n, const float pose[12], BatchItem* out) {
    int rc = check_scan_args(map, points_dev, n, pose);
    if (rc != TSDF_OK) return rc;
    if (((uintptr_t)points_dev & 15u) != 0) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    rc = ensure_acc(map);   // batches use the accumulator reductions
    if (rc != TSDF_OK) return rc;
    rc = ensure_rays(map, n);
    if (rc != TSDF_OK) return rc;
    fill_scan_args(map, points_dev, n, pose, out->a);
    out->m = map->dev;
    out->reduce = map->p.reduce;
    out->w_max = map->p.w_max;
    out->bricks = (uint32_t)map->bricks;
    out->flags = map->p.flags;
    return TSDF_OK;
}

int map_device(const ::tsdf_map* map) { return map->device; }

const long long* map_last_counters(const ::tsdf_map* map) { return &map->dev.ctr->last_valid; }

const volatile long long* map_host_counters(const ::tsdf_map* map) { return map->host_last; }

int map_reserve_points(::tsdf_map* map, int64_t n) {
    if (!map || n < 0 || n > TSDF_MAX_POINTS) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    int rc = ensure_acc(map);
    if (rc != TSDF_OK) return rc;
    return ensure_rays(map, n);
}

int map_reserve_sort(::tsdf_map* map, int64_t n) {
    if (!map || n < 0 || n > TSDF_MAX_POINTS) return TSDF_ERR_INVALID;
    DeviceScope ds(map->device);
    int rc = ensure_rays(map, n);
    if (rc != TSDF_OK) return rc;
    return ensure_sort(map, n);
}

}  // namespace tsdf
