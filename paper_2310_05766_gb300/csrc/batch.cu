// Batched integration: one scan into each of many maps in ONE persistent
// cooperative launch, optionally replayed from a captured CUDA graph.
//
// The kernel runs the five phases of the per-map path (rays, contrib,
// compact, apply, finish; integrate_device.cuh) over all maps of the batch,
// with a grid-wide barrier between phases. Work is spread over the whole GPU:
// CTAs take ray blocks of any map, warps take (32-ray block, k-group) items of
// any map, and so on, so maps of uneven size share the SMs. Per-map offsets
// of the work known on the host (ray blocks, flag words) come with the
// descriptors; those known only on the device (live rays, touched bricks) are
// prefix-summed by every CTA after the barrier.
//
// The barrier is a counter plus generation word; each wait gives up after a
// bounded number of polls, sets the batch's error word and makes every CTA
// return, which the host reports as TSDF_ERR_TIMEOUT.
//
// Descriptors live in device memory, copied from a pinned host buffer by the
// first node of the launch sequence, so one captured graph (copy, barrier
// reset, kernel) serves every later batch: only the pinned buffer changes.
// Two buffer sets alternate so the host can fill one while the GPU reads the
// other.
//
// Tuning (per-scan reduction by accumulator atomics or by sort, warp merge,
// steps per work item, CTA size, CTAs per SM, apply task size) changes speed
// only: results are bit-identical for every setting. The sort configurations add three phases (count, prefix, scatter:
// a counting sort of the emitted pairs by brick, see integrate.cu) and apply
// each brick from its sorted segment. With autotuning on, the first calls
// cycle through the settings, timing each with events, and the fastest is
// kept.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "integrate_device.cuh"
#include "../../include/tsdf.h"

// 1: the atomic configurations apply each brick from registers
// (apply_brick_reg); 0: through shared memory (apply_brick).
#ifndef TSDF_BATCH_APPLY_REG
#define TSDF_BATCH_APPLY_REG 1
#endif
// Voxel pairs per lane in one register-apply task of the atomic configurations
// (8: a warp per brick, 4: per half brick, 2: per quarter brick). Whole bricks
// measured fastest here (quarter bricks: 1.85 against 1.67 ms for 64 maps;
// every task pays a search for its map).
#ifndef TSDF_BATCH_APPLY_PAIRS
#define TSDF_BATCH_APPLY_PAIRS 8
#endif

namespace tsdf {
namespace {

using namespace dev;

constexpr int kBatchMax = 1024;               // maps per batch
constexpr size_t kApplySmemPerWarp = kBrickVoxels * (4 + 8 + 2);   // grid, accumulator, offsets
constexpr int kWarpBrickCacheLog2 = 10;                              // per-warp brick cache in phase 2
constexpr size_t kWarpCacheBytes = 4u << kWarpBrickCacheLog2;
static_assert(kWarpCacheBytes <= kApplySmemPerWarp, "brick cache fits the staging area");
// Phase 2's brick cache shared by a CTA's warps (in the staging areas of its
// first warps), used when every map of the batch has fewer than 2^22 bricks
// and the batch fewer than 1023 maps: map i tags its entries with i << 22.
constexpr int kCtaBrickCacheLog2 = 11;
constexpr uint32_t kTagShift = 22;
static_assert((4u << kCtaBrickCacheLog2) <= 4 * kApplySmemPerWarp, "CTA brick cache fits four warps' staging");
static_assert((4u << kCtaBrickCacheLog2) <= 4 * kWarpCacheBytes, "CTA brick cache fits four warps' caches");

struct BatchHeader {
    int32_t count;
    uint32_t ray_tasks;                      // total CTA ray tasks (THREADS times the configuration's points per thread)
    uint32_t word_tasks;                     // total warp compaction tasks (32 flag words each)
    uint32_t extra_arrivals;                 // test hook: barrier arrivals that never come
    uint32_t cta_cache;                      // 1: phase 2 keeps one brick cache per CTA (map-tagged keys)
    long long spin_limit;                    // polls before a barrier wait gives up
    uint32_t ray_prefix[kBatchMax + 1];      // exclusive prefix of ray tasks per map
    uint32_t word_prefix[kBatchMax + 1];     // exclusive prefix of compaction tasks per map
};

struct BatchSync {
    unsigned arrive;
    unsigned generation;
    unsigned error;
    unsigned pad;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch; false if the batch failed.
__device__ bool grid_barrier(BatchSync* s, unsigned arrivals, long long spin_limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire(&s->generation);
        __threadfence();
        const unsigned prev = atomicAdd(&s->arrive, 1u);
        bool good = true;
        if (prev == arrivals - 1u) {
            atomicExch(&s->arrive, 0u);
            __threadfence();
            atomicAdd(&s->generation, 1u);
        } else {
            long long polls = 0;
            while (ld_acquire(&s->generation) == gen) {
                if (++polls > spin_limit || ld_acquire(&s->error) != 0u) {
                    atomicOr(&s->error, 1u);
                    good = false;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok = good && ld_acquire(&s->error) == 0u;
    }
    __syncthreads();
    return ok != 0;
}

// Index of the map whose segment [prefix[i], prefix[i+1]) holds t.
__device__ __forceinline__ int find_segment(const uint32_t* prefix, int count, uint32_t t) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Block-wide exclusive prefix of per-map values v(i), written to out[0..count].
template <typename F>
__device__ void block_prefix(int count, F v, uint32_t* out) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned lane = threadIdx.x;
        uint32_t carry = 0;
        for (int base = 0; base < count; base += 32) {
            const int i = base + (int)lane;
            const uint32_t x = i < count ? v(i) : 0u;
            uint32_t incl = x;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= (unsigned)o) incl += y;
            }
            if (i < count) out[i] = carry + incl - x;
            carry += __shfl_sync(kFull, incl, 31);
        }
        if (lane == 0) out[count] = carry;
    }
    __syncthreads();
}

// Adds a warp's counter to the map's partial slot (lane 0 after a warp sum).
__device__ __forceinline__ void warp_add(unsigned long long v, unsigned long long* dst) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31u) == 0 && v) atomicAdd(dst, v);
}

// Pair slots written by map i's scan (sort configurations).
__device__ __forceinline__ uint32_t written_slots(const MapDev& m) {
    const unsigned long long n = __ldcg(&m.ctr->slot_count);
    return (uint32_t)(n < m.pair_cap ? n : (unsigned long long)m.pair_cap);
}

// THREADS: CTA size (a ray task is THREADS points of a map); APAIRS: voxel
// pairs per lane of a register-apply task (8: a warp per brick, 2: a quarter).
template <bool MERGE, int KPT, bool SORT, int THREADS, int APAIRS, int RPPT = 1>
__global__ void __launch_bounds__(THREADS, 768 / THREADS) batch_kernel(const BatchItem* __restrict__ items,
                                                                         const BatchHeader* __restrict__ hdr,
                                                                         BatchSync* sync) {
    constexpr int kBatchWarps = THREADS / 32;
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ uint32_t s_prefix[kBatchMax + 1];
    __shared__ uint32_t s_live[kBatchMax];   // phase 2: live rays per map, read once per CTA
    // phases 2 and 4: each warp's copy of its current map's scan arguments and
    // buffers (the march reads them at every sample; from global memory they
    // compete for L1 with the rays and the brick flags); phase 1: slot 0 holds
    // the CTA's task map
    __shared__ ScanArgs s_args[kBatchWarps];
    __shared__ MapDev s_dev[kBatchWarps];
    __shared__ RaysSmemT<kBatchWarps> rsm;
    const int count = hdr->count;
    const unsigned arrivals = gridDim.x + hdr->extra_arrivals;
    const long long spin = hdr->spin_limit;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned w = threadIdx.x >> 5;
    const unsigned gwarp = blockIdx.x * kBatchWarps + w;
    const unsigned nwarps = gridDim.x * kBatchWarps;

    // ---- phase 1: ray set-up and compaction, one CTA task = RPPT THREADS points
    // of a map (RPPT points per thread)
    static_assert(!(SORT && RPPT > 1), "the sort configurations set up one point per thread");
    // (the CTA's task map's arguments are staged in the first warp's slots of
    // s_args / s_dev, read by every thread of the task: 64-map batch 1.15
    // against 1.18 ms)
    int p1_map = -1;
    for (uint32_t t = blockIdx.x; t < hdr->ray_tasks; t += gridDim.x) {
        const int i = find_segment(hdr->ray_prefix, count, t);   // CTA-uniform
        if (i != p1_map) {
            const uint32_t* sa = reinterpret_cast<const uint32_t*>(&items[i].a);
            uint32_t* da = reinterpret_cast<uint32_t*>(&s_args[0]);
            for (int e = (int)threadIdx.x; e < (int)(sizeof(ScanArgs) / 4); e += THREADS) da[e] = sa[e];
            const uint32_t* sm_ = reinterpret_cast<const uint32_t*>(&items[i].m);
            uint32_t* dm = reinterpret_cast<uint32_t*>(&s_dev[0]);
            for (int e = (int)threadIdx.x; e < (int)(sizeof(MapDev) / 4); e += THREADS) dm[e] = sm_[e];
            __syncthreads();   // (the previous task ended with one, so no thread still reads the old copy)
            p1_map = i;
        }
        if constexpr (SORT)
            rays_task<false, SORT, false, kBatchWarps>(s_args[0], s_dev[0], (int)((t - hdr->ray_prefix[i]) * THREADS),
                                                       t, &rsm);
        else
            rays_task_ppt<false, false, kBatchWarps, RPPT>(s_args[0], s_dev[0],
                                                           (int)((t - hdr->ray_prefix[i]) * THREADS * RPPT), t, &rsm);
        __syncthreads();
    }
    if (!grid_barrier(sync, arrivals, spin)) return;

    // ---- phase 2: contributions; per map ceil(live / 32) * ceil((2K+1) / KPT) warp items
    const bool cta_cache = hdr->cta_cache != 0u;
    uint32_t* const ctab = reinterpret_cast<uint32_t*>(dyn);
    if (cta_cache)   // (block_prefix synchronises the CTA before any use)
        for (int e = (int)threadIdx.x; e < (1 << kCtaBrickCacheLog2); e += THREADS) ctab[e] = kNoVoxel;
    block_prefix(count, [&](int i) {
        const unsigned nl = __ldcg(&items[i].m.ctr->live_count);
        s_live[i] = nl;
        return (nl + 31u) / 32u * ((unsigned)(2 * items[i].a.K + KPT) / KPT);
    }, s_prefix);
    {
        unsigned last_brick = kNoVoxel;
        int cur = -1;
        unsigned hits = 0;
        bool ovf = false;
        // the brick cache lives in dynamic shared memory (the apply staging
        // area of the configurations that stage bricks, unused until phase
        // 4): one per CTA whose keys carry the map's tag, or else one per
        // warp, emptied whenever the warp moves to another map. The warps of
        // a CTA take consecutive items (mostly of one map) and mark the same
        // bricks, so a shared cache stops more global flag stores.
        BrickCache bc = cta_cache ? BrickCache{ctab, 32u - kCtaBrickCacheLog2, 0u}
                                  : BrickCache{reinterpret_cast<uint32_t*>(dyn + w * kWarpCacheBytes),
                                               32u - kWarpBrickCacheLog2, 0u};
        for (uint32_t g = gwarp; g < s_prefix[count]; g += nwarps) {   // warp-uniform
            const int i = find_segment(s_prefix, count, g);
            if (i != cur) {
                if (cur >= 0 && items[cur].reduce == 1)
                    warp_add(hits, &items[cur].m.ctr->part[gwarp % kParts].hits);
                if (cur >= 0 && ovf) items[cur].m.ctr->overflow = 1u;
                hits = 0;
                ovf = false;
                last_brick = kNoVoxel;
                cur = i;
                if (cta_cache) {
                    bc.tag = (uint32_t)i << kTagShift;
                } else {
                    for (int e = (int)lane; e < (1 << kWarpBrickCacheLog2); e += 32) bc.tab[e] = kNoVoxel;
                }
                __syncwarp();   // the warp is done with the previous map's copies
                {
                    const uint32_t* sa = reinterpret_cast<const uint32_t*>(&items[i].a);
                    uint32_t* da = reinterpret_cast<uint32_t*>(&s_args[w]);
                    for (int e = (int)lane; e < (int)(sizeof(ScanArgs) / 4); e += 32) da[e] = sa[e];
                    const uint32_t* sm_ = reinterpret_cast<const uint32_t*>(&items[i].m);
                    uint32_t* dm = reinterpret_cast<uint32_t*>(&s_dev[w]);
                    for (int e = (int)lane; e < (int)(sizeof(MapDev) / 4); e += 32) dm[e] = sm_[e];
                }
                __syncwarp();
            }
            const BatchItem& it = items[i];
            const ScanArgs& ia = s_args[w];
            const MapDev& im = s_dev[w];
            const unsigned ngrp = (unsigned)(2 * ia.K + KPT) / KPT;
            const unsigned local = g - s_prefix[i];
            const unsigned nl = s_live[i];
            const unsigned ray = (local / ngrp) * 32u + lane;
            float4 A, B;
            load_rays(im, nl, ray, A, B);
            if (SORT) {
                const uint32_t sslot = ray < nl ? im.ray_slot[ray] : kNoSlot;
                if (it.reduce == 0)
                    contrib_item<0, false, KPT, true>(ia, im, local % ngrp, A, B, hits, last_brick, sslot, &ovf,
                                                      nullptr, bc);
                else contrib_item<1, false, KPT, true>(ia, im, local % ngrp, A, B, hits, last_brick, sslot, &ovf,
                                                       nullptr, bc);
            } else {
                if (it.reduce == 0)
                    contrib_item<0, MERGE, KPT>(ia, im, local % ngrp, A, B, hits, last_brick, kNoSlot, nullptr,
                                                nullptr, bc);
                else contrib_item<1, MERGE, KPT>(ia, im, local % ngrp, A, B, hits, last_brick, kNoSlot, nullptr,
                                                 nullptr, bc);
            }
        }
        if (cur >= 0 && items[cur].reduce == 1) warp_add(hits, &items[cur].m.ctr->part[gwarp % kParts].hits);
        if (cur >= 0 && ovf) items[cur].m.ctr->overflow = 1u;
    }
    if (!grid_barrier(sync, arrivals, spin)) return;

    // ---- phase 3: brick flags -> brick lists, one warp task = 32 flag words of a map
    for (uint32_t t = gwarp; t < hdr->word_tasks; t += nwarps) {
        const int i = find_segment(hdr->word_prefix, count, t);
        const unsigned nwords = (items[i].bricks + 3u) / 4u;
        compact_words(items[i].m, (t - hdr->word_prefix[i]) * 32u + lane, nwords);
    }
    if (!grid_barrier(sync, arrivals, spin)) return;

    if (SORT) {
        // ---- phase 3b: pair counts per brick, one warp task = 128 pair slots of a map
        block_prefix(count, [&](int i) { return (written_slots(items[i].m) + 127u) / 128u; }, s_prefix);
        for (uint32_t g = gwarp; g < s_prefix[count]; g += nwarps) {
            const int i = find_segment(s_prefix, count, g);
            sort_count_warp(items[i].m, (g - s_prefix[i]) * 128u, written_slots(items[i].m));
        }
        if (!grid_barrier(sync, arrivals, spin)) return;
        // ---- phase 3c: segment starts, one CTA per map
        for (int i = blockIdx.x; i < count; i += gridDim.x)
            sort_scan_cta(items[i].m, __ldcg(&items[i].m.ctr->brick_count), s_prefix);
        if (!grid_barrier(sync, arrivals, spin)) return;
        // ---- phase 3d: scatter into the segments (same tasks as the count)
        block_prefix(count, [&](int i) { return (written_slots(items[i].m) + 127u) / 128u; }, s_prefix);
        for (uint32_t g = gwarp; g < s_prefix[count]; g += nwarps) {
            const int i = find_segment(s_prefix, count, g);
            sort_scatter_warp(items[i].m, (g - s_prefix[i]) * 128u, written_slots(items[i].m));
        }
        if (!grid_barrier(sync, arrivals, spin)) return;
    }

    // ---- phase 4: Eq. 1 / Eq. 2 on the touched bricks, one warp task per brick
    // (register apply: per part of a brick, kTaskParts parts each)
    constexpr unsigned kTaskParts = (!SORT && TSDF_BATCH_APPLY_REG) ? 8u / APAIRS : 1u;
    block_prefix(count, [&](int i) { return __ldcg(&items[i].m.ctr->brick_count) * kTaskParts; }, s_prefix);
    {
        uint32_t* s_grid = reinterpret_cast<uint32_t*>(dyn + w * kApplySmemPerWarp);
        unsigned long long* s_acc = reinterpret_cast<unsigned long long*>(dyn + w * kApplySmemPerWarp + 2048);
        uint16_t* s_off = reinterpret_cast<uint16_t*>(dyn + w * kApplySmemPerWarp + 6144);
        int cur = -1;
        unsigned long long touched = 0, hits = 0;
        for (uint32_t g = gwarp; g < s_prefix[count]; g += nwarps) {   // warp-uniform
            const int i = find_segment(s_prefix, count, g);
            if (i != cur) {
                if (cur >= 0) {
                    warp_add(touched, &items[cur].m.ctr->part[gwarp % kParts].touched);
                    if (SORT || items[cur].reduce == 0) warp_add(hits, &items[cur].m.ctr->part[gwarp % kParts].hits);
                }
                touched = hits = 0;
                cur = i;
                __syncwarp();   // (the map's buffers, as in phase 2)
                const uint32_t* sm_ = reinterpret_cast<const uint32_t*>(&items[i].m);
                uint32_t* dm = reinterpret_cast<uint32_t*>(&s_dev[w]);
                for (int e = (int)lane; e < (int)(sizeof(MapDev) / 4); e += 32) dm[e] = sm_[e];
                __syncwarp();
            }
            const BatchItem& it = items[i];
            const MapDev& im = s_dev[w];
            const unsigned local = g - s_prefix[i];
            if (SORT) {
                const bool ovf = __ldcg(&im.ctr->overflow) != 0u;
                if (it.reduce == 0)
                    sort_apply_brick<0>(im, it.w_max, it.flags, local, ovf, s_grid, s_acc, s_off, touched, hits);
                else sort_apply_brick<1>(im, it.w_max, it.flags, local, ovf, s_grid, s_acc, s_off, touched, hits);
            } else {
#if TSDF_BATCH_APPLY_REG
                if (it.reduce == 0)
                    apply_part_reg<0, APAIRS>(im, it.w_max, it.flags, local, touched, hits);
                else apply_part_reg<1, APAIRS>(im, it.w_max, it.flags, local, touched, hits);
#else
                if (it.reduce == 0) apply_brick<0>(im, it.w_max, it.flags, local, s_grid, s_acc, s_off, touched, hits);
                else apply_brick<1>(im, it.w_max, it.flags, local, s_grid, s_acc, s_off, touched, hits);
#endif
            }
        }
        if (cur >= 0) {
            warp_add(touched, &items[cur].m.ctr->part[gwarp % kParts].touched);
            if (SORT || items[cur].reduce == 0) warp_add(hits, &items[cur].m.ctr->part[gwarp % kParts].hits);
        }
    }
    if (!grid_barrier(sync, arrivals, spin)) return;

    // ---- phase 5: publish each map's counters
    for (uint32_t i = gwarp; i < (uint32_t)count; i += nwarps) finish_warp(items[i].m);
}

using BatchKernel = void (*)(const BatchItem*, const BatchHeader*, BatchSync*);

// Tuning configurations: reduction, warp merge and steps per item, then the
// launch shape (CTA size, CTAs per SM -- 0: as many as fit -- and the apply
// task size). Every one gives bit-identical results.
struct Config {
    bool merge;
    int kpt;
    bool sort;
    int threads;
    int ctas_per_sm;
    int apply_pairs;
    int rays_ppt;   // points per thread in the ray set-up
};
constexpr int kP = TSDF_BATCH_APPLY_PAIRS;
const Config kConfigs[] = {
    {false, 4, false, 256, 0, kP, 1}, {false, 2, false, 256, 0, kP, 1}, {false, 1, false, 256, 0, kP, 1},
    {true, 4, false, 256, 0, kP, 1},  {true, 2, false, 256, 0, kP, 1},  {true, 1, false, 256, 0, kP, 1},
    {false, 4, true, 256, 0, kP, 1},  {false, 2, true, 256, 0, kP, 1},
    // launch shapes of the plain atomic configuration
    {false, 4, false, 128, 0, kP, 1}, {false, 4, false, 512, 0, kP, 1}, {false, 4, false, 256, 2, kP, 1},
    {false, 4, false, 256, 0, 2, 1},
    // CTAs of 128 threads, several points per thread in the ray set-up: more
    // point loads in flight for large batches (64 outdoor-sized scans: 1.17-
    // 1.19 against 1.21 ms), a configuration of its own because the form
    // costs registers in the whole kernel (when every configuration had it,
    // 32 served sessions ran at 26 k instead of 30 k scans/s)
    {false, 4, false, 128, 0, kP, kBatchRaysPPT}};
constexpr int kNumConfigs = 13;

// Dynamic shared memory of a configuration: the apply staging area (per warp)
// where the apply stages bricks, else only phase 2's brick caches (one per CTA,
// or one per warp as the fallback). The smaller footprint leaves more of the
// SM's memory to L1, which holds the maps' descriptors that phase 2 reads
// (64-map batch, configuration 0: 1.40 against 1.66 ms).
size_t dyn_smem(const Config& c) {
    const size_t warps = (size_t)(c.threads / 32);
    if (c.sort || !TSDF_BATCH_APPLY_REG) return warps * kApplySmemPerWarp;
    return std::max<size_t>(4u << kCtaBrickCacheLog2, warps * kWarpCacheBytes);
}

template <int T, int AP>
BatchKernel kernel_shape(const Config& c) {
    if (c.sort) return c.kpt == 2 ? batch_kernel<false, 2, true, T, AP> : batch_kernel<false, 4, true, T, AP>;
    if (c.merge)
        return c.kpt == 1 ? batch_kernel<true, 1, false, T, AP>
                          : c.kpt == 2 ? batch_kernel<true, 2, false, T, AP> : batch_kernel<true, 4, false, T, AP>;
    return c.kpt == 1 ? batch_kernel<false, 1, false, T, AP>
                      : c.kpt == 2 ? batch_kernel<false, 2, false, T, AP> : batch_kernel<false, 4, false, T, AP>;
}

BatchKernel kernel_for(const Config& c) {
    if (c.rays_ppt > 1) return batch_kernel<false, 4, false, 128, kP, kBatchRaysPPT>;
    if (c.threads == 128) return batch_kernel<false, 4, false, 128, kP>;
    if (c.threads == 512) return batch_kernel<false, 4, false, 512, kP>;
    if (c.apply_pairs == 2) return batch_kernel<false, 4, false, 256, 2>;
    return kernel_shape<256, kP>(c);
}

}  // namespace
}  // namespace tsdf

using namespace tsdf;

struct tsdf_batch {
    int device = 0;
    int max_count = 0;
    int grid_pct = 100;                    // percentage of each configuration's co-resident CTAs launched
    int grid_max[kNumConfigs] = {};        // co-resident CTAs of each configuration (its launch shape)
    // two alternating descriptor sets
    struct Slot {
        unsigned char* host = nullptr;     // pinned: header + items
        unsigned char* dev = nullptr;
        cudaEvent_t done = nullptr;        // recorded after the set's launch
        bool pending = false;
        cudaGraphExec_t exec[kNumConfigs] = {};
    } slot[2];
    int next_slot = 0;
    BatchSync* sync = nullptr;
    size_t desc_bytes = 0;
    // options
    bool use_graph = true;
    bool autotune = true;
    int config = 0;                        // index into kConfigs
    int extra_arrivals = 0;
    long long spin_limit = 1LL << 24;
    // autotuning state
    int trials_per_config = 2;
    bool tune_sort = true;                 // the autotuner also times the sort configurations
    bool cta_cache = true;                 // phase 2 shares one brick cache per CTA when the maps allow it
    int tuned = -1;                        // chosen config, -1 while tuning
    struct Trial {
        int config;
        cudaEvent_t start, stop;
    };
    std::vector<Trial> trials;
    float best_ms[kNumConfigs] = {};
    int n_timed[kNumConfigs] = {};
    cudaStream_t capture_stream = nullptr;
};

namespace {

int cu_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? TSDF_ERR_OOM : TSDF_ERR_CUDA; }

struct DevScope {
    int prev = -1;
    bool changed = false;
    explicit DevScope(int d) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) changed = cudaSetDevice(d) == cudaSuccess;
    }
    ~DevScope() {
        if (changed) cudaSetDevice(prev);
    }
};

void free_batch(tsdf_batch* b) {
    if (!b) return;
    for (auto& s : b->slot) {
        for (auto& e : s.exec)
            if (e) cudaGraphExecDestroy(e);
        if (s.host) cudaFreeHost(s.host);
        cudaFree(s.dev);
        if (s.done) cudaEventDestroy(s.done);
    }
    for (auto& t : b->trials) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    cudaFree(b->sync);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    delete b;
}

// CTAs launched for configuration `cfg`: its co-resident CTAs (limited to
// ctas_per_sm per SM when set), scaled by the grid-fraction option.
int grid_of(const tsdf_batch* b, int cfg) {
    return std::max(1, (int)((long long)b->grid_max[cfg] * b->grid_pct / 100));
}

// Enqueue copy + barrier reset + cooperative kernel for descriptor slot `si`.
cudaError_t enqueue(tsdf_batch* b, int si, int cfg, cudaStream_t s) {
    tsdf_batch::Slot& sl = b->slot[si];
    cudaError_t e = cudaMemcpyAsync(sl.dev, sl.host, b->desc_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->sync, 0, sizeof(BatchSync), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t lc = {};
    const Config& c = kConfigs[cfg];
    lc.gridDim = dim3((unsigned)grid_of(b, cfg));
    lc.blockDim = dim3((unsigned)c.threads);
    lc.dynamicSmemBytes = dyn_smem(c);
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    const BatchItem* items = reinterpret_cast<const BatchItem*>(sl.dev + sizeof(BatchHeader));
    const BatchHeader* hdr = reinterpret_cast<const BatchHeader*>(sl.dev);
    return cudaLaunchKernelEx(&lc, kernel_for(kConfigs[cfg]), items, hdr, b->sync);
}

// Collect finished autotuning trials; pick the fastest config once all have run.
void harvest_trials(tsdf_batch* b) {
    std::vector<tsdf_batch::Trial> keep;
    for (auto& t : b->trials) {
        if (cudaEventQuery(t.stop) != cudaSuccess) {
            keep.push_back(t);
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
            if (b->n_timed[t.config] == 0 || ms < b->best_ms[t.config]) b->best_ms[t.config] = ms;
            b->n_timed[t.config]++;
        }
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    b->trials.swap(keep);
    bool all = true;
    for (int c = 0; c < kNumConfigs; ++c)
        all = all && (b->n_timed[c] >= b->trials_per_config || (kConfigs[c].sort && !b->tune_sort));
    if (all && b->tuned < 0) {
        int best = 0;
        for (int c = 1; c < kNumConfigs; ++c)
            if (!(kConfigs[c].sort && !b->tune_sort) && b->best_ms[c] < b->best_ms[best]) best = c;
        b->tuned = best;
        b->config = best;
    }
}

}  // namespace

extern "C" {

int tsdf_batch_create(int32_t max_count, tsdf_batch** out) {
    if (!out || max_count < 1 || max_count > kBatchMax) return TSDF_ERR_INVALID;
    *out = nullptr;
    tsdf_batch* b = new tsdf_batch();
    b->max_count = max_count;
    cudaError_t e = cudaGetDevice(&b->device);
    int sms = 0;
    for (int c = 0; c < kNumConfigs && e == cudaSuccess; ++c)
        e = cudaFuncSetAttribute(kernel_for(kConfigs[c]),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem(kConfigs[c]));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    // each configuration's grid must be co-resident (a cooperative launch)
    for (int c = 0; c < kNumConfigs && e == cudaSuccess; ++c) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(kConfigs[c]), kConfigs[c].threads,
                                                          dyn_smem(kConfigs[c]));
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
        if (kConfigs[c].ctas_per_sm > 0) per_sm = std::min(per_sm, kConfigs[c].ctas_per_sm);
        b->grid_max[c] = sms * std::max(per_sm, 1);
    }
    b->desc_bytes = sizeof(BatchHeader) + (size_t)max_count * sizeof(BatchItem);
    for (auto& s : b->slot) {
        if (e == cudaSuccess) e = cudaMallocHost(&s.host, b->desc_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s.dev, b->desc_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) std::memset(s.host, 0, b->desc_bytes);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->sync, sizeof(BatchSync));
    if (e == cudaSuccess) e = cudaMemset(b->sync, 0, sizeof(BatchSync));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_batch(b);
        return cu_fail(e);
    }
    *out = b;
    return TSDF_OK;
}

int tsdf_batch_destroy(tsdf_batch* b) {
    if (!b) return TSDF_OK;
    DevScope ds(b->device);
    cudaDeviceSynchronize();
    free_batch(b);
    return TSDF_OK;
}

int tsdf_batch_set_option(tsdf_batch* b, int32_t option, int64_t value) {
    if (!b) return TSDF_ERR_INVALID;
    switch (option) {
        case TSDF_BATCH_OPT_GRAPH:
            if (value != 0 && value != 1) return TSDF_ERR_INVALID;
            b->use_graph = value != 0;
            return TSDF_OK;
        case TSDF_BATCH_OPT_AUTOTUNE:
            if (value != 0 && value != 1) return TSDF_ERR_INVALID;
            b->autotune = value != 0;
            return TSDF_OK;
        case TSDF_BATCH_OPT_CONFIG:
            if (value < 0 || value >= kNumConfigs) return TSDF_ERR_INVALID;
            b->config = (int)value;
            b->autotune = false;
            return TSDF_OK;
        case TSDF_BATCH_OPT_SPIN_LIMIT:
            if (value < 1) return TSDF_ERR_INVALID;
            b->spin_limit = value;
            return TSDF_OK;
        case TSDF_BATCH_OPT_GRID_FRACTION:
            // percentage of the co-resident CTAs the launch uses (1..100); the
            // captured graphs are rebuilt for the new grid
            if (value < 1 || value > 100) return TSDF_ERR_INVALID;
            {
                if ((int)value != b->grid_pct) {
                    for (auto& sl : b->slot) {
                        if (sl.pending) {
                            cudaEventSynchronize(sl.done);
                            sl.pending = false;
                        }
                        for (auto& e : sl.exec)
                            if (e) {
                                cudaGraphExecDestroy(e);
                                e = nullptr;
                            }
                    }
                    b->grid_pct = (int)value;
                }
            }
            return TSDF_OK;
        case TSDF_BATCH_OPT_TUNE_SORT:
            if (value != 0 && value != 1) return TSDF_ERR_INVALID;
            b->tune_sort = value != 0;
            return TSDF_OK;
        case TSDF_BATCH_OPT_CTA_BRICK_CACHE:
            if (value != 0 && value != 1) return TSDF_ERR_INVALID;
            b->cta_cache = value != 0;
            return TSDF_OK;
        case TSDF_BATCH_OPT_TEST_MISSING_ARRIVALS:
            if (value < 0 || value > 1024) return TSDF_ERR_INVALID;
            b->extra_arrivals = (int)value;
            return TSDF_OK;
        default: return TSDF_ERR_INVALID;
    }
}

int tsdf_batch_get_config(const tsdf_batch* b, int32_t* config, int32_t* merge, int32_t* steps_per_item,
                          int32_t* reduction, int32_t* tuned, int32_t* threads_per_cta, int32_t* ctas,
                          int32_t* apply_voxel_pairs) {
    if (!b) return TSDF_ERR_INVALID;
    if (config) *config = b->config;
    if (threads_per_cta) *threads_per_cta = kConfigs[b->config].threads;
    if (ctas) *ctas = grid_of(b, b->config);
    if (apply_voxel_pairs) *apply_voxel_pairs = kConfigs[b->config].apply_pairs;
    if (reduction) *reduction = kConfigs[b->config].sort ? TSDF_REDUCTION_SORT : TSDF_REDUCTION_ATOMIC;
    if (merge) *merge = kConfigs[b->config].merge ? 1 : 0;
    if (steps_per_item) *steps_per_item = kConfigs[b->config].kpt;
    if (tuned) *tuned = b->tuned >= 0 ? 1 : 0;
    return TSDF_OK;
}

int tsdf_batch_integrate(tsdf_batch* b, tsdf_map* const* maps, const float* const* points_dev, const int64_t* n,
                         const float* poses, int32_t count, void* stream) {
    if (!b || !maps || !points_dev || !n || !poses || count < 0 || count > b->max_count) return TSDF_ERR_INVALID;
    if (count == 0) return TSDF_OK;
    for (int i = 0; i < count; ++i) {
        if (!maps[i] || map_device(maps[i]) != b->device) return TSDF_ERR_INVALID;
        for (int j = 0; j < i; ++j)
            if (maps[j] == maps[i]) return TSDF_ERR_INVALID;   // one scan per map per batch
    }
    DevScope ds(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int si = b->next_slot;
    tsdf_batch::Slot& sl = b->slot[si];
    if (sl.pending) {   // the GPU may still be reading this slot's host buffer
        cudaError_t e = cudaEventSynchronize(sl.done);
        if (e != cudaSuccess) return cu_fail(e);
        sl.pending = false;
    }
    if (b->autotune && b->tuned < 0) harvest_trials(b);
    int cfg = b->config;
    bool timing = false;
    if (b->autotune && b->tuned < 0) {
        // cycle through the configurations until each has been timed enough
        int pending_of[kNumConfigs] = {};
        for (auto& t : b->trials) pending_of[t.config]++;
        for (int c = 0; c < kNumConfigs; ++c) {
            if (kConfigs[c].sort && !b->tune_sort) continue;
            if (b->n_timed[c] + pending_of[c] < b->trials_per_config) {
                cfg = c;
                timing = true;
                break;
            }
        }
    }
    BatchHeader* hdr = reinterpret_cast<BatchHeader*>(sl.host);
    BatchItem* items = reinterpret_cast<BatchItem*>(sl.host + sizeof(BatchHeader));
    uint32_t rt = 0, wt = 0;
    bool small_maps = count < 1023;
    const int64_t task_points = (int64_t)kConfigs[cfg].threads * kConfigs[cfg].rays_ppt;
    for (int i = 0; i < count; ++i) {
        if (kConfigs[cfg].sort) {   // the sort buffers must exist before the descriptors are taken
            int rc = map_reserve_sort(maps[i], n[i]);
            if (rc != TSDF_OK) return rc;
        }
        int rc = prepare_batch_item(maps[i], points_dev[i], n[i], poses + 12 * i, &items[i]);
        if (rc != TSDF_OK) return rc;
        hdr->ray_prefix[i] = rt;
        hdr->word_prefix[i] = wt;
        rt += (uint32_t)((n[i] + task_points - 1) / task_points);
        wt += ((items[i].bricks + 3u) / 4u + 31u) / 32u;
        small_maps = small_maps && items[i].bricks < (1u << kTagShift);
    }
    hdr->ray_prefix[count] = rt;
    hdr->word_prefix[count] = wt;
    hdr->count = count;
    hdr->ray_tasks = rt;
    hdr->word_tasks = wt;
    hdr->extra_arrivals = (uint32_t)b->extra_arrivals;
    hdr->cta_cache = small_maps && b->cta_cache ? 1u : 0u;
    hdr->spin_limit = b->spin_limit;

    cudaError_t e = cudaSuccess;
    tsdf_batch::Trial trial{cfg, nullptr, nullptr};
    if (timing) {
        e = cudaEventCreate(&trial.start);
        if (e == cudaSuccess) e = cudaEventCreate(&trial.stop);
        if (e == cudaSuccess) e = cudaEventRecord(trial.start, s);
    }
    if (e == cudaSuccess) {
        if (b->use_graph) {
            if (!sl.exec[cfg]) {
                // capture copy + reset + kernel once for this slot and config
                cudaGraph_t g = nullptr;
                e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e2 = enqueue(b, si, cfg, b->capture_stream);
                    e = cudaStreamEndCapture(b->capture_stream, &g);
                    if (e == cudaSuccess) e = e2;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.exec[cfg], g, 0);
                if (g) cudaGraphDestroy(g);
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec[cfg], s);
        } else {
            e = enqueue(b, si, cfg, s);
        }
    }
    if (e == cudaSuccess && timing) {
        e = cudaEventRecord(trial.stop, s);
        if (e == cudaSuccess) b->trials.push_back(trial);
    } else if (timing) {
        if (trial.start) cudaEventDestroy(trial.start);
        if (trial.stop) cudaEventDestroy(trial.stop);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, s);
    if (e != cudaSuccess) return cu_fail(e);
    sl.pending = true;
    b->next_slot ^= 1;
    return TSDF_OK;
}

int tsdf_integrate_batch(tsdf_map* const* maps, const float* const* points_dev, const int64_t* n, const float* poses,
                         int32_t count, void* stream) {
    // one batch object per host thread and device, created on first use and
    // destroyed when the thread exits
    struct PerThread {
        tsdf_batch* b[64] = {};
        ~PerThread() {
            for (tsdf_batch* x : b) tsdf_batch_destroy(x);
        }
    };
    static thread_local PerThread per_thread;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TSDF_ERR_CUDA;
    tsdf_batch*& b = per_thread.b[dev];
    if (!b) {
        int rc = tsdf_batch_create(kBatchMax, &b);
        if (rc != TSDF_OK) return rc;
    }
    return tsdf_batch_integrate(b, maps, points_dev, n, poses, count, stream);
}

int tsdf_batch_sync(tsdf_batch* b, void* stream) {
    if (!b) return TSDF_ERR_INVALID;
    DevScope ds(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, &b->sync->error, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cu_fail(e);
    return err ? TSDF_ERR_TIMEOUT : TSDF_OK;
}

}  // extern "C"
