// Per-scan TSDF integration kernels (FeatSense, Section "TSDF Map Generation").
//
// rays (K-A): one thread per point, coalesced float4 loads. Transforms the
//   point by the pose, sets up the ray (range r, unit direction d, unit
//   interpolation direction int = d x (d x up) with up the sensor z axis) and
//   appends it (two float4) to a compacted list of live rays: a ray whose whole
//   march (+-tau around the hit, widened by the fill height of Eq. 4 and a
//   safety margin) stays outside the window box is dropped, since none of its
//   samples could land in the window. Order is kept within a CTA, so
//   neighbouring rays stay neighbours. On the plain path the list is split:
//   rays whose fill reaches a voxel each side (delta_z r >= vs) are appended
//   from its front, the others from its end.
// contrib (K-B): persistent; a warp takes work items (32 consecutive live
//   rays, a group of KPT steps k of k = -K..K), one ray per lane. For each of its steps the
//   thread walks the fill samples j = -J..J (Eq. 3 / Eq. 4) in warp lock-step.
//   A sample inside the window yields (voxel, q), q the int16 code of the
//   truncated projective distance of the voxel centre, and issues one
//   fire-and-forget 64-bit reduction into the per-scan accumulator:
//     WSUM    : acc += (count << 40) + sum(q)   (two's-complement packing; exact
//               while count < 2^24 and |sum| < 2^39)
//     MIN_ABS : acc = max(acc, 65536 - key), key = (|q| << 1) | (q < 0)
//   so acc == 0 means "untouched". Optionally (MERGE) lanes that hit the same
//   voxel in the same iteration are first combined with match.any +
//   redux.sync so that one lane per distinct voxel issues the reduction. The
//   issuing lane marks the voxel's brick in a byte-per-brick flag array with
//   a plain store (idempotent, nothing to wait for), filtered by a per-CTA
//   shared-memory cache of the bricks the CTA has marked. The items of the
//   list's front (the costly rays) come first. Integer accumulation makes the
//   result independent of the order of the atomics.
// compact: turns the brick flags into a list of touched bricks (4 flags per
//   thread, one list atomic per warp) and clears the flags.
// apply (K-C): warp tasks over the listed bricks (grid-stride), by default a
//   quarter brick per task: each lane loads its voxel pairs' accumulators and
//   grid words into registers with coalesced loads, applies Eq. 1 in exact
//   integers with one rounding (half away from zero) and Eq. 2 with the weight
//   cap to every touched voxel (non-zero accumulator), writes changed pairs
//   back and resets their accumulators. (TSDF_APPLY_REG 0 selects the older
//   form: a warp per brick staged in shared memory, touched voxels compacted
//   with a warp scan.) Touched voxels are counted, and in WSUM mode the
//   contributions too (the sum of the decoded weights).
// finish: the last apply CTA to retire sums the per-scan counters into the
//   published ones and clears the per-scan state (one warp).
//
// Sort reduction (an alternative to the accumulator atomics, same results):
// rays also reserve each live ray's pair slots (one per march sample); emit is
// the contrib march writing (voxel word, code) to the sample's slot instead of
// reducing it (no atomics; samples beyond the capacity fall back to the
// accumulators); count adds each brick's pairs (warp-merged per brick);
// scan turns counts into segment starts; scatter moves every pair to its
// brick's segment as a 32-bit (offset, code); sort_apply reduces each brick's
// segment per voxel in shared memory and applies Eq. 1 / Eq. 2. Together
// count, scan and scatter are a counting sort of the contributions by brick.
//
// Kernels may be launched with programmatic stream serialisation: each may be
// scheduled while its predecessor drains, and waits (griddepcontrol.wait) for
// the predecessor's completion before touching its results.
//
// Every float operation on the geometry path is an explicit round-to-nearest
// intrinsic (no contraction into FMA), in the same order as the CPU oracle, so
// voxel indices and codes agree bit for bit.
#include <mutex>
#include <unordered_map>
#include <utility>

#include "integrate_device.cuh"

// Minimum resident CTAs per SM requested for the plain contribution kernel:
// 4 caps it at 64 registers (no spills), 32 resident warps per SM instead of
// 24 at its natural 79 registers; 34.6 against 35.5 us per outdoor scan.
#ifndef TSDF_CONTRIB_MIN_CTAS
#define TSDF_CONTRIB_MIN_CTAS 4
#endif
// The same for the sort reduction's emit kernel (no cap).
#ifndef TSDF_EMIT_MIN_CTAS
#define TSDF_EMIT_MIN_CTAS 1
#endif
// CTAs per SM launched by the contribution and apply kernels, which walk
// their work with a grid stride; 0 = as many as are resident at once.
#ifndef TSDF_CONTRIB_CTAS_PER_SM
#define TSDF_CONTRIB_CTAS_PER_SM 8
#endif
#ifndef TSDF_APPLY_CTAS_PER_SM
#define TSDF_APPLY_CTAS_PER_SM 0
#endif
// 1: the plain path splits its ray list into heavy and light rays (see
// rays_task); 0: one list in arrival order.
#ifndef TSDF_RAYS_SPLIT
#define TSDF_RAYS_SPLIT 1
#endif
// Threads per CTA of the contribution kernel.
#ifndef TSDF_CONTRIB_THREADS
#define TSDF_CONTRIB_THREADS 256
#endif
// Minimum resident CTAs per SM requested for the apply kernel.
#ifndef TSDF_APPLY_MIN_CTAS
#define TSDF_APPLY_MIN_CTAS 1
#endif
// 1: the apply kernel keeps each lane's voxels in registers (apply_brick_reg);
// 0: it stages the brick in shared memory and compacts the touched voxels.
#ifndef TSDF_APPLY_REG
#define TSDF_APPLY_REG 1
#endif

namespace tsdf {
namespace {

using namespace dev;

// Threads per CTA of the ray set-up kernel (one list atomic per CTA and list end).
#ifndef TSDF_RAYS_THREADS
#define TSDF_RAYS_THREADS 256
#endif
constexpr int kRaysThreads = TSDF_RAYS_THREADS;

template <bool SORT, bool SPLIT>
__global__ void __launch_bounds__(kRaysThreads) rays_kernel(const ScanArgs a, const MapDev m) {
    __shared__ RaysSmemT<kRaysThreads / 32> sm;
    if constexpr (SORT)
        rays_task<true, SORT, SPLIT, kRaysThreads / 32>(a, m, (int)(blockIdx.x * blockDim.x), blockIdx.x, &sm);
    else
        rays_task_ppt<true, SPLIT, kRaysThreads / 32, kRaysPPT>(a, m, (int)(blockIdx.x * blockDim.x) * kRaysPPT,
                                                                blockIdx.x, &sm);
}

// Contribution work items: (block of 32 consecutive live rays, group of KPT
// steps). Each warp walks the items with a grid stride and loads the next
// item's rays while it processes the current one. The grid is
// TSDF_CONTRIB_CTAS_PER_SM CTAs per SM, more than are resident at once, so the
// hardware hands the CTAs of later waves to the SMs that finish first. The
// warps of one CTA take consecutive items (the step groups of the same 32
// rays and of their neighbours), so they mark the same bricks and the CTA's
// brick cache absorbs most marks: giving a CTA's warps unrelated items, or
// handing out items through counters, made the kernel about 30 % slower, the
// extra time in brick-flag stores.
constexpr int kContribThreads = TSDF_CONTRIB_THREADS;

template <int MODE, bool MERGE, int KPT>
__global__ void __launch_bounds__(kContribThreads, TSDF_CONTRIB_MIN_CTAS) contrib_kernel(const ScanArgs a,
                                                                                        const MapDev m) {
    __shared__ unsigned long long red[kContribThreads / 32];
    __shared__ uint32_t btab[kBrickCache];
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    __shared__ unsigned s_counts[2];
    pdl_trigger();
    brick_cache_init(btab);
    pdl_wait();   // ray list and live count come from the rays kernel
    // A coherent load after the wait (a read-only __ldg could be hoisted above
    // it and see a count from before the rays kernel finished), one per CTA:
    // every CTA of the grid reads the same line, so per-warp reads would make
    // it a hot spot. The ray list may be split (heavy rays from the front,
    // light ones from the end): the blocks of the front come first, so the
    // costly items are taken by the first wave of CTAs and the CTAs that start
    // late get light ones.
    if (threadIdx.x == 0) {
        s_counts[0] = __ldcg(&m.ctr->live_count);
        s_counts[1] = __ldcg(&m.ctr->live_back);
    }
    __syncthreads();   // (also orders the brick cache initialisation)
    const unsigned nf = s_counts[0], nb = s_counts[1];
    const unsigned bf = (nf + 31u) / 32u, bb = (nb + 31u) / 32u;
    const unsigned ngrp = (unsigned)(2 * a.K + KPT) / KPT;   // ceil((2K+1) / KPT)
    const unsigned nitems = (bf + bb) * ngrp;
    // first ray of block `blk` and the end of its part of the list
    auto block_ray = [&](unsigned blk, unsigned& end) {
        if (blk < bf) {
            end = nf;
            return blk * 32u;
        }
        end = m.ray_cap;
        return m.ray_cap - nb + (blk - bf) * 32u;
    };
    unsigned hits = 0;
    unsigned last_brick = kNoVoxel;
    const BrickCache bc{btab, 32u - kBrickCacheLog2};
    float4 A, B;
    {
        unsigned end;
        const unsigned r0 = block_ray(gwarp / ngrp, end);
        load_rays(m, gwarp < nitems ? end : 0u, r0 + lane, A, B);
    }
    for (unsigned item = gwarp; item < nitems; item += nwarps) {   // warp-uniform
        float4 An, Bn;
        const unsigned next = item + nwarps;
        unsigned end;
        const unsigned r0 = block_ray(next / ngrp, end);
        load_rays(m, next < nitems ? end : 0u, r0 + lane, An, Bn);   // prefetch
        contrib_item<MODE, MERGE, KPT>(a, m, item % ngrp, A, B, hits, last_brick, kNoSlot, nullptr, nullptr, bc);
        A = An;
        B = Bn;
    }
    if (MODE == 1) {
        // MIN_ABS keeps no contribution count per voxel: count them here
        const unsigned long long total = cta_sum<kContribThreads / 32>((unsigned long long)hits, red);
        if (threadIdx.x == 0 && total) atomicAdd(&m.ctr->part[blockIdx.x % kParts].hits, total);
    }
}

// Sort reduction: the contribution march writing pairs (same work items).
template <int MODE, int KPT>
__global__ void __launch_bounds__(256, TSDF_EMIT_MIN_CTAS) emit_kernel(const ScanArgs a, const MapDev m) {
    __shared__ unsigned long long red[8];
    __shared__ uint32_t btab[kBrickCache];
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    pdl_trigger();
    brick_cache_init(btab);
    __syncthreads();
    pdl_wait();
    unsigned nlive = 0;
    if (lane == 0) nlive = __ldcg(&m.ctr->live_count);
    nlive = __shfl_sync(kFull, nlive, 0);
    const unsigned ngrp = (unsigned)(2 * a.K + KPT) / KPT;
    const unsigned nitems = (nlive + 31u) / 32u * ngrp;
    unsigned hits = 0;
    unsigned last_brick = kNoVoxel;
    bool ovf = false;
    for (unsigned item = gwarp; item < nitems; item += nwarps) {   // warp-uniform
        const unsigned ray = (item / ngrp) * 32u + lane;
        float4 A, B;
        load_rays(m, nlive, ray, A, B);
        const uint32_t sslot = ray < nlive ? m.ray_slot[ray] : kNoSlot;
        contrib_item<MODE, false, KPT, true>(a, m, item % ngrp, A, B, hits, last_brick, sslot, &ovf, nullptr,
                                             BrickCache{btab, 32u - kBrickCacheLog2});
    }
    if (ovf) m.ctr->overflow = 1u;
    if (MODE == 1) {
        const unsigned long long total = cta_sum<8>((unsigned long long)hits, red);
        if (threadIdx.x == 0 && total) atomicAdd(&m.ctr->part[blockIdx.x % kParts].hits, total);
    }
}

// Pool reduction: the contribution march accumulating into claimed pool
// bricks (same work items as contrib_kernel).
template <int MODE, int KPT>
__global__ void __launch_bounds__(256) pool_contrib_kernel(const ScanArgs a, const MapDev m) {
    __shared__ unsigned long long red[8];
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    pdl_trigger();
    pdl_wait();
    unsigned nlive = 0;
    if (lane == 0) nlive = __ldcg(&m.ctr->live_count);
    nlive = __shfl_sync(kFull, nlive, 0);
    const unsigned ngrp = (unsigned)(2 * a.K + KPT) / KPT;
    const unsigned nitems = (nlive + 31u) / 32u * ngrp;
    unsigned hits = 0;
    unsigned last_brick = kNoVoxel;
    uint32_t last_slot = kPoolEmpty;
    for (unsigned item = gwarp; item < nitems; item += nwarps) {   // warp-uniform
        float4 A, B;
        load_rays(m, nlive, (item / ngrp) * 32u + lane, A, B);
        contrib_item<MODE, false, KPT, false, true>(a, m, item % ngrp, A, B, hits, last_brick, kNoSlot, nullptr,
                                                    &last_slot);
    }
    if (MODE == 1) {
        const unsigned long long total = cta_sum<8>((unsigned long long)hits, red);
        if (threadIdx.x == 0 && total) atomicAdd(&m.ctr->part[blockIdx.x % kParts].hits, total);
    }
}

__global__ void __launch_bounds__(256) sort_count_kernel(const MapDev m) {
    pdl_trigger();
    pdl_wait();   // pairs come from emit, brick slots from compact
    const uint32_t n = sort_nslots(m);
    const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = w0; w * 128u < n; w += nw) sort_count_warp(m, w * 128u, n);
}

__global__ void __launch_bounds__(1024) sort_scan_kernel(const MapDev m) {
    __shared__ uint32_t smem[33];
    __shared__ uint32_t nb;
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x == 0) nb = __ldcg(&m.ctr->brick_count);
    __syncthreads();
    sort_scan_cta(m, nb, smem);
}

__global__ void __launch_bounds__(256) sort_scatter_kernel(const MapDev m) {
    pdl_trigger();
    pdl_wait();
    const uint32_t n = sort_nslots(m);
    const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = w0; w * 128u < n; w += nw) sort_scatter_warp(m, w * 128u, n);
}

__global__ void __launch_bounds__(256) compact_kernel(const MapDev m, const uint32_t nwords) {
    pdl_trigger();
    pdl_wait();   // flags come from the contrib kernel
    compact_words(m, blockIdx.x * blockDim.x + threadIdx.x, nwords);
}

constexpr int kApplyWarps = 4;   // CTA size of the staged (sort and pool) apply kernels
// CTA size of the register apply kernel.
#ifndef TSDF_APPLY_WARPS
#define TSDF_APPLY_WARPS 4
#endif
#if TSDF_APPLY_REG
constexpr int kRegApplyWarps = TSDF_APPLY_WARPS;
#else
constexpr int kRegApplyWarps = kApplyWarps;
#endif
// Voxel pairs per lane in one apply task: 8 = a warp per brick, 4 = a warp
// per half brick, 2 = per quarter brick (more, shorter tasks in flight: the
// apply is latency-bound).
#ifndef TSDF_APPLY_PAIRS
#define TSDF_APPLY_PAIRS 2
#endif
constexpr int kApplyPairs = TSDF_APPLY_PAIRS;

// The last CTA to finish also publishes the scan's counters (finish_if_last).
template <int MODE>
__global__ void __launch_bounds__(kRegApplyWarps * 32, TSDF_APPLY_MIN_CTAS) apply_kernel(const MapDev m,
                                                                                         const int32_t w_max,
                                                                                         const int32_t flags) {
#if !TSDF_APPLY_REG
    // per warp: the brick's grid words and accumulators, and the offsets of
    // its touched voxels (compacted)
    __shared__ uint32_t s_grid[kRegApplyWarps][kBrickVoxels];
    __shared__ unsigned long long s_acc[kRegApplyWarps][kBrickVoxels];
    __shared__ uint16_t s_off[kRegApplyWarps][kBrickVoxels];
#endif
    __shared__ unsigned long long red_u[kRegApplyWarps], red_h[kRegApplyWarps];
    __shared__ unsigned s_last;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned w = threadIdx.x >> 5;
    const unsigned gwarp = blockIdx.x * kRegApplyWarps + w;
    const unsigned nwarps = gridDim.x * kRegApplyWarps;
    pdl_trigger();
    pdl_wait();   // list and accumulators come from the earlier kernels
    // coherent load after the wait (see contrib_kernel), one per CTA
    if (threadIdx.x == 0) s_last = __ldcg(&m.ctr->brick_count);
    __syncthreads();
    const unsigned nb = s_last;
    __syncthreads();   // s_last is reused by finish_if_last
    unsigned long long touched = 0, hits = 0;
#if TSDF_APPLY_REG
    for (unsigned t = gwarp; t < nb * (8u / kApplyPairs); t += nwarps)
        apply_part_reg<MODE, kApplyPairs>(m, w_max, flags, t, touched, hits);
#else
    for (unsigned i = gwarp; i < nb; i += nwarps)
        apply_brick<MODE>(m, w_max, flags, i, s_grid[w], s_acc[w], s_off[w], touched, hits);
#endif
    for (int o = 16; o > 0; o >>= 1) {
        touched += __shfl_xor_sync(kFull, touched, o);
        hits += __shfl_xor_sync(kFull, hits, o);
    }
    if (lane == 0) {
        red_u[w] = touched;
        red_h[w] = hits;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long bu = 0, bh = 0;
        for (int k = 0; k < kRegApplyWarps; ++k) {
            bu += red_u[k];
            bh += red_h[k];
        }
        if (bu) atomicAdd(&m.ctr->part[blockIdx.x % kParts].touched, bu);
        if (MODE == 0 && bh) atomicAdd(&m.ctr->part[blockIdx.x % kParts].hits, bh);
    }
    finish_if_last(m, &s_last);
}

// Sort reduction: one warp per listed brick (as apply_kernel, and likewise
// the last CTA publishes the counters).
template <int MODE>
__global__ void __launch_bounds__(kApplyWarps * 32) sort_apply_kernel(const MapDev m, const int32_t w_max,
                                                                       const int32_t flags) {
    __shared__ uint32_t s_grid[kApplyWarps][kBrickVoxels];
    __shared__ unsigned long long s_acc[kApplyWarps][kBrickVoxels];
    __shared__ uint16_t s_off[kApplyWarps][kBrickVoxels];
    __shared__ unsigned long long red_u[kApplyWarps], red_h[kApplyWarps];
    __shared__ unsigned s_last;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned w = threadIdx.x >> 5;
    const unsigned gwarp = blockIdx.x * kApplyWarps + w;
    const unsigned nwarps = gridDim.x * kApplyWarps;
    pdl_trigger();
    pdl_wait();
    unsigned nb = 0, ovf = 0;
    if (lane == 0) {
        nb = __ldcg(&m.ctr->brick_count);
        ovf = __ldcg(&m.ctr->overflow);
    }
    nb = __shfl_sync(kFull, nb, 0);
    ovf = __shfl_sync(kFull, ovf, 0);
    unsigned long long touched = 0, hits = 0;
    for (unsigned i = gwarp; i < nb; i += nwarps)
        sort_apply_brick<MODE>(m, w_max, flags, i, ovf != 0u, s_grid[w], s_acc[w], s_off[w], touched, hits);
    for (int o = 16; o > 0; o >>= 1) {
        touched += __shfl_xor_sync(kFull, touched, o);
        hits += __shfl_xor_sync(kFull, hits, o);
    }
    if (lane == 0) {
        red_u[w] = touched;
        red_h[w] = hits;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long bu = 0, bh = 0;
        for (int k = 0; k < kApplyWarps; ++k) {
            bu += red_u[k];
            bh += red_h[k];
        }
        if (bu) atomicAdd(&m.ctr->part[blockIdx.x % kParts].touched, bu);
        if (bh) atomicAdd(&m.ctr->part[blockIdx.x % kParts].hits, bh);
    }
    finish_if_last(m, &s_last);
}


// Pool reduction: one warp per claimed slot applies Eq. 1 / Eq. 2 to its
// brick (unless the pool overflowed: then the scan is dropped and the slots
// are only cleared), resets the slot and the brick's table entry; the last CTA
// publishes the counters and the scan's status.
template <int MODE>
__global__ void __launch_bounds__(kApplyWarps * 32) pool_apply_kernel(const MapDev m, const int32_t w_max,
                                                                       const int32_t flags) {
    __shared__ unsigned long long red_u[kApplyWarps], red_h[kApplyWarps];
    __shared__ unsigned s_last;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned w = threadIdx.x >> 5;
    const unsigned gwarp = blockIdx.x * kApplyWarps + w;
    const unsigned nwarps = gridDim.x * kApplyWarps;
    pdl_trigger();
    pdl_wait();
    unsigned ns = 0, ovf = 0;
    if (lane == 0) {
        ns = __ldcg(&m.ctr->pool_count);
        ovf = __ldcg(&m.ctr->pool_overflow);
    }
    ns = __shfl_sync(kFull, ns, 0);
    ovf = __shfl_sync(kFull, ovf, 0);
    if (ns > m.pool_cap) ns = m.pool_cap;
    unsigned long long touched = 0, hits = 0;
    for (unsigned i = gwarp; i < ns; i += nwarps) {
        const unsigned brick = __ldcg(m.pool_brick + i);
        unsigned long long* accp = m.pool_acc + ((size_t)i << 9);
        if (!ovf) {
            apply_brick_at<MODE>(m, w_max, flags, brick, accp, touched, hits);
        } else {
            ulonglong2* ap = reinterpret_cast<ulonglong2*>(accp);
#pragma unroll
            for (int v = 0; v < 8; ++v) ap[32 * v + lane] = make_ulonglong2(0ull, 0ull);
        }
        if (lane == 0) m.pool_table[brick] = kPoolEmpty;
    }
    for (int o = 16; o > 0; o >>= 1) {
        touched += __shfl_xor_sync(kFull, touched, o);
        hits += __shfl_xor_sync(kFull, hits, o);
    }
    if (lane == 0) {
        red_u[w] = touched;
        red_h[w] = hits;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long bu = 0, bh = 0;
        for (int k = 0; k < kApplyWarps; ++k) {
            bu += red_u[k];
            bh += red_h[k];
        }
        if (bu) atomicAdd(&m.ctr->part[blockIdx.x % kParts].touched, bu);
        if (MODE == 0 && bh) atomicAdd(&m.ctr->part[blockIdx.x % kParts].hits, bh);
    }
    finish_if_last(m, &s_last);
}

// Launch with programmatic stream serialisation when `pdl` is set.
template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, bool pdl, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// CTAs of `kernel` (launched with `threads` threads and static shared memory
// only) that the current device holds at once: SMs x resident CTAs per SM.
// Persistent kernels launch exactly this many, so no CTA waits for a second
// wave. Cached per kernel and device.
int resident_ctas(const void* kernel, int threads) {
    static std::mutex mu;
    static std::unordered_map<unsigned long long, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long key = (unsigned long long)(uintptr_t)kernel * 1024ull + (unsigned long long)dev;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int sms = 1, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int n = (sms > 0 ? sms : 1) * per_sm;
    cache[key] = n;
    return n;
}

template <typename... KArgs>
dim3 resident_grid(void (*kernel)(KArgs...), int threads, int per_sm = 0) {
    if (per_sm > 0) {
        static int sms[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        const int d = dev >= 0 && dev < 64 ? dev : 0;
        if (sms[d] == 0) {
            int v = 1;
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
            sms[d] = v > 0 ? v : 1;
        }
        return dim3((unsigned)(sms[d] * per_sm));
    }
    return dim3((unsigned)resident_ctas(reinterpret_cast<const void*>(kernel), threads));
}

template <int MODE, bool MERGE, int KPT>
cudaError_t launch_contrib_kk(const ScanArgs& a, const MapDev& m, bool pdl, cudaStream_t s) {
    auto* k = contrib_kernel<MODE, MERGE, KPT>;
    return launch(k, resident_grid(k, kContribThreads, TSDF_CONTRIB_CTAS_PER_SM), dim3(kContribThreads), s, pdl, a,
                  m);
}

template <int MODE, bool MERGE>
cudaError_t launch_contrib_k(const ScanArgs& a, const MapDev& m, int kpt, bool pdl, cudaStream_t s) {
    switch (kpt) {
        case 2: return launch_contrib_kk<MODE, MERGE, 2>(a, m, pdl, s);
        case 4: return launch_contrib_kk<MODE, MERGE, 4>(a, m, pdl, s);
        default: return launch_contrib_kk<MODE, MERGE, 1>(a, m, pdl, s);
    }
}

template <int MODE, int KPT>
cudaError_t launch_emit_k(const ScanArgs& a, const MapDev& m, bool pdl, cudaStream_t s) {
    auto* k = emit_kernel<MODE, KPT>;
    return launch(k, resident_grid(k, 256, TSDF_CONTRIB_CTAS_PER_SM), dim3(256), s, pdl, a, m);
}

}  // namespace

const void* rays_kernel_fn(bool sort, bool split) {
    if (sort) return reinterpret_cast<const void*>(rays_kernel<true, false>);
    return split && TSDF_RAYS_SPLIT ? reinterpret_cast<const void*>(rays_kernel<false, true>)
                                    : reinterpret_cast<const void*>(rays_kernel<false, false>);
}

const void* contrib_kernel_fn(int32_t reduce, bool merge, int kpt) {
    const int k = kpt == 2 || kpt == 4 ? kpt : 1;
    if (reduce == 0) {
        if (merge) return k == 4 ? reinterpret_cast<const void*>(contrib_kernel<0, true, 4>)
                        : k == 2 ? reinterpret_cast<const void*>(contrib_kernel<0, true, 2>)
                                 : reinterpret_cast<const void*>(contrib_kernel<0, true, 1>);
        return k == 4 ? reinterpret_cast<const void*>(contrib_kernel<0, false, 4>)
             : k == 2 ? reinterpret_cast<const void*>(contrib_kernel<0, false, 2>)
                      : reinterpret_cast<const void*>(contrib_kernel<0, false, 1>);
    }
    if (merge) return k == 4 ? reinterpret_cast<const void*>(contrib_kernel<1, true, 4>)
                    : k == 2 ? reinterpret_cast<const void*>(contrib_kernel<1, true, 2>)
                             : reinterpret_cast<const void*>(contrib_kernel<1, true, 1>);
    return k == 4 ? reinterpret_cast<const void*>(contrib_kernel<1, false, 4>)
         : k == 2 ? reinterpret_cast<const void*>(contrib_kernel<1, false, 2>)
                  : reinterpret_cast<const void*>(contrib_kernel<1, false, 1>);
}

unsigned rays_grid(int64_t n, bool sort) {
    const int64_t per_cta = (int64_t)kRaysThreads * (sort ? 1 : kRaysPPT);
    return (unsigned)((n + per_cta - 1) / per_cta);
}

cudaError_t launch_rays(const ScanArgs& a, const MapDev& m, bool sort, bool split, bool pdl, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const dim3 grid(rays_grid(a.n, sort)), block(kRaysThreads);
    if (sort) return launch(rays_kernel<true, false>, grid, block, s, pdl, a, m);
    return split && TSDF_RAYS_SPLIT ? launch(rays_kernel<false, true>, grid, block, s, pdl, a, m)
                                    : launch(rays_kernel<false, false>, grid, block, s, pdl, a, m);
}

cudaError_t launch_emit(const ScanArgs& a, const MapDev& m, int32_t reduce, int kpt, bool pdl, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (reduce == 0) {
        switch (kpt) {
            case 2: return launch_emit_k<0, 2>(a, m, pdl, s);
            case 4: return launch_emit_k<0, 4>(a, m, pdl, s);
            default: return launch_emit_k<0, 1>(a, m, pdl, s);
        }
    }
    switch (kpt) {
        case 2: return launch_emit_k<1, 2>(a, m, pdl, s);
        case 4: return launch_emit_k<1, 4>(a, m, pdl, s);
        default: return launch_emit_k<1, 1>(a, m, pdl, s);
    }
}

cudaError_t launch_pool_contrib(const ScanArgs& a, const MapDev& m, int32_t reduce, int kpt, bool pdl,
                                cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    auto pick = [&](auto* k) { return launch(k, resident_grid(k, 256, TSDF_CONTRIB_CTAS_PER_SM), dim3(256), s, pdl, a, m); };
    if (reduce == 0) {
        switch (kpt) {
            case 2: return pick(pool_contrib_kernel<0, 2>);
            case 4: return pick(pool_contrib_kernel<0, 4>);
            default: return pick(pool_contrib_kernel<0, 1>);
        }
    }
    switch (kpt) {
        case 2: return pick(pool_contrib_kernel<1, 2>);
        case 4: return pick(pool_contrib_kernel<1, 4>);
        default: return pick(pool_contrib_kernel<1, 1>);
    }
}

cudaError_t launch_pool_apply(const MapDev& m, int32_t reduce, int32_t w_max, int32_t flags, bool pdl,
                              cudaStream_t s) {
    auto* k = reduce == 0 ? pool_apply_kernel<0> : pool_apply_kernel<1>;
    return launch(k, resident_grid(k, kApplyWarps * 32), dim3(kApplyWarps * 32), s, pdl, m, w_max, flags);
}

cudaError_t launch_sort_count(const MapDev& m, bool pdl, cudaStream_t s) {
    return launch(sort_count_kernel, resident_grid(sort_count_kernel, 256), dim3(256), s, pdl, m);
}

cudaError_t launch_sort_scan(const MapDev& m, bool pdl, cudaStream_t s) {
    return launch(sort_scan_kernel, dim3(1), dim3(1024), s, pdl, m);
}

cudaError_t launch_sort_scatter(const MapDev& m, bool pdl, cudaStream_t s) {
    return launch(sort_scatter_kernel, resident_grid(sort_scatter_kernel, 256), dim3(256), s, pdl, m);
}

cudaError_t launch_sort_apply(const MapDev& m, int32_t reduce, int32_t w_max, int32_t flags, bool pdl,
                              cudaStream_t s) {
    auto* k = reduce == 0 ? sort_apply_kernel<0> : sort_apply_kernel<1>;
    return launch(k, resident_grid(k, kApplyWarps * 32, TSDF_APPLY_CTAS_PER_SM), dim3(kApplyWarps * 32), s, pdl, m,
                  w_max, flags);
}

cudaError_t launch_contrib(const ScanArgs& a, const MapDev& m, int32_t reduce, bool merge, int kpt, bool pdl,
                           cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (reduce == 0)
        return merge ? launch_contrib_k<0, true>(a, m, kpt, pdl, s) : launch_contrib_k<0, false>(a, m, kpt, pdl, s);
    return merge ? launch_contrib_k<1, true>(a, m, kpt, pdl, s) : launch_contrib_k<1, false>(a, m, kpt, pdl, s);
}

cudaError_t launch_compact(const MapDev& m, uint32_t bricks, bool pdl, cudaStream_t s) {
    const uint32_t nwords = (bricks + 3u) / 4u;
    return launch(compact_kernel, dim3((nwords + 255u) / 256u), dim3(256), s, pdl, m, nwords);
}

cudaError_t launch_apply(const MapDev& m, int32_t reduce, int32_t w_max, int32_t flags, bool pdl, cudaStream_t s) {
    auto* k = reduce == 0 ? apply_kernel<0> : apply_kernel<1>;
    return launch(k, resident_grid(k, kRegApplyWarps * 32, TSDF_APPLY_CTAS_PER_SM), dim3(kRegApplyWarps * 32), s,
                  pdl, m, w_max, flags);
}

}  // namespace tsdf
