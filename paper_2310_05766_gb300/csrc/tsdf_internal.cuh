// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

struct tsdf_map;   // host-side map object (defined in api.cu)

namespace tsdf {

constexpr int32_t kQMax = 32767;
constexpr int kBrick = 8;                 // bricks are 8 x 8 x 8 voxels, stored contiguously
constexpr int kBrickVoxels = 512;

constexpr int32_t kFlagStepValue = 1;    // TSDF_FLAG_STEP_VALUE
constexpr int32_t kFlagScanWeight = 2;   // TSDF_FLAG_SCAN_WEIGHT

constexpr int kParts = 32;        // counters are spread over 32 slots, one 128-byte line each

// Per-map device counters (one instance per map, in device memory). The
// counters of the scan in flight are split over kParts slots so that CTAs
// add to different L2 lines; the finish kernel sums them.
struct CounterPart {
    unsigned long long valid;       // valid rays
    unsigned long long hits;        // in-window contributions
    unsigned long long touched;     // voxels updated
    unsigned long long pad[13];
};
struct MapCounters {
    CounterPart part[kParts];
    long long last_valid;           // counters of the last completed scan
    long long last_hits;
    long long last_touched;
    long long last_status;          // 0, or TSDF_ERR_CAPACITY when the scan was dropped (pool full)
    unsigned int live_count;        // rays of the scan in flight that can reach the window (compacted)
    unsigned int brick_count;       // length of the touched-brick list of the scan in flight
    unsigned long long slot_count;  // sort reduction: pair slots reserved by the scan in flight
    unsigned int overflow;          // sort reduction: 1 if some contribution went to the accumulators
    unsigned int apply_done;        // CTAs of the apply kernel that have finished (the last one publishes)
    unsigned long long surface_count;   // points found by the last surface extraction
    unsigned int pool_count;        // pool reduction: slots claimed by the scan in flight (may exceed the capacity)
    unsigned int pool_overflow;     // pool reduction: 1 if a brick found the pool full (the scan is dropped)
    unsigned int live_back;         // split ray list: light rays of the scan in flight, stored from the list's end
    unsigned int pad_;
};

constexpr uint32_t kPoolEmpty = 0xFFFFFFFFu;      // pool table entry of a brick without a slot
constexpr long long kStatusCapacity = -8;        // TSDF_ERR_CAPACITY

constexpr uint32_t kNoSlot = 0xFFFFFFFFu;        // ray without pair slots (all its samples overflow)
constexpr uint32_t kRaySlotLimit = 1u << 20;      // rays with more samples than this overflow
constexpr uint32_t kPairCapMax = 1u << 28;        // largest pair capacity of a map

// Device-side view of one map. The window is bricked and ring addressed:
// global voxel g lives in brick ((g >> 3) mod (dims / 8)) at offset
// ((g.z & 7) * 8 + (g.y & 7)) * 8 + (g.x & 7).
struct MapDev {
    uint32_t* grid;                 // value (low 16) | weight (high 16), 512 words per brick
    unsigned long long* acc;        // packed per-scan accumulators, same layout; all zero between scans
    uint8_t* brick_flag;            // one byte per brick (padded to 4): 1 = touched by the scan in flight
    uint32_t* brick_list;           // touched bricks of the scan in flight, built by the compaction kernel
    float4* ray_a;                  // per live ray (compacted): (dir.x, dir.y, dir.z, r)
    float4* ray_b;                  // per live ray (compacted): (int.x, int.y, int.z, fill ? 1 : 0)
    uint32_t ray_cap;               // entries of ray_a / ray_b (the split list fills them from both ends)
    MapCounters* ctr;
    long long* host_last;           // mapped pinned host copy of last_valid / hits / touched / status, or null
    // sort reduction (null / 0 when the map has no sort buffers)
    uint32_t* brick_slot;           // per brick: its position in the brick list (touched bricks only)
    uint32_t* seg_count;            // per list position: pair count, then the scatter cursor; zero between scans
    uint32_t* seg_start;            // per list position: first entry of the brick's segment in `sorted`
    uint32_t* ray_slot;             // per live ray: first pair slot, or kNoSlot
    uint2* pairs;                   // emitted (voxel word, code) per sample; word kNoVoxel = outside the window
    uint32_t* sorted;               // (offset in brick << 16) | (code & 0xFFFF), grouped by brick
    uint32_t pair_cap;              // capacity of `pairs` and `sorted`
    // pool reduction (null / 0 when the map has no pool)
    uint32_t* pool_table;           // per brick: its slot in the pool, kPoolEmpty between scans
    uint32_t* pool_brick;           // per slot: the brick that claimed it
    unsigned long long* pool_acc;   // per slot: 512 packed accumulators, all zero between scans
    uint32_t pool_cap;              // slots
};

// Everything the kernels need about one scan, passed by value.
struct ScanArgs {
    const float4* pts;
    int32_t n;
    int32_t K;                      // march steps on each side of the hit
    float R[9];                     // row-major rotation, sensor -> world
    float t[3];                     // sensor position in the world
    float vs, inv_vs, tau, qs, dz, rmin, rmax;
    int32_t fill;                   // delta_z > 0
    float win_lo[3], win_hi[3];     // window box in metres (rounded outward), for ray culling
    float fo[3];                    // window origin as float (exact: |origin| <= 2^23)
    float fe[3];                    // origin + dims as float (exact)
    uint32_t cmask[3];              // dims / 8 - 1 per axis
    uint32_t lcx, lcxy;             // log2(dims.x / 8), log2(dims.x / 8 * dims.y / 8)
    uint32_t dmask[3];              // dims - 1 per axis
    uint32_t omod[3];               // origin mod dims per axis (ring offset of the window origin)
    int32_t flags;                  // TSDF_FLAG_* bits
    // Derived constants of the lean contribution march, in pairs for the
    // packed (x, y) arithmetic (set by fill_lean_args).
    float2 l_t;                     // (t.x, t.y)
    float2 l_nt;                    // (-t.x, -t.y)
    float2 l_inv;                   // (1 / vs, 1 / vs)
    float2 l_vs;                    // (vs, vs)
    float2 l_m;                     // 1.5 * 2^23 - origin, x and y (exact: origins are multiples of 8)
    float l_mz;                     // the same for z
    float l_ntz;                    // -t.z
    uint32_t l_dim[3];              // window size per axis
    uint32_t l_omb[3];              // (origin mod dims) - 0x4B400000 per axis, modulo 2^32
    uint32_t l_cy, l_cz;            // 2^(lcx + 9) - 64 and 2^(lcxy + 9) - 512 (brick strides in the word index)
};

// Fill the lean-march constants of `a` from its other fields (host side,
// after t, vs, inv_vs, fo, dmask, omod, lcx and lcxy are set).
inline void fill_lean_args(ScanArgs& a) {
    a.l_t = make_float2(a.t[0], a.t[1]);
    a.l_nt = make_float2(-a.t[0], -a.t[1]);
    a.l_inv = make_float2(a.inv_vs, a.inv_vs);
    a.l_vs = make_float2(a.vs, a.vs);
    a.l_m = make_float2(12582912.0f - a.fo[0], 12582912.0f - a.fo[1]);
    a.l_mz = 12582912.0f - a.fo[2];
    a.l_ntz = -a.t[2];
    for (int i = 0; i < 3; ++i) {
        a.l_dim[i] = a.dmask[i] + 1u;
        a.l_omb[i] = a.omod[i] - 0x4B400000u;
    }
    a.l_cy = (1u << (a.lcx + 9u)) - 64u;
    a.l_cz = (1u << (a.lcxy + 9u)) - 512u;
}

// One brick slot that changes owner during a shift.
struct ShiftItem {
    uint32_t brick;                 // ring brick index
    uint32_t pad0;
    unsigned long long out_ptr;     // address of the shift's candidate slot with this item's index
    unsigned long long in_ptr;      // store address of the entering brick, 0 = zero fill
    unsigned long long pad1;
};

// One 2048-byte chunk copy (device addresses).
struct ChunkCopy {
    unsigned long long dst;
    unsigned long long src;
};

struct WindowGeom {
    uint32_t dims[3];
    uint32_t cmask[3];
    uint32_t lcx, lcxy;
};

// One scan of a batch: everything the batched kernel needs about it.
struct BatchItem {
    ScanArgs a;
    MapDev m;
    int32_t reduce;
    int32_t w_max;
    uint32_t bricks;
    int32_t flags;
};


// Host helpers implemented in api.cu for the batched path: validate a scan for
// `map`, grow its ray buffers if needed and fill the batch item.
int prepare_batch_item(::tsdf_map* map, const float* points_dev, int64_t n, const float pose[12], BatchItem* out);
int map_device(const ::tsdf_map* map);
// Device address of the map's published counters (last_valid, last_hits,
// last_touched: three contiguous int64).
const long long* map_last_counters(const ::tsdf_map* map);
// Host address of the mapped pinned copy of those counters, which the last CTA
// of every integration (per-map or batched) writes; null when the map has none.
const volatile long long* map_host_counters(const ::tsdf_map* map);
// Grow the map's per-ray buffers to hold n points (synchronous allocation).
int map_reserve_points(::tsdf_map* map, int64_t n);

// Grow the map's ray and sort-reduction buffers for scans of n points
// (synchronous allocation on first use or growth).
int map_reserve_sort(::tsdf_map* map, int64_t n);

// Launchers (return the cudaError_t of the launch).
// sort: reserve pair slots per ray (sort reduction); split: heavy rays (fill
// of at least one voxel each side) from the list's front, the others from
// its end (the plain contribution kernel takes heavy work first).
cudaError_t launch_rays(const ScanArgs& a, const MapDev& m, bool sort, bool split, bool pdl, cudaStream_t s);
// CTAs of the ray set-up kernel for a scan of n points.
unsigned rays_grid(int64_t n, bool sort);
// The kernel functions that launch_rays / launch_contrib launch for these
// arguments (to find their nodes in a captured graph).
const void* rays_kernel_fn(bool sort, bool split);
const void* contrib_kernel_fn(int32_t reduce, bool merge, int kpt);
cudaError_t launch_contrib(const ScanArgs& a, const MapDev& m, int32_t reduce, bool merge, int kpt, bool pdl,
                           cudaStream_t s);
cudaError_t launch_compact(const MapDev& m, uint32_t bricks, bool pdl, cudaStream_t s);
cudaError_t launch_apply(const MapDev& m, int32_t reduce, int32_t w_max, int32_t flags, bool pdl, cudaStream_t s);
// Sort reduction: emit pairs, count per brick, prefix, scatter, reduce + apply.
cudaError_t launch_emit(const ScanArgs& a, const MapDev& m, int32_t reduce, int kpt, bool pdl, cudaStream_t s);
cudaError_t launch_sort_count(const MapDev& m, bool pdl, cudaStream_t s);
// Pool reduction: the contribution march into claimed pool bricks, and the
// apply over the claimed slots (which also publishes the counters).
cudaError_t launch_pool_contrib(const ScanArgs& a, const MapDev& m, int32_t reduce, int kpt, bool pdl,
                                cudaStream_t s);
cudaError_t launch_pool_apply(const MapDev& m, int32_t reduce, int32_t w_max, int32_t flags, bool pdl,
                              cudaStream_t s);
cudaError_t launch_sort_scan(const MapDev& m, bool pdl, cudaStream_t s);
cudaError_t launch_sort_scatter(const MapDev& m, bool pdl, cudaStream_t s);
cudaError_t launch_sort_apply(const MapDev& m, int32_t reduce, int32_t w_max, int32_t flags, bool pdl,
                              cudaStream_t s);
// The leaving brick of each item that holds a non-zero voxel claims the next
// candidate slot (*claimed counts them, from 0) and is copied to
// items[claim].out_ptr; claim[item] is that index or -1 (the brick held no
// data). claim may point to mapped host memory.
cudaError_t launch_shift(uint32_t* grid, const ShiftItem* items, int count, unsigned* claimed, int* claim,
                         cudaStream_t s);
cudaError_t launch_copy_chunks(const ChunkCopy* items, int count, cudaStream_t s);
cudaError_t launch_register(const float* pts_dev, int n, const float pose[12], const uint32_t* grid,
                            const WindowGeom& geo, const long long origin[3], float vs, float inv_vs, float tau,
                            int min_w, double* out_dev, cudaStream_t s);
bool register_step(const double sys[29], float pose[12], double* step_norm);
cudaError_t launch_mesh(const uint32_t* grid, const WindowGeom& geo, const long long origin[3], int min_w, float vs,
                        float* out, unsigned long long cap, unsigned long long* count, cudaStream_t s);
cudaError_t launch_surface(const uint32_t* grid, const WindowGeom& geo, const long long origin[3], int min_w, float vs,
                           float4* out, unsigned long long cap, unsigned long long* count, cudaStream_t s);
cudaError_t launch_read_box(const uint32_t* grid, const long long lo[3], const uint32_t box[3],
                            const WindowGeom& g, int16_t* v, int16_t* w, cudaStream_t s);
cudaError_t launch_write_box(uint32_t* grid, const long long lo[3], const uint32_t box[3], const WindowGeom& g,
                             const int16_t* v, const int16_t* w, cudaStream_t s);

}  // namespace tsdf
