// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tsdf {

constexpr int32_t kQMax = 32767;
constexpr unsigned kEmptySlot = 0xFFFFFFFFu;

// Per-map device counters (one instance per map, in device memory).
struct MapCounters {
    unsigned long long cur_valid;   // valid rays of the scan in flight
    unsigned long long cur_hits;    // in-window contributions of the scan in flight
    unsigned int touched_count;     // length of the touched list of the scan in flight
    unsigned int apply_done;        // CTAs of the apply kernel that have finished
    long long last_valid;           // counters of the last completed scan
    long long last_hits;
    long long last_touched;
    unsigned int error;             // sticky device-side error word (0 = none)
    unsigned int pad;
};

// Device-side view of one map.
struct MapDev {
    uint32_t* grid;                 // X*Y*Z words: value (low 16) | weight (high 16), ring addressed
    unsigned long long* acc;        // X*Y*Z packed per-scan accumulators, all zero between scans
    uint32_t* touched;              // slots touched by the scan in flight (first-touch order)
    MapCounters* ctr;
};

// Everything the contribution kernel needs about one scan, passed by value.
struct ScanArgs {
    const float4* pts;
    int32_t n;
    int32_t K;                      // march steps on each side of the hit
    float R[9];                     // row-major rotation, sensor -> world
    float t[3];                     // sensor position in the world
    float vs, inv_vs, tau, qs, dz, rmin, rmax;
    int32_t fill;                   // delta_z > 0
    int32_t reduce;                 // 0 = WSUM, 1 = MIN_ABS
    long long ox, oy, oz;           // window origin (global voxel coordinates)
    uint32_t dimx, dimy, dimz;      // powers of two
    uint32_t shx, shxy;             // log2(dimx), log2(dimx*dimy)
    int32_t w_max;
};

// One 8^3 chunk slot that changes owner during a shift.
struct ShiftItem {
    uint32_t chunk_slot;            // (cz * CY + cy) * CX + cx in ring (slot) chunk coordinates
    uint32_t pad0;
    unsigned long long out_ptr;     // store address for the leaving chunk (2048 B), 0 = discard
    unsigned long long in_ptr;      // store address of the entering chunk, 0 = zero fill
    unsigned long long pad1;
};

// Launchers (return the cudaError_t of the launch).
cudaError_t launch_contrib(const ScanArgs& a, const MapDev& m, cudaStream_t s);
cudaError_t launch_apply(const MapDev& m, int32_t reduce, int32_t w_max, int num_ctas, cudaStream_t s);
cudaError_t launch_shift(uint32_t* grid, const ShiftItem* items, int count, uint32_t dimx, uint32_t dimy,
                         cudaStream_t s);
cudaError_t launch_read_box(const uint32_t* grid, const long long lo[3], const uint32_t box[3],
                            uint32_t dimx, uint32_t dimy, uint32_t dimz, int16_t* v, int16_t* w,
                            cudaStream_t s);
cudaError_t launch_write_box(uint32_t* grid, const long long lo[3], const uint32_t box[3], uint32_t dimx,
                             uint32_t dimy, uint32_t dimz, const int16_t* v, const int16_t* w,
                             cudaStream_t s);

}  // namespace tsdf
