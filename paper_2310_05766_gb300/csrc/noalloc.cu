// tsdf_integrate_static: one scan integration that allocates no memory.
//
// Some callers cannot allocate device memory once they are running: a
// real-time mapping loop on a robot that reserves all of its memory at
// start-up (a cudaMalloc may synchronise the device and take unbounded time),
// or a host process whose device memory is entirely owned by another
// allocator. This entry point serves them. The caller passes the voxel grid
// (in/out) and the points (in); every other buffer the integration needs (the
// per-scan accumulator, brick flags and list, per-ray data and counters) lives
// in one file-scope __device__ array of fixed size, which every GPU that loads
// the library keeps until the process exits.
//
// The kernels are the library's integration kernels (rays, contrib, compact,
// and apply, whose last CTA publishes the counters); only the origin of their
// scratch memory differs.
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "tsdf_internal.cuh"
#include "../../include/tsdf.h"

using namespace tsdf;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

constexpr size_t kMaxVoxels = (size_t)TSDF_STATIC_MAX_VOXELS;
constexpr size_t kMaxPoints = (size_t)TSDF_STATIC_MAX_POINTS;
constexpr size_t kMaxBricks = kMaxVoxels / kBrickVoxels;

// Layout of the scratch array (offsets in bytes, each 256-byte aligned).
constexpr size_t kOffCtr = 0;
constexpr size_t kOffAcc = kOffCtr + round_up(sizeof(MapCounters));
constexpr size_t kOffFlag = kOffAcc + round_up(kMaxVoxels * sizeof(unsigned long long));
constexpr size_t kOffList = kOffFlag + round_up(kMaxBricks);
constexpr size_t kOffRayA = kOffList + round_up(kMaxBricks * sizeof(uint32_t));
constexpr size_t kOffRayB = kOffRayA + round_up(kMaxPoints * sizeof(float4));
constexpr size_t kScratchBytes = kOffRayB + round_up(kMaxPoints * sizeof(float4));

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Device address of g_static_scratch per device, resolved once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
// Per device: a call failed after its contribution kernel may have written
// accumulators or brick flags, so the next call clears them. (A call that
// completes leaves both all zero: the compaction clears the flags it lists
// and the apply resets every accumulator it reads; a freshly loaded module's
// array is zero.)
bool g_dirty[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out, int* dev_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TSDF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        // In host code the symbol is only a host-side stand-in: the kernels
        // must get the device address, looked up with this device current.
        unsigned char* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
        if (e != cudaSuccess || !p) return TSDF_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    *dev_out = dev;
    return TSDF_OK;
}

bool pow2(int32_t v) { return v > 0 && (v & (v - 1)) == 0; }
uint32_t ilog2(uint32_t v) {
    uint32_t s = 0;
    while ((1u << s) < v) ++s;
    return s;
}

int check_params(const tsdf_params* p) {
    if (!p) return TSDF_ERR_INVALID;
    size_t voxels = 1;
    for (int a = 0; a < 3; ++a) {
        if (!pow2(p->dims[a]) || p->dims[a] < 8 || p->dims[a] > 32768) return TSDF_ERR_INVALID;
        voxels *= (size_t)p->dims[a];
        if (p->origin[a] % 8 != 0 || p->origin[a] > (1LL << 23) || p->origin[a] < -(1LL << 23)) return TSDF_ERR_INVALID;
    }
    if (voxels > kMaxVoxels) return TSDF_ERR_INVALID;   // beyond the static scratch
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

}  // namespace

extern "C" int tsdf_integrate_static(uint32_t* grid_dev, const tsdf_params* params, const float* points_dev,
                                     int64_t n, const float pose[12], tsdf_scan_stats* stats_host, void* stream) {
    int rc = check_params(params);
    if (rc != TSDF_OK) return rc;
    if (!grid_dev || ((uintptr_t)grid_dev & 15u) != 0 || !pose) return TSDF_ERR_INVALID;
    if (n < 0 || (size_t)n > kMaxPoints) return TSDF_ERR_INVALID;   // beyond the static scratch
    if (n > 0 && (!points_dev || ((uintptr_t)points_dev & 15u) != 0)) return TSDF_ERR_INVALID;
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(pose[i])) return TSDF_ERR_INVALID;
    unsigned char* base = nullptr;
    int dev = 0;
    rc = scratch_for_current_device(&base, &dev);
    if (rc != TSDF_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t voxels = (size_t)params->dims[0] * params->dims[1] * params->dims[2];
    const size_t bricks = voxels / kBrickVoxels;

    MapDev md{};
    md.grid = grid_dev;
    md.ctr = reinterpret_cast<MapCounters*>(base + kOffCtr);
    md.acc = reinterpret_cast<unsigned long long*>(base + kOffAcc);
    md.brick_flag = base + kOffFlag;
    md.brick_list = reinterpret_cast<uint32_t*>(base + kOffList);
    md.ray_a = reinterpret_cast<float4*>(base + kOffRayA);
    md.ray_b = reinterpret_cast<float4*>(base + kOffRayB);
    md.ray_cap = (uint32_t)kMaxPoints;

    // The array keeps the previous call's contents: the counters are cleared
    // on every call; the brick flags and accumulators (zero after any call
    // that completed) only after a failed call, and then over the whole array.
    cudaError_t e = cudaMemsetAsync(md.ctr, 0, sizeof(MapCounters), s);
    bool dirty = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        dirty = g_dirty[dev];
    }
    if (dirty) {
        if (e == cudaSuccess) e = cudaMemsetAsync(md.brick_flag, 0, round_up(kMaxBricks), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(md.acc, 0, kMaxVoxels * sizeof(unsigned long long), s);
        if (e == cudaSuccess) {
            std::lock_guard<std::mutex> lk(g_mu);
            g_dirty[dev] = false;
        }
    }

    ScanArgs a{};
    a.pts = reinterpret_cast<const float4*>(points_dev);
    a.n = (int32_t)n;
    a.K = (int)std::floor((double)params->tau / (double)params->voxel_size + 1e-9);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) a.R[r * 3 + c] = pose[r * 4 + c];
        a.t[r] = pose[r * 4 + 3];
    }
    a.vs = params->voxel_size;
    a.inv_vs = (float)(1.0 / (double)params->voxel_size);
    a.tau = params->tau;
    a.qs = (float)((double)kQMax / (double)params->tau);
    a.dz = params->delta_z;
    a.rmin = params->r_min;
    a.rmax = params->r_max;
    a.fill = params->delta_z > 0.f ? 1 : 0;
    for (int ax = 0; ax < 3; ++ax) {
        const double lo = (double)params->origin[ax] * (double)params->voxel_size;
        const double hi = (double)(params->origin[ax] + params->dims[ax]) * (double)params->voxel_size;
        a.win_lo[ax] = std::nextafter((float)lo, -INFINITY);
        a.win_hi[ax] = std::nextafter((float)hi, INFINITY);
        a.fo[ax] = (float)params->origin[ax];
        a.fe[ax] = (float)(params->origin[ax] + params->dims[ax]);
        a.cmask[ax] = (uint32_t)params->dims[ax] / 8u - 1u;
        a.dmask[ax] = (uint32_t)params->dims[ax] - 1u;
        a.omod[ax] = (uint32_t)((unsigned long long)params->origin[ax] & (unsigned long long)(params->dims[ax] - 1));
    }
    a.lcx = ilog2((uint32_t)params->dims[0] / 8u);
    a.lcxy = a.lcx + ilog2((uint32_t)params->dims[1] / 8u);
    a.flags = params->flags;
    fill_lean_args(a);

    if (e == cudaSuccess) e = launch_rays(a, md, false, true, true, s);
    bool launched_contrib = false;
    if (e == cudaSuccess) {
        e = launch_contrib(a, md, params->reduce, false, 4, true, s);
        launched_contrib = true;
    }
    if (e == cudaSuccess) e = launch_compact(md, (uint32_t)bricks, true, s);
    if (e == cudaSuccess) e = launch_apply(md, params->reduce, params->w_max, params->flags, true, s);
    if (e == cudaSuccess && stats_host) {
        long long last[3] = {0, 0, 0};
        e = cudaMemcpyAsync(last, &md.ctr->last_valid, sizeof(last), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) {
            stats_host->valid_rays = last[0];
            stats_host->hits = last[1];
            stats_host->touched = last[2];
        }
    }
    if (e != cudaSuccess && launched_contrib) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_dirty[dev] = true;
    }
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TSDF_ERR_OOM : TSDF_ERR_CUDA;
    return TSDF_OK;
}
