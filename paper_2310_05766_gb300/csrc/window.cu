// Local-map window kernels: ring-buffer shift and box read/write.
//
// The window is ring addressed (Kintinuous-style, cited in the paper's
// related work): global voxel g lives in slot g mod dims, so a shift moves no
// data inside the overlap. Only the 8^3 chunks whose slot changes owner are
// touched: their old contents go to the global store and the entering
// contents come from the store or are zero (Introduction: the local map is
// shifted after a movement threshold; map parts leaving it are written out and
// previously mapped parts are read back in).
#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

// One CTA of 128 threads per chunk: a chunk is 64 rows of 8 voxels (32 B);
// each thread moves one 16-byte half row. The store keeps a chunk as 512
// words in [z][y][x] order, so thread t's 16 B live at byte offset 16 t.
__global__ void __launch_bounds__(128) shift_kernel(uint32_t* __restrict__ grid, const ShiftItem* __restrict__ items,
                                                     int count, uint32_t dimx, uint32_t dimy) {
    const uint32_t cdx = dimx >> 3, cdy = dimy >> 3;
    const int t = threadIdx.x;
    const int row = t >> 1, half = t & 1;
    const int z = row >> 3, y = row & 7;
    for (int it = blockIdx.x; it < count; it += gridDim.x) {
        const ShiftItem s = items[it];
        const uint32_t cx = s.chunk_slot % cdx;
        const uint32_t cy = (s.chunk_slot / cdx) % cdy;
        const uint32_t cz = s.chunk_slot / (cdx * cdy);
        const size_t gidx = ((size_t)(cz * 8 + z) * dimy + (cy * 8 + y)) * dimx + cx * 8 + half * 4;
        uint4* gp = reinterpret_cast<uint4*>(grid + gidx);
        const uint4 old = *gp;
        if (s.out_ptr) reinterpret_cast<uint4*>(s.out_ptr)[t] = old;
        uint4 nv = make_uint4(0u, 0u, 0u, 0u);
        if (s.in_ptr) nv = reinterpret_cast<const uint4*>(s.in_ptr)[t];
        *gp = nv;
    }
}

__device__ __forceinline__ size_t slot_of(long long gx, long long gy, long long gz, uint32_t dimx, uint32_t dimy,
                                          uint32_t dimz) {
    const size_t sx = (size_t)((unsigned long long)gx & (dimx - 1u));
    const size_t sy = (size_t)((unsigned long long)gy & (dimy - 1u));
    const size_t sz = (size_t)((unsigned long long)gz & (dimz - 1u));
    return (sz * dimy + sy) * dimx + sx;
}

__global__ void read_box_kernel(const uint32_t* __restrict__ grid, long long lx, long long ly, long long lz,
                                uint32_t bx, uint32_t by, size_t total, uint32_t dimx, uint32_t dimy, uint32_t dimz,
                                int16_t* __restrict__ v, int16_t* __restrict__ w) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t x = i % bx, y = (i / bx) % by, z = i / ((size_t)bx * by);
        const uint32_t word = grid[slot_of(lx + (long long)x, ly + (long long)y, lz + (long long)z, dimx, dimy, dimz)];
        if (v) v[i] = (int16_t)(word & 0xFFFFu);
        if (w) w[i] = (int16_t)(word >> 16);
    }
}

__global__ void write_box_kernel(uint32_t* __restrict__ grid, long long lx, long long ly, long long lz, uint32_t bx,
                                 uint32_t by, size_t total, uint32_t dimx, uint32_t dimy, uint32_t dimz,
                                 const int16_t* __restrict__ v, const int16_t* __restrict__ w) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t x = i % bx, y = (i / bx) % by, z = i / ((size_t)bx * by);
        grid[slot_of(lx + (long long)x, ly + (long long)y, lz + (long long)z, dimx, dimy, dimz)] =
            (uint32_t)(uint16_t)v[i] | ((uint32_t)(uint16_t)w[i] << 16);
    }
}

int grid_for(size_t total) {
    size_t b = (total + 255) / 256;
    if (b > 65536) b = 65536;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_shift(uint32_t* grid, const ShiftItem* items, int count, uint32_t dimx, uint32_t dimy,
                         cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int blocks = count < 65536 ? count : 65536;
    shift_kernel<<<blocks, 128, 0, s>>>(grid, items, count, dimx, dimy);
    return cudaGetLastError();
}

cudaError_t launch_read_box(const uint32_t* grid, const long long lo[3], const uint32_t box[3], uint32_t dimx,
                            uint32_t dimy, uint32_t dimz, int16_t* v, int16_t* w, cudaStream_t s) {
    const size_t total = (size_t)box[0] * box[1] * box[2];
    if (total == 0) return cudaSuccess;
    read_box_kernel<<<grid_for(total), 256, 0, s>>>(grid, lo[0], lo[1], lo[2], box[0], box[1], total, dimx, dimy,
                                                    dimz, v, w);
    return cudaGetLastError();
}

cudaError_t launch_write_box(uint32_t* grid, const long long lo[3], const uint32_t box[3], uint32_t dimx,
                             uint32_t dimy, uint32_t dimz, const int16_t* v, const int16_t* w, cudaStream_t s) {
    const size_t total = (size_t)box[0] * box[1] * box[2];
    if (total == 0) return cudaSuccess;
    write_box_kernel<<<grid_for(total), 256, 0, s>>>(grid, lo[0], lo[1], lo[2], box[0], box[1], total, dimx, dimy,
                                                     dimz, v, w);
    return cudaGetLastError();
}

}  // namespace tsdf
