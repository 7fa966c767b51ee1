// Local-map window kernels: ring-buffer shift and box read/write.
//
// The window is ring addressed (the Kintinuous-style ring buffer cited in the
// paper's related work) and bricked: global voxel g lives in brick
// (g >> 3) mod (dims / 8), 512 contiguous words per brick. A shift therefore
// moves no data inside the overlap: only the bricks whose ring slot changes
// owner are touched; their old contents go to the global store and the
// entering contents come from the store or are zero (Introduction: the local
// map is shifted after a movement threshold; map parts leaving it are written
// out and previously mapped parts are read back in).
#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

// One warp per brick (4 per CTA): each lane moves 4 x 16 bytes of the
// 2048-byte brick, issuing all of its loads (the leaving brick and the
// entering one) before any store, so that each lane has 128 bytes in flight.
// A leaving brick with some non-zero voxel claims the next of the shift's
// candidate store slots (one atomic per such brick; candidate c's address is
// items[c].out_ptr) and is written there; claim[item] receives the
// candidate's index, or -1 for a brick that held no data (not written). The store keeps a brick in the same [z][y][x] order; a
// slot may lie in pinned host memory, which the kernel reads and writes in
// place.
__global__ void __launch_bounds__(128) shift_kernel(uint32_t* __restrict__ grid, const ShiftItem* __restrict__ items,
                                                     int count, unsigned* __restrict__ claimed, int* __restrict__ claim) {
    const int lane = threadIdx.x & 31;
    for (int it = blockIdx.x * 4 + (threadIdx.x >> 5); it < count; it += gridDim.x * 4) {
        const ShiftItem s = items[it];
        uint4* gp = reinterpret_cast<uint4*>(grid + ((size_t)s.brick << 9));
        uint4 old[4], nv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) old[v] = gp[32 * v + lane];
#pragma unroll
        for (int v = 0; v < 4; ++v)
            nv[v] = s.in_ptr ? reinterpret_cast<const uint4*>(s.in_ptr)[32 * v + lane] : make_uint4(0u, 0u, 0u, 0u);
        unsigned any = 0u;
#pragma unroll
        for (int v = 0; v < 4; ++v) any |= old[v].x | old[v].y | old[v].z | old[v].w;
        const bool keep = __any_sync(0xFFFFFFFFu, any != 0u);
        int c = -1;
        if (keep && claimed) {
            if (lane == 0) c = (int)atomicAdd(claimed, 1u);
            c = __shfl_sync(0xFFFFFFFFu, c, 0);
            uint4* dst = reinterpret_cast<uint4*>(items[c].out_ptr);
#pragma unroll
            for (int v = 0; v < 4; ++v) dst[32 * v + lane] = old[v];
        }
        if (claim && lane == 0) claim[it] = c;
#pragma unroll
        for (int v = 0; v < 4; ++v) gp[32 * v + lane] = nv[v];
    }
}

// One CTA of 128 threads per chunk: copies 2048 bytes from src to dst.
__global__ void __launch_bounds__(128) copy_chunks_kernel(const ChunkCopy* __restrict__ items, int count) {
    const int t = threadIdx.x;
    for (int it = blockIdx.x; it < count; it += gridDim.x) {
        const ChunkCopy c = items[it];
        reinterpret_cast<uint4*>(c.dst)[t] = reinterpret_cast<const uint4*>(c.src)[t];
    }
}

__device__ __forceinline__ size_t word_of(long long gx, long long gy, long long gz, const WindowGeom& g) {
    const size_t bx = (size_t)((unsigned long long)(gx >> 3) & g.cmask[0]);
    const size_t by = (size_t)((unsigned long long)(gy >> 3) & g.cmask[1]);
    const size_t bz = (size_t)((unsigned long long)(gz >> 3) & g.cmask[2]);
    const size_t brick = (bz << g.lcxy) | (by << g.lcx) | bx;
    return (brick << 9) | (size_t)(((gz & 7) << 6) | ((gy & 7) << 3) | (gx & 7));
}

__global__ void read_box_kernel(const uint32_t* __restrict__ grid, long long lx, long long ly, long long lz,
                                uint32_t bx, uint32_t by, size_t total, const WindowGeom g, int16_t* __restrict__ v,
                                int16_t* __restrict__ w) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t x = i % bx, y = (i / bx) % by, z = i / ((size_t)bx * by);
        const uint32_t word = grid[word_of(lx + (long long)x, ly + (long long)y, lz + (long long)z, g)];
        v[i] = (int16_t)(word & 0xFFFFu);
        w[i] = (int16_t)(word >> 16);
    }
}

__global__ void write_box_kernel(uint32_t* __restrict__ grid, long long lx, long long ly, long long lz, uint32_t bx,
                                 uint32_t by, size_t total, const WindowGeom g, const int16_t* __restrict__ v,
                                 const int16_t* __restrict__ w) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t x = i % bx, y = (i / bx) % by, z = i / ((size_t)bx * by);
        grid[word_of(lx + (long long)x, ly + (long long)y, lz + (long long)z, g)] =
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

cudaError_t launch_copy_chunks(const ChunkCopy* items, int count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    copy_chunks_kernel<<<count < 4096 ? count : 4096, 128, 0, s>>>(items, count);
    return cudaGetLastError();
}

cudaError_t launch_shift(uint32_t* grid, const ShiftItem* items, int count, unsigned* claimed, int* claim,
                         cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int need = (count + 3) / 4;
    const int blocks = need < 65536 ? need : 65536;
    shift_kernel<<<blocks, 128, 0, s>>>(grid, items, count, claimed, claim);
    return cudaGetLastError();
}

cudaError_t launch_read_box(const uint32_t* grid, const long long lo[3], const uint32_t box[3], const WindowGeom& g,
                            int16_t* v, int16_t* w, cudaStream_t s) {
    const size_t total = (size_t)box[0] * box[1] * box[2];
    if (total == 0) return cudaSuccess;
    read_box_kernel<<<grid_for(total), 256, 0, s>>>(grid, lo[0], lo[1], lo[2], box[0], box[1], total, g, v, w);
    return cudaGetLastError();
}

cudaError_t launch_write_box(uint32_t* grid, const long long lo[3], const uint32_t box[3], const WindowGeom& g,
                             const int16_t* v, const int16_t* w, cudaStream_t s) {
    const size_t total = (size_t)box[0] * box[1] * box[2];
    if (total == 0) return cudaSuccess;
    write_box_kernel<<<grid_for(total), 256, 0, s>>>(grid, lo[0], lo[1], lo[2], box[0], box[1], total, g, v, w);
    return cudaGetLastError();
}

}  // namespace tsdf
