// Zero crossings of the TSDF: a consumer of the map (the paper's outlook puts
// mesh extraction and TSDF-based registration after the map generation).
//
// For every pair of 6-connected window voxels a and b = a + e_axis with both
// weights >= min_weight and values of different sign ((v_a < 0) != (v_b < 0)),
// one surface point is emitted where the linear interpolation of the stored
// codes between the two voxel centres is zero:
//   t = v_a / (v_a - v_b)                       (one IEEE division, round to nearest)
//   p_axis = ((float)g_axis + 0.5 + t) * vs      (the other two: ((float)g + 0.5) * vs)
// in world metres, with the axis index in the fourth component. One thread
// per window voxel reads it and its +x, +y, +z neighbours through the ring
// addressing; points are appended with one atomic per warp.
#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

__device__ __forceinline__ size_t surface_word(long long gx, long long gy, long long gz, const WindowGeom& g) {
    const size_t bx = (size_t)((unsigned long long)(gx >> 3) & g.cmask[0]);
    const size_t by = (size_t)((unsigned long long)(gy >> 3) & g.cmask[1]);
    const size_t bz = (size_t)((unsigned long long)(gz >> 3) & g.cmask[2]);
    const size_t brick = (bz << g.lcxy) | (by << g.lcx) | bx;
    return (brick << 9) | (size_t)(((gz & 7) << 6) | ((gy & 7) << 3) | (gx & 7));
}

__global__ void __launch_bounds__(256) surface_kernel(const uint32_t* __restrict__ grid, const WindowGeom geo,
                                                      long long ox, long long oy, long long oz, int min_w, float vs,
                                                      float4* __restrict__ out, unsigned long long cap,
                                                      unsigned long long* __restrict__ count) {
    const size_t total = (size_t)geo.dims[0] * geo.dims[1] * geo.dims[2];
    const unsigned lane = threadIdx.x & 31u;
    // the loop bound is uniform per warp so that every lane reaches the shuffles
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
        const size_t i = base + lane;
        float4 pt[3];
        unsigned n = 0;
        if (i < total) {
            const long long x = (long long)(i % geo.dims[0]);
            const long long y = (long long)((i / geo.dims[0]) % geo.dims[1]);
            const long long z = (long long)(i / ((size_t)geo.dims[0] * geo.dims[1]));
            const long long g[3] = {ox + x, oy + y, oz + z};
            const long long rel[3] = {x, y, z};
            const uint32_t wa = grid[surface_word(g[0], g[1], g[2], geo)];
            const int va = (int)(int16_t)(wa & 0xFFFFu);
            if ((int)(int16_t)(wa >> 16) >= min_w) {
                const float c[3] = {__fmul_rn(__fadd_rn((float)g[0], 0.5f), vs), __fmul_rn(__fadd_rn((float)g[1], 0.5f), vs),
                                    __fmul_rn(__fadd_rn((float)g[2], 0.5f), vs)};
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    if (rel[ax] + 1 >= (long long)geo.dims[ax]) continue;
                    const uint32_t wb = grid[surface_word(g[0] + (ax == 0), g[1] + (ax == 1), g[2] + (ax == 2), geo)];
                    const int vb = (int)(int16_t)(wb & 0xFFFFu);
                    if ((int)(int16_t)(wb >> 16) < min_w || ((va < 0) == (vb < 0))) continue;
                    const float t = __fdiv_rn((float)va, (float)(va - vb));
                    const float p = __fmul_rn(__fadd_rn(__fadd_rn((float)g[ax], 0.5f), t), vs);
                    pt[n] = make_float4(ax == 0 ? p : c[0], ax == 1 ? p : c[1], ax == 2 ? p : c[2], (float)ax);
                    ++n;
                }
            }
        }
        unsigned incl = n;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(kFullMask, incl, o);
            if (lane >= (unsigned)o) incl += v;
        }
        const unsigned tot = __shfl_sync(kFullMask, incl, 31);
        if (tot == 0u) continue;
        unsigned long long b = 0;
        if (lane == 31) b = atomicAdd(count, (unsigned long long)tot);
        b = __shfl_sync(kFullMask, b, 31) + (incl - n);
        for (unsigned k = 0; k < n; ++k)
            if (b + k < cap) out[b + k] = pt[k];
    }
}

}  // namespace

cudaError_t launch_surface(const uint32_t* grid, const WindowGeom& geo, const long long origin[3], int min_w, float vs,
                           float4* out, unsigned long long cap, unsigned long long* count, cudaStream_t s) {
    const size_t total = (size_t)geo.dims[0] * geo.dims[1] * geo.dims[2];
    size_t blocks = (total + 255) / 256;
    if (blocks > 16384) blocks = 16384;
    surface_kernel<<<(unsigned)blocks, 256, 0, s>>>(grid, geo, origin[0], origin[1], origin[2], min_w, vs, out, cap,
                                                     count);
    return cudaGetLastError();
}

}  // namespace tsdf
