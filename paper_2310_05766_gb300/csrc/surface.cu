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

// ---- marching tetrahedra (see tsdf_extract_mesh in the public header): one
// thread per dual cube (corner voxel a = window origin + (x, y, z), x + 1 <
// dims.x and so on). The cube's 8 codes are read once; the triangles are
// counted, the warp reserves space with one atomic, and the cube writes them.
__constant__ int kTetAxesDev[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

__device__ __forceinline__ void tet_corners(int tt, int off[4][3]) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) off[k][a] = k == 3 ? 1 : 0;
    off[1][kTetAxesDev[tt][0]] = 1;
    off[2][kTetAxesDev[tt][0]] = 1;
    off[2][kTetAxesDev[tt][1]] = 1;
}

// Vertex on the edge from the negative corner P to the positive corner Q.
__device__ __forceinline__ void mt_vertex(const long long gp[3], int vp, const long long gq[3], int vq, float vs,
                                          float* o) {
    const float t = __fdiv_rn((float)vp, (float)(vp - vq));
#pragma unroll
    for (int a = 0; a < 3; ++a)
        o[a] = __fmul_rn(__fadd_rn(__fadd_rn((float)gp[a], 0.5f), __fmul_rn(t, (float)(gq[a] - gp[a]))), vs);
}

__device__ __forceinline__ void mt_emit(const float tri[3][3], const double dir[3], float* out,
                                        unsigned long long slot, unsigned long long cap) {
    const double e1[3] = {(double)tri[1][0] - tri[0][0], (double)tri[1][1] - tri[0][1], (double)tri[1][2] - tri[0][2]};
    const double e2[3] = {(double)tri[2][0] - tri[0][0], (double)tri[2][1] - tri[0][1], (double)tri[2][2] - tri[0][2]};
    const double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2],
                 nz = e1[0] * e2[1] - e1[1] * e2[0];
    const bool flip = nx * dir[0] + ny * dir[1] + nz * dir[2] < 0.0;
    if (slot >= cap) return;
    float* o = out + 9 * slot;
    const int order[3] = {0, flip ? 2 : 1, flip ? 1 : 2};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) o[3 * c + a] = tri[order[c]][a];
}

__global__ void __launch_bounds__(256) mesh_kernel(const uint32_t* __restrict__ grid, const WindowGeom geo,
                                                   long long ox, long long oy, long long oz, int min_w, float vs,
                                                   float* __restrict__ out, unsigned long long cap,
                                                   unsigned long long* __restrict__ count) {
    const size_t total = (size_t)geo.dims[0] * geo.dims[1] * geo.dims[2];
    const unsigned lane = threadIdx.x & 31u;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
        const size_t i = base + lane;
        int val[8];
        bool ok = false;
        long long g0[3] = {0, 0, 0};
        if (i < total) {
            const long long x = (long long)(i % geo.dims[0]);
            const long long y = (long long)((i / geo.dims[0]) % geo.dims[1]);
            const long long z = (long long)(i / ((size_t)geo.dims[0] * geo.dims[1]));
            ok = x + 1 < (long long)geo.dims[0] && y + 1 < (long long)geo.dims[1] && z + 1 < (long long)geo.dims[2];
            g0[0] = ox + x;
            g0[1] = oy + y;
            g0[2] = oz + z;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (!ok) break;
                const uint32_t w = grid[surface_word(g0[0] + (c & 1), g0[1] + ((c >> 1) & 1), g0[2] + (c >> 2), geo)];
                val[c] = (int)(int16_t)(w & 0xFFFFu);
                if ((int)(int16_t)(w >> 16) < min_w) ok = false;
            }
        }
        // triangles of this cube
        unsigned n = 0;
        if (ok) {
            for (int tt = 0; tt < 6; ++tt) {
                int off[4][3];
                tet_corners(tt, off);
                int neg = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) neg += val[off[k][0] | (off[k][1] << 1) | (off[k][2] << 2)] < 0 ? 1 : 0;
                n += (neg == 1 || neg == 3) ? 1u : (neg == 2 ? 2u : 0u);
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
        if (n == 0) continue;
        for (int tt = 0; tt < 6; ++tt) {
            int off[4][3];
            tet_corners(tt, off);
            long long g[4][3];
            int v[4];
            int neg = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
#pragma unroll
                for (int a = 0; a < 3; ++a) g[k][a] = g0[a] + off[k][a];
                v[k] = val[off[k][0] | (off[k][1] << 1) | (off[k][2] << 2)];
                neg += v[k] < 0 ? 1 : 0;
            }
            if (neg == 0 || neg == 4) continue;
            double dir[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) dir[a] += (v[k] < 0 ? -1.0 / neg : 1.0 / (4 - neg)) * (double)off[k][a];
            float tri[3][3];
            if (neg == 1 || neg == 3) {
                int lone = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if ((v[k] < 0) == (neg == 1)) lone = k;
                int e = 0;
                for (int k = 0; k < 4; ++k) {
                    if (k == lone) continue;
                    if (neg == 1) mt_vertex(g[lone], v[lone], g[k], v[k], vs, tri[e]);
                    else mt_vertex(g[k], v[k], g[lone], v[lone], vs, tri[e]);
                    ++e;
                }
                mt_emit(tri, dir, out, b++, cap);
            } else {
                int ng[2], ps[2], na = 0, nb = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (v[k] < 0) ng[na++] = k;
                    else ps[nb++] = k;
                }
                float ac[3], ad[3], bd[3], bc[3];
                mt_vertex(g[ng[0]], v[ng[0]], g[ps[0]], v[ps[0]], vs, ac);
                mt_vertex(g[ng[0]], v[ng[0]], g[ps[1]], v[ps[1]], vs, ad);
                mt_vertex(g[ng[1]], v[ng[1]], g[ps[1]], v[ps[1]], vs, bd);
                mt_vertex(g[ng[1]], v[ng[1]], g[ps[0]], v[ps[0]], vs, bc);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    tri[0][a] = ac[a];
                    tri[1][a] = ad[a];
                    tri[2][a] = bd[a];
                }
                mt_emit(tri, dir, out, b++, cap);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    tri[1][a] = bd[a];
                    tri[2][a] = bc[a];
                }
                mt_emit(tri, dir, out, b++, cap);
            }
        }
    }
}

}  // namespace

cudaError_t launch_mesh(const uint32_t* grid, const WindowGeom& geo, const long long origin[3], int min_w, float vs,
                        float* out, unsigned long long cap, unsigned long long* count, cudaStream_t s) {
    const size_t total = (size_t)geo.dims[0] * geo.dims[1] * geo.dims[2];
    size_t blocks = (total + 255) / 256;
    if (blocks > 16384) blocks = 16384;
    mesh_kernel<<<(unsigned)blocks, 256, 0, s>>>(grid, geo, origin[0], origin[1], origin[2], min_w, vs, out, cap,
                                                  count);
    return cudaGetLastError();
}

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
