// Scan-to-map registration on the TSDF (a consumer of the map; the paper's
// outlook names registration against the TSDF map). Gauss-Newton on
//   E(T) = sum_i d(T p_i)^2,
// d the trilinear interpolation of the stored truncated distances at a point,
// with the pose update q' = Exp(w) q + v (w, v in the world frame).
//
// The kernel evaluates, for the current pose, the normal equations of all
// points: one thread per point computes q = R p + t and u = q / vs - 0.5 in
// binary32 (explicit round-to-nearest, the ray set-up's order), takes the 8
// voxels i0 + {0,1}^3 with i0 = floor(u), and if all lie in the window with
// weights >= min_w and |d| < tau adds J = [q x grad d, grad d] (binary64) to
// H = sum J J^T, g = sum J d, the cost and the count. Sums go through warp
// shuffles and shared memory to one binary64 atomic per CTA and entry. The
// host solves H xi = -g (Cholesky) and updates the pose.
#include <cmath>
#include <cstring>

#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

constexpr unsigned kFullMaskR = 0xFFFFFFFFu;
constexpr int kSysN = 29;   // 21 (H upper triangle) + 6 (g) + cost + count

struct RegArgs {
    const float4* pts;
    int n;
    float R[9];
    float t[3];
    float vs, inv_vs;
    double scale;            // tau / 32767
    double tau;
    int min_w;
    long long o[3];          // window origin
    WindowGeom geo;
};

__device__ __forceinline__ size_t reg_word(long long gx, long long gy, long long gz, const WindowGeom& g) {
    const size_t bx = (size_t)((unsigned long long)(gx >> 3) & g.cmask[0]);
    const size_t by = (size_t)((unsigned long long)(gy >> 3) & g.cmask[1]);
    const size_t bz = (size_t)((unsigned long long)(gz >> 3) & g.cmask[2]);
    const size_t brick = (bz << g.lcxy) | (by << g.lcx) | bx;
    return (brick << 9) | (size_t)(((gz & 7) << 6) | ((gy & 7) << 3) | (gx & 7));
}

// Contribution of point i to the system, in `acc` (zero when it is not used).
__device__ __forceinline__ void reg_point(const RegArgs& a, const uint32_t* __restrict__ grid, int i, double* acc) {
    const float4 p = a.pts[i];
    if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) return;
    float q[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        q[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(a.R[3 * r], p.x), __fmul_rn(a.R[3 * r + 1], p.y)),
                                   __fmul_rn(a.R[3 * r + 2], p.z)),
                         a.t[r]);
    long long i0[3];
    double f[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float u = __fsub_rn(__fmul_rn(q[r], a.inv_vs), 0.5f);
        const float fl = floorf(u);
        i0[r] = (long long)fl;
        f[r] = (double)__fsub_rn(u, fl);
    }
    double c[2][2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const long long g[3] = {i0[0] + dx, i0[1] + dy, i0[2] + dz};
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    if (g[r] < a.o[r] || g[r] >= a.o[r] + (long long)a.geo.dims[r]) return;
                const uint32_t w = grid[reg_word(g[0], g[1], g[2], a.geo)];
                if ((int)(int16_t)(w >> 16) < a.min_w) return;
                c[dz][dy][dx] = (double)(int16_t)(w & 0xFFFFu) * a.scale;
            }
    const double fx = f[0], fy = f[1], fz = f[2];
    double cx[2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) cx[dz][dy] = c[dz][dy][0] * (1 - fx) + c[dz][dy][1] * fx;
    const double cy0 = cx[0][0] * (1 - fy) + cx[0][1] * fy, cy1 = cx[1][0] * (1 - fy) + cx[1][1] * fy;
    const double d = cy0 * (1 - fz) + cy1 * fz;
    if (!(fabs(d) < a.tau)) return;
    double gu[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
            gu[0] += ((dy ? fy : 1 - fy) * (dz ? fz : 1 - fz)) * (c[dz][dy][1] - c[dz][dy][0]);
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
            gu[1] += ((dx ? fx : 1 - fx) * (dz ? fz : 1 - fz)) * (c[dz][1][dx] - c[dz][0][dx]);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
            gu[2] += ((dx ? fx : 1 - fx) * (dy ? fy : 1 - fy)) * (c[1][dy][dx] - c[0][dy][dx]);
    const double vsd = (double)a.vs;
    const double gr[3] = {gu[0] / vsd, gu[1] / vsd, gu[2] / vsd};
    const double qd[3] = {(double)q[0], (double)q[1], (double)q[2]};
    const double J[6] = {qd[1] * gr[2] - qd[2] * gr[1], qd[2] * gr[0] - qd[0] * gr[2], qd[0] * gr[1] - qd[1] * gr[0],
                         gr[0], gr[1], gr[2]};
    int k = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int cc = r; cc < 6; ++cc) acc[k++] += J[r] * J[cc];
#pragma unroll
    for (int r = 0; r < 6; ++r) acc[21 + r] += J[r] * d;
    acc[27] += d * d;
    acc[28] += 1.0;
}

__global__ void __launch_bounds__(256) register_kernel(const RegArgs a, const uint32_t* __restrict__ grid,
                                                       double* __restrict__ out) {
    __shared__ double red[8][kSysN];
    double acc[kSysN];
#pragma unroll
    for (int k = 0; k < kSysN; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) reg_point(a, grid, i, acc);
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSysN; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMaskR, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSysN) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        if (v != 0.0) atomicAdd(out + threadIdx.x, v);
    }
}

}  // namespace

cudaError_t launch_register(const float* pts_dev, int n, const float pose[12], const uint32_t* grid,
                            const WindowGeom& geo, const long long origin[3], float vs, float inv_vs, float tau,
                            int min_w, double* out_dev, cudaStream_t s) {
    RegArgs a{};
    a.pts = reinterpret_cast<const float4*>(pts_dev);
    a.n = n;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) a.R[3 * r + c] = pose[4 * r + c];
        a.t[r] = pose[4 * r + 3];
        a.o[r] = origin[r];
    }
    a.vs = vs;
    a.inv_vs = inv_vs;
    a.scale = (double)tau / 32767.0;
    a.tau = (double)tau;
    a.min_w = min_w;
    a.geo = geo;
    cudaError_t e = cudaMemsetAsync(out_dev, 0, kSysN * sizeof(double), s);
    if (e != cudaSuccess || n <= 0) return e;
    int blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    register_kernel<<<blocks, 256, 0, s>>>(a, grid, out_dev);
    return cudaGetLastError();
}

// One Gauss-Newton step on the host: solve H xi = -g by Cholesky (binary64),
// then R' = Exp(w) R, t' = Exp(w) t + v. Returns false if H is not positive
// definite.
bool register_step(const double sys[29], float pose[12], double* step_norm) {
    double H[6][6];
    int k = 0;
    for (int r = 0; r < 6; ++r)
        for (int c = r; c < 6; ++c) H[r][c] = H[c][r] = sys[k++];
    double L[6][6] = {};
    for (int j = 0; j < 6; ++j) {
        double s = H[j][j];
        for (int p = 0; p < j; ++p) s -= L[j][p] * L[j][p];
        if (!(s > 0.0)) return false;
        L[j][j] = std::sqrt(s);
        for (int i = j + 1; i < 6; ++i) {
            double t = H[i][j];
            for (int p = 0; p < j; ++p) t -= L[i][p] * L[j][p];
            L[i][j] = t / L[j][j];
        }
    }
    double y[6], xi[6];
    for (int i = 0; i < 6; ++i) {
        double t = -sys[21 + i];
        for (int p = 0; p < i; ++p) t -= L[i][p] * y[p];
        y[i] = t / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double t = y[i];
        for (int p = i + 1; p < 6; ++p) t -= L[p][i] * xi[p];
        xi[i] = t / L[i][i];
    }
    const double w[3] = {xi[0], xi[1], xi[2]};
    const double th = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    const double K[3][3] = {{0, -w[2], w[1]}, {w[2], 0, -w[0]}, {-w[1], w[0], 0}};
    double K2[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            K2[r][c] = 0.0;
            for (int p = 0; p < 3; ++p) K2[r][c] += K[r][p] * K[p][c];
        }
    const double a = th < 1e-12 ? 1.0 : std::sin(th) / th;
    const double b = th < 1e-12 ? 0.0 : (1.0 - std::cos(th)) / (th * th);
    double E[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) E[r][c] = (r == c ? 1.0 : 0.0) + a * K[r][c] + b * K2[r][c];
    double P[3][4];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) P[r][c] = (double)pose[4 * r + c];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            double v = 0.0;
            for (int p = 0; p < 3; ++p) v += E[r][p] * P[p][c];
            pose[4 * r + c] = (float)v;
        }
        double v = xi[3 + r];
        for (int p = 0; p < 3; ++p) v += E[r][p] * P[p][3];
        pose[4 * r + 3] = (float)v;
    }
    double n2 = 0.0;
    for (int i = 0; i < 6; ++i) n2 += xi[i] * xi[i];
    *step_norm = std::sqrt(n2);
    return true;
}

}  // namespace tsdf
