// Per-scan TSDF integration kernels (FeatSense, Section "TSDF Map Generation").
//
// contrib: one thread per point. The thread transforms its point by the pose,
//   sets up the ray (range, unit direction, unit interpolation direction
//   int = d x (d x up), Eq. 3 / Eq. 4) and walks the steps k = -K..K and the
//   fill samples j = -J..J in warp lock-step. Every sample that lands in the
//   window yields (slot, q) with q the int16 code of the truncated projective
//   distance of the voxel centre. Lanes of a warp that hit the same voxel in
//   the same iteration are merged with match.any + redux.sync, and one lane
//   per distinct voxel issues a single 64-bit atomic into the per-scan
//   accumulator:
//     WSUM    : acc += (count << 40) + sum(q)      (two's-complement packing;
//               exact while count < 2^24 and |sum| < 2^39)
//     MIN_ABS : acc = max(acc, 65536 - key), key = (|q| << 1) | (q < 0)
//   so acc == 0 means "untouched". The lane that turned an accumulator from 0
//   to non-zero appends the slot to the touched list (one list atomic per warp
//   iteration). Integer accumulation makes the result independent of the
//   order in which atomics land.
// apply: one thread per touched voxel, grid-stride. Eq. 1 in exact integers
//   with one rounding (half away from zero), Eq. 2 with the weight cap, and
//   the accumulator is reset to 0. The last CTA to finish publishes the scan
//   counters and clears the per-scan state.
//
// Every float operation on the geometry path is an explicit round-to-nearest
// intrinsic (no contraction into FMA), in the same order as the CPU oracle, so
// voxel indices and codes agree bit for bit.
#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }

template <int MODE>
__global__ void __launch_bounds__(256) contrib_kernel(const ScanArgs a, const MapDev m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;

    // ---- transform + ray set-up (Section "TSDF Map Generation")
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool in = i < a.n;
    if (in) p = __ldg(a.pts + i);
    const float tx = a.t[0], ty = a.t[1], tz = a.t[2];
    const float pwx = fa(fa(fa(fm(a.R[0], p.x), fm(a.R[1], p.y)), fm(a.R[2], p.z)), tx);
    const float pwy = fa(fa(fa(fm(a.R[3], p.x), fm(a.R[4], p.y)), fm(a.R[5], p.z)), ty);
    const float pwz = fa(fa(fa(fm(a.R[6], p.x), fm(a.R[7], p.y)), fm(a.R[8], p.z)), tz);
    const float vx = fs(pwx, tx), vy = fs(pwy, ty), vz = fs(pwz, tz);
    const float r2 = fa(fa(fm(vx, vx), fm(vy, vy)), fm(vz, vz));
    const float r = __fsqrt_rn(r2);
    const bool valid = in && (r >= a.rmin) && (r <= a.rmax);
    const unsigned vmask = __ballot_sync(kFull, valid);
    if (vmask == 0u) return;   // warp-uniform exit

    float dx = 0.f, dy = 0.f, dz = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
    bool fill = false;
    if (valid) {
        dx = __fdiv_rn(vx, r);
        dy = __fdiv_rn(vy, r);
        dz = __fdiv_rn(vz, r);
        const float ux = a.R[2], uy = a.R[5], uz = a.R[8];   // sensor z axis in the world
        const float ax = fs(fm(dy, uz), fm(dz, uy));
        const float ay = fs(fm(dz, ux), fm(dx, uz));
        const float az = fs(fm(dx, uy), fm(dy, ux));
        const float ivx = fs(fm(dy, az), fm(dz, ay));
        const float ivy = fs(fm(dz, ax), fm(dx, az));
        const float ivz = fs(fm(dx, ay), fm(dy, ax));
        const float n2 = fa(fa(fm(ivx, ivx), fm(ivy, ivy)), fm(ivz, ivz));
        if (a.fill && n2 >= 1e-12f) {
            const float nn = __fsqrt_rn(n2);
            fill = true;
            hx = __fdiv_rn(ivx, nn);
            hy = __fdiv_rn(ivy, nn);
            hz = __fdiv_rn(ivz, nn);
        }
    }

    const unsigned mx = a.dimx - 1u, my = a.dimy - 1u, mz = a.dimz - 1u;
    unsigned long long warp_hits = 0;

    for (int k = -a.K; k <= a.K; ++k) {
        const float l = fa(r, fm((float)k, a.vs));
        const bool lv = valid && (l > 0.f);
        int J = 0;
        if (lv && fill) J = __float2int_rd(fm(fm(a.dz, l), a.inv_vs));
        const int Jw = __reduce_max_sync(kFull, lv ? J : -1);
        if (Jw < 0) continue;
        const float bx = fa(tx, fm(dx, l));
        const float by = fa(ty, fm(dy, l));
        const float bz = fa(tz, fm(dz, l));
        for (int j = -Jw; j <= Jw; ++j) {
            unsigned slot = kEmptySlot;
            int q = 0;
            if (lv && j >= -J && j <= J) {
                const float jd = fm((float)j, a.vs);
                const float qx = fa(bx, fm(hx, jd));
                const float qy = fa(by, fm(hy, jd));
                const float qz = fa(bz, fm(hz, jd));
                const long long gx = __float2ll_rd(fm(qx, a.inv_vs));
                const long long gy = __float2ll_rd(fm(qy, a.inv_vs));
                const long long gz = __float2ll_rd(fm(qz, a.inv_vs));
                if ((unsigned long long)(gx - a.ox) < a.dimx && (unsigned long long)(gy - a.oy) < a.dimy &&
                    (unsigned long long)(gz - a.oz) < a.dimz) {
                    slot = ((unsigned)gz & mz) << a.shxy | ((unsigned)gy & my) << a.shx | ((unsigned)gx & mx);
                    const float cx = fm(fa(__ll2float_rn(gx), 0.5f), a.vs);
                    const float cy = fm(fa(__ll2float_rn(gy), 0.5f), a.vs);
                    const float cz = fm(fa(__ll2float_rn(gz), 0.5f), a.vs);
                    const float proj = fa(fa(fm(fs(cx, tx), dx), fm(fs(cy, ty), dy)), fm(fs(cz, tz), dz));
                    float d = fs(r, proj);
                    d = fminf(fmaxf(d, -a.tau), a.tau);
                    q = __float2int_rn(fm(d, a.qs));
                    q = max(-kQMax, min(kQMax, q));
                }
            }
            const bool act = slot != kEmptySlot;
            const unsigned amask = __ballot_sync(kFull, act);
            if (amask == 0u) continue;
            warp_hits += __popc(amask);
            const unsigned peers = __match_any_sync(kFull, slot);
            bool first = false;
            if (act) {
                const unsigned leader = __ffs(peers) - 1u;
                if (MODE == 0) {
                    const int s = __reduce_add_sync(peers, q);
                    if (lane == leader) {
                        const unsigned long long add =
                            ((unsigned long long)__popc(peers) << 40) + (unsigned long long)(long long)s;
                        first = atomicAdd(m.acc + slot, add) == 0ull;
                    }
                } else {
                    const unsigned key = ((unsigned)abs(q) << 1) | (q < 0 ? 1u : 0u);
                    const unsigned kmin = __reduce_min_sync(peers, key);
                    if (lane == leader) first = atomicMax(m.acc + slot, 65536ull - kmin) == 0ull;
                }
            }
            const unsigned fmask = __ballot_sync(kFull, first);
            if (fmask) {
                unsigned base = 0;
                if (lane == 0) base = atomicAdd(&m.ctr->touched_count, (unsigned)__popc(fmask));
                base = __shfl_sync(kFull, base, 0);
                if (first) m.touched[base + __popc(fmask & lt_mask)] = slot;
            }
        }
    }
    if (lane == 0) {
        atomicAdd(&m.ctr->cur_valid, (unsigned long long)__popc(vmask));
        atomicAdd(&m.ctr->cur_hits, warp_hits);
    }
}

template <int MODE>
__global__ void __launch_bounds__(256) apply_kernel(const MapDev m, const int32_t w_max) {
    const unsigned U = *(volatile unsigned*)&m.ctr->touched_count;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < U; i += stride) {
        const unsigned slot = m.touched[i];
        const unsigned long long P = m.acc[slot];
        m.acc[slot] = 0ull;
        long long S, W;
        if (MODE == 0) {
            S = ((long long)(P << 24)) >> 24;               // sign-extended low 40 bits
            W = (long long)((P - (unsigned long long)S) >> 40);
        } else {
            const unsigned key = 65536u - (unsigned)P;
            const int mag = (int)(key >> 1);
            S = (key & 1u) ? -mag : mag;
            W = 1;
        }
        const uint32_t word = m.grid[slot];
        const long long gv = (long long)(int16_t)(word & 0xFFFFu);
        const long long gw = (long long)(int16_t)(word >> 16);
        // Eq. 1: (gv*gw + S) / (gw + W), rounded half away from zero
        const long long num = gv * gw + S;
        const long long den = gw + W;
        const long long an = num < 0 ? -num : num;
        const long long qv = (2 * an + den) / (2 * den);
        const long long nv = num < 0 ? -qv : qv;
        // Eq. 2: min(w_max, gw + W)
        const long long nw = den > w_max ? (long long)w_max : den;
        m.grid[slot] = (uint32_t)(uint16_t)(int16_t)nv | ((uint32_t)nw << 16);
    }
    // The last CTA publishes the counters and clears the per-scan state.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&m.ctr->apply_done, 1u);
        if (done == gridDim.x - 1u) {
            MapCounters* c = m.ctr;
            c->last_valid = (long long)c->cur_valid;
            c->last_hits = (long long)c->cur_hits;
            c->last_touched = (long long)U;
            c->cur_valid = 0ull;
            c->cur_hits = 0ull;
            c->touched_count = 0u;
            c->apply_done = 0u;
            __threadfence();
        }
    }
}

}  // namespace

cudaError_t launch_contrib(const ScanArgs& a, const MapDev& m, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (a.n + threads - 1) / threads;
    if (a.reduce == 0) contrib_kernel<0><<<blocks, threads, 0, s>>>(a, m);
    else contrib_kernel<1><<<blocks, threads, 0, s>>>(a, m);
    return cudaGetLastError();
}

cudaError_t launch_apply(const MapDev& m, int32_t reduce, int32_t w_max, int num_ctas, cudaStream_t s) {
    if (reduce == 0) apply_kernel<0><<<num_ctas, 256, 0, s>>>(m, w_max);
    else apply_kernel<1><<<num_ctas, 256, 0, s>>>(m, w_max);
    return cudaGetLastError();
}

}  // namespace tsdf
