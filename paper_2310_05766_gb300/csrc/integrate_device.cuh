// Device-side bodies of the integration phases, shared by the per-map kernels
// (integrate.cu) and the batched persistent kernel (batch.cu), so that both
// run the same arithmetic. See integrate.cu for the method.
#pragma once

#include "tsdf_internal.cuh"

namespace tsdf {
namespace dev {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr unsigned kNoVoxel = 0xFFFFFFFFu;

// Shared-memory cache of bricks already marked in the scan's brick flags
// (direct mapped on a multiplicative hash of the brick index). A null table
// sends every mark to global memory. An entry holds brick + tag: a table that
// serves several maps gives each map its own tag, so that keys of different
// maps never coincide (nor equal kNoVoxel, the empty entry).
struct BrickCache {
    uint32_t* tab = nullptr;
    unsigned shift = 32;          // 32 - log2(entries)
    uint32_t tag = 0;
};

// The per-map contribution kernels keep one cache per CTA.
constexpr int kBrickCacheLog2 = 11;
constexpr int kBrickCache = 1 << kBrickCacheLog2;

// Empty the CTA's brick cache (every thread calls it; a __syncthreads
// must follow before the first use).
__device__ __forceinline__ void brick_cache_init(uint32_t* btab) {
    for (int i = threadIdx.x; i < kBrickCache; i += blockDim.x) btab[i] = kNoVoxel;
}

#ifndef TSDF_MARK_SHFL
#define TSDF_MARK_SHFL 0
#endif
// 1: the plain atomic contribution march runs lean_march (fewer instructions
// per sample, same results); 0: the general march
#ifndef TSDF_LEAN_MARCH
#define TSDF_LEAN_MARCH 1
#endif

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }

// Programmatic dependent launch: wait for the preceding grid's completion
// (and visibility of its writes) / let the next grid be scheduled early.
// Both are no-ops for a grid launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Sum of a 64-bit value over the CTA (every thread must call it); the result
// is valid in thread 0.
template <int NWARPS>
__device__ __forceinline__ unsigned long long cta_sum(unsigned long long v, unsigned long long* smem) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31u) == 0) smem[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NWARPS; ++w) s += smem[w];
    return s;
}

// Exact integer value of an integer-valued float x with 0 <= x < 2^22 (and of
// rint(x) for |x| < 2^22), via one float add and one integer subtract: the
// add places the integer in the low mantissa bits.
__device__ __forceinline__ int small_int(float x) { return __float_as_int(fa(x, 12582912.0f)) - 0x4B400000; }

// Fill half-height J of march step k of a ray of range r (Eq. 3 / Eq. 4):
// J = floor(delta_z * l / vs) at l = r + k vs; -1 when the step is skipped
// (l <= 0 or a dead ray). The contribution march and the slot count of the
// sort reduction both use exactly this arithmetic.
__device__ __forceinline__ int step_fill(const ScanArgs& a, float r, bool fill, int k, float& l) {
    l = fa(r, fm((float)k, a.vs));
    const bool lv = (r >= 0.f) && (l > 0.f);
    if (!lv) return -1;
    return fill ? __float2int_rd(fm(fm(a.dz, l), a.inv_vs)) : 0;
}

// Sort reduction: pair slots of one ray, one per (k, j) sample of its march,
// or kNoSlot when it has more than kRaySlotLimit (its samples then overflow).
__device__ __forceinline__ uint32_t ray_slots(const ScanArgs& a, float r, bool fill) {
    uint32_t n = 0;
    for (int k = -a.K; k <= a.K; ++k) {
        float l;
        const int J = step_fill(a, r, fill, k, l);
        if (J < 0) continue;
        if ((uint32_t)J >= kRaySlotLimit) return kNoSlot;
        n += 2u * (uint32_t)J + 1u;
        if (n > kRaySlotLimit) return kNoSlot;
    }
    return n;
}

template <int NW>
struct RaysSmemT {
    // per warp: live (split: heavy) rays, valid rays, pair slots, light rays
    // (split list); thread 0 turns them into exclusive prefixes over the warps
    unsigned wl[NW], wv[NW], ws[NW], wb[NW];
    unsigned base;                  // the CTA's first ray-list entry
    unsigned bbase;                 // split list: the CTA's first light-ray entry, counted from the end
    unsigned long long sbase;       // the CTA's first pair slot (sort reduction)
};
using RaysSmem = RaysSmemT<8>;

// One point of a scan (sensor frame; `in`: the point exists): world transform,
// range test, unit direction, fill direction (Eq. 3 / Eq. 4) and the
// conservative window culling. ra = (dir, r) with r = -1 for an invalid ray,
// rb = (fill direction, 1) or zeros without fill.
__device__ __forceinline__ void ray_setup(const ScanArgs& a, float4 p, bool in, float4& ra, float4& rb, bool& valid,
                                          bool& live) {
    const float tx = a.t[0], ty = a.t[1], tz = a.t[2];
    const float pwx = fa(fa(fa(fm(a.R[0], p.x), fm(a.R[1], p.y)), fm(a.R[2], p.z)), tx);
    const float pwy = fa(fa(fa(fm(a.R[3], p.x), fm(a.R[4], p.y)), fm(a.R[5], p.z)), ty);
    const float pwz = fa(fa(fa(fm(a.R[6], p.x), fm(a.R[7], p.y)), fm(a.R[8], p.z)), tz);
    const float vx = fs(pwx, tx), vy = fs(pwy, ty), vz = fs(pwz, tz);
    const float r2 = fa(fa(fm(vx, vx), fm(vy, vy)), fm(vz, vz));
    const float r = __fsqrt_rn(r2);
    valid = in && (r >= a.rmin) && (r <= a.rmax);

    ra = make_float4(0.f, 0.f, 0.f, -1.f);
    rb = make_float4(0.f, 0.f, 0.f, 0.f);
    live = false;
    if (valid) {
        const float dx = __fdiv_rn(vx, r), dy = __fdiv_rn(vy, r), dz = __fdiv_rn(vz, r);
        const float ux = a.R[2], uy = a.R[5], uz = a.R[8];   // sensor z axis in the world
        const float ax = fs(fm(dy, uz), fm(dz, uy));
        const float ay = fs(fm(dz, ux), fm(dx, uz));
        const float az = fs(fm(dx, uy), fm(dy, ux));
        const float ivx = fs(fm(dy, az), fm(dz, ay));
        const float ivy = fs(fm(dz, ax), fm(dx, az));
        const float ivz = fs(fm(dx, ay), fm(dy, ax));
        const float n2 = fa(fa(fm(ivx, ivx), fm(ivy, ivy)), fm(ivz, ivz));
        const bool fill = a.fill && n2 >= 1e-12f;
        if (fill) {
            const float nn = __fsqrt_rn(n2);
            rb = make_float4(__fdiv_rn(ivx, nn), __fdiv_rn(ivy, nn), __fdiv_rn(ivz, nn), 1.f);
        }
        // conservative culling: distance from the hit to the window box against
        // the reach of the march (tau + fill height + margin)
        const float hx = tx + dx * r, hy = ty + dy * r, hz = tz + dz * r;
        const float ex = fmaxf(fmaxf(a.win_lo[0] - hx, hx - a.win_hi[0]), 0.f);
        const float ey = fmaxf(fmaxf(a.win_lo[1] - hy, hy - a.win_hi[1]), 0.f);
        const float ez = fmaxf(fmaxf(a.win_lo[2] - hz, hz - a.win_hi[2]), 0.f);
        const float reach = a.tau + (fill ? a.dz * (r + a.tau) : 0.f) + 2.f * a.vs +
                            1e-4f * (fabsf(tx) + fabsf(ty) + fabsf(tz) + r);
        live = ex * ex + ey * ey + ez * ez <= reach * reach;
        ra = make_float4(dx, dy, dz, r);
    }
}

// ---- rays: the CTA's 32 NW threads set up points [base, base + 32 NW) of a
// scan and append the live ones to the map's ray list. With SORT each live ray also
// reserves its pair slots (one 64-bit atomic per CTA). With SPLIT the rays
// whose fill reaches at least one voxel each side at the hit (delta_z r >= vs,
// the costly ones) go to the front of the list and the others to its end
// (entry ray_cap - 1 - j for the j-th), so that the contribution kernel can
// take the costly work first; with both ends counted, they never meet. With
// PDL the wait for the preceding grid comes before the first access to the
// map's counters and ray list.
template <bool PDL, bool SORT, bool SPLIT = false, int NW = 8>
__device__ __forceinline__ void rays_task(const ScanArgs& a, const MapDev& m, int base, unsigned part,
                                          RaysSmemT<NW>* sm) {
    static_assert(!(SORT && SPLIT), "the sort reduction keeps one list");
    const int i = base + (int)threadIdx.x;
    const unsigned lane = threadIdx.x & 31u;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool in = i < a.n;
    if (in) p = __ldg(a.pts + i);   // the caller's points: no dependency on earlier grids
    if (PDL) pdl_trigger();
    float4 ra, rb;
    bool valid, live;
    ray_setup(a, p, in, ra, rb, valid, live);
    // pair slots of this ray (sort reduction): an inclusive warp scan
    uint32_t nslot = 0, sincl = 0;
    if (SORT) {
        nslot = live ? ray_slots(a, ra.w, rb.w != 0.f) : 0u;
        const uint32_t own = nslot == kNoSlot ? 0u : nslot;
        sincl = own;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, sincl, o);
            if (lane >= (unsigned)o) sincl += y;
        }
    }
    // CTA-level compaction of the live rays: one list atomic per CTA (per end)
    const unsigned warp = threadIdx.x >> 5;
    const bool heavy = !SPLIT || (live && rb.w != 0.f && fm(fm(a.dz, ra.w), a.inv_vs) >= 1.f);
    const unsigned lmask = __ballot_sync(kFull, live && heavy);
    const unsigned bmask = SPLIT ? __ballot_sync(kFull, live && !heavy) : 0u;
    const unsigned vmask = __ballot_sync(kFull, valid);
    if (lane == 0) {
        sm->wl[warp] = __popc(lmask);
        sm->wv[warp] = __popc(vmask);
        if (SPLIT) sm->wb[warp] = __popc(bmask);
    }
    if (SORT && lane == 31) sm->ws[warp] = sincl;
    __syncthreads();
    if (PDL) pdl_wait();   // the previous scan's finish kernel resets live_count and the counters
    if (threadIdx.x == 0) {
        unsigned tl = 0, tv = 0, tb = 0, ts32 = 0;
        unsigned long long ts = 0;
        for (int w = 0; w < NW; ++w) {
            const unsigned l = sm->wl[w], b = SPLIT ? sm->wb[w] : 0u, q = SORT ? sm->ws[w] : 0u;
            sm->wl[w] = tl;
            tl += l;
            tv += sm->wv[w];
            if (SPLIT) {
                sm->wb[w] = tb;
                tb += b;
            }
            if (SORT) {
                sm->ws[w] = ts32;
                ts32 += q;
                ts += q;
            }
        }
        sm->base = tl ? atomicAdd(&m.ctr->live_count, tl) : 0u;
        if (SPLIT) sm->bbase = tb ? atomicAdd(&m.ctr->live_back, tb) : 0u;
        if (tv) atomicAdd(&m.ctr->part[part % kParts].valid, (unsigned long long)tv);
        if (SORT) sm->sbase = ts ? atomicAdd(&m.ctr->slot_count, ts) : 0ull;
    }
    __syncthreads();
    if (live) {
        const unsigned below = (1u << lane) - 1u;
        unsigned off;
        if (heavy) {
            off = sm->base + sm->wl[warp] + __popc(lmask & below);
        } else {
            off = m.ray_cap - 1u - (sm->bbase + sm->wb[warp] + __popc(bmask & below));
        }
        m.ray_a[off] = ra;
        m.ray_b[off] = rb;
        if (SORT) {
            const unsigned long long first = sm->sbase + sm->ws[warp] + (sincl - (nslot == kNoSlot ? 0u : nslot));
            // slots at or beyond the capacity overflow, sample by sample
            m.ray_slot[off] = nslot == kNoSlot ? kNoSlot
                                                : (uint32_t)(first < m.pair_cap ? first : (unsigned long long)m.pair_cap);
        }
    }
}

// Points per thread of the plain path's ray set-up (rays_task_ppt): in the
// per-map ray kernel, whose CTAs are all resident at once, one (4 measured
// 1.6 us slower per outdoor scan: a quarter of the CTAs, each thread's four
// points set up one after another); in the batched kernel, whose fixed grid
// walks the ray tasks of all maps, four in one of its configurations (64-map
// batch 1.17-1.19 against 1.21 ms: four point loads in flight per thread), one
// in the others.
#ifndef TSDF_RAYS_PPT
#define TSDF_RAYS_PPT 1
#endif
#ifndef TSDF_BATCH_RAYS_PPT
#define TSDF_BATCH_RAYS_PPT 4
#endif
constexpr int kRaysPPT = TSDF_RAYS_PPT;
constexpr int kBatchRaysPPT = TSDF_BATCH_RAYS_PPT;

// The plain path's ray set-up with PPT consecutive points per thread: the
// CTA's threads set up points [base, base + 32 NW PPT), thread t the points
// base + PPT t .. base + PPT t + PPT - 1, whose loads are all in flight at
// once, and append the live ones (in point order) to the map's ray list with
// one list atomic per CTA and list end, as rays_task does for one point per
// thread. Same rays, same per-ray results; only fewer CTAs and atomics.
template <bool PDL, bool SPLIT, int NW, int PPT>
__device__ __forceinline__ void rays_task_ppt(const ScanArgs& a, const MapDev& m, int base, unsigned part,
                                              RaysSmemT<NW>* sm) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned warp = threadIdx.x >> 5;
    const int i0 = base + PPT * (int)threadIdx.x;
    float4 p[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {   // the caller's points: no dependency on earlier grids
        p[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i0 + k < a.n) p[k] = __ldg(a.pts + i0 + k);
    }
    if (PDL) pdl_trigger();
    float4 ra[PPT], rb[PPT];
    unsigned hv = 0, lv = 0;   // bit k: point k is a live heavy (front) / light (end) ray
    unsigned cv = 0;           // valid rays
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        bool valid, live;
        ray_setup(a, p[k], i0 + k < a.n, ra[k], rb[k], valid, live);
        const bool heavy = !SPLIT || (live && rb[k].w != 0.f && fm(fm(a.dz, ra[k].w), a.inv_vs) >= 1.f);
        if (live && heavy) hv |= 1u << k;
        if (live && !heavy) lv |= 1u << k;
        cv += valid ? 1u : 0u;
    }
    // CTA-level compaction: inclusive warp scans of the per-thread counts
    const unsigned cl = __popc(hv), cb = __popc(lv);
    unsigned il = cl, ib = cb;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned yl = __shfl_up_sync(kFull, il, o);
        const unsigned yb = __shfl_up_sync(kFull, ib, o);
        if (lane >= (unsigned)o) {
            il += yl;
            ib += yb;
        }
    }
    const unsigned wv = __reduce_add_sync(kFull, cv);
    if (lane == 31) {
        sm->wl[warp] = il;
        sm->wb[warp] = ib;
        sm->wv[warp] = wv;
    }
    __syncthreads();
    if (PDL) pdl_wait();   // the previous scan's finish kernel resets live_count and the counters
    if (threadIdx.x == 0) {
        unsigned tl = 0, tv = 0, tb = 0;
        for (int w = 0; w < NW; ++w) {
            const unsigned l = sm->wl[w], b = sm->wb[w];
            sm->wl[w] = tl;
            tl += l;
            sm->wb[w] = tb;
            tb += b;
            tv += sm->wv[w];
        }
        sm->base = tl ? atomicAdd(&m.ctr->live_count, tl) : 0u;
        sm->bbase = SPLIT && tb ? atomicAdd(&m.ctr->live_back, tb) : 0u;
        if (tv) atomicAdd(&m.ctr->part[part % kParts].valid, (unsigned long long)tv);
    }
    __syncthreads();
    unsigned off_l = sm->base + sm->wl[warp] + il - cl;     // first front entry of this thread
    unsigned off_b = sm->bbase + sm->wb[warp] + ib - cb;    // first end entry (counted from the end)
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (hv & (1u << k)) {
            m.ray_a[off_l] = ra[k];
            m.ray_b[off_l] = rb[k];
            ++off_l;
        } else if (lv & (1u << k)) {
            m.ray_a[m.ray_cap - 1u - off_b] = ra[k];
            m.ray_b[m.ray_cap - 1u - off_b] = rb[k];
            ++off_b;
        }
    }
}

// ---- contrib: rays of one 32-ray block (one per lane, dead lanes r = -1);
// `ray` is live when below `end`
__device__ __forceinline__ void load_rays(const MapDev& m, unsigned end, unsigned ray, float4& A, float4& B) {
    A = make_float4(0.f, 0.f, 0.f, -1.f);
    B = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ray < end) {
        A = m.ray_a[ray];
        B = m.ray_b[ray];
    }
}

// One warp: the steps of k-group `grp` (KPT steps) of its 32 rays.
// SORT (sort reduction, MERGE off): each sample of a lane's ray is written to
// the ray's pair slot sslot + (its index in the ray's march) instead of being
// reduced: (voxel word, code) inside the window, kNoVoxel outside. Samples
// whose slot is at or beyond the capacity (or whose ray has none) take the
// accumulator reduction instead and set `ovf`.
// Pool reduction: slot of `brick` in the map's pool, claimed on first touch.
// Lanes of the active set that need the same brick share one claim (match).
// The claimer moves the brick's table entry from empty to a "claiming" mark
// with a CAS, takes the next slot from the counter and publishes it; other
// warps that meet the mark wait for the slot (a bounded wait: the claimer
// depends on nothing, and a wait that runs out drops the scan like a full
// pool). So every slot holds a distinct brick. Returns kPoolEmpty when the
// pool is full (the scan is then dropped and reported).
constexpr uint32_t kPoolClaiming = 0xFFFFFFFEu;
constexpr long long kPoolSpinLimit = 1LL << 20;

__device__ __forceinline__ uint32_t pool_slot(const MapDev& m, unsigned brick) {
    uint32_t s = __ldcg(m.pool_table + brick);
    if (s < kPoolClaiming) return s;
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, brick);
    const unsigned leader = (unsigned)(__ffs(peers) - 1);
    if ((threadIdx.x & 31u) == leader) {
        long long spins = 0;
        for (;;) {
            if (__ldcg(&m.ctr->pool_overflow) != 0u) {
                s = kPoolEmpty;
                break;
            }
            s = __ldcg(m.pool_table + brick);
            if (s < kPoolClaiming) break;
            if (s == kPoolEmpty) {
                if (atomicCAS(m.pool_table + brick, kPoolEmpty, kPoolClaiming) != kPoolEmpty) continue;
                const uint32_t ns = atomicAdd(&m.ctr->pool_count, 1u);
                if (ns < m.pool_cap) {
                    m.pool_brick[ns] = brick;
                    atomicExch(m.pool_table + brick, ns);
                    s = ns;
                } else {
                    atomicExch(&m.ctr->pool_overflow, 1u);
                    atomicExch(m.pool_table + brick, kPoolEmpty);
                    s = kPoolEmpty;
                }
                break;
            }
            if (++spins > kPoolSpinLimit) {   // another warp is claiming it
                atomicExch(&m.ctr->pool_overflow, 1u);
                s = kPoolEmpty;
                break;
            }
            __nanosleep(32);
        }
    }
    return __shfl_sync(peers, s, leader);
}

// ---- lean march of the plain atomic reduction (no sort, pool or merge).
//
// The same samples, voxels and codes as the general march below, with fewer
// instructions per sample:
//  * window test and ring index from one float add per axis: for the
//    integer-valued float f = floor(q / vs), RN(f + (1.5 * 2^23 - o)) is
//    exact whenever f - o lies in [-2^22, 2^22), and its bit pattern minus
//    that of 1.5 * 2^23 is then f - o; outside that range the difference is
//    at least 2^22 as an unsigned number. So `rel < dims` (unsigned) is
//    exactly the window test o <= f < o + dims, and (rel + o mod dims) mod
//    dims the ring index, for any finite f;
//  * x and y in packed binary32 pairs (each lane of a pair is an IEEE
//    round-to-nearest operation, as the scalar ones);
//  * fill samples +j and -j share the offset B * (j vs): the oracle's
//    b + B * (-(j vs)) is exactly b - B * (j vs), and the j = 0 sample is b
//    itself (b + B * 0 rounds to b, up to the sign of a zero, which changes
//    neither the floor, the window test nor the voxel centre);
//  * no clamp of the code: |d| <= tau gives |d * qs| <= 32767.002, whose
//    rounding never leaves [-32767, 32767].
constexpr uint32_t kMagicBits = 0x4B400000u;   // bit pattern of 1.5 * 2^23

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

// Packed (x, y) binary32 add and multiply, each component round-to-nearest.
// TSDF_LEAN_PACKED selects where packed pairs are used: bit 0 for the sample
// position (b, q, q / vs, the window add), bit 1 for the voxel centre and the
// projection; 0 = scalar operations throughout.
#ifndef TSDF_LEAN_PACKED
#define TSDF_LEAN_PACKED 0
#endif
template <bool PACKED>
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    if (PACKED) return __fadd2_rn(a, b);
    return make_float2(fa(a.x, b.x), fa(a.y, b.y));
}
template <bool PACKED>
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    if (PACKED) return __fmul2_rn(a, b);
    return make_float2(fm(a.x, b.x), fm(a.y, b.y));
}
constexpr bool kPackPos = (TSDF_LEAN_PACKED & 1) != 0;
constexpr bool kPackCtr = (TSDF_LEAN_PACKED & 2) != 0;

// One sample at q = (qxy, qz) of a ray (direction A, range r): voxel, code,
// reduction and brick mark. `mine` = the lane's ray has this sample.
template <int MODE, bool SV>
__device__ __forceinline__ void lean_sample(const ScanArgs& a, const MapDev& m, float2 qxy,
                                            float qz, const float4& A, float dstep, bool mine, unsigned& hits,
                                            unsigned& last_brick, const BrickCache& bc) {
    const float2 yxy = mul2<kPackPos>(qxy, a.l_inv);
    const float yz = fm(qz, a.inv_vs);
    const float fx = floorf(yxy.x), fy = floorf(yxy.y), fz = floorf(yz);
    const float2 uxy = add2<kPackPos>(f2(fx, fy), a.l_m);
    const float uz = fa(fz, a.l_mz);
    const uint32_t bx = __float_as_uint(uxy.x), by = __float_as_uint(uxy.y), bz = __float_as_uint(uz);
    const bool act = mine && (bx - kMagicBits < a.l_dim[0]) && (by - kMagicBits < a.l_dim[1]) &&
                     (bz - kMagicBits < a.l_dim[2]);
    // ring coordinates and the bricked word index:
    // word = sx + 8 sy + 64 sz + 504 (sx >> 3) + cy (sy >> 3) + cz (sz >> 3)
    const uint32_t sx = (bx + a.l_omb[0]) & a.dmask[0];
    const uint32_t sy = (by + a.l_omb[1]) & a.dmask[1];
    const uint32_t sz = (bz + a.l_omb[2]) & a.dmask[2];
    const uint32_t word = sx + (sy << 3) + (sz << 6) + (sx >> 3) * 504u + (sy >> 3) * a.l_cy + (sz >> 3) * a.l_cz;
    float d;
    if (SV) {
        d = dstep;
    } else {
        // projective distance of the voxel centre (f + 0.5) vs
        const float2 cxy = mul2<kPackCtr>(add2<kPackCtr>(f2(fx, fy), f2(0.5f, 0.5f)), a.l_vs);
        const float cz = fm(fa(fz, 0.5f), a.vs);
        const float2 exy = mul2<kPackCtr>(add2<kPackCtr>(cxy, a.l_nt), f2(A.x, A.y));
        const float ez = fm(fa(cz, a.l_ntz), A.z);
        d = fs(A.w, fa(fa(exy.x, exy.y), ez));
    }
    d = fminf(fmaxf(d, -a.tau), a.tau);
    const int q = small_int(fm(d, a.qs));
    if (act) {
        if (MODE == 0) {
            atomicAdd(m.acc + word, (1ull << 40) + (unsigned long long)(long long)q);
        } else {
            const unsigned key = ((unsigned)abs(q) << 1) | (q < 0 ? 1u : 0u);
            atomicMax(m.acc + word, 65536ull - key);
            ++hits;
        }
        // mark the brick unless this lane marked it last; with a brick cache
        // the global flag store only on a cache miss (see contrib_item)
        const unsigned brick = word >> 9;
        if (brick != last_brick) {
            last_brick = brick;
            if (bc.tab) {
                const unsigned h = (brick * 2654435761u) >> bc.shift;
                if (bc.tab[h] != brick + bc.tag) {
                    bc.tab[h] = brick + bc.tag;
                    m.brick_flag[brick] = 1;
                }
            } else {
                m.brick_flag[brick] = 1;
            }
        }
    }
}

// The steps k0 .. k0 + KPT - 1 (at most K) of the warp's 32 rays.
template <int MODE, int KPT, bool SV>
__device__ __forceinline__ void lean_march(const ScanArgs& a, const MapDev& m, int k0, const float4& A,
                                           const float4& B, unsigned& hits, unsigned& last_brick,
                                           const BrickCache& bc) {
    const float r = A.w;                // dead lanes carry r = -1
    const bool rfill = B.w != 0.f;
#pragma unroll 1
    for (int kk = 0; kk < KPT; ++kk) {
        const int k = k0 + kk;
        if (k > a.K) break;   // uniform
        float l;
        const int J = step_fill(a, r, rfill, k, l);   // -1: no sample
        const int Jw = __reduce_max_sync(kFull, J);
        if (Jw < 0) continue;   // uniform
        const float2 bxy = add2<kPackPos>(a.l_t, mul2<kPackPos>(f2(A.x, A.y), f2(l, l)));
        const float bz = fa(a.t[2], fm(A.z, l));
        const float dstep = fs(r, l);
        lean_sample<MODE, SV>(a, m, bxy, bz, A, dstep, J >= 0, hits, last_brick, bc);
        for (int j = 1; j <= Jw; ++j) {   // warp-uniform bounds
            const float jd = fm((float)j, a.vs);
            const float2 oxy = mul2<kPackPos>(f2(B.x, B.y), f2(jd, jd));
            const float oz = fm(B.z, jd);
            const bool mine = j <= J;
            lean_sample<MODE, SV>(a, m, add2<kPackPos>(bxy, oxy), fa(bz, oz), A, dstep, mine, hits, last_brick, bc);
            lean_sample<MODE, SV>(a, m, add2<kPackPos>(bxy, f2(-oxy.x, -oxy.y)), fs(bz, oz), A, dstep, mine, hits,
                                  last_brick, bc);
        }
    }
}

template <int MODE, bool MERGE, int KPT, bool SORT = false, bool POOL = false>
__device__ __forceinline__ void contrib_item(const ScanArgs& a, const MapDev& m, unsigned grp, const float4 A,
                                             const float4 B, unsigned& hits, unsigned& last_brick,
                                             uint32_t sslot = kNoSlot, bool* ovf = nullptr,
                                             uint32_t* last_slot = nullptr, BrickCache bc = BrickCache{}) {
    static_assert(!(SORT && MERGE), "the sort reduction emits every sample");
    static_assert(!(POOL && (SORT || MERGE)), "the pool reduction is a variant of the plain atomic one");
#if TSDF_LEAN_MARCH
    if constexpr (!SORT && !POOL && !MERGE) {
        const int k0l = (int)grp * KPT - a.K;
        if (a.flags & kFlagStepValue) lean_march<MODE, KPT, true>(a, m, k0l, A, B, hits, last_brick, bc);
        else lean_march<MODE, KPT, false>(a, m, k0l, A, B, hits, last_brick, bc);
        return;
    }
#endif
    const unsigned lane = threadIdx.x & 31u;
    const float tx = a.t[0], ty = a.t[1], tz = a.t[2];
    const float r = A.w;                // dead lanes carry r = -1
    const bool rfill = B.w != 0.f;
    const int k0 = (int)grp * KPT - a.K;
    uint32_t sidx = 0;                  // SORT: index of the step's first sample in the ray's march
    if (SORT && sslot != kNoSlot) {
        for (int k = -a.K; k < k0; ++k) {
            float l;
            const int J = step_fill(a, r, rfill, k, l);
            if (J >= 0) sidx += 2u * (uint32_t)J + 1u;
        }
    }
#pragma unroll 1
    for (int kk = 0; kk < KPT; ++kk) {
        const int k = k0 + kk;
        if (k > a.K) break;   // uniform
        float l;
        const int Jr = step_fill(a, r, rfill, k, l);
        const bool lv = Jr >= 0;
        const int J = lv ? Jr : 0;
        const int Jw = __reduce_max_sync(kFull, lv ? J : -1);   // -1: no live lane
        const float bx = fa(tx, fm(A.x, l));
        const float by = fa(ty, fm(A.y, l));
        const float bz = fa(tz, fm(A.z, l));
        const float dstep = fs(r, l);   // the step's own distance (TSDF_FLAG_STEP_VALUE)
        for (int j = -Jw; j <= Jw; ++j) {   // warp-uniform bounds
            // every lane evaluates the sample; lanes outside their own fill
            // range or outside the window are masked out (no divergent branches)
            const float jd = fm((float)j, a.vs);
            const float fx = floorf(fm(fa(bx, fm(B.x, jd)), a.inv_vs));
            const float fy = floorf(fm(fa(by, fm(B.y, jd)), a.inv_vs));
            const float fz = floorf(fm(fa(bz, fm(B.z, jd)), a.inv_vs));
            const bool act = lv && j >= -J && j <= J && fx >= a.fo[0] && fx < a.fe[0] && fy >= a.fo[1] &&
                             fy < a.fe[1] && fz >= a.fo[2] && fz < a.fe[2];
            // window-relative index (exact: both integers below 2^24), then the ring slot
            const unsigned rx = ((unsigned)small_int(fs(fx, a.fo[0])) + a.omod[0]) & a.dmask[0];
            const unsigned ry = ((unsigned)small_int(fs(fy, a.fo[1])) + a.omod[1]) & a.dmask[1];
            const unsigned rz = ((unsigned)small_int(fs(fz, a.fo[2])) + a.omod[2]) & a.dmask[2];
            const unsigned brick = ((rz >> 3) << a.lcxy) | ((ry >> 3) << a.lcx) | (rx >> 3);
            const unsigned word = (brick << 9) | ((rz & 7u) << 6) | ((ry & 7u) << 3) | (rx & 7u);
            // voxel centre: (float)g + 0.5 is fx + 0.5 exactly (|g| < 2^24)
            const float cx = fm(fa(fx, 0.5f), a.vs);
            const float cy = fm(fa(fy, 0.5f), a.vs);
            const float cz = fm(fa(fz, 0.5f), a.vs);
            const float proj = fa(fa(fm(fs(cx, tx), A.x), fm(fs(cy, ty), A.y)), fm(fs(cz, tz), A.z));
            const float d = fminf(fmaxf((a.flags & kFlagStepValue) ? dstep : fs(r, proj), -a.tau), a.tau);
            // rint (ties to even) of |d qs| <= 32767.x < 2^22, as an exact float add
            int q = small_int(fm(d, a.qs));
            q = max(-kQMax, min(kQMax, q));
            bool leader = act;
            if (POOL) {
                // the lane's last brick and its slot are cached: the table is
                // read only when the lane moves to another brick
                if (act && brick != last_brick) {
                    *last_slot = pool_slot(m, brick);
                    last_brick = brick;
                }
                if (act && *last_slot != kPoolEmpty) {
                    unsigned long long* pa = m.pool_acc + (((size_t)*last_slot) << 9) + (word & 511u);
                    if (MODE == 0) atomicAdd(pa, (1ull << 40) + (unsigned long long)(long long)q);
                    else atomicMax(pa, 65536ull - (((unsigned)abs(q) << 1) | (q < 0 ? 1u : 0u)));
                }
                if (MODE == 1) hits += act ? 1u : 0u;
                continue;   // no brick flags: the claimed slots list the touched bricks
            } else if (SORT) {
                const bool mine = lv && j >= -J && j <= J;
                const uint32_t slot = sslot + sidx + (uint32_t)(j + J);   // no wrap: sslot <= cap, sidx < 2^21
                if (mine && sslot != kNoSlot && slot < m.pair_cap) {
                    m.pairs[slot] = act ? make_uint2(word, (uint32_t)q) : make_uint2(kNoVoxel, 0u);
                } else if (act) {
                    if (MODE == 0) atomicAdd(m.acc + word, (1ull << 40) + (unsigned long long)(long long)q);
                    else atomicMax(m.acc + word, 65536ull - (((unsigned)abs(q) << 1) | (q < 0 ? 1u : 0u)));
                    if (MODE == 1) ++hits;
                    *ovf = true;
                }
            } else if (MERGE) {
                if (__ballot_sync(kFull, act) == 0u) continue;   // warp-uniform
                const unsigned peers = __match_any_sync(kFull, act ? word : kNoVoxel);
                leader = act && lane == (unsigned)(__ffs(peers) - 1);
                if (MODE == 0) {
                    const int s = __reduce_add_sync(peers, q);
                    if (leader)
                        atomicAdd(m.acc + word,
                                  ((unsigned long long)__popc(peers) << 40) + (unsigned long long)(long long)s);
                } else {
                    const unsigned key = ((unsigned)abs(q) << 1) | (q < 0 ? 1u : 0u);
                    const unsigned kmin = __reduce_min_sync(peers, key);
                    if (leader) atomicMax(m.acc + word, 65536ull - kmin);
                }
            } else {
                if (MODE == 0) {
                    if (act) atomicAdd(m.acc + word, (1ull << 40) + (unsigned long long)(long long)q);
                } else {
                    const unsigned key = ((unsigned)abs(q) << 1) | (q < 0 ? 1u : 0u);
                    if (act) atomicMax(m.acc + word, 65536ull - key);
                }
            }
            if (MODE == 1 && !SORT) hits += act ? 1u : 0u;
            // mark the brick unless this lane marked it last (same-address
            // byte stores of a warp merge into one transaction); optionally
            // also skip when the lane below marks the same brick now. With a
            // brick cache the global store is issued only on a cache miss:
            // many lanes and warps touch the same few bricks, and same-address
            // stores from every SM are what makes the marking costly. (Any
            // thread that puts a brick into the cache also stores its flag,
            // so a hit never hides an unmarked brick.)
#if TSDF_MARK_SHFL
            const unsigned below = __shfl_up_sync(kFull, leader ? brick : kNoVoxel, 1);
            if (leader && brick != last_brick && (lane == 0 || below != brick)) {
#else
            if (leader && brick != last_brick) {
#endif
                last_brick = brick;
                if (bc.tab) {
                    const unsigned h = (brick * 2654435761u) >> bc.shift;
                    if (bc.tab[h] != brick + bc.tag) {
                        bc.tab[h] = brick + bc.tag;
                        m.brick_flag[brick] = 1;
                    }
                } else {
                    m.brick_flag[brick] = 1;
                }
            }
        }
        if (SORT && lv) sidx += 2u * (uint32_t)J + 1u;
    }
}

// Eq. 1 / Eq. 2 for one voxel. Returns the new grid word.
__device__ __forceinline__ uint32_t update_voxel(uint32_t word, long long S, long long W, int32_t w_max) {
    const long long gv = (long long)(int16_t)(word & 0xFFFFu);
    const long long gw = (long long)(int16_t)(word >> 16);
    const long long num = gv * gw + S;
    const long long den = gw + W;
    const unsigned long long an = (unsigned long long)(num < 0 ? -num : num);
    const unsigned long long top = 2ull * an + (unsigned long long)den;
    const unsigned long long bot = 2ull * (unsigned long long)den;
    const unsigned long long qv = top / bot;
    const long long nv = num < 0 ? -(long long)qv : (long long)qv;
    const long long nw = den > w_max ? (long long)w_max : den;
    return (uint32_t)(uint16_t)(int16_t)nv | ((uint32_t)nw << 16);
}

// Eq. 1 / Eq. 2 when the scan's average S/W counts as one observation of
// weight 1 (TSDF_FLAG_SCAN_WEIGHT): (gv gw W + S) / ((gw + 1) W), one rounding.
__device__ __forceinline__ uint32_t update_voxel_scan(uint32_t word, long long S, long long W, int32_t w_max) {
    const long long gv = (long long)(int16_t)(word & 0xFFFFu);
    const long long gw = (long long)(int16_t)(word >> 16);
    const long long num = gv * gw * W + S;
    const long long den = (gw + 1) * W;
    const unsigned long long an = (unsigned long long)(num < 0 ? -num : num);
    const unsigned long long qv = (2ull * an + (unsigned long long)den) / (2ull * (unsigned long long)den);
    const long long nv = num < 0 ? -(long long)qv : (long long)qv;
    const long long nw = gw + 1 > w_max ? (long long)w_max : gw + 1;
    return (uint32_t)(uint16_t)(int16_t)nv | ((uint32_t)nw << 16);
}

// Decode one accumulator and update its voxel; returns the voxel's number of
// contributions (WSUM) or 1 (MIN_ABS), 0 if untouched. WSUM accumulators
// whose sum fits 31 bits and count fits 15 bits (the common case) take an
// all-32-bit path with the same result as the 64-bit one.
// Eq. 1 / Eq. 2 in 32-bit integers, exact while |gv gw + S| < 2^31 - 2^17
// and gw + W < 2^16 (then 2 |num| + den < 2^32).
__device__ __forceinline__ uint32_t eq12_small(uint32_t word, int S, unsigned W, int32_t w_max) {
    const int gv = (int)(int16_t)(word & 0xFFFFu);
    const int gw = (int)(int16_t)(word >> 16);
    const int num = gv * gw + S;
    const unsigned den = (unsigned)gw + W;
    const unsigned an = (unsigned)(num < 0 ? -num : num);
    const unsigned q = (2u * an + den) / (2u * den);
    const int nv = num < 0 ? -(int)q : (int)q;
    const unsigned nw = den > (unsigned)w_max ? (unsigned)w_max : den;
    return (uint32_t)(uint16_t)(int16_t)nv | (nw << 16);
}

// WSUM cases outside the 32-bit range, and the per-scan weight reading, in
// 64-bit integers; rare, so kept out of line (fewer registers in the callers).
static __device__ __noinline__ uint32_t decode_apply_wide(unsigned long long P, uint32_t word, int32_t w_max,
                                                   int32_t flags) {
    const long long S = ((long long)(P << 24)) >> 24;   // sign-extended low 40 bits
    const long long W = (long long)((P - (unsigned long long)S) >> 40);
    return (flags & kFlagScanWeight) ? update_voxel_scan(word, S, W, w_max) : update_voxel(word, S, W, w_max);
}

template <int MODE>
__device__ __forceinline__ unsigned decode_apply(unsigned long long P, uint32_t& word, int32_t w_max,
                                                 int32_t flags = 0) {
    if (P == 0ull) return 0u;
    if (MODE == 0) {
        const unsigned lo = (unsigned)P, hi = (unsigned)(P >> 32);
        const unsigned hb = hi & 0xFFu;   // bits 32..39 of the 40-bit sum
        const bool small = ((hb == 0u) && (int)lo >= 0) || ((hb == 0xFFu) && (int)lo < 0);
        const int S32 = (int)lo;
        const unsigned W32 = (hi >> 8) + (S32 < 0 ? 1u : 0u);   // exact when `small`
        const int gw = (int)(int16_t)(word >> 16);
        if (!(flags & kFlagScanWeight) && small && W32 < 32768u && gw >= 0 && S32 > -(1 << 30) &&
            S32 < (1 << 30)) {
            word = eq12_small(word, S32, W32, w_max);   // |gv gw| < 2^30, |S| < 2^30
            return W32;
        }
        word = decode_apply_wide(P, word, w_max, flags);
        const long long S = ((long long)(P << 24)) >> 24;
        return (unsigned)((P - (unsigned long long)S) >> 40);
    } else {
        // |S| <= 32767 and W = 1: always inside the 32-bit range
        const unsigned key = 65536u - (unsigned)P;
        const int mag = (int)(key >> 1);
        word = eq12_small(word, (key & 1u) ? -mag : mag, 1u, w_max);
        return 1u;
    }
}

// ---- compact: lane i of the warp turns flag word i (4 bricks) into list
// entries and clears it; the warp takes one list atomic.
__device__ __forceinline__ void compact_words(const MapDev& m, unsigned i, unsigned nwords) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned f = 0;
    if (i < nwords) f = reinterpret_cast<const uint32_t*>(m.brick_flag)[i];
    // bytes are 0 or 1: one bit per touched brick in bits 0, 8, 16, 24
    const unsigned bits = (f & 1u) | ((f >> 7) & 2u) | ((f >> 14) & 4u) | ((f >> 21) & 8u);
    const unsigned cnt = __popc(bits);
    unsigned incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(kFull, incl, o);
        if (lane >= (unsigned)o) incl += v;
    }
    const unsigned total = __shfl_sync(kFull, incl, 31);
    if (total == 0u) return;   // warp-uniform
    unsigned base = 0;
    if (lane == 31) base = atomicAdd(&m.ctr->brick_count, total);
    base = __shfl_sync(kFull, base, 31) + incl - cnt;
    if (bits) {
        reinterpret_cast<uint32_t*>(m.brick_flag)[i] = 0u;
        for (unsigned b = 0; b < 4; ++b) {
            if (bits & (1u << b)) {
                if (m.brick_slot) m.brick_slot[4u * i + b] = base;
                m.brick_list[base++] = 4u * i + b;
            }
        }
    }
}

// Apply part shared by both reductions: the brick's grid words and per-scan
// accumulators are staged in shared memory; nz (bit 2v / 2v+1 of lane l) marks
// voxel 2(32 v + l) / +1 as touched. Compacts the touched voxels, applies
// Eq. 1 / Eq. 2 to each (one per lane) and writes the brick back.
template <int MODE>
__device__ __forceinline__ void apply_staged(const MapDev& m, int32_t w_max, int32_t flags, unsigned brick,
                                             unsigned nz, uint32_t* s_grid, const unsigned long long* s_acc,
                                             uint16_t* s_off, unsigned long long& touched,
                                             unsigned long long& hits) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned cnt = __popc(nz);
    unsigned incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(kFull, incl, o);
        if (lane >= (unsigned)o) incl += t;
    }
    const unsigned total = __shfl_sync(kFull, incl, 31);
    unsigned pos = incl - cnt;
    for (unsigned bits = nz; bits; bits &= bits - 1u) {
        const unsigned b = __ffs(bits) - 1u;
        s_off[pos++] = (uint16_t)(2u * (32u * (b >> 1) + lane) + (b & 1u));
    }
    __syncwarp();
    // Eq. 1 / Eq. 2 over the touched voxels only, one per lane
    for (unsigned e = lane; e < total; e += 32u) {
        const unsigned off = s_off[e];
        uint32_t word = s_grid[off];
        hits += decode_apply<MODE>(s_acc[off], word, w_max, flags);
        s_grid[off] = word;
    }
    touched += lane == 0 ? total : 0u;
    __syncwarp();
    uint4* gpw = reinterpret_cast<uint4*>(m.grid + ((size_t)brick << 9));
    const uint4* sg4 = reinterpret_cast<const uint4*>(s_grid);
#pragma unroll
    for (int v = 0; v < 4; ++v) gpw[32 * v + lane] = sg4[32 * v + lane];
}

// ---- apply, register form: one warp updates grid brick `brick` from the 512
// accumulators at `accp` (a brick of the dense accumulator or a pool slot).
// Lane l holds voxels 2(32 v + l) and +1 (v = 0..7) as eight 8-byte grid pairs
// and eight 16-byte accumulator pairs, all loaded at once; every touched voxel
// is decoded in place (16 independent updates per lane), and only changed
// pairs are written back and reset.
// NV voxel pairs per lane, starting at pair row v0: NV = 8 is the whole
// brick, NV = 4 (v0 = 0 or 4) one half, NV = 2 a quarter.
template <int MODE, int NV = 8>
__device__ __forceinline__ void apply_brick_at(const MapDev& m, int32_t w_max, int32_t flags, unsigned brick,
                                               unsigned long long* accp, unsigned long long& touched,
                                               unsigned long long& hits, unsigned v0 = 0) {
    static_assert(NV == 8 || NV == 4 || NV == 2, "whole, half or quarter bricks");
    const unsigned lane = threadIdx.x & 31u;
    uint2* gp = reinterpret_cast<uint2*>(m.grid + ((size_t)brick << 9)) + 32 * v0;
    ulonglong2* ap = reinterpret_cast<ulonglong2*>(accp) + 32 * v0;
    ulonglong2 acc[NV];
    uint2 g[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = ap[32 * v + lane];
#pragma unroll
    for (int v = 0; v < NV; ++v) g[v] = gp[32 * v + lane];
    unsigned cnt = 0;
    unsigned long long h = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (acc[v].x != 0ull) {
            h += decode_apply<MODE>(acc[v].x, g[v].x, w_max, flags);
            ++cnt;
        }
        if (acc[v].y != 0ull) {
            h += decode_apply<MODE>(acc[v].y, g[v].y, w_max, flags);
            ++cnt;
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if ((acc[v].x | acc[v].y) != 0ull) {
            gp[32 * v + lane] = g[v];
            ap[32 * v + lane] = make_ulonglong2(0ull, 0ull);
        }
    }
    touched += cnt;
    hits += h;
}

template <int MODE>
__device__ __forceinline__ void apply_brick_reg(const MapDev& m, int32_t w_max, int32_t flags, unsigned i,
                                                unsigned long long& touched, unsigned long long& hits) {
    const unsigned brick = m.brick_list[i];
    apply_brick_at<MODE>(m, w_max, flags, brick, m.acc + ((size_t)brick << 9), touched, hits);
}

// Part t % P of listed brick t / P (P = 8 / NV parts per brick).
template <int MODE, int NV>
__device__ __forceinline__ void apply_part_reg(const MapDev& m, int32_t w_max, int32_t flags, unsigned t,
                                               unsigned long long& touched, unsigned long long& hits) {
    constexpr unsigned P = 8 / NV;
    const unsigned brick = m.brick_list[t / P];
    apply_brick_at<MODE, NV>(m, w_max, flags, brick, m.acc + ((size_t)brick << 9), touched, hits, (t % P) * NV);
}

// ---- apply: one warp updates listed brick number i of the map. Shared
// memory per warp: s_grid[512] words, s_acc[512] accumulators, s_off[512].
template <int MODE>
__device__ __forceinline__ void apply_brick(const MapDev& m, int32_t w_max, int32_t flags, unsigned i,
                                            uint32_t* s_grid, unsigned long long* s_acc, uint16_t* s_off,
                                            unsigned long long& touched, unsigned long long& hits) {
    const unsigned lane = threadIdx.x & 31u;
    uint4* sg4 = reinterpret_cast<uint4*>(s_grid);
    ulonglong2* sa2 = reinterpret_cast<ulonglong2*>(s_acc);
    const unsigned brick = m.brick_list[i];
    // coalesced, bank-conflict-free 16-byte copies of the brick into shared
    // memory: accumulator pair p = 32 v + lane holds voxels 2p and 2p + 1
    const uint4* gp = reinterpret_cast<const uint4*>(m.grid + ((size_t)brick << 9));
    ulonglong2* ap = reinterpret_cast<ulonglong2*>(m.acc + ((size_t)brick << 9));
    unsigned nz = 0;   // bit 2v (2v+1): voxel 2(32 v + lane) (+1) has a non-zero accumulator
#pragma unroll
    for (int v = 0; v < 4; ++v) sg4[32 * v + lane] = gp[32 * v + lane];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const ulonglong2 a2 = ap[32 * v + lane];
        sa2[32 * v + lane] = a2;
        nz |= (a2.x != 0ull ? 1u : 0u) << (2 * v);
        nz |= (a2.y != 0ull ? 1u : 0u) << (2 * v + 1);
    }
    apply_staged<MODE>(m, w_max, flags, brick, nz, s_grid, s_acc, s_off, touched, hits);
    if (nz) {
#pragma unroll
        for (int v = 0; v < 8; ++v)
            if (nz & (3u << (2 * v))) ap[32 * v + lane] = make_ulonglong2(0ull, 0ull);
    }
    __syncwarp();
}

// ---- sort reduction (counting sort of the emitted pairs by touched brick,
// then a per-brick segmented reduction in shared memory)

// Pair slots of the scan in flight that were written: min(reserved, capacity).
// A coherent load (see the per-map kernels), lane 0 then broadcast.
__device__ __forceinline__ uint32_t sort_nslots(const MapDev& m) {
    unsigned long long n = 0;
    if ((threadIdx.x & 31u) == 0) n = __ldcg(&m.ctr->slot_count);
    n = __shfl_sync(kFull, n, 0);
    return (uint32_t)(n < m.pair_cap ? n : (unsigned long long)m.pair_cap);
}

// One warp: pairs [s, s + 128) add to their bricks' counts; each lane loads
// four pairs and their brick slots before any warp operation, so the loads
// overlap. Lanes holding the same brick (usually neighbouring samples of one
// ray) are merged first.
__device__ __forceinline__ void sort_count_warp(const MapDev& m, uint32_t s, uint32_t nslots) {
    const unsigned lane = threadIdx.x & 31u;
    uint32_t word[4], seg[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint32_t slot = s + 32u * u + lane;
        word[u] = slot < nslots ? m.pairs[slot].x : kNoVoxel;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) seg[u] = word[u] != kNoVoxel ? m.brick_slot[word[u] >> 9] : kNoVoxel;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (__ballot_sync(kFull, seg[u] != kNoVoxel) == 0u) continue;   // warp-uniform
        const unsigned peers = __match_any_sync(kFull, seg[u]);
        if (seg[u] != kNoVoxel && lane == (unsigned)(__ffs(peers) - 1))
            atomicAdd(m.seg_count + seg[u], (uint32_t)__popc(peers));
    }
}

// The CTA turns the per-brick counts of the map's nb listed bricks into
// segment starts (exclusive prefix) and scatter cursors (seg_count := start).
// blockDim.x must be a multiple of 32, at most 1024. smem: 33 words.
__device__ __forceinline__ void sort_scan_cta(const MapDev& m, uint32_t nb, uint32_t* smem) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const unsigned nw = blockDim.x >> 5;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < nb ? m.seg_count[i] : 0u;
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= (unsigned)o) incl += y;
        }
        if (lane == 31) smem[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = lane < nw ? smem[lane] : 0u, ti = t;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, ti, o);
                if (lane >= (unsigned)o) ti += y;
            }
            if (lane < nw) smem[lane] = ti - t;        // exclusive prefix of the warp totals
            if (lane == 31) smem[32] = ti;             // block total
        }
        __syncthreads();
        if (i < nb) {
            const uint32_t start = carry + smem[warp] + incl - x;
            m.seg_start[i] = start;
            m.seg_count[i] = start;
        }
        carry += smem[32];
        __syncthreads();
    }
}

// One warp: pairs [s, s + 128) go to their bricks' segments as
// (offset in brick << 16) | (code & 0xFFFF); loads first (four per lane),
// then one returning atomic per distinct brick of each 32-pair group, the
// four groups' atomics in flight together.
__device__ __forceinline__ void sort_scatter_warp(const MapDev& m, uint32_t s, uint32_t nslots) {
    const unsigned lane = threadIdx.x & 31u;
    uint2 p[4];
    uint32_t seg[4], pos[4];
    unsigned peers[4], leader[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint32_t slot = s + 32u * u + lane;
        p[u] = slot < nslots ? m.pairs[slot] : make_uint2(kNoVoxel, 0u);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) seg[u] = p[u].x != kNoVoxel ? m.brick_slot[p[u].x >> 9] : kNoVoxel;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        peers[u] = __match_any_sync(kFull, seg[u]);
        leader[u] = (unsigned)(__ffs(peers[u]) - 1);
        pos[u] = 0u;
        if (seg[u] != kNoVoxel && lane == leader[u]) pos[u] = atomicAdd(m.seg_count + seg[u], (uint32_t)__popc(peers[u]));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint32_t b = __shfl_sync(kFull, pos[u], leader[u]);
        if (seg[u] != kNoVoxel)
            m.sorted[b + __popc(peers[u] & ((1u << lane) - 1u))] = ((p[u].x & 511u) << 16) | (p[u].y & 0xFFFFu);
    }
}

// One warp: listed brick i. Its segment of `sorted` is reduced per voxel in
// shared memory (the same packed accumulators as the atomic reduction), the
// accumulators of overflowed samples are merged when `ovf`, and Eq. 1 / Eq. 2
// are applied as in apply_brick. Resets the brick's count for the next scan.
template <int MODE>
__device__ __forceinline__ void sort_apply_brick(const MapDev& m, int32_t w_max, int32_t flags, unsigned i, bool ovf,
                                                 uint32_t* s_grid, unsigned long long* s_acc, uint16_t* s_off,
                                                 unsigned long long& touched, unsigned long long& hits) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned brick = m.brick_list[i];
    const uint32_t start = m.seg_start[i], end = m.seg_count[i];
    uint4* sg4 = reinterpret_cast<uint4*>(s_grid);
    ulonglong2* sa2 = reinterpret_cast<ulonglong2*>(s_acc);
    const uint4* gp = reinterpret_cast<const uint4*>(m.grid + ((size_t)brick << 9));
    ulonglong2* ap = reinterpret_cast<ulonglong2*>(m.acc + ((size_t)brick << 9));
    unsigned onz = 0;   // global accumulators that held overflowed samples
#pragma unroll
    for (int v = 0; v < 4; ++v) sg4[32 * v + lane] = gp[32 * v + lane];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        ulonglong2 a2 = make_ulonglong2(0ull, 0ull);
        if (ovf) {
            a2 = ap[32 * v + lane];
            onz |= (a2.x != 0ull || a2.y != 0ull ? 1u : 0u) << v;
        }
        sa2[32 * v + lane] = a2;
    }
    __syncwarp();
    // four entries per lane in flight per round
    for (uint32_t e0 = start; e0 < end; e0 += 128u) {
        uint32_t val[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t e = e0 + 32u * u + lane;
            val[u] = e < end ? m.sorted[e] : kNoVoxel;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (val[u] == kNoVoxel) continue;
            const unsigned off = val[u] >> 16;
            const int q = (int)(int16_t)(val[u] & 0xFFFFu);
            if (MODE == 0) atomicAdd(s_acc + off, (1ull << 40) + (unsigned long long)(long long)q);
            else atomicMax(s_acc + off, 65536ull - (((unsigned)abs(q) << 1) | (q < 0 ? 1u : 0u)));
        }
    }
    if (MODE == 1 && lane == 0) hits += end - start;
    if (lane == 0) m.seg_count[i] = 0u;
    __syncwarp();
    unsigned nz = 0;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const ulonglong2 a2 = sa2[32 * v + lane];
        nz |= (a2.x != 0ull ? 1u : 0u) << (2 * v);
        nz |= (a2.y != 0ull ? 1u : 0u) << (2 * v + 1);
    }
    if (MODE == 0) {
        apply_staged<MODE>(m, w_max, flags, brick, nz, s_grid, s_acc, s_off, touched, hits);
    } else {
        unsigned long long voxels = 0;   // MIN_ABS decode counts voxels, not contributions
        apply_staged<MODE>(m, w_max, flags, brick, nz, s_grid, s_acc, s_off, touched, voxels);
    }
    if (onz) {
#pragma unroll
        for (int v = 0; v < 8; ++v)
            if (onz & (1u << v)) ap[32 * v + lane] = make_ulonglong2(0ull, 0ull);
    }
    __syncwarp();
}

// ---- finish: one warp (lane = counter slot) publishes the scan's counters
// and clears the per-scan state.
__device__ __forceinline__ void finish_warp(const MapDev& m) {
    MapCounters* c = m.ctr;
    const unsigned lane = threadIdx.x & 31u;
    // coherent loads: the partial counters were added by other CTAs' atomics
    unsigned long long v = __ldcg(&c->part[lane].valid), h = __ldcg(&c->part[lane].hits),
                       u = __ldcg(&c->part[lane].touched);
    c->part[lane].valid = 0ull;
    c->part[lane].hits = 0ull;
    c->part[lane].touched = 0ull;
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(kFull, v, o);
        h += __shfl_xor_sync(kFull, h, o);
        u += __shfl_xor_sync(kFull, u, o);
    }
    if (lane == 0) {
        // a pool-reduction scan that found the pool full was dropped
        const long long st = __ldcg(&c->pool_overflow) != 0u ? kStatusCapacity : 0;
        if (st != 0) h = u = 0ull;
        c->last_valid = (long long)v;
        c->last_hits = (long long)h;
        c->last_touched = (long long)u;
        c->last_status = st;
        if (m.host_last) {   // also into host memory: reading them needs no copy
            m.host_last[0] = (long long)v;
            m.host_last[1] = (long long)h;
            m.host_last[2] = (long long)u;
            m.host_last[3] = st;
        }
        c->live_count = 0u;
        c->brick_count = 0u;
        c->slot_count = 0ull;
        c->overflow = 0u;
        c->apply_done = 0u;
        c->pool_count = 0u;
        c->pool_overflow = 0u;
        c->live_back = 0u;
    }
}

// The calling CTA (all threads) counts itself done; the last CTA of the grid
// then publishes the scan's counters with its first warp (finish_warp). The
// caller must have added its partial counters before the call.
__device__ __forceinline__ void finish_if_last(const MapDev& m, unsigned* s_last) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *s_last = atomicAdd(&m.ctr->apply_done, 1u) == gridDim.x - 1u ? 1u : 0u;
    }
    __syncthreads();
    if (*s_last && threadIdx.x < 32) {
        __threadfence();
        finish_warp(m);
    }
}

}  // namespace dev
}  // namespace tsdf
