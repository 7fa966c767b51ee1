// TEST INFRASTRUCTURE -- CPU oracle for the per-scan TSDF integration path.
//
// A plain, slow, single-threaded restatement of FeatSense's TSDF map
// generation (Section "TSDF Map Generation": the ray traversal from the scan
// pose to each scan point, the per-scan volume V, Eq. 1 and Eq. 2, the
// vertical interpolation vector and Eq. 3 / Eq. 4) plus the local-map shift
// of the Introduction (a window that is shifted after a movement threshold,
// with map parts written out to and loaded back from a global store).
//
// Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may load
// this library. It shares no code, header or constant with the CUDA library.
//
// Conventions (each one a reading of the paper, stated once):
//  * Floating point: IEEE binary32, round to nearest even, evaluated in the
//    exact operation order written below; compiled with -ffp-contract=off so
//    no multiply-add is fused. Constants that need a division are derived in
//    binary64 and rounded once to binary32.
//  * The map window is a dense array indexed by (g - origin): no ring
//    addressing here; a shift physically rebuilds the window.
//  * Per-scan volume V: WSUM keeps sum(q) and the hit count per voxel (each
//    hit has weight 1); MIN_ABS keeps the quantised distance of smallest
//    magnitude (tie -> the positive one), the paper's "smallest distance of
//    all rays" with weight 1.
//  * Eq. 1 is evaluated exactly in integers with one rounding, half away
//    from zero. Eq. 2 clamps the summed weight at weight_max.
//  * Two alternative readings selected by flags: bit 1, every sample of a
//    march step takes that step's own distance r - l (the fill copies the
//    step's value); bit 2, a WSUM scan's averaged
//    value enters Eq. 1 / Eq. 2 as one observation of weight 1.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <array>
#include <unordered_map>
#include <vector>

extern "C" {

// Map parameters, same field order as the library's public struct but an
// independent definition.
struct orc_params {
    int32_t dims[3];
    float voxel_size;
    float tau;
    int32_t w_max;
    float delta_z;
    float r_min;
    float r_max;
    int32_t reduce;   // 0 = WSUM, 1 = MIN_ABS
    int32_t flags;    // 1: step-valued fill, 2: one observation per scan (WSUM)
    int64_t origin[3];
};

}  // extern "C"

namespace {

const int32_t QMAX = 32767;

struct Derived {
    float inv_vs;   // 1 / voxel_size
    float qs;       // QMAX / tau
    int K;          // number of march steps on each side of the hit
};

Derived derive(const orc_params& p) {
    Derived d;
    d.inv_vs = (float)(1.0 / (double)p.voxel_size);
    d.qs = (float)((double)QMAX / (double)p.tau);
    d.K = (int)std::floor((double)p.tau / (double)p.voxel_size + 1e-9);
    return d;
}

struct Cell {
    int16_t v;
    int16_t w;
};

struct Ray {
    bool valid;
    bool fill;      // vertical interpolation active for this ray
    float r;        // range from the sensor to the scan point
    float t[3];     // sensor position (pose translation)
    float dir[3];   // unit ray direction
    float ih[3];    // unit interpolation direction
};

// Transform a sensor-frame point by the pose and set up its ray.
// Section "TSDF Map Generation": ray from the scan position to the scan
// point; interpolation vector int = d x (d x up), up = the sensor's z axis,
// the direction orthogonal to the scan lines.
Ray ray_setup(const float pose[12], const float pt[4], float r_min, float r_max, float delta_z) {
    Ray ry;
    const float R00 = pose[0], R01 = pose[1], R02 = pose[2], tx = pose[3];
    const float R10 = pose[4], R11 = pose[5], R12 = pose[6], ty = pose[7];
    const float R20 = pose[8], R21 = pose[9], R22 = pose[10], tz = pose[11];
    const float x = pt[0], y = pt[1], z = pt[2];
    float pwx = ((R00 * x + R01 * y) + R02 * z) + tx;
    float pwy = ((R10 * x + R11 * y) + R12 * z) + ty;
    float pwz = ((R20 * x + R21 * y) + R22 * z) + tz;
    float vx = pwx - tx, vy = pwy - ty, vz = pwz - tz;
    float r2 = (vx * vx + vy * vy) + vz * vz;
    float r = std::sqrt(r2);
    ry.r = r;
    ry.t[0] = tx; ry.t[1] = ty; ry.t[2] = tz;
    ry.valid = (r >= r_min) && (r <= r_max);   // false for NaN and inf
    ry.fill = false;
    ry.dir[0] = ry.dir[1] = ry.dir[2] = 0.f;
    ry.ih[0] = ry.ih[1] = ry.ih[2] = 0.f;
    if (!ry.valid) return ry;
    float dx = vx / r, dy = vy / r, dz = vz / r;
    ry.dir[0] = dx; ry.dir[1] = dy; ry.dir[2] = dz;
    const float ux = R02, uy = R12, uz = R22;
    // a = d x up
    float ax = dy * uz - dz * uy;
    float ay = dz * ux - dx * uz;
    float az = dx * uy - dy * ux;
    // iv = d x a = d x (d x up)
    float ivx = dy * az - dz * ay;
    float ivy = dz * ax - dx * az;
    float ivz = dx * ay - dy * ax;
    float n2 = (ivx * ivx + ivy * ivy) + ivz * ivz;
    if (delta_z > 0.f && n2 >= 1e-12f) {
        float n = std::sqrt(n2);
        ry.fill = true;
        ry.ih[0] = ivx / n; ry.ih[1] = ivy / n; ry.ih[2] = ivz / n;
    }
    return ry;
}

// Quantise a truncated signed distance to the int16 fixed-point code:
// clamp to [-tau, tau], scale by QMAX / tau, round to nearest even, clamp.
int32_t quantize(float d, float tau, float qs) {
    if (d < -tau) d = -tau;
    if (d > tau) d = tau;
    float s = d * qs;
    long q = std::lrint(s);
    if (q > QMAX) q = QMAX;
    if (q < -QMAX) q = -QMAX;
    return (int32_t)q;
}

// Eq. 1 and Eq. 2 with v.value = S / W and v.weight = 1 (one observation per
// scan): value (gv*gw + S/W) / (gw + 1) = (gv*gw*W + S) / ((gw + 1) * W).
void eq12_scan(int32_t gv, int32_t gw, int64_t S, int64_t W, int32_t w_max, int32_t* nv, int32_t* nw) {
    int64_t num = (int64_t)gv * (int64_t)gw * W + S;
    int64_t den = ((int64_t)gw + 1) * W;
    int64_t a = num < 0 ? -num : num;
    int64_t q = (2 * a + den) / (2 * den);
    *nv = (int32_t)(num < 0 ? -q : q);
    int64_t w = (int64_t)gw + 1;
    *nw = (int32_t)(w > w_max ? w_max : w);
}

// Eq. 1 and Eq. 2 with v.value * v.weight = S and v.weight = W.
void eq12(int32_t gv, int32_t gw, int64_t S, int64_t W, int32_t w_max, int32_t* nv, int32_t* nw) {
    int64_t num = (int64_t)gv * (int64_t)gw + S;
    int64_t den = (int64_t)gw + W;
    int64_t a = num < 0 ? -num : num;
    int64_t q = (2 * a + den) / (2 * den);   // floor(|num|/den + 1/2)
    *nv = (int32_t)(num < 0 ? -q : q);
    int64_t w = (int64_t)gw + W;
    *nw = (int32_t)(w > w_max ? w_max : w);
}

// Visit every (voxel, quantised distance) contribution of one ray, in march
// order (k outer, j inner). Eq. 3 gives delta_z; Eq. 4 the fill height
// h = delta_z * l at step distance l; voxels are taken at spacing voxel_size
// along +-int up to h. The distance of a voxel is the projective distance of
// its centre along the ray: r - (c - s) . dir (or, with flag 1, the step's
// own distance r - l).
template <class F>
void for_each_hit(const Ray& ry, const orc_params& p, const Derived& dv, F&& f) {
    if (!ry.valid) return;
    const float vs = p.voxel_size;
    const float tx = ry.t[0], ty = ry.t[1], tz = ry.t[2];
    const float dx = ry.dir[0], dy = ry.dir[1], dz = ry.dir[2];
    for (int k = -dv.K; k <= dv.K; ++k) {
        float l = ry.r + (float)k * vs;
        if (!(l > 0.f)) continue;
        int J = 0;
        if (ry.fill) J = (int)std::floor((p.delta_z * l) * dv.inv_vs);
        float bx = tx + dx * l;
        float by = ty + dy * l;
        float bz = tz + dz * l;
        for (int j = -J; j <= J; ++j) {
            float jd = (float)j * vs;
            float qx = bx + ry.ih[0] * jd;
            float qy = by + ry.ih[1] * jd;
            float qz = bz + ry.ih[2] * jd;
            float fx = std::floor(qx * dv.inv_vs);
            float fy = std::floor(qy * dv.inv_vs);
            float fz = std::floor(qz * dv.inv_vs);
            const float LIM = 4.0e18f;   // far outside any window: skip
            if (!(std::fabs(fx) < LIM && std::fabs(fy) < LIM && std::fabs(fz) < LIM)) continue;
            int64_t g[3] = {(int64_t)fx, (int64_t)fy, (int64_t)fz};
            float cx = ((float)g[0] + 0.5f) * vs;
            float cy = ((float)g[1] + 0.5f) * vs;
            float cz = ((float)g[2] + 0.5f) * vs;
            float proj = (((cx - tx) * dx) + ((cy - ty) * dy)) + ((cz - tz) * dz);
            float d = (p.flags & 1) ? ry.r - l : ry.r - proj;
            f(g, quantize(d, p.tau, dv.qs), k);
        }
    }
}

struct Acc {
    int64_t S = 0;
    int64_t W = 0;
};

struct OracleMap {
    orc_params p;
    Derived dv;
    int64_t origin[3];
    std::vector<Cell> win;
    std::map<std::array<int64_t, 3>, std::vector<Cell>> store;   // global chunk -> 8^3 cells
    int64_t st_valid = 0, st_hits = 0, st_touched = 0;

    int64_t X() const { return p.dims[0]; }
    int64_t Y() const { return p.dims[1]; }
    int64_t Z() const { return p.dims[2]; }
    bool inside(const int64_t g[3]) const {
        for (int a = 0; a < 3; ++a)
            if (g[a] < origin[a] || g[a] >= origin[a] + p.dims[a]) return false;
        return true;
    }
    int64_t lin(const int64_t g[3]) const {
        return ((g[2] - origin[2]) * Y() + (g[1] - origin[1])) * X() + (g[0] - origin[0]);
    }
};

bool params_ok(const orc_params& p) {
    for (int a = 0; a < 3; ++a) {
        if (p.dims[a] < 8 || p.dims[a] % 8 != 0) return false;
        if (p.origin[a] % 8 != 0) return false;
    }
    if (!(p.voxel_size > 0.f) || !(p.tau >= p.voxel_size)) return false;
    if (p.w_max < 1 || p.w_max > 32767) return false;
    if (!(p.delta_z >= 0.f)) return false;
    if (!(p.r_min >= 0.f) || !(p.r_max >= p.r_min)) return false;
    if (p.reduce != 0 && p.reduce != 1) return false;
    if ((p.flags & ~3) != 0) return false;
    return true;
}

// Apply a per-scan volume to the window: Eq. 1 / Eq. 2 for every touched
// voxel. Returns the number of voxels updated.
int64_t apply_volume(OracleMap* m, const std::unordered_map<int64_t, Acc>& vol,
                     const std::unordered_map<int64_t, int32_t>& best) {
    if (m->p.reduce == 0) {
        for (const auto& kv : vol) {
            Cell& c = m->win[kv.first];
            int32_t nv, nw;
            if (m->p.flags & 2) eq12_scan(c.v, c.w, kv.second.S, kv.second.W, m->p.w_max, &nv, &nw);
            else eq12(c.v, c.w, kv.second.S, kv.second.W, m->p.w_max, &nv, &nw);
            c.v = (int16_t)nv;
            c.w = (int16_t)nw;
        }
        return (int64_t)vol.size();
    } else {
        for (const auto& kv : best) {
            Cell& c = m->win[kv.first];
            int32_t nv, nw;
            eq12(c.v, c.w, kv.second, 1, m->p.w_max, &nv, &nw);
            c.v = (int16_t)nv;
            c.w = (int16_t)nw;
        }
        return (int64_t)best.size();
    }
}

// MIN_ABS order: smaller magnitude wins; equal magnitude -> the positive value.
bool min_abs_better(int32_t a, int32_t b) {
    int32_t aa = a < 0 ? -a : a, bb = b < 0 ? -b : b;
    if (aa != bb) return aa < bb;
    return a > b;
}

}  // namespace

extern "C" {

void* orc_create(const orc_params* p) {
    if (!p || !params_ok(*p)) return nullptr;
    OracleMap* m = new OracleMap();
    m->p = *p;
    m->dv = derive(*p);
    for (int a = 0; a < 3; ++a) m->origin[a] = p->origin[a];
    m->win.assign((size_t)p->dims[0] * p->dims[1] * p->dims[2], Cell{0, 0});
    return m;
}

void orc_destroy(void* h) { delete (OracleMap*)h; }

void orc_derived(const orc_params* p, float* inv_vs, float* qs, int32_t* K) {
    Derived d = derive(*p);
    *inv_vs = d.inv_vs;
    *qs = d.qs;
    *K = d.K;
}

// Ray-major integration of one scan (points: float[n][4], sensor frame).
int orc_integrate(void* h, const float* pts, int64_t n, const float pose[12]) {
    OracleMap* m = (OracleMap*)h;
    if (!m || n < 0 || (n > 0 && !pts) || !pose) return -1;
    std::unordered_map<int64_t, Acc> vol;
    std::unordered_map<int64_t, int32_t> best;
    int64_t valid = 0, hits = 0;
    for (int64_t i = 0; i < n; ++i) {
        Ray ry = ray_setup(pose, pts + 4 * i, m->p.r_min, m->p.r_max, m->p.delta_z);
        if (!ry.valid) continue;
        ++valid;
        for_each_hit(ry, m->p, m->dv, [&](const int64_t g[3], int32_t q, int) {
            if (!m->inside(g)) return;
            ++hits;
            int64_t key = m->lin(g);
            if (m->p.reduce == 0) {
                Acc& a = vol[key];
                a.S += q;
                a.W += 1;
            } else {
                auto it = best.find(key);
                if (it == best.end()) best.emplace(key, q);
                else if (min_abs_better(q, it->second)) it->second = q;
            }
        });
    }
    m->st_touched = apply_volume(m, vol, best);
    m->st_valid = valid;
    m->st_hits = hits;
    return 0;
}

// The same scan on `threads` host threads, partitioned by voxel: every
// thread enumerates all rays (the cheap part) but keeps only the
// contributions to the voxels it owns (a hash of the window index), then
// applies Eq. 1 / Eq. 2 to those voxels. Owners are disjoint, so nothing is
// merged and the result is identical to orc_integrate. Used to time the
// oracle on all host cores (the paper's CPU baseline is multithreaded).
int orc_integrate_parallel(void* h, const float* pts, int64_t n, const float pose[12], int32_t threads) {
    OracleMap* m = (OracleMap*)h;
    if (!m || n < 0 || (n > 0 && !pts) || !pose || threads < 1) return -1;
    std::vector<int64_t> valid((size_t)threads, 0), hits((size_t)threads, 0), touched((size_t)threads, 0);
    auto owner = [threads](int64_t key) {
        return (int)(((uint64_t)key * 0x9E3779B97F4A7C15ull) >> 40) % threads;
    };
    auto work = [&](int t) {
        std::unordered_map<int64_t, Acc> vol;
        std::unordered_map<int64_t, int32_t> best;
        for (int64_t i = 0; i < n; ++i) {
            Ray ry = ray_setup(pose, pts + 4 * i, m->p.r_min, m->p.r_max, m->p.delta_z);
            if (!ry.valid) continue;
            if (t == 0) ++valid[0];
            for_each_hit(ry, m->p, m->dv, [&](const int64_t g[3], int32_t q, int) {
                if (!m->inside(g)) return;
                const int64_t key = m->lin(g);
                if (owner(key) != t) return;
                ++hits[(size_t)t];
                if (m->p.reduce == 0) {
                    Acc& a = vol[key];
                    a.S += q;
                    a.W += 1;
                } else {
                    auto it = best.find(key);
                    if (it == best.end()) best.emplace(key, q);
                    else if (min_abs_better(q, it->second)) it->second = q;
                }
            });
        }
        touched[(size_t)t] = apply_volume(m, vol, best);   // disjoint cells per thread
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
    int64_t h_all = 0, u_all = 0;
    for (int t = 0; t < threads; ++t) {
        h_all += hits[(size_t)t];
        u_all += touched[(size_t)t];
    }
    m->st_valid = valid[0];
    m->st_hits = h_all;
    m->st_touched = u_all;
    return 0;
}

// Voxel-major brute force of the same scan: for every window voxel, scan all
// rays and all (k, j) steps and collect the contributions that land on it.
// Loop order differs from orc_integrate on purpose. Tiny inputs only.
int orc_integrate_bruteforce(void* h, const float* pts, int64_t n, const float pose[12]) {
    OracleMap* m = (OracleMap*)h;
    if (!m || n < 0 || (n > 0 && !pts) || !pose) return -1;
    std::vector<Ray> rays;
    int64_t valid = 0;
    for (int64_t i = 0; i < n; ++i) {
        Ray ry = ray_setup(pose, pts + 4 * i, m->p.r_min, m->p.r_max, m->p.delta_z);
        if (ry.valid) ++valid;
        rays.push_back(ry);
    }
    const float vs = m->p.voxel_size;
    std::vector<Cell> next = m->win;
    int64_t hits = 0, touched = 0;
    for (int64_t gz = m->origin[2]; gz < m->origin[2] + m->Z(); ++gz)
    for (int64_t gy = m->origin[1]; gy < m->origin[1] + m->Y(); ++gy)
    for (int64_t gx = m->origin[0]; gx < m->origin[0] + m->X(); ++gx) {
        int64_t S = 0, W = 0;
        bool any = false;
        int32_t bq = 0;
        for (const Ray& ry : rays) {
            if (!ry.valid) continue;
            for (int k = -m->dv.K; k <= m->dv.K; ++k) {
                float l = ry.r + (float)k * vs;
                if (!(l > 0.f)) continue;
                int J = ry.fill ? (int)std::floor((m->p.delta_z * l) * m->dv.inv_vs) : 0;
                for (int j = -J; j <= J; ++j) {
                    float jd = (float)j * vs;
                    float qx = (ry.t[0] + ry.dir[0] * l) + ry.ih[0] * jd;
                    float qy = (ry.t[1] + ry.dir[1] * l) + ry.ih[1] * jd;
                    float qz = (ry.t[2] + ry.dir[2] * l) + ry.ih[2] * jd;
                    if ((int64_t)std::floor(qx * m->dv.inv_vs) != gx) continue;
                    if ((int64_t)std::floor(qy * m->dv.inv_vs) != gy) continue;
                    if ((int64_t)std::floor(qz * m->dv.inv_vs) != gz) continue;
                    float cx = ((float)gx + 0.5f) * vs;
                    float cy = ((float)gy + 0.5f) * vs;
                    float cz = ((float)gz + 0.5f) * vs;
                    float d = (m->p.flags & 1) ? ry.r - l
                                               : ry.r - ((((cx - ry.t[0]) * ry.dir[0]) + ((cy - ry.t[1]) * ry.dir[1])) +
                                                         ((cz - ry.t[2]) * ry.dir[2]));
                    int32_t q = quantize(d, m->p.tau, m->dv.qs);
                    S += q;
                    W += 1;
                    if (!any || min_abs_better(q, bq)) bq = q;
                    any = true;
                }
            }
        }
        if (!any) continue;
        ++touched;
        hits += W;
        int64_t g[3] = {gx, gy, gz};
        Cell& c = next[m->lin(g)];
        int32_t nv, nw;
        if (m->p.reduce == 0 && (m->p.flags & 2)) eq12_scan(c.v, c.w, S, W, m->p.w_max, &nv, &nw);
        else if (m->p.reduce == 0) eq12(c.v, c.w, S, W, m->p.w_max, &nv, &nw);
        else eq12(c.v, c.w, bq, 1, m->p.w_max, &nv, &nw);
        c.v = (int16_t)nv;
        c.w = (int16_t)nw;
    }
    m->win.swap(next);
    m->st_valid = valid;
    m->st_hits = hits;
    m->st_touched = touched;
    return 0;
}

// Every contribution of a scan, in enumeration order, whether or not it lands
// in the window: out_g int64[cap][3], out_q int32[cap]. Returns the count
// (which may exceed cap; only the first cap are written).
int64_t orc_hits(const orc_params* p, const float* pts, int64_t n, const float pose[12],
                 int64_t* out_g, int32_t* out_q, int64_t* out_ray, int32_t* out_k, int64_t cap) {
    Derived dv = derive(*p);
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        Ray ry = ray_setup(pose, pts + 4 * i, p->r_min, p->r_max, p->delta_z);
        for_each_hit(ry, *p, dv, [&](const int64_t g[3], int32_t q, int k) {
            if (cnt < cap) {
                out_g[3 * cnt + 0] = g[0];
                out_g[3 * cnt + 1] = g[1];
                out_g[3 * cnt + 2] = g[2];
                out_q[cnt] = q;
                if (out_ray) out_ray[cnt] = i;
                if (out_k) out_k[cnt] = k;
            }
            ++cnt;
        });
    }
    return cnt;
}

// Ray set-up of one point, for pin tests: out[0]=valid, [1]=fill, [2]=r,
// [3..5]=dir, [6..8]=ih.
void orc_ray(const float pose[12], const float pt[4], float r_min, float r_max, float delta_z, float out[9]) {
    Ray ry = ray_setup(pose, pt, r_min, r_max, delta_z);
    out[0] = ry.valid ? 1.f : 0.f;
    out[1] = ry.fill ? 1.f : 0.f;
    out[2] = ry.r;
    for (int a = 0; a < 3; ++a) {
        out[3 + a] = ry.dir[a];
        out[6 + a] = ry.ih[a];
    }
}

int32_t orc_quantize(float d, float tau, float qs) { return quantize(d, tau, qs); }

void orc_eq12(int32_t gv, int32_t gw, int64_t S, int64_t W, int32_t w_max, int32_t* nv, int32_t* nw) {
    eq12(gv, gw, S, W, w_max, nv, nw);
}

void orc_eq12_scan(int32_t gv, int32_t gw, int64_t S, int64_t W, int32_t w_max, int32_t* nv, int32_t* nw) {
    eq12_scan(gv, gw, S, W, w_max, nv, nw);
}

// Move the window to new_origin (multiples of 8). Chunks (8^3 voxels) that
// leave are kept in the global store when any of their cells is non-zero;
// cells that enter are loaded from the store, else (0, 0).
int orc_shift(void* h, const int64_t no[3]) {
    OracleMap* m = (OracleMap*)h;
    if (!m || !no) return -1;
    for (int a = 0; a < 3; ++a)
        if (no[a] % 8 != 0) return -1;
    const int64_t X = m->X(), Y = m->Y(), Z = m->Z();
    // 1. evict chunks of the old window that are not inside the new one
    for (int64_t cz = m->origin[2]; cz < m->origin[2] + Z; cz += 8)
    for (int64_t cy = m->origin[1]; cy < m->origin[1] + Y; cy += 8)
    for (int64_t cx = m->origin[0]; cx < m->origin[0] + X; cx += 8) {
        bool stays = cx >= no[0] && cx < no[0] + X && cy >= no[1] && cy < no[1] + Y &&
                     cz >= no[2] && cz < no[2] + Z;
        if (stays) continue;
        std::vector<Cell> cells(512);
        bool nonzero = false;
        for (int z = 0; z < 8; ++z)
        for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x) {
            int64_t g[3] = {cx + x, cy + y, cz + z};
            Cell c = m->win[m->lin(g)];
            cells[(z * 8 + y) * 8 + x] = c;
            if (c.v != 0 || c.w != 0) nonzero = true;
        }
        std::array<int64_t, 3> key = {cx / 8, cy / 8, cz / 8};
        if (nonzero) m->store[key] = cells;
        else m->store.erase(key);
    }
    // 2. build the new window: copy the overlap, load or zero the rest
    std::vector<Cell> next((size_t)(X * Y * Z), Cell{0, 0});
    for (int64_t gz = no[2]; gz < no[2] + Z; ++gz)
    for (int64_t gy = no[1]; gy < no[1] + Y; ++gy)
    for (int64_t gx = no[0]; gx < no[0] + X; ++gx) {
        int64_t g[3] = {gx, gy, gz};
        Cell c{0, 0};
        if (m->inside(g)) {
            c = m->win[m->lin(g)];
        } else {
            auto fl = [](int64_t v) { return v >= 0 ? v / 8 : -((-v + 7) / 8); };
            std::array<int64_t, 3> key = {fl(gx), fl(gy), fl(gz)};
            auto it = m->store.find(key);
            if (it != m->store.end()) {
                int64_t x = gx - key[0] * 8, y = gy - key[1] * 8, z = gz - key[2] * 8;
                c = it->second[(z * 8 + y) * 8 + x];
            }
        }
        next[(size_t)(((gz - no[2]) * Y + (gy - no[1])) * X + (gx - no[0]))] = c;
    }
    m->win.swap(next);
    for (int a = 0; a < 3; ++a) m->origin[a] = no[a];
    return 0;
}

// Copy the global box [lo, hi) (inside the window) to v/w in [z][y][x] order.
int orc_read(void* h, const int64_t lo[3], const int64_t hi[3], int16_t* v, int16_t* w) {
    OracleMap* m = (OracleMap*)h;
    if (!m) return -1;
    for (int a = 0; a < 3; ++a)
        if (lo[a] < m->origin[a] || hi[a] > m->origin[a] + m->p.dims[a] || hi[a] < lo[a]) return -1;
    int64_t i = 0;
    for (int64_t gz = lo[2]; gz < hi[2]; ++gz)
    for (int64_t gy = lo[1]; gy < hi[1]; ++gy)
    for (int64_t gx = lo[0]; gx < hi[0]; ++gx, ++i) {
        int64_t g[3] = {gx, gy, gz};
        Cell c = m->win[m->lin(g)];
        if (v) v[i] = c.v;
        if (w) w[i] = c.w;
    }
    return 0;
}

// Overwrite the window's cells from v/w in [z][y][x] window order (test set-up).
int orc_load_window(void* h, const int16_t* v, const int16_t* w) {
    OracleMap* m = (OracleMap*)h;
    if (!m) return -1;
    for (size_t i = 0; i < m->win.size(); ++i) m->win[i] = Cell{v[i], w[i]};
    return 0;
}

void orc_origin(void* h, int64_t out[3]) {
    OracleMap* m = (OracleMap*)h;
    for (int a = 0; a < 3; ++a) out[a] = m->origin[a];
}

void orc_stats(void* h, int64_t out[3]) {
    OracleMap* m = (OracleMap*)h;
    out[0] = m->st_valid;
    out[1] = m->st_hits;
    out[2] = m->st_touched;
}

int64_t orc_store_chunks(void* h) { return (int64_t)((OracleMap*)h)->store.size(); }

// Zero crossings of the window (a consumer of the map): for each voxel a (z,
// y, x order) and each axis x, y, z with b = a + e_axis inside the window,
// both weights >= min_w and (v_a < 0) != (v_b < 0): the point where the
// linear interpolation of v between the centres is zero, t = v_a / (v_a -
// v_b), coordinate along the axis ((float)g_a + 0.5 + t) * vs. Writes up to
// cap points as (x, y, z, axis); returns the number found.
int64_t orc_surface(void* h, int32_t min_w, float* out, int64_t cap) {
    OracleMap* m = (OracleMap*)h;
    const float vs = m->p.voxel_size;
    int64_t n = 0;
    for (int64_t z = 0; z < m->Z(); ++z)
    for (int64_t y = 0; y < m->Y(); ++y)
    for (int64_t x = 0; x < m->X(); ++x) {
        const int64_t ga[3] = {m->origin[0] + x, m->origin[1] + y, m->origin[2] + z};
        const Cell a = m->win[m->lin(ga)];
        if (a.w < min_w) continue;
        for (int ax = 0; ax < 3; ++ax) {
            int64_t gb[3] = {ga[0], ga[1], ga[2]};
            gb[ax] += 1;
            if (!m->inside(gb)) continue;
            const Cell b = m->win[m->lin(gb)];
            if (b.w < min_w || ((a.v < 0) == (b.v < 0))) continue;
            const float t = (float)a.v / (float)(a.v - b.v);
            float p[3];
            for (int k = 0; k < 3; ++k) p[k] = ((float)ga[k] + 0.5f) * vs;
            p[ax] = (((float)ga[ax] + 0.5f) + t) * vs;
            if (n < cap) {
                out[4 * n + 0] = p[0];
                out[4 * n + 1] = p[1];
                out[4 * n + 2] = p[2];
                out[4 * n + 3] = (float)ax;
            }
            ++n;
        }
    }
    return n;
}

// Triangle mesh of the zero level set by marching tetrahedra (a consumer of
// the map). Cubes of the dual grid: corners at the centres of voxels
// a + {0,1}^3, all 8 inside the window with weights >= min_w. Each cube is
// split into 6 tetrahedra sharing its diagonal 000-111, one per axis order
// (i, j, k): 000, e_i, e_i + e_j, 111 (orders in lexicographic order of
// (i, j, k)). In a tetrahedron with corner signs n = (v < 0): one corner
// against three gives a triangle on the three edges leaving it; two against
// two a quad on the four mixed edges (two triangles: (a,c),(a,d),(b,d) and
// (a,c),(b,d),(b,c) for negatives a < b and positives c < d in tetrahedron
// order). A vertex on edge P-Q, P the negative end (so a shared edge gives
// the same vertex in every tetrahedron): t = v_P / (v_P - v_Q), coordinate
// ((float)g_P + 0.5 + t * (g_Q - g_P)) * vs per axis (binary32). Each
// triangle is oriented so that its normal (binary64 cross product of its
// binary32 vertices) points towards the tetrahedron's positive corners.
// Writes up to cap triangles as 9 floats; returns the number found.
namespace {
const int kTetAxes[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
}

int64_t orc_mesh(void* h, int32_t min_w, float* out, int64_t cap) {
    OracleMap* m = (OracleMap*)h;
    const float vs = m->p.voxel_size;
    int64_t n = 0;
    auto vertex = [&](const int64_t gp[3], int vp, const int64_t gq[3], int vq, float* o) {
        const float t = (float)vp / (float)(vp - vq);
        for (int a = 0; a < 3; ++a) o[a] = (((float)gp[a] + 0.5f) + t * (float)(gq[a] - gp[a])) * vs;
    };
    for (int64_t z = 0; z + 1 < m->Z(); ++z)
    for (int64_t y = 0; y + 1 < m->Y(); ++y)
    for (int64_t x = 0; x + 1 < m->X(); ++x) {
        const int64_t base[3] = {m->origin[0] + x, m->origin[1] + y, m->origin[2] + z};
        int val[2][2][2];
        bool ok = true;
        for (int dz = 0; dz < 2 && ok; ++dz)
        for (int dy = 0; dy < 2 && ok; ++dy)
        for (int dx = 0; dx < 2 && ok; ++dx) {
            const int64_t g[3] = {base[0] + dx, base[1] + dy, base[2] + dz};
            const Cell c = m->win[m->lin(g)];
            if (c.w < min_w) ok = false;
            val[dz][dy][dx] = c.v;
        }
        if (!ok) continue;
        for (int tt = 0; tt < 6; ++tt) {
            int off[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
            off[1][kTetAxes[tt][0]] = 1;
            off[2][kTetAxes[tt][0]] = 1;
            off[2][kTetAxes[tt][1]] = 1;
            int64_t g[4][3];
            int v[4];
            int neg = 0;
            for (int k = 0; k < 4; ++k) {
                for (int a = 0; a < 3; ++a) g[k][a] = base[a] + off[k][a];
                v[k] = val[off[k][2]][off[k][1]][off[k][0]];
                neg += v[k] < 0 ? 1 : 0;
            }
            if (neg == 0 || neg == 4) continue;
            float tri[2][3][3];
            int nt = 0;
            if (neg == 1 || neg == 3) {
                int lone = 0;
                for (int k = 0; k < 4; ++k)
                    if ((v[k] < 0) == (neg == 1)) lone = k;
                int e = 0;   // every edge is interpolated from its negative end
                for (int k = 0; k < 4; ++k) {
                    if (k == lone) continue;
                    if (neg == 1) vertex(g[lone], v[lone], g[k], v[k], tri[0][e++]);
                    else vertex(g[k], v[k], g[lone], v[lone], tri[0][e++]);
                }
                nt = 1;
            } else {
                int ng[2], ps[2], a = 0, b = 0;
                for (int k = 0; k < 4; ++k) {
                    if (v[k] < 0) ng[a++] = k;
                    else ps[b++] = k;
                }
                float ac[3], ad[3], bd[3], bc[3];
                vertex(g[ng[0]], v[ng[0]], g[ps[0]], v[ps[0]], ac);
                vertex(g[ng[0]], v[ng[0]], g[ps[1]], v[ps[1]], ad);
                vertex(g[ng[1]], v[ng[1]], g[ps[1]], v[ps[1]], bd);
                vertex(g[ng[1]], v[ng[1]], g[ps[0]], v[ps[0]], bc);
                for (int a2 = 0; a2 < 3; ++a2) {
                    tri[0][0][a2] = ac[a2]; tri[0][1][a2] = ad[a2]; tri[0][2][a2] = bd[a2];
                    tri[1][0][a2] = ac[a2]; tri[1][1][a2] = bd[a2]; tri[1][2][a2] = bc[a2];
                }
                nt = 2;
            }
            // direction towards the positive corners: their mean minus the negatives' mean
            double dir[3] = {0, 0, 0};
            for (int k = 0; k < 4; ++k)
                for (int a2 = 0; a2 < 3; ++a2)
                    dir[a2] += (v[k] < 0 ? -1.0 / neg : 1.0 / (4 - neg)) * (double)off[k][a2];
            for (int r = 0; r < nt; ++r) {
                const double e1[3] = {(double)tri[r][1][0] - tri[r][0][0], (double)tri[r][1][1] - tri[r][0][1],
                                      (double)tri[r][1][2] - tri[r][0][2]};
                const double e2[3] = {(double)tri[r][2][0] - tri[r][0][0], (double)tri[r][2][1] - tri[r][0][1],
                                      (double)tri[r][2][2] - tri[r][0][2]};
                const double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2],
                             nz = e1[0] * e2[1] - e1[1] * e2[0];
                const bool flip = nx * dir[0] + ny * dir[1] + nz * dir[2] < 0.0;
                if (n < cap) {
                    const int order[3] = {0, flip ? 2 : 1, flip ? 1 : 2};
                    for (int c = 0; c < 3; ++c)
                        for (int a2 = 0; a2 < 3; ++a2) out[9 * n + 3 * c + a2] = tri[r][order[c]][a2];
                }
                ++n;
            }
        }
    }
    return n;
}

// Scan-to-map registration system (a consumer of the map): for every point,
// q = R p + t (binary32, the ray set-up's order), u = q / vs - 0.5 (binary32:
// fm then fs), i0 = floor(u), f = u - i0. If the 8 voxels i0 + {0,1}^3 lie in
// the window with weights >= min_w and the trilinear interpolation d of their
// distances (code * tau / 32767, binary64) has |d| < tau, the point adds its
// residual r = d and Jacobian J = [q x grad d, grad d] (binary64; the pose
// update q' = q + w x q + v) to H = sum J J^T (21 upper-triangle entries, row
// by row), g = sum J r (6), cost = sum r^2 and the point count: out[0..28].
void orc_register_system(void* h, const float* pts, int64_t n, const float pose[12], int32_t min_w, double* out) {
    OracleMap* m = (OracleMap*)h;
    for (int i = 0; i < 29; ++i) out[i] = 0.0;
    const float vs = m->p.voxel_size;
    const float inv = m->dv.inv_vs;
    const double scale = (double)m->p.tau / 32767.0;
    const double tau = (double)m->p.tau;
    for (int64_t i = 0; i < n; ++i) {
        const float x = pts[4 * i], y = pts[4 * i + 1], z = pts[4 * i + 2];
        if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z)) continue;
        float q[3];
        for (int a = 0; a < 3; ++a)
            q[a] = ((pose[4 * a] * x + pose[4 * a + 1] * y) + pose[4 * a + 2] * z) + pose[4 * a + 3];
        int64_t i0[3];
        double f[3];
        for (int a = 0; a < 3; ++a) {
            const float u = q[a] * inv - 0.5f;
            const float fl = std::floor(u);
            i0[a] = (int64_t)fl;
            f[a] = (double)(u - fl);
        }
        double c[2][2][2];
        bool ok = true;
        for (int dz = 0; dz < 2 && ok; ++dz)
        for (int dy = 0; dy < 2 && ok; ++dy)
        for (int dx = 0; dx < 2 && ok; ++dx) {
            const int64_t g[3] = {i0[0] + dx, i0[1] + dy, i0[2] + dz};
            if (!m->inside(g)) { ok = false; break; }
            const Cell cell = m->win[m->lin(g)];
            if (cell.w < min_w) { ok = false; break; }
            c[dz][dy][dx] = (double)cell.v * scale;
        }
        if (!ok) continue;
        const double fx = f[0], fy = f[1], fz = f[2];
        // interpolation along x, then y, then z
        double cx[2][2];
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy) cx[dz][dy] = c[dz][dy][0] * (1 - fx) + c[dz][dy][1] * fx;
        const double cy0 = cx[0][0] * (1 - fy) + cx[0][1] * fy, cy1 = cx[1][0] * (1 - fy) + cx[1][1] * fy;
        const double d = cy0 * (1 - fz) + cy1 * fz;
        if (!(std::fabs(d) < tau)) continue;
        // gradient with respect to u, then q
        double gu[3] = {0, 0, 0};
        for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy) {
            const double wyz = (dy ? fy : 1 - fy) * (dz ? fz : 1 - fz);
            gu[0] += wyz * (c[dz][dy][1] - c[dz][dy][0]);
        }
        for (int dz = 0; dz < 2; ++dz)
        for (int dx = 0; dx < 2; ++dx) {
            const double wxz = (dx ? fx : 1 - fx) * (dz ? fz : 1 - fz);
            gu[1] += wxz * (c[dz][1][dx] - c[dz][0][dx]);
        }
        for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            const double wxy = (dx ? fx : 1 - fx) * (dy ? fy : 1 - fy);
            gu[2] += wxy * (c[1][dy][dx] - c[0][dy][dx]);
        }
        const double gr[3] = {gu[0] / (double)vs, gu[1] / (double)vs, gu[2] / (double)vs};
        const double qd[3] = {(double)q[0], (double)q[1], (double)q[2]};
        const double J[6] = {qd[1] * gr[2] - qd[2] * gr[1], qd[2] * gr[0] - qd[0] * gr[2], qd[0] * gr[1] - qd[1] * gr[0],
                             gr[0], gr[1], gr[2]};
        int k = 0;
        for (int r = 0; r < 6; ++r)
            for (int cc = r; cc < 6; ++cc) out[k++] += J[r] * J[cc];
        for (int r = 0; r < 6; ++r) out[21 + r] += J[r] * d;
        out[27] += d * d;
        out[28] += 1.0;
    }
}

// The global map as non-empty 8^3 chunks: every window chunk with a non-zero
// cell, then every stored chunk outside the window (a stored copy of a chunk
// that is back in the window is stale). Writes up to `cap` chunks: key (the
// chunk's first voxel / 8) and 512 values and weights in (z * 8 + y) * 8 + x
// order. Returns the number of chunks.
int64_t orc_global_chunks(void* h, int64_t* keys, int16_t* v, int16_t* w, int64_t cap) {
    OracleMap* m = (OracleMap*)h;
    int64_t n = 0;
    auto emit = [&](const std::array<int64_t, 3>& key, const std::vector<Cell>& cells) {
        if (n < cap) {
            for (int a = 0; a < 3; ++a) keys[3 * n + a] = key[a];
            for (int i = 0; i < 512; ++i) {
                v[512 * n + i] = cells[i].v;
                w[512 * n + i] = cells[i].w;
            }
        }
        ++n;
    };
    for (int64_t cz = m->origin[2]; cz < m->origin[2] + m->Z(); cz += 8)
    for (int64_t cy = m->origin[1]; cy < m->origin[1] + m->Y(); cy += 8)
    for (int64_t cx = m->origin[0]; cx < m->origin[0] + m->X(); cx += 8) {
        std::vector<Cell> cells(512);
        bool nonzero = false;
        for (int z = 0; z < 8; ++z)
        for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x) {
            int64_t g[3] = {cx + x, cy + y, cz + z};
            Cell c = m->win[m->lin(g)];
            cells[(z * 8 + y) * 8 + x] = c;
            if (c.v != 0 || c.w != 0) nonzero = true;
        }
        if (nonzero) emit({cx / 8, cy / 8, cz / 8}, cells);
    }
    for (const auto& kv : m->store) {
        const int64_t g[3] = {kv.first[0] * 8, kv.first[1] * 8, kv.first[2] * 8};
        if (m->inside(g)) continue;
        emit(kv.first, kv.second);
    }
    return n;
}

}  // extern "C"
