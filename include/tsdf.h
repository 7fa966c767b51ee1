/*
 * tsdf.h -- C ABI of the GB300 TSDF map-generation library (libtsdf_gb300.so).
 *
 * The library integrates registered LiDAR scans into a truncated signed
 * distance field held on one GPU as a fixed-point, ring-addressed local map,
 * as described in FeatSense (Gaal et al.), Section "TSDF Map Generation":
 * each voxel is a (value, weight) pair of 16 bits each; a scan is traversed
 * ray by ray from the scan pose to each point; every voxel within +-tau of a
 * hit receives the truncated signed distance of its centre; neighbouring
 * scan lines are bridged by the vertical interpolation of Eq. 3 / Eq. 4; the
 * per-scan volume is merged into the map with the weighted average of Eq. 1
 * and the clamped weight of Eq. 2. The local map is shifted as the sensor
 * moves (Introduction: a local map that is shifted after a movement
 * threshold, its parts written to and read back from a global map).
 *
 * Conventions for every function:
 *  - Return value: TSDF_OK (0) or a negative TSDF_ERR_* code. On error no
 *    state visible through this API has changed unless stated otherwise.
 *  - Device pointers must come from the same CUDA device the map was created
 *    on (the device current at tsdf_map_create). The library makes that
 *    device current for the duration of each call.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream. Calls marked "asynchronous" only enqueue work on `stream`; calls
 *    on one map must be serialised by the caller (one stream, or events).
 *  - All sizes are counts of elements unless named *_bytes.
 *  - Thread safety: different maps may be used from different host threads;
 *    one map must not be used by two host threads at once.
 *
 * Fixed-point encoding: value code q in [-32767, 32767] stands for the
 * truncated signed distance q * tau / 32767 metres, positive in front of the
 * surface (on the sensor side). Weight 0 means "never observed".
 */
#ifndef TSDF_GB300_H
#define TSDF_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define TSDF_OK              0
#define TSDF_ERR_INVALID    -1  /* bad argument: null pointer, bad dims/params, misaligned points, n out of range, box outside the window */
#define TSDF_ERR_OOM        -2  /* a device or pinned-host allocation failed */
#define TSDF_ERR_CUDA       -3  /* a CUDA runtime call or kernel launch failed; see tsdf_last_cuda_error() */
#define TSDF_ERR_TIMEOUT    -4  /* a bounded device-side wait expired */
#define TSDF_ERR_ADMISSION  -5  /* a session would exceed the device-memory budget */
#define TSDF_ERR_BUSY       -6  /* the resource is in use (e.g. an outstanding request) */
#define TSDF_ERR_IO         -7  /* a file could not be opened, read or written, or is not a map file */
#define TSDF_ERR_DEGENERATE -9  /* registration: too few usable points or no curvature along some direction */
#define TSDF_ERR_CAPACITY   -8  /* the last scan needed more accumulator bricks than the pool holds; it was
                                   dropped whole (the map is unchanged) */

/* ---- per-scan reduction of the contributions to one voxel ----------------- */
#define TSDF_REDUCE_WSUM     0  /* sum of weight * distance and sum of weights (weight 1 per contribution) */
#define TSDF_REDUCE_MIN_ABS  1  /* the paper's "smallest distance of all rays": smallest |q|, ties -> positive; weight 1 */

/* ---- alternative readings of the paper (tsdf_params.flags) ---------------- */
#define TSDF_FLAG_STEP_VALUE   1  /* every sample of a march step (the step's voxel and its fill samples) gets the
                                     step's own truncated distance r - l (the fill copies the step's value, Section
                                     "TSDF Map Generation"); default: the projective distance of the voxel's centre */
#define TSDF_FLAG_SCAN_WEIGHT  2  /* WSUM: a scan's averaged value S/W enters Eq. 1 / Eq. 2 as one observation of
                                     weight 1: value (gv*gw*W + S) / ((gw + 1) * W), weight min(w_max, gw + 1);
                                     default: weight W (its contribution count) */

/* Largest number of points accepted by one integrate call. A ray's samples
 * lie on a square lattice of spacing voxel_size (march steps along the ray,
 * fill samples along the interpolation direction); among any five points of
 * such a lattice two are at least two spacings apart, more than a voxel's
 * diagonal, so at most four samples of one ray fall in one voxel (four do
 * occur). With weight 1 per contribution a voxel's per-scan count is then at
 * most 4 * (2^22 - 1) < 2^24 and its distance sum below 2^39: both fit the
 * packed 64-bit accumulator exactly. (The bound assumes binary32 rounding
 * moves a sample by far less than a voxel, which holds while ranges and
 * coordinates stay below about 2^17 voxels.) */
#define TSDF_MAX_POINTS      ((1LL << 22) - 1)

/* Map parameters. */
typedef struct tsdf_params {
    int32_t dims[3];      /* window size in voxels (x, y, z): each a power of two, 8..32768; product <= 2^31 */
    float   voxel_size;   /* voxel edge length in metres, > 0 */
    float   tau;          /* truncation distance in metres, voxel_size <= tau <= 1024 voxels */
    int32_t w_max;        /* weight cap of Eq. 2, 1..32767 */
    float   delta_z;      /* Eq. 3, tan(vfov / hlines) computed by the caller; 0 disables vertical interpolation; 0..1 */
    float   r_min;        /* points with range < r_min are skipped, >= 0 */
    float   r_max;        /* points with range > r_max are skipped, r_min <= r_max <= 1e5 */
    int32_t reduce;       /* TSDF_REDUCE_WSUM or TSDF_REDUCE_MIN_ABS */
    int32_t flags;        /* TSDF_FLAG_* bits; 0 selects the default readings */
    int64_t origin[3];    /* initial window origin in global voxel coordinates; multiples of 8, |origin| <= 2^23 */
} tsdf_params;

/* Counters of the most recent integrate call on a map. */
typedef struct tsdf_scan_stats {
    int64_t valid_rays;   /* points with a finite range inside [r_min, r_max] */
    int64_t hits;         /* (ray, voxel) contributions that fell inside the window */
    int64_t touched;      /* distinct voxels updated by Eq. 1 / Eq. 2 */
} tsdf_scan_stats;

typedef struct tsdf_map tsdf_map;   /* opaque; owns all of its device memory */

/* Create a map on the current CUDA device. The window starts at
 * params->origin with every voxel (0, 0). Allocates the voxel grid (4 bytes
 * per voxel: int16 value, int16 weight) and a touched-brick flag array and
 * list (bricks of 8^3 voxels). The per-scan accumulator (8 bytes per voxel,
 * kept all-zero between calls) is allocated by the first integrate call that
 * uses the atomic or sort reduction (the pool reduction keeps a smaller one of
 * its own), and the per-ray buffers (32 bytes per point) by the first
 * integrate call that needs them. Synchronous. On success *out receives the
 * handle, which the caller releases with tsdf_map_destroy. Errors: INVALID,
 * OOM, CUDA. */
int tsdf_map_create(const tsdf_params* params, tsdf_map** out);

/* Release a map and all of its device memory. Waits for the map's work to
 * finish (device synchronisation). NULL is accepted and ignored. */
int tsdf_map_destroy(tsdf_map* map);

/* Integrate one registered scan (Section "TSDF Map Generation": ray march
 * within +-tau of each point, vertical interpolation of Eq. 3 / Eq. 4,
 * per-scan volume, Eq. 1 / Eq. 2). Asynchronous on `stream`.
 *   points_dev : device pointer to n float4 values (x, y, z, unused) in the
 *                sensor frame, 16-byte aligned, any point order (beam-major
 *                for locality). Non-finite points and points out of
 *                [r_min, r_max] are skipped. Owned by the caller, who keeps
 *                it alive until the stream has passed this call.
 *   n          : 0 <= n <= TSDF_MAX_POINTS; n = 0 only records zero counters.
 *   pose       : host pointer to 12 floats, the row-major 3x4 sensor-to-world
 *                transform [R | t]; R's third column is the direction
 *                orthogonal to the scan lines. Copied at call time.
 * The result is bit-identical to a serial evaluation in any launch order.
 * When n exceeds every earlier n of this map, the per-ray buffers grow first
 * (a synchronous reallocation). Errors: INVALID, OOM, CUDA. */
int tsdf_integrate(tsdf_map* map, const float* points_dev, int64_t n, const float pose[12], void* stream);

/* As tsdf_integrate, but points_host is a HOST pointer (pinned or pageable)
 * to n float4 values. Pinned memory that is mapped into the device (16-byte
 * aligned) is read in place by the first kernel over the host link
 * (TSDF_OPT_HOST_ZERO_COPY); otherwise the points are copied into a map-owned
 * device buffer on `stream` first. Either way the buffer must stay valid and
 * unchanged until the stream has passed the call. Returns once the work has
 * been enqueued (for pageable memory the CUDA runtime may wait for the copy).
 * Errors: INVALID, OOM, CUDA. */
int tsdf_integrate_host(tsdf_map* map, const float* points_host, int64_t n, const float pose[12], void* stream);

/* Move the window to new_origin (global voxel coordinates, multiples of 8,
 * |new_origin| <= 2^23). Voxels inside both windows keep their values (ring
 * addressing: no data moves). Chunks of 8^3 voxels that leave the window are
 * written to the map's global store if any of their voxels is non-zero (the
 * others are dropped); chunks that enter are read back from the store (and
 * leave it, freeing their slot), or set to (0, 0) if not stored. (Introduction
 * of the paper: the local map is shifted, map parts leaving it are written out
 * and previously mapped parts are read back.)
 * The store has two tiers of 2 KiB slots (a third, a file, on request): device memory, up to
 * TSDF_OPT_STORE_DEVICE_CHUNKS slots, and pinned host memory mapped into the
 * device, which the shift kernel reads and writes in place. When the device
 * tier is full, its chunks stored longest ago move to the host tier first
 * (and, with TSDF_OPT_STORE_SPILL_AGE, any chunk stored that many shifts ago).
 * Asynchronous on `stream`, except that it waits for the previous shift's
 * kernel (whose per-chunk "held data" flags it needs), and that growing a tier
 * allocates synchronously (8 MiB segments; see tsdf_map_reserve_store to
 * allocate the device tier up front). With a file tier
 * (tsdf_map_set_store_file) the host-tier chunks beyond its limit are queued
 * for the file first, and entering file-tier chunks are read back into host
 * slots before the kernel is enqueued. Errors: INVALID, OOM, CUDA, IO (a file
 * write failed earlier, or an entering file-tier chunk could not be read or
 * given a host slot: the shift is done all the same and that chunk enters as
 * (0, 0); the error is then IO, OOM or CUDA). */
int tsdf_shift(tsdf_map* map, const int64_t new_origin[3], void* stream);

/* Allocate the device tier of the map's global store now: `device_chunks`
 * slots (2 KiB each, rounded up to whole 8 MiB segments), which also become
 * its limit (TSDF_OPT_STORE_DEVICE_CHUNKS), so that later shifts allocate no
 * device memory (chunks beyond it go to the host tier). device_chunks >= 1.
 * Synchronous. Errors: INVALID, OOM, CUDA. */
int tsdf_map_reserve_store(tsdf_map* map, int64_t device_chunks);

/* Global-store counters of a map (waits for the last shift's kernel). */
typedef struct tsdf_store_stats {
    int64_t device_chunks;      /* chunks held in device memory */
    int64_t device_capacity;    /* device-tier slots allocated */
    int64_t host_chunks;        /* chunks held in pinned host memory */
    int64_t host_capacity;      /* host-tier slots allocated */
    int64_t spilled;            /* chunks moved from device to host memory so far */
    int64_t dropped;            /* leaving chunks found empty (all voxels zero) and not stored, so far */
    int64_t file_chunks;        /* chunks held in the file tier */
    int64_t to_file;            /* chunks moved from host memory to the file so far */
    int64_t from_file;          /* file-tier chunks read back when they re-entered the window, so far */
} tsdf_store_stats;
int tsdf_get_store_stats(tsdf_map* map, tsdf_store_stats* out);

/* Give the map's global store a third tier in a file, for maps larger than
 * host memory (the paper keeps the global map on disk: map parts that leave
 * the local window are written out and earlier parts read back; Introduction,
 * and the Evaluation's closing remarks on an SSD). From the next shift on, at
 * the start of every shift the host tier keeps at most `host_chunks` chunks
 * (host_chunks >= 0; it may hold more until the next shift); the chunks that
 * entered it longest ago move to the file. Writes are asynchronous: a writer
 * thread of the map writes them while the caller goes on (up to 4096 chunks,
 * 8 MiB, wait to be written; a shift that queues more waits for room). A chunk
 * that re-enters the window is read back from the file (or from its queued
 * copy) by the shift. `path` must not exist: the call creates it; it holds
 * 2 KiB records and no header (tsdf_map_save writes the map file), and it is
 * removed by tsdf_map_destroy. Once per map. Errors: INVALID (null map or
 * path, host_chunks < 0, a file already set), IO (the path exists or the file
 * cannot be created). */
int tsdf_map_set_store_file(tsdf_map* map, const char* path, int64_t host_chunks);

/* Copy the global voxel box [lo, hi) (must lie inside the current window) to
 * the host in [z][y][x] order: value_host and weight_host each receive
 * (hi-lo).x*(hi-lo).y*(hi-lo).z int16 values; either may be NULL. Enqueued on
 * `stream`, then synchronises `stream`. Errors: INVALID, OOM, CUDA. */
int tsdf_read(tsdf_map* map, const int64_t lo[3], const int64_t hi[3], int16_t* value_host,
              int16_t* weight_host, void* stream);

/* Overwrite the global box [lo, hi) (inside the window) from host arrays in
 * [z][y][x] order (restore / test set-up). Weights must be in [0, w_max].
 * Synchronises `stream`. Errors: INVALID, OOM, CUDA. */
int tsdf_write(tsdf_map* map, const int64_t lo[3], const int64_t hi[3], const int16_t* value_host,
               const int16_t* weight_host, void* stream);

/* Counters of the most recent integrate call (zero before the first).
 * Synchronises `stream`. Returns TSDF_ERR_CAPACITY (hits and touched 0) when
 * that scan was dropped by the pool reduction. Errors: INVALID, CUDA. */
int tsdf_stats(tsdf_map* map, tsdf_scan_stats* out, void* stream);

/* Tuning options (no effect on results, which are bit-identical for every
 * setting; only on speed). */
#define TSDF_OPT_WARP_MERGE  1  /* 1: lanes of a warp that hit the same voxel in the same step are merged
                                   (match.any + redux) before one accumulator atomic; 0 (default): every
                                   contribution issues its own atomic */
#define TSDF_OPT_STEPS_PER_THREAD 2  /* march steps k handled by one contribution work item: 1, 2 or 4 (default) */
#define TSDF_OPT_PDL         3  /* 1 (default): the kernels of one integrate call use programmatic dependent
                                   launch, so each may be scheduled while the previous one drains; 0: plain
                                   stream order */
#define TSDF_OPT_REDUCTION   4  /* how a scan's contributions are combined per voxel (the per-scan volume of
                                   Section "TSDF Map Generation"): TSDF_REDUCTION_ATOMIC (default) or
                                   TSDF_REDUCTION_SORT. Both give bit-identical maps and counters. */
#define TSDF_OPT_SORT_CAPACITY 5  /* sort reduction: pair slots held by the map (each 12 bytes of device
                                   memory); 0 (default): 32 per point of the largest scan so far, at least
                                   2^20; otherwise 1024 .. 2^28. Samples beyond the capacity are reduced
                                   with accumulator atomics instead (same result, slower). */

#define TSDF_OPT_HOST_ZERO_COPY 6  /* 1 (default): tsdf_integrate_host reads points that lie in pinned host memory
                                     mapped into the device (cudaHostAlloc / cudaHostRegister) in place over
                                     the host link instead of copying them first; 0: always stage a copy */

#define TSDF_REDUCTION_ATOMIC 0  /* each contribution is one 64-bit reduction into a per-voxel accumulator */
#define TSDF_REDUCTION_SORT   1  /* contributions are written as (voxel, code) pairs, counting-sorted by brick
                                   and reduced per voxel in shared memory; no per-contribution atomics. Buffers
                                   are allocated on the first integrate call that uses it (synchronous). */
#define TSDF_REDUCTION_POOL   2  /* sparse per-scan accumulator: a brick gets a 4 KiB accumulator slot from a
                                   pool on its first contribution of the scan (brick -> slot table, 4 B per
                                   brick) and the apply walks the claimed slots; the dense 8 B/voxel
                                   accumulator is never allocated for a map used only this way. A scan that
                                   needs more bricks than the pool holds is dropped whole and tsdf_stats
                                   returns TSDF_ERR_CAPACITY. Same results as the other reductions. */
#define TSDF_REDUCTION_AUTO   3  /* the atomic, sort and pool reductions are each run once untimed and then
                                   timed (CUDA events) on the next calls; once every trial has finished
                                   the fastest is used from then on (tsdf_get_reduction tells which). A pool
                                   trial that overflows is dropped like any pool scan: do not use AUTO with a
                                   pool too small for the scans */
#define TSDF_OPT_POOL_BRICKS  7  /* pool reduction: slots of the pool (64 .. bricks of the window); 0 (default):
                                   an eighth of the window's bricks, at least 16384 */
#define TSDF_OPT_STORE_DEVICE_CHUNKS 8  /* global store: most slots of its device tier (2 KiB each); 0 (default):
                                          as many as the window has bricks. Chunks beyond it go to pinned host
                                          memory. Lowering it frees nothing already allocated. */
#define TSDF_OPT_STORE_SPILL_AGE 9  /* global store: a chunk stored this many shifts ago moves from device to
                                      host memory at the next shift; 0 (default): only when the device tier is
                                      full */
#define TSDF_OPT_LAUNCH_GRAPH 10  /* 1: the atomic reduction's four kernels are captured once into a CUDA
                                    graph (again after buffers or options change) and each scan sets the
                                    graph's arguments and launches it once: less host time per scan, for
                                    callers whose thread is the bottleneck; 0 (default): four launches per
                                    scan, which let consecutive scans overlap on the device. Scans while
                                    profiling is enabled or while the caller's stream is being captured use
                                    four launches. */

/* Device memory held by the map (grid, per-scan buffers of the reductions
 * that have been used, ray buffers, global store) in bytes. Host-side.
 * Errors: INVALID. */
int tsdf_map_device_bytes(const tsdf_map* map, int64_t* out);

/* The reduction in use: the option's value, or for TSDF_REDUCTION_AUTO the
 * one chosen (TSDF_REDUCTION_AUTO while the trials still run). Host-side
 * (looks at finished trial events without waiting). Errors: INVALID. */
int tsdf_get_reduction(tsdf_map* map, int32_t* reduction);

/* Set a tuning option of a map; takes effect for later calls. Host-side
 * state only (the sort buffers are allocated by the next integrate call).
 * Errors: INVALID (unknown option or value). */
int tsdf_set_option(tsdf_map* map, int32_t option, int64_t value);

/* Current window origin (host-side state; no synchronisation). */
int tsdf_get_origin(const tsdf_map* map, int64_t out[3]);

/* Device pointer of the voxel grid: uint32 words, value in the low 16 bits,
 * weight in the high 16 bits, bricked and ring addressed: global voxel g
 * lives in brick b = ((bz * CY) + by) * CX + bx with (bx, by, bz) =
 * (g >> 3) mod (dims / 8) and (CX, CY) = dims.xy / 8, at word
 * b * 512 + ((g.z & 7) * 8 + (g.y & 7)) * 8 + (g.x & 7). Valid until destroy. */
int tsdf_grid_device_ptr(const tsdf_map* map, void** out);

/* Per-kernel device time of this map's launches, measured with CUDA events
 * recorded on the launching stream around each kernel while profiling is on. */
typedef struct tsdf_kernel_time {
    char    name[24];     /* "rays", "contrib", "apply" (brick compaction, update, counters) or "shift" */
    int64_t launches;     /* kernel launches since profiling was enabled */
    double  total_ms;     /* summed event-to-event device time */
} tsdf_kernel_time;

/* Turn per-kernel event timing on (enable != 0) or off, and reset the
 * accumulated times. Host-side state only. Errors: INVALID. */
int tsdf_profile_enable(tsdf_map* map, int32_t enable);

/* Accumulated per-kernel times: writes up to `capacity` entries to out and
 * the number of kernels with launches to *count. Waits for the recorded
 * events (host blocks until the profiled launches have finished).
 * Errors: INVALID, CUDA. */
int tsdf_profile_read(tsdf_map* map, tsdf_kernel_time* out, int32_t capacity, int32_t* count);

/* ---- persistence (checkpoint / resume of the whole global map) --------------
 * The paper keeps the local map small and writes map parts that leave it to
 * storage, reading them back when the sensor returns (Introduction). Here the
 * parts live in a device-resident store while the process runs; these calls
 * write the whole global map (window + store) to a file and rebuild a map from
 * one, bit for bit.
 *
 * File format (little-endian): a 128-byte header, then one 2072-byte record
 * per non-empty 8^3 chunk.
 *   header: char magic[8] = "TSDFMAP1"; uint32 version = 1; uint32 header_bytes
 *           = 128; tsdf_params params (72 bytes; origin = the window origin at
 *           save time); int64 chunk_count; 32 zero bytes.
 *   record: int64 chunk[3] (the chunk's first voxel in global coordinates,
 *           divided by 8); uint32 word[512], word (z * 8 + y) * 8 + x holding
 *           voxel chunk * 8 + (x, y, z) as value (low 16 bits, int16) and
 *           weight (high 16 bits, int16).
 * A chunk is non-empty when any of its words is non-zero. */
#define TSDF_FILE_HEADER_BYTES 128
#define TSDF_FILE_RECORD_BYTES 2072

/* Write `map` to `path` (created or truncated). Synchronises `stream` first
 * (all earlier work on the map must be on it); uses a pinned staging buffer.
 * Errors: INVALID, IO, OOM, CUDA. */
int tsdf_map_save(tsdf_map* map, const char* path, void* stream);

/* Create a map from a file written by tsdf_map_save: same parameters, window
 * at the saved origin, every chunk back in the window or the store. The new
 * map is ready when the call returns (it synchronises `stream`). The file is
 * checked (magic, version, sizes, parameters) before any device memory is
 * allocated. Errors: INVALID, IO, OOM, CUDA. */
int tsdf_map_load(const char* path, tsdf_map** out, void* stream);

/* ---- map consumers ------------------------------------------------------------
 * Surface points: one per pair of 6-connected window voxels a, b = a + e_axis
 * (axis 0, 1, 2 = x, y, z) whose weights are both >= min_weight and whose
 * values differ in sign ((v_a < 0) != (v_b < 0)), placed where the linear
 * interpolation of the two codes between the voxel centres is zero:
 * t = v_a / (v_a - v_b) (IEEE binary32 division), coordinate along the axis
 * ((float)g_a + 0.5 + t) * voxel_size, the other two ((float)g + 0.5) *
 * voxel_size, in world metres. out_dev: device float4 array (x, y, z, axis),
 * 16-byte aligned, `capacity` points; the order is unspecified. *count gets
 * the number of points found (those beyond capacity are not written).
 * Synchronises `stream`. Errors: INVALID, CUDA. */
int tsdf_extract_surface(tsdf_map* map, int32_t min_weight, float* out_dev, int64_t capacity, int64_t* count,
                         void* stream);

/* Triangle mesh of the window's zero level set by marching tetrahedra. Dual
 * cubes have their corners at the centres of voxels a + {0,1}^3 (all 8 in the
 * window with weights >= min_weight); each is split into 6 tetrahedra around
 * its 000-111 diagonal, one per axis order (i, j, k) in lexicographic order:
 * 000, e_i, e_i + e_j, 111. A tetrahedron whose corners differ in sign
 * (v < 0) gives one triangle (one corner against three) or two (two against
 * two: negatives a < b, positives c < d in tetrahedron order: (a,c),(a,d),(b,d)
 * and (a,c),(b,d),(b,c)). A vertex on the edge from the negative corner P to
 * the positive corner Q: t = v_P / (v_P - v_Q), coordinate ((float)g_P + 0.5
 * + t (g_Q - g_P)) * voxel_size (binary32), so a shared edge gives the same
 * vertex in every tetrahedron and the mesh is closed where the surface is.
 * Triangles face the positive side. out_dev: device floats, 9 per triangle
 * (3 vertices x y z, world metres); `capacity` triangles; the order is
 * unspecified; *count gets the number found. Synchronises `stream`.
 * Errors: INVALID, CUDA. */
int tsdf_extract_mesh(tsdf_map* map, int32_t min_weight, float* out_dev, int64_t capacity, int64_t* count,
                      void* stream);

/* Scan-to-map registration (Gauss-Newton on the map): minimises
 * sum_i d(T p_i)^2, d the trilinear interpolation of the stored distances
 * (code * tau / 32767, metres) of the 8 voxels around a point, using the
 * points whose 8 voxels lie in the window with weights >= min_weight and
 * whose |d| < tau. Pose update q' = Exp(w) q + v (world frame); residual
 * Jacobian J = [q x grad d, grad d].
 *
 * tsdf_register_system: the normal equations at `pose` (host, row-major
 * 3x4): out_host[0..20] = H = sum J J^T (upper triangle, row by row),
 * [21..26] = g = sum J d, [27] = sum d^2, [28] = points used (binary64; the
 * point position math is binary32 in a fixed order, the rest binary64).
 * points_dev: n device float4 (16-byte aligned). Synchronises `stream`.
 *
 * tsdf_register: up to `iterations` steps from pose_inout (updated in
 * place after each successful step; solve by Cholesky, stops when the step
 * norm falls below 1e-7). result may be NULL. Returns TSDF_ERR_DEGENERATE
 * (pose_inout keeping the last good pose) when a step finds fewer than 6
 * points or a singular system. Errors: INVALID, DEGENERATE, CUDA. */
typedef struct tsdf_register_result {
    int64_t used_points;  /* points in the last evaluated system */
    double  rms;          /* sqrt(sum d^2 / points) of the last evaluated system, metres */
    double  step;         /* norm of the last step (w in rad, v in m) */
    int32_t iterations;   /* steps taken */
    int32_t reserved;
} tsdf_register_result;

int tsdf_register_system(tsdf_map* map, const float* points_dev, int64_t n, const float pose[12],
                         int32_t min_weight, double* out_host, void* stream);
int tsdf_register(tsdf_map* map, const float* points_dev, int64_t n, float pose_inout[12], int32_t iterations,
                  int32_t min_weight, tsdf_register_result* result, void* stream);

/* ---- measurement ------------------------------------------------------------
 * Sustained rate (operations per second) of fire-and-forget 64-bit integer
 * reductions into L2-resident device memory on the current device, the
 * operation the contribution kernel issues once per in-window sample:
 * pattern 0 = each warp's lanes on 32 consecutive words, 1 = scattered words.
 * Allocates and frees a 64 MiB scratch buffer; synchronises `stream`.
 * Errors: INVALID, OOM, CUDA. */
int tsdf_probe_reduction_rate(int32_t pattern, double* per_second, void* stream);

/* ---- batched integration ---------------------------------------------------
 * Integrates one scan into each of many maps in a single persistent
 * cooperative launch: the phases of tsdf_integrate (ray set-up, contributions,
 * brick compaction, Eq. 1 / Eq. 2 update, counters) run over all maps of the
 * batch with a grid-wide barrier between phases, so maps of uneven size share
 * the whole GPU and a batch costs one launch instead of five per map. Each map's
 * result is bit-identical to tsdf_integrate of the same scan. The launch (a
 * descriptor copy, a barrier reset and the kernel) is captured once into a CUDA
 * graph and replayed; the descriptors are the only thing that changes. */
typedef struct tsdf_batch tsdf_batch;   /* opaque; owns pinned and device descriptor buffers */

#define TSDF_BATCH_OPT_GRAPH      1  /* 1 (default): replay a captured CUDA graph; 0: plain launches */
#define TSDF_BATCH_OPT_AUTOTUNE   2  /* 1 (default): time every tuning configuration on the first calls and keep the fastest */
#define TSDF_BATCH_OPT_CONFIG     3  /* fix the tuning configuration; turns autotuning off. 0..5: atomic reduction,
                                        {no merge, merge} x {4, 2, 1} steps per item; 6, 7: sort reduction
                                        (TSDF_REDUCTION_SORT) with 4, 2 steps per item (all with CTAs of 256
                                        threads, as many per SM as fit, whole-brick apply tasks); 8..11: atomic
                                        reduction, no merge, 4 steps per item, with CTAs of 128 threads, of 512
                                        threads, of 256 threads but 2 per SM, or quarter-brick apply tasks; 12:
                                        as 8 with four points per thread in the ray set-up */
#define TSDF_BATCH_OPT_SPIN_LIMIT 4  /* polls before a grid-barrier wait gives up (default 2^24, about a second) */
#define TSDF_BATCH_OPT_TEST_MISSING_ARRIVALS 5  /* test hook: the barrier waits for this many CTAs that do not exist (default 0) */
#define TSDF_BATCH_OPT_GRID_FRACTION 6  /* percent (1..100, default 100) of the device's co-resident CTAs the launch uses,
                                           so that launches on several streams can be resident together */
#define TSDF_BATCH_OPT_TUNE_SORT  7  /* 1 (default): the autotuner also times the sort configurations, whose first use
                                        allocates each map's sort buffers; 0: only the atomic ones (no allocation) */
#define TSDF_BATCH_OPT_CTA_BRICK_CACHE 8  /* 1 (default): the warps of a CTA share one cache of the bricks they
                                              marked (keys tagged with the map), when every map has fewer than
                                              2^22 bricks and the batch fewer than 1023 maps; 0: one cache per
                                              warp. Speed only: results are identical. */

/* Create a batch object for up to max_count (1..1024) maps per call, on the
 * current device. Synchronous. Errors: INVALID, OOM, CUDA. */
int tsdf_batch_create(int32_t max_count, tsdf_batch** out);

/* Release a batch object (waits for the device). NULL is ignored. */
int tsdf_batch_destroy(tsdf_batch* batch);

/* Set an option (TSDF_BATCH_OPT_*). Host-side state. Errors: INVALID. */
int tsdf_batch_set_option(tsdf_batch* batch, int32_t option, int64_t value);

/* The tuning configuration in use: index, warp merge (0/1), steps per work
 * item, reduction (TSDF_REDUCTION_*), whether autotuning has finished, and the
 * launch shape: threads per CTA, CTAs launched, and voxel pairs per lane of
 * an apply task (8: a warp per brick, 2: a quarter brick). Any pointer may be
 * NULL. */
int tsdf_batch_get_config(const tsdf_batch* batch, int32_t* config, int32_t* merge, int32_t* steps_per_item,
                          int32_t* reduction, int32_t* tuned, int32_t* threads_per_cta, int32_t* ctas,
                          int32_t* apply_voxel_pairs);

/* Integrate scan i (points_dev[i]: n[i] device float4 points, 16-byte
 * aligned; poses + 12*i: host row-major 3x4 pose) into maps[i], for i <
 * count (count <= max_count). The maps must be distinct and live on the batch's
 * device; each keeps its own window (shift them separately). Asynchronous on
 * `stream`; calls on one batch object must be serialised on one stream, and
 * while a batch is in flight its maps must not be used on other streams.
 * Per-map counters are available through tsdf_stats afterwards. A device-side
 * barrier timeout is reported by tsdf_batch_sync; the maps of that batch are
 * then in an undefined state. Errors: INVALID, OOM, CUDA. */
int tsdf_batch_integrate(tsdf_batch* batch, tsdf_map* const* maps, const float* const* points_dev, const int64_t* n,
                         const float* poses, int32_t count, void* stream);

/* Convenience form of tsdf_batch_integrate with a batch object per host thread
 * and device, created on first use and destroyed when the thread exits (up to
 * 1024 maps per call). */
int tsdf_integrate_batch(tsdf_map* const* maps, const float* const* points_dev, const int64_t* n, const float* poses,
                         int32_t count, void* stream);

/* Wait for `stream` and report the last batch launch's status: TSDF_OK, or
 * TSDF_ERR_TIMEOUT if a grid-barrier wait gave up. Errors: INVALID, CUDA. */
int tsdf_batch_sync(tsdf_batch* batch, void* stream);

/* ---- serving: continuous batching over many map sessions -------------------
 * A server keeps every session's map resident on the device and admits
 * sessions against a device-memory budget. Requests are queued per session;
 * a worker thread forms batches from the requests that have arrived (at most
 * one per session per batch, at most one batch per session in flight, so each
 * map sees its scans in submission order) and runs each batch as one batched
 * integration on one of several streams, so that batches overlap on the
 * device. A session's map is bit-identical whether its scans ran alone or in
 * any mix of sessions. */
typedef struct tsdf_server tsdf_server;   /* opaque; owns its sessions' maps, streams and pinned slabs */

typedef struct tsdf_server_config {
    int64_t hbm_budget_bytes;   /* device memory the sessions may take (grid, accumulator, ray buffers, the device
                                   tier of each session's global store) */
    int64_t max_points;         /* largest scan accepted, 1..TSDF_MAX_POINTS */
    int32_t max_batch;          /* most sessions in one batch, 1..1024 */
    int32_t streams;            /* batches that may be in flight together, 1..8 */
    int32_t max_outstanding;    /* submitted requests not yet waited for (pinned slabs of max_points points) */
    int32_t store_chunks;       /* device-tier slots of each session's global store, allocated when the session
                                   opens and charged to the budget (2 KiB each); 0: an eighth of the window's
                                   bricks. Shifts never allocate device memory; chunks beyond it go to pinned
                                   host memory. */
} tsdf_server_config;

typedef struct tsdf_request_result {
    uint64_t ticket;
    int32_t session;
    int32_t status;             /* TSDF_OK or the error of the request */
    int32_t batch_size;         /* requests in the batch that carried it */
    int32_t reserved;
    tsdf_scan_stats stats;      /* counters of the scan */
    double t_submit_us;         /* host steady-clock microseconds: submitted, */
    double t_start_us;          /* launched on the GPU, */
    double t_done_us;           /* and seen complete by the worker */
} tsdf_request_result;

typedef struct tsdf_server_stats {
    int32_t sessions;
    int32_t reserved;
    int64_t used_bytes;         /* device memory reserved by the sessions */
    int64_t completed;          /* requests completed */
    int64_t batches;            /* batches launched */
    int64_t queued;             /* requests waiting to be batched */
    double mean_batch;          /* requests per batch */
} tsdf_server_stats;

/* Create a server on the current device and start its worker thread.
 * Allocates per stream a batch object and a device staging buffer of
 * max_batch x max_points points, and max_outstanding pinned host slabs.
 * Errors: INVALID, OOM, CUDA. */
int tsdf_server_create(const tsdf_server_config* config, tsdf_server** out);

/* Stop the worker, wait for the device and free everything, including the
 * sessions' maps. Outstanding requests are dropped. NULL is ignored. */
int tsdf_server_destroy(tsdf_server* server);

/* Admit a session with a new map (params as for tsdf_map_create) if its memory
 * fits the remaining budget. Synchronous (allocates). Errors: ADMISSION (over
 * budget; retry after a session closes), INVALID, OOM, CUDA. */
int tsdf_server_open_session(tsdf_server* server, const tsdf_params* params, int32_t* session);

/* Close a session and free its map and budget. Errors: BUSY (requests not yet
 * waited for), INVALID. */
int tsdf_server_close_session(tsdf_server* server, int32_t session);

/* Queue a scan for a session: n <= max_points host float4 points (copied
 * before the call returns; points in pinned host memory mapped into the device
 * and 16-byte aligned are instead read in place by the batch and must stay
 * unchanged until tsdf_server_wait has returned for the ticket), a host
 * pose, and optionally a new window origin
 * (multiples of 8; the window is shifted before the scan is integrated).
 * Returns a ticket for tsdf_server_wait. Errors: BUSY (max_outstanding
 * requests not yet waited for), INVALID, or a previous worker error. */
int tsdf_server_submit(tsdf_server* server, int32_t session, const float* points_host, int64_t n,
                       const float pose[12], const int64_t* new_origin, uint64_t* ticket);

/* Submit `count` scans at once (no window shifts), in order, as
 * tsdf_server_submit with sessions[k], points_host[k], n[k], poses + 12 k,
 * writing tickets[k]. Stops at the first error, which it returns; *submitted
 * says how many were queued. */
int tsdf_server_submit_many(tsdf_server* server, int32_t count, const int32_t* sessions,
                            const float* const* points_host, const int64_t* n, const float* poses,
                            uint64_t* tickets, int32_t* submitted);

/* Wait up to timeout_us (negative: forever) for a request and take its
 * result (each ticket can be waited for once). Returns the request's status,
 * or TIMEOUT (the request is still pending), or INVALID (unknown ticket). */
int tsdf_server_wait(tsdf_server* server, uint64_t ticket, tsdf_request_result* out, int64_t timeout_us);

/* tsdf_server_wait for every ticket of tickets[0..count) in order (each with
 * timeout_us), results into out[0..count); out[i].status is the request's
 * status, or TIMEOUT / INVALID for a ticket that was not taken (a timed-out
 * ticket stays pending and can be waited for again). Returns TSDF_OK, or the
 * first non-OK status met. */
int tsdf_server_wait_many(tsdf_server* server, int32_t count, const uint64_t* tickets, tsdf_request_result* out,
                          int64_t timeout_us);

/* The session's map, for tsdf_read and tsdf_stats once all of its requests
 * have been waited for. Errors: INVALID. */
int tsdf_server_session_map(tsdf_server* server, int32_t session, tsdf_map** out);

/* Server-wide counters. Errors: INVALID. */
int tsdf_server_get_stats(tsdf_server* server, tsdf_server_stats* out);

/* ---- integration without device allocation ---------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory once they run: for example a real-time
 * mapping loop that reserves all of its memory at start-up (cudaMalloc may
 * synchronise the device and take unbounded time), or a process whose device
 * memory is owned by another allocator. It allocates nothing: it calls no
 * cudaMalloc or cudaFree and no allocating library routine. Its working memory
 * is one fixed file-scope device array of about 20 MiB (accumulators for up to
 * TSDF_STATIC_MAX_VOXELS voxels, per-ray data for up to TSDF_STATIC_MAX_POINTS
 * points, brick flags and list, counters) that every GPU which loads the
 * library keeps until the process exits. */
#define TSDF_STATIC_MAX_VOXELS  (1LL << 21)   /* window voxels (dims product) accepted */
#define TSDF_STATIC_MAX_POINTS  (1LL << 17)   /* points per call accepted (one 128 x 1024 scan) */

/* Integrate one scan into a caller-owned voxel grid, with the same result as
 * tsdf_integrate on a map with these parameters and origin.
 *   grid_dev   : device pointer, in/out, dims.x*dims.y*dims.z uint32 words in
 *                the layout tsdf_grid_device_ptr describes (value low 16 bits,
 *                weight high 16 bits, bricked, ring addressed); 16-byte
 *                aligned. All zero for an empty map.
 *   params     : window and method parameters; params->origin is the window
 *                origin (this call never shifts). dims product must not exceed
 *                TSDF_STATIC_MAX_VOXELS.
 *   points_dev : n float4 points as for tsdf_integrate; n <= TSDF_STATIC_MAX_POINTS.
 *   pose       : host, 12 floats, as for tsdf_integrate.
 *   stats_host : if not NULL, receives the scan's counters; the call then
 *                synchronises `stream`. If NULL the call is asynchronous.
 * Set-up: the first call on each device looks up the device address of the
 * scratch array (cudaGetSymbolAddress) with that device current, so make that
 * first call before any stream capture. The address is kept for the process:
 * after cudaDeviceReset (which unloads the library's device code) this entry
 * point must not be called again in that process.
 * The array keeps the last call's contents: each call clears the counters;
 * accumulators and brick flags are left all zero by every call that completes
 * and are cleared in full by the call that follows a failed one.
 * All calls share the one scratch array: calls that overlap on the GPU
 * (different streams, or different host threads, on one device) race and give
 * undefined results; serialise them.
 * Errors: INVALID (null or misaligned pointers, bad parameters, window larger
 * than TSDF_STATIC_MAX_VOXELS voxels, n < 0 or n > TSDF_STATIC_MAX_POINTS),
 * CUDA. */
int tsdf_integrate_static(uint32_t* grid_dev, const tsdf_params* params, const float* points_dev, int64_t n,
                          const float pose[12], tsdf_scan_stats* stats_host, void* stream);

/* Static description of an error code. Never NULL. */
const char* tsdf_error_string(int code);

/* The last CUDA error seen by the library on this host thread (cudaError_t
 * as int, 0 if none). */
int tsdf_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TSDF_GB300_H */
