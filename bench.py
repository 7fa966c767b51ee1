#!/usr/bin/env python
"""Benchmark of the TSDF integration path on the OS1-128-shaped outdoor sequence.

Workload (one step = one scan): 128 beams over [-22.5, 22.5] deg x 1024
azimuths = 131072 points per scan, range [0.5, 100] m, sigma 0.01 m, a seeded
outdoor scene (ground plane, 200 boxes, 50 cylinders), 100 scans at 10 Hz on a
seeded 1 m/s trajectory, a 512 x 512 x 128 window at 0.064 m with tau 0.6 m,
re-centred (ring-buffer shift) after each 1 m of motion. Steps walk the
100-scan sequence forward then backward (ping-pong), so the window keeps
shifting as a vehicle's would. A step is one tsdf_integrate call, preceded by
tsdf_shift when the window has to move.

Timing: all scans are resident in HBM before the timed region; L2 is flushed
before every timed step (a 512 MiB device write, then a 512 MiB read so that
the write's dirty lines are written back before the step) and the flush is
excluded by per-step CUDA events on the launching stream. Per-kernel times come from the
library's own events around each launch. The end-to-end figure goes through
tsdf_integrate_host from pinned host memory and reads the scan counters back
(tsdf_stats) every step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): one independent replica per rank (the path shards by
map; no collective on the data path); value = all ranks' voxel updates / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TSDF voxel updates/s (OS1-128-shaped scan)"
# DRAM bytes (read + write) per launch from the committed ncu summaries of these
# kernels on the outdoor workload, the default one (under profiles/); other
# workloads report none. Reset an entry to None whenever its kernel changes.
NCU_DRAM_BYTES = {"contrib": 13.201e6, "apply": 27.350e6, "rays": None}
UNIT = "voxel_updates/s"
N_SEQ = 100


class L2Flush:
    """Flush of the 129 MB L2 between timed steps: a 512 MiB device write, then
    a 512 MiB read of another buffer, so that the write's own dirty lines are
    written back before the step starts (a write alone leaves the L2 full of
    dirty lines whose eviction would land inside the next timed step)."""

    DESCRIPTION = ("flushed before every timed step: 512 MiB write, then a 512 MiB read so the flush's dirty lines "
                   "are written back before the step; flush excluded by per-step events")

    def __init__(self, torch, device):
        self.torch = torch
        self.w = torch.empty(512 << 20, dtype=torch.uint8, device=device)
        self.r = torch.ones(128 << 20, dtype=torch.float32, device=device)
        self.acc = torch.empty(1, dtype=torch.float32, device=device)

    def __call__(self):
        self.w.zero_()
        self.torch.sum(self.r, dim=0, keepdim=True, out=self.acc)


def ping_pong(n_steps: int, n: int = N_SEQ):
    """Scan indices 0..n-1, n-2..1, 0..n-1, ... of length n_steps."""
    period = 2 * n - 2
    out = []
    for s in range(n_steps):
        k = s % period
        out.append(k if k < n else period - k)
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.t0 = self.t1 = None
        cmd = ["nvidia-smi", f"--query-gpu=timestamp,{self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = []
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            rows.append(parts)
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, val in zip(names, r[6:10]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        # samples under load: the highest-clock half of the window (the timed
        # region is bracketed by idle host work)
        loaded = sorted(sm)[len(sm) // 2:] if sm else []
        return dict(sm_mhz=statistics.median(loaded) if loaded else None,
                    sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(rows))


# ---------------------------------------------------------------- oracle timing (CPU)

def oracle_sample(w, budget_s: float, stride: int = 1, order=None, threads: int = 0):
    """Time the oracle on scans of the sequence until `budget_s` is used.

    One oracle window per distinct window origin of the sequence, so no shift
    is needed (shifts are not part of this timed sample). threads > 0 splits
    each scan's rays over that many host threads (identical result). Returns
    (hits per second, scans used, hits, seconds)."""
    import oracle
    maps = {}
    hits = 0
    t_used = 0.0
    n_used = 0
    order = list(range(len(w.scans))) if order is None else order
    for i in order:
        o = tuple(w.origins[i])
        if o not in maps:
            maps[o] = oracle.OracleMap(dict(w.params, origin=o))
        pts = w.scans[i][::stride]
        t0 = time.perf_counter()
        maps[o].integrate(pts, w.poses[i], threads=threads)
        t_used += time.perf_counter() - t0
        hits += maps[o].stats()["hits"]
        n_used += 1
        if t_used >= budget_s:
            break
    return hits / max(t_used, 1e-9), n_used, hits, t_used


# ---------------------------------------------------------------- multi-rank aggregation

def aggregate_ranks(units, times, device=None):
    """Whole-job figures over the ranks of the default process group: the sum
    of each entry of `units` and the max of each entry of `times`. Without an
    initialised group (one process) the inputs are returned unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(units), list(times)
    u = torch.tensor(units, dtype=torch.float64, device=device)
    t = torch.tensor(times, dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return u.cpu().tolist(), t.cpu().tolist()


# ---------------------------------------------------------------- main GPU arm

def sequence_workload(name: str):
    """The scan sequence of a per-map workload and its description."""
    from paper_2310_05766_gb300 import synth
    if name == "corridor":
        w = synth.workload_corridor(n_scans=50)
        return w, ("high-resolution corridor: 128x2048 beams, 50 scans at 10 Hz, 0.5 m/s, window 1024x1024x256 "
                   "at 0.02 m (1 GiB grid), tau 0.1 m, shift every 0.5 m (ping-pong over the sequence)")
    w = synth.workload_outdoor(n_scans=N_SEQ)
    return w, ("outdoor OS1-128 sequence: 128x1024 beams, 100 scans at 10 Hz, 1 m/s, window 512x512x128 at "
               "0.064 m, tau 0.6 m, shift every 1 m (ping-pong over the sequence)")


def run_gpu(args, rank: int, world: int, local_rank: int):
    import torch
    from paper_2310_05766_gb300 import binding as b, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    b.lib()
    w, wdesc = sequence_workload(args.workload)
    n_seq = len(w.scans)
    p = w.params
    scans_dev = [torch.from_numpy(s).to(dev) for s in w.scans]
    scans_pin = [torch.from_numpy(s).pin_memory() for s in w.scans]
    flush = L2Flush(torch, dev)
    stream = torch.cuda.current_stream(dev)

    m = b.TsdfMap(p)
    h = m.handle
    sort = args.reduction == "sort"
    red_opt = {"atomic": None, "sort": b.TSDF_REDUCTION_SORT, "pool": b.TSDF_REDUCTION_POOL}[args.reduction]
    for opt, val in ((b.TSDF_OPT_WARP_MERGE, args.merge), (b.TSDF_OPT_STEPS_PER_THREAD, args.kpt),
                     (b.TSDF_OPT_PDL, args.pdl), (b.TSDF_OPT_REDUCTION, red_opt),
                     (b.TSDF_OPT_HOST_ZERO_COPY, args.zero_copy),
                     (b.TSDF_OPT_LAUNCH_GRAPH, getattr(args, "graph", None))):
        if val is not None:
            b.tsdf_set_option(h, opt, val)
    cur = tuple(p["origin"])
    origins = [tuple(int(v) for v in o) for o in w.origins]   # (outside the timed steps)

    def step(i, host=False):
        nonlocal cur
        o = origins[i]
        if o != cur:
            b.tsdf_shift(h, o, stream)
            cur = o
        if host:
            b.tsdf_integrate_host(h, scans_pin[i].data_ptr(), scans_pin[i].shape[0], w.poses[i], stream)
        else:
            b.tsdf_integrate(h, scans_dev[i], scans_dev[i].shape[0], w.poses[i], stream)

    # per-scan counters (they depend only on the scan, its pose and the window origin)
    hits = np.zeros(n_seq, np.int64)
    touched = np.zeros(n_seq, np.int64)
    for i in range(n_seq):
        step(i)
        st = b.tsdf_stats(h, stream)
        hits[i], touched[i] = st["hits"], st["touched"]

    schedule = ping_pong(args.warmup + args.steps, n_seq)
    for i in schedule[:args.warmup]:
        step(i)
    torch.cuda.synchronize()

    timed = schedule[args.warmup:]
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in timed]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in timed]
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid) if rank == 0 else None

    def timed_pass(profile: bool):
        """K steps, L2 flushed before each, each step bracketed by events.
        With profile=True the library also records events around each kernel
        (which serialises the kernels of a step: headline timing uses False)."""
        b.tsdf_profile_enable(h, profile)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, i in enumerate(timed):
            flush()
            ev0[k].record(stream)
            step(i)
            ev1[k].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t0
        if world > 1:
            torch.distributed.barrier()
        prof = b.tsdf_profile_read(h) if profile else None
        b.tsdf_profile_enable(h, False)
        return [ev0[k].elapsed_time(ev1[k]) for k in range(len(timed))], t_wall, prof

    if clocks:
        clocks.mark_start()
    step_ms, t_wall, _ = timed_pass(False)          # headline: no per-kernel events
    if clocks:
        clocks.mark_end()
    # the sampler stops with the timed region: its nvidia-smi queries share the
    # driver with the host calls that the end-to-end steps below time
    clk = clocks.stop() if clocks else None
    prof_step_ms, _, prof = timed_pass(True)        # same steps again, per-kernel events on
    dev_ms = float(sum(step_ms))
    hits_timed = int(sum(hits[i] for i in timed))
    touched_timed = int(sum(touched[i] for i in timed))
    n_shift_timed = prof.get("shift", (0, 0.0))[0]

    # ---- end to end through host buffers (pinned), counters read back each step;
    # at least 200 steps of the ping-pong schedule (one in ten shifts the window),
    # so that the figure does not hang on two or three shifts
    n_e2e = max(min(len(timed), 400), 200)
    e2e_sched = ping_pong(args.warmup + n_e2e, n_seq)[args.warmup:]
    t_e2e = 0.0
    for i in e2e_sched:
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(i, host=True)
        b.tsdf_stats(h, stream)
        t_e2e += time.perf_counter() - t0
    e2e_hits = int(sum(hits[i] for i in e2e_sched))
    map_bytes = b.tsdf_map_device_bytes(h)
    m.close()

    # ---- reduce over ranks: total units / slowest rank
    (hits_all, e2e_hits_all), (dev_ms_max, t_e2e_max) = aggregate_ranks(
        [float(hits_timed), float(e2e_hits)], [dev_ms, t_e2e], dev if world > 1 else None)
    if rank != 0:
        return None

    value = hits_all / (dev_ms_max / 1e3)
    K = len(timed)
    # roofline of the dominant kernel
    peak, peak_kind = peaks()
    n_pts = scans_dev[0].shape[0]
    # (the sort group -- compaction, count, prefix, scatter -- only reorders
    # contributions and has no algorithmic bytes of its own)
    kern = max(((k, v) for k, v in prof.items() if k in ("contrib", "emit", "apply")), key=lambda kv: kv[1][1])
    kname, (klaunch, kms) = kern

    def hbm_fig(name):
        """HBM figure of one kernel with the algorithmic bytes it owns: the
        march reads the scan's points (16 B each), the apply read-modify-writes
        the grid (4 + 4 B per touched voxel)."""
        if name not in prof:
            return None
        nl, ms = prof[name]
        alg = (16.0 * n_pts * K if name in ("contrib", "emit", "rays") else 8.0 * touched_timed) / nl
        ach = alg / (ms / nl / 1e3) / 1e9
        return dict(kernel=name, achieved=ach, peak=peak, unit="GB/s", frac=ach / peak,
                    peak_source=f"{peak_kind} hbm_gbs",
                    alg_bytes_def=("16 B per point of the scan" if name in ("contrib", "emit", "rays")
                                   else "8 B per touched voxel (grid read-modify-write)"),
                    alg_bytes_per_launch=alg, avg_launch_us=1e3 * ms / nl,
                    traffic=(NCU_DRAM_BYTES.get(name) if args.reduction == "atomic" and args.workload == "outdoor"
                             else None))
    # the binding roofline of the contribution kernel: its 64-bit L2
    # reductions (one per in-window contribution) against the rate the
    # reduction probe measures in this run
    l2red = None
    if "contrib" in prof:
        rate_coal = b.tsdf_probe_reduction_rate(0, stream)
        rate_scat = b.tsdf_probe_reduction_rate(1, stream)
        c_launch, c_ms = prof["contrib"]
        red_rate = hits_timed / (c_ms / 1e3) if c_launch == K else float("nan")
        l2red = dict(kernel="contrib", bound="l2_reduction", achieved=red_rate, peak=rate_scat,
                     unit="reductions/s", frac=red_rate / rate_scat,
                     peak_coalesced=rate_coal, peak_scattered=rate_scat,
                     frac_coalesced=red_rate / rate_coal, frac_scattered=red_rate / rate_scat,
                     avg_launch_us=1e3 * c_ms / c_launch,
                     peak_source="tsdf_probe_reduction_rate, measured in this run (64-bit red.add into a 64 MiB "
                                 "L2-resident buffer, GPU-filling grid; scattered: every lane its own hashed word)",
                     traffic=(NCU_DRAM_BYTES.get("contrib") if args.reduction == "atomic" and args.workload == "outdoor"
                              else None))
    if l2red is not None:
        roof = dict(l2red)
        roof["hbm"] = hbm_fig("contrib")
        roof["apply_hbm"] = hbm_fig("apply")
    else:
        roof = hbm_fig(kname)
        roof["bound"] = "hbm"
    kernels = {k: dict(launches=v[0], total_ms=round(v[1], 4), avg_us=round(1e3 * v[1] / v[0], 3),
                       share=round(v[1] / sum(x[1] for x in prof.values()), 4)) for k, v in prof.items()}

    cpu = cpu_par = None
    if world == 1 and not args.no_cpu_baseline:
        rate, n_used, h_used, t_used = oracle_sample(w, args.cpu_budget)
        cpu = dict(value=rate, unit=UNIT, cores=1, kind="oracle",
                   sample=f"first {n_used} scans of the {n_seq}-scan sequence, all {n_pts} points each, "
                          f"{h_used} voxel updates in {t_used:.1f} s, single-threaded C++ oracle; "
                          f"window re-centring by pre-placed oracle windows (shift not timed)")
        nthr = os.cpu_count() or 1
        prate, pn, ph, pt = oracle_sample(w, args.cpu_budget, threads=nthr)
        cpu_par = dict(value=prate, unit=UNIT, cores=nthr, kind="oracle, rays split over host threads",
                       sample=f"first {pn} scans, {ph} voxel updates in {pt:.1f} s on {nthr} threads "
                              f"(per-thread per-scan volumes merged exactly; same result as the serial oracle)")

    out = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=K, warmup=args.warmup,
        ms_per_step=dev_ms_max / K, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32 geometry, int64 accumulation, int16 map", data="synthetic",
        config=dict(workload=wdesc, seed=w.meta.get("seed"),
                    points_per_scan=int(n_pts), voxel_size=p["voxel_size"], tau=p["tau"], dims=list(p["dims"]),
                    reduce="WSUM", reduction=args.reduction, map_device_bytes=map_bytes, l2=L2Flush.DESCRIPTION,
                    parallelism=f"replicas x{world}"),
        scans_per_s=K * world / (dev_ms_max / 1e3),
        us_per_scan=dict(mean=1e3 * dev_ms_max / K, p50=1e3 * float(np.percentile(step_ms, 50)),
                         p99=1e3 * float(np.percentile(step_ms, 99))),
        applied_updates_per_s=touched_timed * world / (dev_ms_max / 1e3),
        hits_per_scan=hits_timed / K, touched_per_scan=touched_timed / K, shifts_timed=int(n_shift_timed),
        kernels=kernels,
        kernels_note="per-kernel times from a second pass over the same timed steps with library events around "
                     "each kernel (that pass: %.1f us/scan; events serialise the kernels of a step)" %
                     (1e3 * float(sum(prof_step_ms)) / K),
        roofline=roof,
        e2e=dict(value=e2e_hits_all / t_e2e_max, unit=UNIT, h2d_bytes_per_step=int(16 * n_pts),
                 d2h_bytes_per_step=24, steps=n_e2e,
                 zero_copy=args.zero_copy != 0,
                 note="tsdf_integrate_host from pinned memory (read in place by the first kernel over the host "
                      "link unless --zero-copy 0) + tsdf_stats read-back, host wall clock"),
        # library launches: one per profiled entry, plus the compaction that shares
        # the apply entry (atomic) or compact + count + prefix + scatter sharing
        # the sort entry (sort); the pool reduction has no compaction
        gpu_launches=int(sum(v[0] for v in prof.values()) +
                         {"atomic": 1, "sort": 3, "pool": 0}[args.reduction] * K),
        clocks=clk,
        wall_s_timed=t_wall,
        cpu_baseline=cpu,
        cpu_baseline_parallel=cpu_par,
    )
    return out


# ---------------------------------------------------------------- the other configured workloads

def run_room_bench(steps: int = 200):
    """Box room, one 16 x 360 scan into a 256 x 256 x 64 window at 0.05 m: the
    same scan integrated `steps` times, L2 flushed before each, per-step events
    (a latency-bound workload: reported in microseconds per scan)."""
    import torch
    from paper_2310_05766_gb300 import binding as b, synth
    w = synth.workload_room()
    pts = torch.from_numpy(w.scans[0]).cuda()
    flush = L2Flush(torch, "cuda")
    stream = torch.cuda.current_stream()
    m = b.TsdfMap(w.params)
    try:
        b.tsdf_integrate(m.handle, pts, pts.shape[0], w.poses[0], stream)
        hits = m.stats()["hits"]
        for _ in range(10):
            b.tsdf_integrate(m.handle, pts, pts.shape[0], w.poses[0], stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for e0, e1 in ev:
            flush()
            e0.record(stream)
            b.tsdf_integrate(m.handle, pts, pts.shape[0], w.poses[0], stream)
            e1.record(stream)
        torch.cuda.synchronize()
        us = np.array([1e3 * e0.elapsed_time(e1) for e0, e1 in ev])
    finally:
        m.close()
    return dict(workload="box room: 16 x 360 beams (5760 points), 256x256x64 window at 0.05 m, tau 0.2 m, "
                         "the same scan integrated every step",
                seed=1, steps=steps, us_per_scan=dict(mean=float(us.mean()), p50=float(np.percentile(us, 50)),
                                              p99=float(np.percentile(us, 99))),
                scans_per_s=1e6 / float(us.mean()), voxel_updates_per_s=hits / (float(us.mean()) / 1e6),
                hits_per_scan=hits, note="latency-bound (a few microseconds of work per scan); not judged by roofline")


def run_drive_bench(n_pos: int = 1000, file_host_chunks=None):
    """A 1 km drive of the outdoor window (512 x 512 x 128 at 0.064 m), a scan and
    a shift every metre: the global store's device tier fills to its limit (the
    window's brick count) and the oldest chunks move to pinned host memory.
    Reports the shift's host time and device time (events on the stream) and
    the map's device memory. Scans: the first 20 of the outdoor sequence, each
    placed at the next metre (a synthetic drive, not a ray-cast of a 1 km scene).
    With `file_host_chunks` the store has a file tier (a scratch file in the
    temporary directory) behind a host tier of that many chunks, and the drive
    goes n_pos / 2 metres out and the same way back, so that chunks are both
    written to and read back from the file."""
    import tempfile
    import torch
    from paper_2310_05766_gb300 import binding as b, synth
    w = synth.workload_outdoor(n_scans=20)
    pts = [torch.from_numpy(x).cuda() for x in w.scans]
    dims, vs = w.params["dims"], w.params["voxel_size"]
    stream = torch.cuda.current_stream()
    m = b.TsdfMap(w.params)
    host_us, dev_us, dev_bytes = [], [], []
    tmpdir = tempfile.TemporaryDirectory() if file_host_chunks is not None else None
    try:
        if tmpdir is not None:
            b.tsdf_map_set_store_file(m.handle, os.path.join(tmpdir.name, "store.bin"), file_host_chunks)
        cur = tuple(w.params["origin"])
        for k in range(n_pos):
            j = k % len(pts)
            pose = np.array(w.poses[j], np.float32).reshape(3, 4).copy()
            x = float(k) if tmpdir is None or k < n_pos // 2 else float(n_pos - 1 - k)
            pose[:, 3] = (x, 0.0, 0.0)
            o = synth.window_origin(pose[:, 3].astype(np.float64), dims, vs)
            if o != cur:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                t0 = time.perf_counter()
                b.tsdf_shift(m.handle, o, stream)
                host_us.append(1e6 * (time.perf_counter() - t0))
                e1.record(stream)
                torch.cuda.synchronize()
                dev_us.append(1e3 * e0.elapsed_time(e1))
                dev_bytes.append(b.tsdf_map_device_bytes(m.handle))
                cur = o
            b.tsdf_integrate(m.handle, pts[j], pts[j].shape[0], pose.reshape(12), stream)
        torch.cuda.synchronize()
        st = b.tsdf_get_store_stats(m.handle)
    finally:
        m.close()
        if tmpdir is not None:
            tmpdir.cleanup()
    pct = lambda v, q: float(np.percentile(v, q))
    if tmpdir is None:
        wl = ("1 km drive, window 512x512x128 at 0.064 m, a scan (128x1024) and a 1 m shift every metre; "
              "store device tier limited to the window's brick count, the rest in pinned host memory")
    else:
        wl = (f"{n_pos // 2} m out and back, window 512x512x128 at 0.064 m, a scan (128x1024) and a 1 m shift every "
              f"metre; store device tier limited to the window's brick count, host tier to {file_host_chunks} chunks "
              f"at each shift, the rest in a scratch file (temporary directory) written by the map's writer thread")
    return dict(workload=wl,
                seed=w.meta.get("seed"),
                shifts=len(host_us), shift_host_us=dict(p50=pct(host_us, 50), p99=pct(host_us, 99), mean=float(np.mean(host_us))),
                shift_device_us=dict(p50=pct(dev_us, 50), p99=pct(dev_us, 99), mean=float(np.mean(dev_us)),
                                     note="from the start event to the end of the shift kernel, including its host time"),
                map_device_bytes=dict(first=dev_bytes[0], max=max(dev_bytes), last=dev_bytes[-1]),
                store=st)


def run_configs(args):
    """The configured workloads besides the headline one, each short, as
    sub-records of the default line: box room (us per scan), the 64-map batch
    against 64 plain calls, the high-resolution corridor, a 1 km drive through
    the global store's device and host tiers and a drive out and back through
    its file tier (shift latency), and a 32-session serving run at
    Poisson 500 scans/s (p50 / p99 latency)."""
    import copy
    out = {}
    out["room"] = run_room_bench(200)
    a = copy.copy(args)
    a.workload, a.steps, a.warmup, a.no_cpu_baseline = "corridor", 100, 5, True
    c = run_gpu(a, 0, 1, 0)
    out["corridor"] = dict(workload=c["config"]["workload"], seed=c["config"].get("seed"), steps=c["steps"], value=c["value"], unit=c["unit"],
                           us_per_scan=c["us_per_scan"], scans_per_s=c["scans_per_s"],
                           hits_per_scan=c["hits_per_scan"], contrib_avg_us=c["kernels"]["contrib"]["avg_us"],
                           l2_reductions_frac_scattered=c["roofline"].get("frac_scattered"),
                           e2e=c["e2e"]["value"], map_device_bytes=c["config"]["map_device_bytes"])
    if not args.no_cpu_baseline:
        # the single-threaded oracle per scan beside the GPU figures (room: its
        # one scan; corridor: its first scans, about a second of host time)
        from paper_2310_05766_gb300 import synth
        for key, wk, budget in (("room", synth.workload_room(), 0.0),
                                ("corridor", synth.workload_corridor(n_scans=3), 1.0)):
            rate, n_used, hits, t = oracle_sample(wk, budget)
            out[key]["cpu_baseline"] = dict(value=rate, unit=UNIT, cores=1, kind="oracle",
                                            ms_per_scan=1e3 * t / n_used,
                                            sample=f"first {n_used} scan(s) of the workload, {hits} voxel updates "
                                                   f"in {t:.2f} s, single-threaded C++ oracle")
    a = copy.copy(args)
    a.steps, a.warmup = 20, 16
    bt = run_batch_bench(a)
    out["batch"] = dict(workload=bt["config"]["workload"], seed=bt["config"].get("seed"), steps=bt["steps"], ms_per_batch=bt["ms_per_step"],
                        value=bt["value"], unit=bt["unit"], scans_per_s=bt["scans_per_s"],
                        plain_ms_per_64_scans=bt["plain_per_scan_launches"]["ms_per_step"],
                        speedup_vs_plain=bt["batch_speedup_vs_plain"], tuned_config=bt["config"]["tuned_config"])
    out["drive"] = run_drive_bench(1000)
    out["drive_file_tier"] = run_drive_bench(500, file_host_chunks=16384)
    a = copy.copy(args)
    a.serve_seconds, a.serve_rate, a.serve_pinned = 6.0, 500.0, 1
    sv = run_serving_bench(a)
    out["serving"] = dict(workload=sv["config"]["workload"], requests=sv["steps"], scans_per_s=sv["value"],
                          p50_ms=sv["latency_ms"]["p50"], p99_ms=sv["latency_ms"]["p99"],
                          mean_ms=sv["latency_ms"]["mean"], voxel_updates_per_s=sv["voxel_updates_per_s"],
                          mean_batch=sv["mean_batch"], sessions=sv["sessions"])
    # the same sessions saturated (every request due at once, bursts of 1024
    # outstanding): where continuous batching shows
    a = copy.copy(args)
    a.serve_seconds, a.serve_rate, a.serve_pinned = 2.0, 0.0, 1
    ss = run_serving_bench(a)
    out["serving_saturated"] = dict(workload=ss["config"]["workload"], requests=ss["steps"], scans_per_s=ss["value"],
                                    p50_ms=ss["latency_ms"]["p50"], p99_ms=ss["latency_ms"]["p99"],
                                    voxel_updates_per_s=ss["voxel_updates_per_s"], mean_batch=ss["mean_batch"])
    return out


# ---------------------------------------------------------------- reference arm (the oracle)

def run_reference(args, rank: int, world: int):
    if rank != 0:
        return None
    from paper_2310_05766_gb300 import synth
    import oracle
    w = synth.workload_outdoor(n_scans=N_SEQ)
    schedule = ping_pong(args.warmup + args.steps)
    # calibrate one full scan, then pick a point stride that keeps the run near the budget
    rate, _, _, t_full = oracle_sample(w, 0.0)
    per_step = args.ref_budget / max(1, len(schedule))
    stride = max(1, int(math.ceil(t_full / per_step)))
    maps = {}

    def one(i):
        o = tuple(w.origins[i])
        if o not in maps:
            maps[o] = oracle.OracleMap(dict(w.params, origin=o))
        t0 = time.perf_counter()
        maps[o].integrate(w.scans[i][::stride], w.poses[i])
        dt = time.perf_counter() - t0
        return maps[o].stats()["hits"], dt

    for i in schedule[:args.warmup]:
        one(i)
    hits = 0
    t = 0.0
    for i in schedule[args.warmup:]:
        h, dt = one(i)
        hits += h
        t += dt
    K = len(schedule) - args.warmup
    value = hits / max(t, 1e-9)
    sample = (f"every {stride}th point of each scan ({131072 // stride} of 131072), one scan per step in "
              f"ping-pong order over the 100-scan sequence, single-threaded C++ oracle; window re-centring "
              f"by pre-placed oracle windows (shift not timed)")
    return dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=K, warmup=args.warmup,
                ms_per_step=1e3 * t / K, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32 geometry, int64 accumulation, int16 map", data="synthetic", impl="reference",
                config=dict(workload="outdoor OS1-128 sequence: 128x1024 beams, 100 scans at 10 Hz, 1 m/s, "
                                     "window 512x512x128 at 0.064 m, tau 0.6 m, shift every 1 m (ping-pong over the sequence)",
                            seed=2, points_per_step=131072 // stride, parallelism="host cores"),
                cpu_baseline=dict(kind="oracle", cores=1, sample=sample, value=value, unit=UNIT),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))


# ---------------------------------------------------------------- batched workload (64 maps)

def run_batch_bench(args):
    """64 maps, one scan each (beams {16,32,64,128} x azimuths {512,1024,2048},
    grids 256^3 / 512x512x128 at 0.064 m, tau 0.6 m): one batched launch per step
    (graph replay, autotuned) against 64 plain tsdf_integrate calls per step, with
    L2 flushed before every step and excluded by per-step events."""
    import torch
    from paper_2310_05766_gb300 import binding as b, synth
    torch.cuda.set_device(0)
    b.lib()
    ws = synth.workload_batch(n_maps=64, seed=3)
    pts = [torch.from_numpy(w.scans[0]).cuda() for w in ws]
    poses = [w.poses[0] for w in ws]
    maps = [b.TsdfMap(w.params) for w in ws]
    flush = L2Flush(torch, "cuda")
    stream = torch.cuda.current_stream()
    batch = b.tsdf_batch_create(64)
    hits = 0
    for m, p_, pose in zip(maps, pts, poses):
        m.integrate(p_, pose)
        hits += m.stats()["hits"]

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for e0, e1 in ev:
            flush()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in ev]

    def plain():
        for m, p_, pose in zip(maps, pts, poses):
            b.tsdf_integrate(m.handle, p_, p_.shape[0], pose, stream)

    def batched():
        b.tsdf_batch_integrate(batch, maps, pts, poses, stream)

    for _ in range(max(args.warmup, 16)):
        batched()
    # the autotuner's trials (each configuration timed twice) end before the
    # timed steps: they are not part of the steady state being measured
    for _ in range(200):
        assert b.tsdf_batch_sync(batch, stream) == b.TSDF_OK
        if b.tsdf_batch_get_config(batch)["tuned"]:
            break
        batched()
    for _ in range(3):
        batched()
    assert b.tsdf_batch_sync(batch, stream) == b.TSDF_OK
    plain()
    K = max(10, min(args.steps, 200))
    t_plain = timed(plain, K)
    t_batch = timed(batched, K)
    cfg = b.tsdf_batch_get_config(batch)
    b.tsdf_batch_destroy(batch)
    for m in maps:
        m.close()
    ms_b = float(np.mean(t_batch))
    ms_p = float(np.mean(t_plain))
    return dict(metric="TSDF voxel updates/s, 64-map batch (one persistent launch, graph replay)",
                value=hits / (ms_b / 1e3), unit=UNIT, n_gpus=1, steps=K, warmup=args.warmup, ms_per_step=ms_b,
                higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32 geometry, int64 accumulation, int16 map", data="synthetic",
                config=dict(workload="64 maps, beams {16,32,64,128} x azimuths {512,1024,2048}, grids 256^3 / "
                                     "512x512x128 at 0.064 m, tau 0.6 m, one scan per map per step",
                            seed=3, l2=L2Flush.DESCRIPTION, tuned_config=cfg),
                scans_per_s=64 / (ms_b / 1e3), plain_per_scan_launches=dict(ms_per_step=ms_p, value=hits / (ms_p / 1e3)),
                batch_speedup_vs_plain=ms_p / ms_b, hits_per_step=hits)


# ---------------------------------------------------------------- serving workload (32 sessions)

def run_serving_bench(args):
    """32 sessions (grids 256^3 / 512x512x128, voxel 0.05-0.1 m, tau 0.2-0.6 m),
    Poisson arrivals at an aggregate 500 scans/s with scan sizes {16,32,64,128} x
    {1024,2048}, 20 s, the first 2 s discarded; HBM budget 120 GB."""
    import threading
    import torch
    from paper_2310_05766_gb300 import binding as b, synth
    torch.cuda.set_device(0)
    b.lib()
    duration = args.serve_seconds
    sess = synth.serving_sessions(32, seed=100)
    rng = synth.SplitMix64(777)
    scans = []
    for i, sp in enumerate(sess):
        beams = [16, 32, 64, 128][int(rng.integers(1, 0, 4)[0])]
        az = [1024, 2048][int(rng.integers(1, 0, 2)[0])]
        w = synth.workload_outdoor(n_scans=2, seed=sp["seed"], beams=beams, azimuths=az, dims=sp["dims"],
                                   voxel_size=sp["voxel_size"], tau=sp["tau"])
        if args.serve_pinned:   # points in pinned host memory: the server reads them in place
            w.scans = [torch.from_numpy(x).pin_memory() for x in w.scans]
        scans.append(w)
    srv = b.tsdf_server_create(hbm_budget_bytes=120 * 10**9, max_points=128 * 2048, max_batch=32, streams=2,
                               max_outstanding=1024)
    sids = [b.tsdf_server_open_session(srv, w.params) for w in scans]
    rate = args.serve_rate
    if rate > 0:
        times, who = synth.poisson_arrivals(rate, duration, 32, seed=101)
    else:
        # saturation: every request is due at once (submitted as fast as the
        # server's back-pressure allows); sessions drawn like the arrivals
        _, who = synth.poisson_arrivals(20000.0, duration, 32, seed=101)
        times = np.zeros(len(who))
    # everything a request needs is laid out before the run (pointers, sizes,
    # sessions, poses; result buffers), so that each burst of submissions or
    # waits is a single library call
    import ctypes
    nreq = len(who)
    ptr = np.array([(scans[who[i]].scans[i % 2].data_ptr() if args.serve_pinned else
                     scans[who[i]].scans[i % 2].ctypes.data) for i in range(nreq)], np.uint64)
    nn = np.array([scans[who[i]].scans[i % 2].shape[0] for i in range(nreq)], np.int64)
    ses = np.array([sids[who[i]] for i in range(nreq)], np.int32)
    pz = np.ascontiguousarray(np.stack([np.asarray(scans[who[i]].poses[i % 2], np.float32).reshape(12)
                                        for i in range(nreq)]), np.float32)
    tk = np.zeros(nreq, np.uint64)
    res = (b.tsdf_request_result * nreq)()
    L = b.lib()
    P = ctypes.POINTER
    submitted = [0]
    done_flag = [False]

    def submitter():
        t0 = time.perf_counter()
        k = 0
        done = ctypes.c_int32()
        while k < nreq:
            now = time.perf_counter() - t0
            if times[k] > now:
                time.sleep(min(times[k] - now, 0.0005))
                continue
            e = int(np.searchsorted(times, now, side="right"))
            e = max(k + 1, min(e, k + 256))
            rc = L.tsdf_server_submit_many(
                srv, e - k, ses[k:].ctypes.data_as(P(ctypes.c_int32)), ptr[k:].ctypes.data_as(P(ctypes.c_void_p)),
                nn[k:].ctypes.data_as(P(ctypes.c_int64)), pz[k:].ctypes.data_as(P(ctypes.c_float)),
                tk[k:].ctypes.data_as(P(ctypes.c_uint64)), ctypes.byref(done))
            if rc not in (b.TSDF_OK, b.TSDF_ERR_BUSY):
                raise b.TsdfError(rc, "tsdf_server_submit_many")
            k += done.value
            submitted[0] = k
            if rc == b.TSDF_ERR_BUSY:
                time.sleep(0.0002)   # back-pressure: results must be taken first
        done_flag[0] = True

    def collector():
        i = 0
        while i < nreq:
            avail = submitted[0]
            if avail <= i:
                time.sleep(0.0002)
                continue
            cnt = min(avail - i, 256)
            rc = L.tsdf_server_wait_many(srv, cnt, tk[i:].ctypes.data_as(P(ctypes.c_uint64)),
                                         ctypes.cast(ctypes.addressof(res) + i * ctypes.sizeof(b.tsdf_request_result),
                                                     P(b.tsdf_request_result)), -1)
            if rc != b.TSDF_OK:
                raise b.TsdfError(rc, "tsdf_server_wait_many")
            i += cnt

    if rate > 0:
        th_s = threading.Thread(target=submitter)
        th_c = threading.Thread(target=collector)
        th_s.start()
        th_c.start()
        th_s.join()
        th_c.join()
    else:
        # saturation, closed loop: fill the server's window of outstanding
        # requests with one call, wait for all of them with one call, repeat
        done = ctypes.c_int32()
        k = 0
        while k < nreq:
            cnt = min(1024, nreq - k)
            rc = L.tsdf_server_submit_many(
                srv, cnt, ses[k:].ctypes.data_as(P(ctypes.c_int32)), ptr[k:].ctypes.data_as(P(ctypes.c_void_p)),
                nn[k:].ctypes.data_as(P(ctypes.c_int64)), pz[k:].ctypes.data_as(P(ctypes.c_float)),
                tk[k:].ctypes.data_as(P(ctypes.c_uint64)), ctypes.byref(done))
            if rc not in (b.TSDF_OK, b.TSDF_ERR_BUSY) or done.value == 0:
                raise b.TsdfError(rc, "tsdf_server_submit_many")
            rc = L.tsdf_server_wait_many(srv, done.value, tk[k:].ctypes.data_as(P(ctypes.c_uint64)),
                                         ctypes.cast(ctypes.addressof(res) + k * ctypes.sizeof(b.tsdf_request_result),
                                                     P(b.tsdf_request_result)), -1)
            if rc != b.TSDF_OK:
                raise b.TsdfError(rc, "tsdf_server_wait_many")
            k += done.value
    st = b.tsdf_server_get_stats(srv)
    b.tsdf_server_destroy(srv)
    results = [(float(times[i]), b._result_dict(res[i])) for i in range(nreq)]
    # steady state: arrivals after the first 2 s (at most a fifth of the run;
    # saturation: all but the first 10 % of the requests)
    if rate > 0:
        skip = min(2.0, 0.2 * duration)
        keep = [r for ta, r in results if ta >= skip]
    else:
        keep = [r for _, r in results[len(results) // 10:]]
    lat = np.array([r["t_done_us"] - r["t_submit_us"] for r in keep])
    hits = sum(r["stats"]["hits"] for r in keep)
    span = (max(r["t_done_us"] for r in keep) - min(r["t_submit_us"] for r in keep)) / 1e6
    load = ("Poisson %g scans/s" % rate if rate > 0 else
            "saturating closed loop (bursts of 1024 requests submitted at once, then waited for)")
    return dict(metric="served scan latency (p50 / p99) and throughput, 32 sessions, " + load,
                value=len(keep) / span, unit="scans/s", n_gpus=1, steps=len(keep), warmup=0,
                ms_per_step=float(np.mean(lat)) / 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32 geometry, int64 accumulation, int16 map", data="synthetic",
                config=dict(workload="32 sessions, grids 256^3 / 512x512x128, voxel 0.05-0.1 m, tau 0.2-0.6 m, "
                                     "%s, scans {16,32,64,128} x {1024,2048}, %g s of arrivals, warm-up discarded, "
                                     "HBM budget 120 GB, 2 streams, batches up to 32, scans %s" %
                                     (load, duration, "pinned (read in place)" if args.serve_pinned else
                                      "pageable (copied at submission)"),
                            seeds=dict(sessions=100, arrivals=101)),
                latency_ms=dict(p50=float(np.percentile(lat, 50)) / 1e3, p99=float(np.percentile(lat, 99)) / 1e3,
                                mean=float(np.mean(lat)) / 1e3, max=float(np.max(lat)) / 1e3),
                voxel_updates_per_s=hits / span, mean_batch=st["mean_batch"], batches=st["batches"],
                sessions=st["sessions"], used_bytes=st["used_bytes"])


def spawn_ranks(n: int, argv) -> int:
    """Re-run this script as n ranks on one node (torch.distributed.run, one
    process per GPU, rendezvous on 127.0.0.1); returns the launcher's exit
    code. Each rank then reads RANK / LOCAL_RANK / WORLD_SIZE."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--merge", type=int, default=None, help="tuning: warp match-merge (0/1)")
    ap.add_argument("--kpt", type=int, default=None, help="tuning: march steps per contribution thread (1/2/4)")
    ap.add_argument("--pdl", type=int, default=None, help="tuning: programmatic dependent launch (0/1)")
    ap.add_argument("--graph", type=int, default=None,
                    help="tuning: one graph launch per scan (1) or four kernel launches (0, library default)")
    ap.add_argument("--zero-copy", type=int, default=None,
                    help="e2e: pinned host points read in place (1, library default) or staged (0)")
    ap.add_argument("--reduction", default="atomic", choices=["atomic", "sort", "pool"],
                    help="per-scan reduction: accumulator atomics or counting sort by brick")
    ap.add_argument("--workload", default="outdoor", choices=["outdoor", "corridor", "batch", "serving"],
                    help="outdoor: the headline sequence; batch / serving: the 64-map batch and 32-session serving runs")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-rate", type=float, default=500.0,
                    help="serving: aggregate Poisson arrival rate, scans/s (0: saturating closed loop)")
    ap.add_argument("--serve-pinned", type=int, default=1,
                    help="serving: scans in pinned host memory read in place (1) or pageable, copied (0)")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="headline workload only (skip the room, batch, corridor and serving sub-records)")
    ap.add_argument("--cpu-budget", type=float, default=10.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=120.0, help="seconds of oracle time for --impl reference")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: run this same command under torch.distributed.run
        sys.exit(spawn_ranks(args.gpus, sys.argv[1:]))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "batch":
        out = run_batch_bench(args) if rank == 0 else None
    elif args.workload == "serving":
        out = run_serving_bench(args) if rank == 0 else None
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        out = run_gpu(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        elif args.workload == "outdoor" and not args.no_extra_configs and out is not None:
            out["configs"] = run_configs(args)
    if out is not None and rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
