#!/usr/bin/env python
"""Throughput of the CUDA TPC sector tracker on the central-like workload.

The workload is the central-like event (16000 primaries + 3000 secondaries, 20 % noise, 36
sectors x 159 rows, about 3.3 M clusters) through every stage of the hot path: ingest and
per-row grids, neighbours finder, evolution and start hits, tracklet construction,
selection, output in canonical order.

value: one step = one call tracking --events-per-call (3) central-like events in one pass
of every stage (tpc_track_batch); --inflight (2) calls are on the device at once, each on
its own tracker and stream, as a stream of events is served.  Inputs (12 distinct events,
more than L2 together) are resident in HBM before the timed region, which is bracketed by
CUDA events on the streams; value = events / device time.  Every tracker's workspace and
result buffers are allocated before timing (tpc_tracker_reserve, tpc_tracker_reserve_results)
and the warm-up runs the timed pattern itself, so the timed calls allocate nothing and the
value does not depend on --steps; Python's garbage collector is off while a region is timed.  Beside it in the same line: the same stream with one event
per call, one event at a time with L2 flushed before each (latency), the step's call alone
(per-stage times and the per-stage and total rooflines), the optional stages, the end-to-end
figure from pinned host buffers through tpc_track_batch_host with the results copied back,
and Poisson-arrival serving latency through the native serving loop.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle (the reference
arm of this build) on the host cores, on the same resident events.
"""
from __future__ import annotations

import argparse
import collections
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "central-like events/s"
WORKLOAD = ("central-like event: 16000 primary + 3000 secondary helices (vertex radius U[0,60] cm), "
            "pT > 0.05 GeV, 20% noise, 36 sectors x 159 pad rows, Bz 0.5 T, seed 1")
PROFILE_JSON = os.path.join(ROOT, "profiles", "construct_traffic.json")
CONSTRUCT_SRC = [os.path.join(ROOT, "paper_1712_09407_gb300", "csrc", f) for f in ("k_construct.cu", "kf.cuh", "common.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="length of each serving run")
    ap.add_argument("--serve-pool", type=int, default=32, help="events of the batched workload the arrivals draw from")
    ap.add_argument("--workload", default="central", choices=["central", "batch", "sector", "full"],
                    help="central: the metric's workload (default); batch: 64 events per call vs one at a time; "
                         "sector / full: the single-sector (200 tracks) and 36-sector (4000 tracks) events, one per call")
    ap.add_argument("--batch-events", type=int, default=64)
    ap.add_argument("--inflight", type=int, default=2, help="tracker calls on the device at once (one stream each)")
    ap.add_argument("--events-per-call", type=int, default=3,
                    help="central events tracked by one call (tpc_track_batch); a step is one call")
    ap.add_argument("--resident", type=int, default=12, help="distinct resident central events (> L2 together)")
    ap.add_argument("--tuning", default="", help="launch choices for every tracker, e.g. construct_block=64")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(x: float, world: int, device: str = "cpu") -> float:
    """Maximum of x over all ranks (the slowest replica sets the job time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(max_total_s: float, steps: int, world: int) -> float:
    """Whole-job events/s: every rank tracks `steps` events of its own (weak scaling)."""
    return world * steps / max_total_s


def replica_event(rank: int) -> int:
    """Event index of the central-like workload a rank tracks (replicas do not share events)."""
    return rank


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons every 50 ms, started well before
    the timed region (so that its start-up does not coincide with it); stop() summarises the
    samples taken inside the marked window."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.windows = []

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def mark(self, t0, t1):
        """A timed window in time.time() seconds."""
        self.windows.append((t0, t1))

    def stop(self, window=-1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        import datetime
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                rows.append([ts] + parts[1:])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        t0, t1 = self.windows[window] if self.windows else (rows[0][0], rows[-1][0])
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        if not inside:                                     # a window shorter than the sampling period
            inside = sorted(rows, key=lambda r: abs(r[0] - 0.5 * (t0 + t1)))[:2]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[2]) for r in inside if num(r[2])]
        mx = max(num(r[3]) or 0 for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(inside), "power_w_max": max(num(r[4]) or 0 for r in inside),
                "sampling": "every 50 ms; samples within the timed region"}


# ------------------------------------------------------------------------------------------------
# roofline bookkeeping
# ------------------------------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Algorithmic bytes of each stage per work unit: every stage reads its inputs and writes its
# outputs once.  N clusters, T tracklets, V construction row visits, K candidates read in them,
# Htl clusters of the claiming tracklets, H output hits, M output tracks.
STAGE_BYTES = {
    "ingest": ("25 B per cluster (9 B in, 12 B sorted out, 4 B bin key)", lambda u: 25 * u["N"]),
    "neighbours": ("32 B per cluster (8 B own, 16 B rows k+-1, 8 B links)", lambda u: 32 * u["N"]),
    "evolution": ("24 B per cluster + 4 B per tracklet", lambda u: 24 * u["N"] + 4 * u["T"]),
    "construction": ("(12 + 8 k) B per row visit (k candidates per visit) + 100 B per tracklet",
                     lambda u: 12 * u["V"] + 8 * u["K"] + 100 * u["T"]),
    "selection": ("20 B per tracklet cluster (8 B atomic, 8 B re-read, 4 B index)", lambda u: 20 * u["Htl"]),
    "output": ("4 B per kept hit + 100 B per track", lambda u: 4 * u["H"] + 100 * u["M"]),
}
STAGE_INDEX = {"ingest": 1, "neighbours": 2, "evolution": 3, "construction": 4, "selection": 5, "output": 6}


def units_of(stats):
    """Work units of one call from its counters (tpc_result_stats)."""
    return dict(N=int(stats["clusters"]), T=int(stats["tracklets"]), V=int(stats["row_visits"]),
                K=int(stats["candidates"]), Htl=int(stats["tracklet_hits"]), H=int(stats["hits"]),
                M=int(stats["tracks"]))


def stage_roofline(units, stage_ms, call_ms, peak):
    """Algorithmic bytes / CUDA-event time of each stage against the HBM peak, the whole path's
    total, and the compulsory input/output traffic as a lower bound."""
    stages, tot_b, tot_ms = {}, 0, 0.0
    for name, (formula, f) in STAGE_BYTES.items():
        b = int(f(units))
        ms = float(stage_ms[STAGE_INDEX[name]])
        gbs = b / (ms * 1e-3) / 1e9 if ms > 0 else None
        stages[name] = {"bytes": b, "ms": round(ms, 4), "achieved_gbs": gbs,
                        "frac": gbs / peak if gbs else None, "per_unit": formula}
        tot_b += b
        tot_ms += ms
    compulsory = 9 * units["N"] + 4 * units["H"] + 112 * units["M"]
    total = {"bytes": tot_b, "ms_stages": round(tot_ms, 4), "achieved_gbs": tot_b / (tot_ms * 1e-3) / 1e9,
             "frac": tot_b / (tot_ms * 1e-3) / 1e9 / peak, "ms_call": round(call_ms, 4),
             "frac_of_call": tot_b / (call_ms * 1e-3) / 1e9 / peak,
             "bytes_per_cluster": tot_b / max(1, units["N"])}
    comp = {"bytes": compulsory, "bytes_per_cluster": compulsory / max(1, units["N"]),
            "what": "9 B per input cluster in, 4 B per output hit + 112 B per output track out",
            "frac_of_call": compulsory / (call_ms * 1e-3) / 1e9 / peak}
    return stages, total, comp


def construct_bytes_touched(stats):
    """Bytes the constructor's loads and stores touch (a wider model than the algorithmic bytes
    above, kept beside them): per row visit 16 B unit record + 8 B grid size + 16 B grid
    origin/scale + 8 B per z-row of cells + 2 B of fitted-cluster index, 8 B per candidate read, per
    tracklet 16 B start record, three 8 B seed points, 4 B input index and 100 B of results."""
    V, K, T = stats["row_visits"], stats["candidates"], stats["tracklets"]
    return V * (16 + 8 + 16 + 8) + 8 * K + T * (16 + 24 + 4 + 100) + 4 * V // 2


def construct_source_hash():
    """Hash of the sources that make up k_construct (its file and the headers it inlines), with
    comments and whitespace removed, so that only a change of the code invalidates the counters."""
    import re
    h = hashlib.sha256()
    for f in CONSTRUCT_SRC:
        src = open(f).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def traffic_for_current_kernel():
    """DRAM bytes and warp instructions of one k_construct launch from the committed ncu record,
    or None when the kernel's sources changed since the capture."""
    if not os.path.exists(PROFILE_JSON):
        return None, None, None
    d = json.load(open(PROFILE_JSON))
    h = construct_source_hash()
    if d.get("source_sha256_16") != h:
        return None, None, "kernel changed since capture"
    return d.get("dram_bytes_per_launch"), d.get("warp_instructions"), d.get("note")


# ------------------------------------------------------------------------------------------------
# workload (identical in both arms)
# ------------------------------------------------------------------------------------------------
def workload_config(n_resident, n_mean, world):
    return {"workload": WORKLOAD, "resident_events": n_resident, "clusters_per_event": int(round(n_mean)),
            "event_seeds": "(1, %d) .. (1, %d)" % (0, n_resident - 1),
            "l2": "inputs larger than L2 (%d resident events, %.0f MB); no flush" % (n_resident, n_resident * n_mean * 9 / 1e6),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def resident_events(n, first_event, pin):
    """The resident central-like events (about 30 MB each), generated in parallel."""
    from paper_1712_09407_gb300.serving import event_pool
    return event_pool(n, cfg=2, first_event=first_event, pin=pin)


# ------------------------------------------------------------------------------------------------
# CPU oracle legs
# ------------------------------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the architecture)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_steps(pool, n_steps, max_seconds, cfg=None):
    """The float-mode oracle over the resident events in turn (OpenMP over the 36 sectors):
    at most n_steps events and about max_seconds of CPU time.  Returns (events, seconds)."""
    import oracle
    from paper_1712_09407_gb300 import eventgen
    cfg = cfg or oracle.config_for(eventgen.Geometry())
    t0 = time.perf_counter()
    k = 0
    while k < n_steps and (k == 0 or time.perf_counter() - t0 < max_seconds):
        y, z, row, counts, _ = pool[k % len(pool)]
        oracle.track_event(cfg, y.numpy(), z.numpy(), row.numpy(), counts, precision=32)
        k += 1
    return k, time.perf_counter() - t0


def oracle_timing(pool, seconds=12.0):
    """The oracle on the host cores over the resident events (a bounded sample), then one event
    on one thread."""
    import oracle
    from paper_1712_09407_gb300 import eventgen
    oracle_steps(pool, 1, 0.0)                                  # first call: page-in, thread start-up
    k, dt = oracle_steps(pool, 10 ** 6, seconds)
    cores = os.cpu_count()
    y, z, row, counts, n = pool[0]
    t0 = time.perf_counter()
    oracle.track_event(oracle.config_for(eventgen.Geometry(), n_threads=1), y.numpy(), z.numpy(), row.numpy(),
                       counts, precision=32)
    t_one = time.perf_counter() - t0
    return dict(value=k / dt, unit="events/s", cores=cores, kind="oracle",
                sample="%d of the resident central-like events in turn (float-mode C oracle, OpenMP over the 36 "
                       "sectors on %d threads), %.1f s" % (k, cores, dt),
                single_thread={"value": 1.0 / t_one, "unit": "events/s", "sample": "one event on one thread"},
                cpu_model=cpu_model())


def run_reference(args):
    """The reference arm: the CPU oracle on the same resident events as our arm, one event per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    pool = resident_events(args.resident, 0, pin=False)
    n_mean = float(np.mean([p[4] for p in pool]))
    oracle_steps(pool, max(1, args.warmup), 1e9)
    steps, dt = oracle_steps(pool, args.steps, 90.0)
    v = steps / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "events/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(len(pool), n_mean, world),
            "cpu_baseline": {"value": v, "unit": "events/s", "cores": cores, "kind": "oracle",
                             "sample": "%d of the resident central-like events in turn, one per step, float-mode "
                                       "C oracle, OpenMP over 36 sectors on %d host threads" % (steps, cores)},
            "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
QDEPTH = 16    # calls each tracker has outstanding in the streamed legs (its result ring holds one more): about
              # 120 ms of queued device work over two streams, so that a host pause does not starve the device
PREROLL_CYCLES = 10_000_000   # about 5 ms at 2 GHz
E2E_DEPTH = 3                  # calls outstanding per tracker in the end-to-end leg
STAGES = ["setup", "ingest", "neighbours", "evolution", "construction", "selection", "output", "global", "merge"]


def apply_tuning(tracker, spec):
    """Launch choices from a "field=value,..." string (none: the library's defaults)."""
    if spec:
        tracker.set_tuning({k: (float(v) if "." in v else int(v)) for k, v in (kv.split("=") for kv in spec.split(","))})


class Streamer:
    """A stream of tracker calls round-robin over trackers, one CUDA stream each, keeping QDEPTH
    calls per tracker outstanding (the oldest is retired on the host while the device works)."""

    def __init__(self, torch, trackers, streams, world):
        self.torch, self.trackers, self.streams, self.world = torch, trackers, streams, world

    def barrier(self):
        self.torch.cuda.synchronize()
        if self.world > 1:
            self.torch.distributed.barrier()
        self.torch.cuda.synchronize()

    def run(self, n_calls, submit, timed):
        torch = self.torch
        nt = len(self.trackers)
        gc_was = gc.isenabled()
        gc.disable()                   # no collector pause may starve the device queue while timing
        launches, tracks = 0, []
        start = ends = None
        if timed:
            self.barrier()
            self.t_host = time.time()
            start = torch.cuda.Event(enable_timing=True)
            ends = [torch.cuda.Event(enable_timing=True) for _ in self.streams]
            # untimed pre-roll: the device spins for about 5 ms before the start event, so that the
            # first calls are already queued when the region starts (the host's enqueue time of the
            # first calls is not device time; the end-to-end leg measures the host path)
            with torch.cuda.stream(self.streams[0]):
                torch.cuda._sleep(PREROLL_CYCLES)
            start.record(self.streams[0])
            for s_ in self.streams[1:]:
                s_.wait_event(start)
        pend = collections.deque()

        def retire(r):
            nonlocal launches
            r.sync()
            launches += r.stats()["kernel_launches"]
            tracks.append(r.n_tracks)
            r.release()

        for k in range(n_calls):
            i = k % nt
            with torch.cuda.stream(self.streams[i]):
                pend.append(submit(self.trackers[i], k, self.streams[i]))
            if len(pend) > nt * QDEPTH:
                retire(pend.popleft())
        if timed:
            for e, s_ in zip(ends, self.streams):
                e.record(s_)
        self.barrier()
        while pend:
            retire(pend.popleft())
        total_s = max(start.elapsed_time(e) for e in ends) / 1e3 if timed else None
        if timed:
            self.t_host_end = time.time()
        if gc_was:
            gc.enable()
        return total_s, launches, tracks


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from __graft_entry__ import build
    build()
    from paper_1712_09407_gb300 import eventgen
    from paper_1712_09407_gb300.serving import page_in_mapped_files
    from paper_1712_09407_gb300.tracker import Tracker

    # Resident inputs: `resident` different central-like events (together more than the 129 MB L2),
    # copied to HBM before any timing; rank r tracks its own events (replicas)
    clocks = ClockSampler(local)
    clocks.start()                   # long before the timed region; only its samples are kept
    pool = resident_events(args.resident, replica_event(rank) * args.resident, pin=True)
    geo = eventgen.Geometry()
    dev = [(p[0].cuda(), p[1].cuda(), p[2].cuda(), p[3], p[4]) for p in pool]
    n_mean = float(np.mean([p[4] for p in pool]))
    # calls of B consecutive resident events (inputs concatenated on the device and, for the
    # end-to-end leg, in pinned host memory, before any timing)
    B = max(1, args.events_per_call)
    calls = []
    for j in range(max(1, len(pool) // B)):
        ps = [pool[(j * B + i) % len(pool)] for i in range(B)]
        ds = [dev[(j * B + i) % len(dev)] for i in range(B)]
        calls.append(dict(y=torch.cat([d[0] for d in ds]), z=torch.cat([d[1] for d in ds]),
                          row=torch.cat([d[2] for d in ds]), counts=np.concatenate([p[3] for p in ps]),
                          n=sum(p[4] for p in ps), hy=torch.cat([p[0] for p in ps]).pin_memory(),
                          hz=torch.cat([p[1] for p in ps]).pin_memory(), hr=torch.cat([p[2] for p in ps]).pin_memory()))
    # B-event calls and one-event calls on separate trackers (each keeps one executable graph); every
    # tracker's workspace and result buffers are allocated here, so the timed calls allocate nothing
    trackers = [Tracker.for_geometry(geo) for _ in range(args.inflight)]
    for t in trackers:
        apply_tuning(t, args.tuning)
        t.reserve(max(c_["n"] for c_ in calls), B, results=QDEPTH + 1)
    trackers1 = [Tracker.for_geometry(geo) for _ in range(args.inflight)]
    for t in trackers1:
        apply_tuning(t, args.tuning)
        t.reserve(max(p[4] for p in pool), 1, results=QDEPTH + 1)
    streams = [torch.cuda.Stream() for _ in range(args.inflight)]
    stream = streams[0]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def call_b(t, k, s_):
        c_ = calls[k % len(calls)]
        if B == 1:
            return t.track(c_["y"], c_["z"], c_["row"], c_["counts"], stream=s_)
        return t.track_batch(c_["y"], c_["z"], c_["row"], c_["counts"], B, stream=s_)

    def call_1(t, k, s_):
        d = dev[k % len(dev)]
        return t.track(d[0], d[1], d[2], d[3], stream=s_)

    sb = Streamer(torch, trackers, streams, world)
    s1 = Streamer(torch, trackers1, streams, world)
    # warm-up: the timed pattern itself (same trackers, streams, call shape and depth of outstanding
    # calls), so that graphs, staging buffers and result buffers are all in use before timing; the
    # process's mapped files are read once first, so that no page of them is fetched mid-region
    page_in_mapped_files()
    n_warm = max(args.warmup, args.inflight * (QDEPTH + 2))
    sb.run(n_warm, call_b, timed=False)
    s1.run(n_warm, call_1, timed=False)

    # ---- timed region (the value): a stream of calls of B central-like events each, `inflight` calls
    # on the device at once (one tracker and stream each); per-call stage timing stays off here
    t_wall = time.perf_counter()
    total_s, launches, tracks = sb.run(args.steps, call_b, timed=True)
    wall = time.perf_counter() - t_wall
    clocks.mark(sb.t_host, sb.t_host_end)
    clk = clocks.stop()
    total_s = reduce_max(total_s, world, "cuda")
    value = replica_throughput(total_s, args.steps * B, world)

    # the same stream with one event per call (tpc_track_event), for comparison
    n_one = max(args.steps * B, 3 * args.inflight * QDEPTH)
    one_s, _, _ = s1.run(n_one, call_1, timed=True)
    one_s = reduce_max(one_s, world, "cuda")
    one_per_call = {"events_per_s": replica_throughput(one_s, n_one, world), "events": n_one,
                    "inflight_calls": args.inflight, "path": "tpc_track_event, one event per call"}

    # ---- one event at a time on one stream, L2 flushed (untimed) before each: latency and stages
    tr1 = trackers1[0]
    tr1.set_timing(True)
    n_serial = min(max(args.steps, 10), 40)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_serial)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_serial)]
    stage_ms = np.zeros(9)
    stats_all = []
    sb.barrier()
    with torch.cuda.stream(stream):
        for k in range(n_serial):
            flush.fill_(float(k))
            starts[k].record(stream)
            r = call_1(tr1, k, stream)
            ends[k].record(stream)
            r.sync()
            st = r.stats()
            stats_all.append(st)
            stage_ms += np.array(st["ms"])
            r.release()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    serial = {"events_per_s": n_serial / (sum(step_ms) / 1e3), "ms_per_event": float(np.mean(step_ms)), "steps": n_serial,
              "ms_per_event_p50": float(np.median(step_ms)), "l2": "flushed before every event (512 MB write, untimed)"}
    tr1.set_timing(False)
    # the step's own call (B events) one at a time, L2 flushed before each: stage times and rooflines
    trb = trackers[0]
    trb.set_timing(True)
    n_bs = min(max(args.steps, 6), 12)
    b_stats, b_ms = [], []
    with torch.cuda.stream(stream):
        for k in range(n_bs + 1):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = call_b(trb, k, stream)
            b.record(stream)
            r.sync()
            if k > 0:                        # the first call builds the timed graph
                b_stats.append(r.stats())
                b_ms.append(a.elapsed_time(b))
            r.release()
    trb.set_timing(False)
    b_stage = np.mean([np.array(s_["ms"]) for s_ in b_stats], axis=0)
    b_units = {k: int(np.mean([units_of(s_)[k] for s_ in b_stats])) for k in units_of(b_stats[0])}

    # ---- optional stages on the same events, one at a time, L2 flushed (untimed)
    def extra_pass(**flags):
        xtr = Tracker.for_geometry(geo, **flags)
        apply_tuning(xtr, args.tuning)
        xtr.reserve(max(p[4] for p in pool), 1, results=2)
        n_x = min(max(args.steps, 10), 20)
        x_ms, x_stats = [], []
        with torch.cuda.stream(stream):
            for k in range(args.warmup):
                r = call_1(xtr, k, stream)
                r.sync()
                r.release()
            xtr.set_timing(True)
            for k in range(n_x + 1):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = call_1(xtr, k, stream)
                b.record(stream)
                r.sync()
                if k > 0:
                    x_stats.append(r.stats())
                    x_ms.append(a.elapsed_time(b))
                r.release()
        xtr.close()
        st_ms = np.mean([np.array(s_["ms"]) for s_ in x_stats], axis=0)
        return n_x, x_ms, x_stats, st_ms

    n_g, g_ms, g_stats, g_stage = extra_pass(global_tracking=True)
    plain_hits = {k % len(dev): stats_all[k]["hits"] for k in range(n_serial)}     # event -> hits without
    added = [g_stats[j]["hits"] - plain_hits[(j + 1) % len(dev)] for j in range(n_g) if (j + 1) % len(dev) in plain_hits]
    global_line = {
        "events_per_s": n_g / (sum(g_ms) / 1e3), "ms_per_event": float(np.mean(g_ms)), "steps": n_g,
        "stages_ms": {n: round(float(v), 4) for n, v in zip(STAGES, g_stage)},
        "clusters_found_per_event": float(np.mean([s_["global_found"] for s_ in g_stats])),
        "clusters_added_per_event": float(np.mean(added)) if added else None,
        "tracks_per_event": float(np.mean([s_["tracks"] for s_ in g_stats])),
        "l2": "flushed before every event (512 MB write, untimed)"}
    n_m, m_ms, m_stats, m_stage = extra_pass(global_tracking=True, merge=True)
    merge_line = {
        "what": "global tracking + track merger with refit",
        "events_per_s": n_m / (sum(m_ms) / 1e3), "ms_per_event": float(np.mean(m_ms)), "steps": n_m,
        "stages_ms": {n: round(float(v), 4) for n, v in zip(STAGES, m_stage)},
        "sector_tracks_per_event": float(np.mean([s_["sector_tracks"] for s_ in m_stats])),
        "merged_tracks_per_event": float(np.mean([s_["tracks"] for s_ in m_stats])),
        "l2": "flushed before every event (512 MB write, untimed)"}

    # ---- end to end through the host-buffer entry point: every call copies its events from pinned
    # host memory, tracks them and copies the result back (all inside the timed region), `inflight`
    # calls in flight on their trackers and streams; the one-event-at-a-time figure beside it
    e2e = None
    if not args.no_e2e:
        e2e = e2e_leg(args, torch, pool, calls, trackers, streams, tr1, stream, flush, B, world)

    serving = None
    if not args.no_serving and world == 1:
        for t in trackers + trackers1:
            t.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        serving = serving_leg(args, torch)

    if rank != 0:
        return 0
    peak, peak_kind = measured_peaks()
    stages_rf, total_rf, comp_rf = stage_roofline(b_units, b_stage, float(np.mean(b_ms)), peak)
    con = stages_rf["construction"]
    traffic, winst, tnote = traffic_for_current_kernel()
    seeded = B * n_mean / 20 > 2 * 152 * 5 * 128
    roof = {"kernel": "k_construct (A5 tracklet construction; %s)" % (
                "pre-seeded, lanes meeting per row" if seeded else "seeds walked per lane"),
            "bound": "hbm", "achieved": con["achieved_gbs"], "peak": peak, "unit": "GB/s", "frac": con["frac"],
            "peak_source": peak_kind + " (hbm_gbs, burst copy)", "traffic": traffic,
            "algorithmic_bytes": con["bytes"], "per_unit": con["per_unit"], "launch_ms": con["ms"],
            "bytes_touched": construct_bytes_touched(
                {"row_visits": b_units["V"], "candidates": b_units["K"], "tracklets": b_units["T"]}),
            "timed_in": "the step's call (%d events) one at a time, L2 flushed before each; construction stage "
                        "(work order, seeds and the constructor), CUDA events on the call's stream" % B,
            "units": b_units, "stages": stages_rf, "total": total_rf, "compulsory_io": comp_rf}
    if tnote:
        roof["traffic_note"] = tnote
    if winst:
        sm_mhz = clk.get("sm_mhz") or 2070.0
        issue_peak = 152 * 4 * sm_mhz * 1e6
        roof["issue"] = {"achieved": winst / (con["ms"] * 1e-3), "peak": issue_peak, "unit": "warp instructions/s",
                         "frac": winst / (con["ms"] * 1e-3) / issue_peak, "warp_instructions": winst,
                         "peak_source": "152 SMs x 4 schedulers x sampled SM clock"}
    line = {"metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(len(pool), n_mean, world),
            "launch": {"events_per_call": B, "inflight_calls": args.inflight, "calls_outstanding_per_tracker": QDEPTH,
                       "tuning": args.tuning or "library defaults",
                       "warmup_calls": n_warm, "allocation": "workspace and %d result buffers per tracker "
                                                             "preallocated (tpc_tracker_reserve_results)" % (QDEPTH + 1)},
            "clusters_per_s": value * n_mean, "tracks_per_event": int(np.mean(tracks)),
            "one_event_per_call": one_per_call, "one_event_at_a_time": serial,
            "stages_ms": {n: round(float(v), 4) for n, v in zip(STAGES, stage_ms / n_serial)},
            "one_call_at_a_time": {"ms_per_call": float(np.mean(b_ms)), "events_per_call": B,
                                   "stages_ms": {n: round(float(v), 4) for n, v in zip(STAGES, b_stage)},
                                   "l2": "flushed before every call (512 MB write, untimed)"},
            "global_tracking": global_line, "global_tracking_and_merger": merge_line,
            "gpu_launches": launches, "e2e": e2e, "serving": serving, "roofline": roof, "clocks": clk,
            "wall_s_timed_region": wall}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_timing(pool)
    print(json.dumps(line))
    return 0


def e2e_leg(args, torch, pool, calls, trackers, streams, tr1, stream, flush, B, world):
    from paper_1712_09407_gb300.tracker import tpc_result_copy_to_host

    def host_bufs(bufs, M, H):
        if bufs is None or bufs["par"].shape[0] < M or bufs["hits"].shape[0] < H:
            bufs = dict(par=torch.empty((M + 1024, 5)).pin_memory(), cov=torch.empty((M + 1024, 15)).pin_memory(),
                        x_ref=torch.empty(M + 1024).pin_memory(), alpha=torch.empty(M + 1024).pin_memory(),
                        chi2=torch.empty(M + 1024).pin_memory(),
                        **{n: torch.empty(M + 1024, dtype=torch.int32).pin_memory()
                           for n in ("ndf", "nhits", "first", "sector", "event")},
                        hits=torch.empty(H + 65536, dtype=torch.int32).pin_memory())
        return bufs

    # one at a time
    bufs = None
    times = []
    with torch.cuda.stream(stream):
        for k in range(args.warmup + min(max(args.steps, 10), 40)):
            hy, hz, hr, counts, _ = pool[k % len(pool)]
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = tr1.track_host(hy, hz, hr, counts, stream=stream)
            M, H = r.sync()
            bufs = host_bufs(bufs, M, H)
            tpc_result_copy_to_host(r.handle, bufs)
            t1 = time.perf_counter()
            r.release()
            if k >= args.warmup:
                times.append(t1 - t0)
    serial_e2e = replica_throughput(reduce_max(sum(times), world, "cuda"), len(times), world)

    # a stream of calls through the trackers, E2E_DEPTH calls outstanding per tracker (the host
    # submits the next calls, host input and all, while earlier ones compute, and copies each
    # result back as soon as it is done); timed in the steady state, from the result of one call
    # to the result of the call n_e2e calls later, so the window holds n_e2e submissions (each with
    # its host-to-device copy) and n_e2e results copied back
    nf = len(trackers)
    hb = [None] * nf
    moved = {"h2d": 0, "d2h": 0}
    n_warm = 2 * E2E_DEPTH * nf
    n_e2e = max(args.steps, 40)
    n_total = n_warm + n_e2e + E2E_DEPTH * nf
    done_t = {}
    pend = collections.deque()

    def retire():
        k, i, r = pend.popleft()
        M, H = r.sync()
        hb[i] = host_bufs(hb[i], M, H)
        tpc_result_copy_to_host(r.handle, hb[i])
        r.release()
        done_t[k] = time.perf_counter()
        if n_warm <= k < n_warm + n_e2e:
            moved["d2h"] += M * (5 + 15 + 3 + 5) * 4 + H * 4 + 48

    torch.cuda.synchronize()
    gc.disable()
    for k in range(n_total):
        if len(pend) >= nf * E2E_DEPTH:
            retire()
        i = k % nf
        c_ = calls[k % len(calls)]
        pend.append((k, i, trackers[i].track_batch_host(c_["hy"], c_["hz"], c_["hr"], c_["counts"], B, stream=streams[i])))
        if n_warm <= k < n_warm + n_e2e:
            moved["h2d"] += c_["n"] * 9
    while pend:
        retire()
    gc.enable()
    wall_e2e = done_t[n_warm + n_e2e - 1] - done_t[n_warm - 1]
    e2e_v = replica_throughput(reduce_max(wall_e2e, world, "cuda"), n_e2e * B, world)
    return {"value": e2e_v, "unit": "events/s", "h2d_bytes_per_step": int(moved["h2d"] / n_e2e),
            "d2h_bytes_per_step": int(moved["d2h"] / n_e2e), "steps": n_e2e, "events_per_step": B,
            "path": "tpc_track_batch_host (pinned host input, %d events per call) + tpc_result_copy_to_host, "
                    "wall clock between results %d calls apart in the steady state, %d calls outstanding on "
                    "each of %d trackers" % (B, n_e2e, E2E_DEPTH, nf),
            "one_event_at_a_time": serial_e2e}


def serving_leg(args, torch):
    """Poisson arrivals of events of the batched workload (primaries log-uniform 500-16000, noise
    5-20 %) through the native serving loop with continuous batching, and through the same loop
    with one lane and one event per batch (the plain one-event-at-a-time path); a fixed 40 GB budget.
    Latency runs from the scheduled arrival to the result in host memory."""
    from paper_1712_09407_gb300 import eventgen
    from paper_1712_09407_gb300.serving import (NativeServer, event_pool, latency_report, make_requests,
                                                poisson_arrivals, run_stream_native)
    pool = event_pool(args.serve_pool, cfg=3)
    geo = eventgen.Geometry()
    out = {"duration_s": args.serve_seconds, "pool_events": len(pool), "budget_gb": 40,
           "workload": "events of the batched workload (primaries log-uniform 500-16000, noise 5-20 %%, seeds (1, i), "
                       "i < %d), drawn with replacement" % len(pool),
           "latency": "scheduled Poisson arrival to the event's result in host memory (copies included)"}
    runs = [(200.0, "continuous_batching"), (200.0, "one_event_at_a_time"), (1000.0, "continuous_batching")]
    for rate, mode in runs:
        lanes, mb = (3, 16) if mode == "continuous_batching" else (1, 1)
        srv = NativeServer(geo, lanes=lanes, hbm_budget=40 << 30, max_batch=mb, keep_results=False)
        srv.warm(make_requests(pool, np.zeros(len(pool)), seed=99))
        reqs = make_requests(pool, poisson_arrivals(rate, args.serve_seconds, seed=int(rate)), seed=int(rate))
        wall = run_stream_native(srv, reqs)
        rep = latency_report(reqs, wall)
        rep.update(lanes=lanes, max_batch=mb)
        out["%d_hz_%s" % (int(rate), mode)] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in rep.items()}
        srv.close()
        torch.cuda.synchronize()
    return out


def run_batch(args):
    """64 events of the batched workload (primaries log-uniform in [500, 16000], noise 5-20 %)
    tracked by one call (every stage launched once over all sectors of all events) against the
    same events tracked one call each; both from HBM-resident inputs, L2 flushed before each
    timed call."""
    import torch
    from __graft_entry__ import build
    build()
    from paper_1712_09407_gb300 import eventgen
    from paper_1712_09407_gb300.serving import event_pool
    from paper_1712_09407_gb300.tracker import Tracker

    pool = event_pool(args.batch_events)
    n_tot = sum(p[4] for p in pool)
    y = torch.cat([p[0] for p in pool]).cuda()
    z = torch.cat([p[1] for p in pool]).cuda()
    row = torch.cat([p[2] for p in pool]).cuda()
    counts = np.concatenate([p[3] for p in pool])
    offs = np.concatenate([[0], np.cumsum([p[4] for p in pool])])
    tr = Tracker.for_geometry(eventgen.Geometry())
    apply_tuning(tr, args.tuning)
    tr.reserve(n_tot, len(pool))
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(fn, reps):
        ms = []
        with torch.cuda.stream(stream):
            for k in range(args.warmup + reps):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                rs = fn()
                b.record(stream)
                for r in rs:
                    r.sync()
                    r.release()
                if k >= args.warmup:
                    ms.append(a.elapsed_time(b))
        return float(np.median(ms))

    def batched():
        return [tr.track_batch(y, z, row, counts, len(pool), stream=stream)]

    def singles():
        out = []
        for i in range(len(pool)):
            out.append(tr.track(y[offs[i]:offs[i + 1]], z[offs[i]:offs[i + 1]], row[offs[i]:offs[i + 1]],
                                pool[i][3], stream=stream))
        return out

    reps = max(3, min(args.steps, 10))
    t_b = timed(batched, reps)
    t_s = timed(singles, reps)

    # time against input size (the paper's Fig. "gp_eventstat": linear, with a small offset on the
    # GPU): every event alone, L2 flushed, median of 3; least-squares t = a + b n
    per = []
    with torch.cuda.stream(stream):
        for i in range(len(pool)):
            ms = []
            for k in range(3):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = tr.track(y[offs[i]:offs[i + 1]], z[offs[i]:offs[i + 1]], row[offs[i]:offs[i + 1]], pool[i][3],
                             stream=stream)
                b.record(stream)
                r.sync()
                r.release()
                ms.append(a.elapsed_time(b))
            per.append((pool[i][4], float(np.median(ms))))
    nn = np.array([p[0] for p in per], dtype=np.float64)
    tt = np.array([p[1] for p in per])
    slope, offset = np.polyfit(nn, tt, 1)
    resid = tt - (offset + slope * nn)
    r2 = 1.0 - float((resid ** 2).sum() / ((tt - tt.mean()) ** 2).sum())
    scaling = {"offset_ms": float(offset), "ms_per_million_clusters": float(slope * 1e6), "r2": r2,
               "clusters_min": int(nn.min()), "clusters_max": int(nn.max()),
               "events": [[int(a_), round(b_, 4)] for a_, b_ in per]}
    line = {"metric": "batched events/s", "value": len(pool) / (t_b / 1e3), "unit": "events/s", "n_gpus": 1,
            "steps": reps, "warmup": args.warmup, "ms_per_step": t_b, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%d events, primaries log-uniform 500-16000, noise 5-20 %%, 36 sectors, seeds (1, i)"
                                   % len(pool), "clusters": int(n_tot), "l2": "flushed before every step"},
            "one_at_a_time": {"value": len(pool) / (t_s / 1e3), "ms_per_step": t_s},
            "speedup_vs_one_at_a_time": t_s / t_b, "time_vs_clusters": scaling}
    print(json.dumps(line))
    return 0


def run_small(args):
    """The single-sector or the 36-sector event (configs of 200 and 4000 tracks), one event per
    call: a stream with 2 calls in flight on 2 trackers (12 distinct events, seeds (1, i)), one
    event at a time (L2 flushed), and the float oracle on the host cores."""
    import torch
    from __graft_entry__ import build
    build()
    from paper_1712_09407_gb300 import eventgen
    from paper_1712_09407_gb300.tracker import Tracker
    cfg = 0 if args.workload == "sector" else 1
    evs = [eventgen.config_event(cfg, event=i) for i in range(args.resident)]
    geo = evs[0].geometry
    dev = [(torch.from_numpy(e.y).cuda(), torch.from_numpy(e.z).cuda(), torch.from_numpy(e.row).cuda(), e.counts)
           for e in evs]
    trackers = [Tracker.for_geometry(geo) for _ in range(args.inflight)]
    for t in trackers:
        apply_tuning(t, args.tuning)
        t.reserve(max(e.n for e in evs), 1, results=QDEPTH + 1)
    streams = [torch.cuda.Stream() for _ in range(args.inflight)]

    def call_1(t, k, s_):
        d = dev[k % len(dev)]
        return t.track(d[0], d[1], d[2], d[3], stream=s_)

    st = Streamer(torch, trackers, streams, 1)
    st.run(max(args.warmup, args.inflight * (QDEPTH + 2)), call_1, timed=False)
    total_s, launches, _ = st.run(args.steps, call_1, timed=True)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ms = []
    with torch.cuda.stream(streams[0]):
        for k in range(min(max(args.steps, 10), 40)):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(streams[0])
            r = call_1(trackers[0], k, streams[0])
            b.record(streams[0])
            r.sync()
            r.release()
            ms.append(a.elapsed_time(b))
    import oracle
    ocfg = oracle.config_for(geo)
    oracle.track_event(ocfg, evs[0].y, evs[0].z, evs[0].row, evs[0].counts, precision=32)
    t0, k = time.perf_counter(), 0
    while k < 200 and (k < 3 or time.perf_counter() - t0 < 10.0):
        e = evs[k % len(evs)]
        oracle.track_event(ocfg, e.y, e.z, e.row, e.counts, precision=32)
        k += 1
    n_mean = float(np.mean([e.n for e in evs]))
    line = {"metric": "events/s", "value": args.steps / total_s, "unit": "events/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("single sector (both z halves), 200 primaries, 5% noise" if cfg == 0 else
                                    "36 sectors, 4000 primaries, 10% noise"), "resident_events": len(evs),
                       "clusters_per_event": int(round(n_mean)), "inflight_calls": args.inflight},
            "clusters_per_s": args.steps / total_s * n_mean, "gpu_launches": launches,
            "one_event_at_a_time": {"ms_per_event": float(np.median(ms)), "l2": "flushed before every event"},
            "cpu_baseline": {"value": k / (time.perf_counter() - t0), "unit": "events/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": "%d events, float-mode C oracle, OpenMP over sectors" % k}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload in ("sector", "full"):
        return run_small(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
