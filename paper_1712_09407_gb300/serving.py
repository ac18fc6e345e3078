"""Continuous-batching serving loop for the sector tracker.

Events arrive at HLT-like rates (the paper's requirement is more than 200 central Pb-Pb events
per second, abstract).  The server keeps ``lanes`` trackers, each with its own preallocated
device workspace, device input buffer and CUDA stream.  Whenever a lane is free it takes the
pending events that fit its reservation (at most ``max_batch`` events and ``lane_clusters``
clusters) as one batch: their clusters are copied into the lane's input buffer and every stage
runs once over all sectors of all of them (``tpc_track_batch``).  Lanes run concurrently on the
device, so requests that arrive while others are on the GPU are admitted as soon as a lane
frees up, and their work overlaps.

Admission by memory budget: the HBM budget is split over the lanes; each lane reserves its
workspace, input buffer and result space for ``lane_clusters`` clusters up front, so the
steady state allocates nothing new.  An event larger than a lane's reservation is refused
(status ``"rejected"``).  A batch that fails on the device (for example a pool overflow on a
noise-filled sector, Section 6) is split and its events retried one by one; an event that
fails alone is reported with its status.

Results are identical whether an event is tracked alone or inside a batch (every stage works
per sector; the only coupling, the output order, is per event).
"""
from __future__ import annotations

import collections
import dataclasses
import math
import os
import stat
import time

import numpy as np

from .tracker import (Tracker, TrackerError, server_result_arrays, tpc_result_copy_to_host, tpc_server_create,
                      tpc_server_destroy, tpc_server_get, tpc_server_now_ns, tpc_server_poll, tpc_server_release,
                      tpc_server_submit)

# device bytes per reserved cluster: workspace (about 246 B), the lane's preallocated result
# (about 32 B), input (9 B), with a margin
BYTES_PER_CLUSTER = 300


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds since the start of the run
    y: object                      # pinned torch float32 [n]
    z: object
    row: object                    # pinned torch uint8 [n]
    counts: np.ndarray             # int32 [36 * 159]
    n: int
    t_start: float = math.nan      # launch time
    t_done: float = math.nan
    status: str = "pending"
    result: dict | None = None
    batch_size: int = 0
    arrival_ns: int = 0            # native server: scheduled arrival, submission, launch, done (server clock)
    t_submit_ns: int = 0
    t_launch_ns: int = 0
    t_done_ns: int = 0


class Lane:
    def __init__(self, geometry, lane_clusters, max_batch, budget, device="cuda"):
        import torch
        self.tracker = Tracker.for_geometry(geometry, budget=budget)
        self.tracker.reserve(lane_clusters, max_batch)
        self.stream = torch.cuda.Stream()
        self.y = torch.empty(lane_clusters, dtype=torch.float32, device=device)
        self.z = torch.empty(lane_clusters, dtype=torch.float32, device=device)
        self.row = torch.empty(lane_clusters, dtype=torch.uint8, device=device)
        self.cap = lane_clusters
        self.max_batch = max_batch
        self.busy = False
        self.result = None
        self.batch = []
        self.offsets = []
        self.launches = 0
        self.host = None              # pinned result buffers, grown on demand
        self.host_m = self.host_h = 0

    def _host_buffers(self, M, H):
        import torch
        if self.host is None or M > self.host_m or H > self.host_h:
            m, h = max(M, 2 * self.host_m, 1024), max(H, 2 * self.host_h, 65536)
            f = lambda *shape: torch.empty(shape, dtype=torch.float32).pin_memory()
            i = lambda n: torch.empty(n, dtype=torch.int32).pin_memory()
            self.host = dict(par=f(m, 5), cov=f(m, 15), x_ref=f(m), alpha=f(m), chi2=f(m), ndf=i(m), nhits=i(m),
                             first=i(m), sector=i(m), event=i(m), hits=i(h))
            self.host_m, self.host_h = m, h
        return self.host

    def launch(self, batch, now, retry=False):
        import torch
        self.batch = batch
        self.offsets = []
        off = 0
        with torch.cuda.stream(self.stream):
            for r in batch:
                self.y[off:off + r.n].copy_(r.y, non_blocking=True)
                self.z[off:off + r.n].copy_(r.z, non_blocking=True)
                self.row[off:off + r.n].copy_(r.row, non_blocking=True)
                self.offsets.append(off)
                off += r.n
                r.t_start = now
                r.batch_size = len(batch)
            counts = np.concatenate([r.counts for r in batch])
            self.result = self.tracker.track_batch(self.y[:off], self.z[:off], self.row[:off], counts, len(batch),
                                                   stream=self.stream)
        self.busy = True
        self.launches += 1

    def ready(self):
        return self.busy and self.result.ready()

    def collect(self, now):
        """Finished batch: split the output per event.  Returns (done, failed) request lists."""
        res, batch, offs = self.result, self.batch, self.offsets
        self.busy = False
        self.result = None
        try:
            M, H = res.sync()
        except TrackerError as e:
            res.release()
            for r in batch:
                r.status = "error %d" % e.status
            return [], batch
        hb = self._host_buffers(M, H)
        tpc_result_copy_to_host(res.handle, hb)
        res.release()
        o = {k: v.numpy() for k, v in hb.items()}
        ev, first, nh = o["event"][:M], o["first"][:M], o["nhits"][:M]
        bounds = np.searchsorted(ev, np.arange(len(batch) + 1))    # tracks are sorted by event
        for i, r in enumerate(batch):
            t0, t1 = int(bounds[i]), int(bounds[i + 1])
            h0 = int(first[t0]) if t1 > t0 else 0
            h1 = int(first[t1 - 1] + nh[t1 - 1]) if t1 > t0 else 0
            r.result = dict(par=o["par"][t0:t1].copy(), cov=o["cov"][t0:t1].copy(), x_ref=o["x_ref"][t0:t1].copy(),
                            chi2=o["chi2"][t0:t1].copy(), ndf=o["ndf"][t0:t1].copy(), nhits=nh[t0:t1].copy(),
                            first=first[t0:t1] - h0, sector=o["sector"][t0:t1].copy(),
                            hits=o["hits"][h0:h1] - offs[i])
            r.t_done = now
            r.status = "done"
        return batch, []


class Server:
    def __init__(self, geometry, lanes=3, hbm_budget=40 << 30, max_batch=16, lane_clusters=None):
        if lane_clusters is None:
            lane_clusters = int(hbm_budget / lanes / BYTES_PER_CLUSTER)
        self.lanes = [Lane(geometry, lane_clusters, max_batch, hbm_budget // lanes) for _ in range(lanes)]
        self.lane_clusters = lane_clusters
        self.max_batch = max_batch
        self.pending = collections.deque()
        self.retry = collections.deque()
        self.done = []
        self.rejected = []
        self.high_water = 0

    def submit(self, r: Request):
        if r.n > self.lane_clusters:
            r.status = "rejected"
            self.rejected.append(r)
            return False
        self.pending.append(r)
        self.high_water = max(self.high_water, len(self.pending))
        return True

    def _form_batch(self):
        if self.retry:                     # events of a failed batch go alone
            return [self.retry.popleft()]
        batch, tot = [], 0
        while self.pending and len(batch) < self.max_batch and tot + self.pending[0].n <= self.lane_clusters:
            r = self.pending.popleft()
            batch.append(r)
            tot += r.n
        return batch

    def poll(self, now):
        """Collect finished lanes and launch new batches on free ones.  Returns True if anything moved."""
        moved = False
        for lane in self.lanes:
            if lane.ready():
                ok, failed = lane.collect(now)
                self.done.extend(ok)
                if len(failed) > 1:
                    self.retry.extend(failed)
                else:
                    self.done.extend(failed)
                moved = True
        for lane in self.lanes:
            if not lane.busy and (self.pending or self.retry):
                batch = self._form_batch()
                if batch:
                    lane.launch(batch, now)
                    moved = True
        return moved

    def busy(self):
        return any(l.busy for l in self.lanes) or bool(self.pending) or bool(self.retry)

    def warm(self, requests):
        """Run one full batch through every lane, so that no lane pays its first-use costs (result
        pool growth, pinned host buffers, the executable graph) on a live request."""
        page_in_mapped_files()
        for lane in self.lanes:
            batch, tot = [], 0
            for r in requests:
                if len(batch) < self.max_batch and tot + r.n <= self.lane_clusters:
                    batch.append(r)
                    tot += r.n
            if batch:
                lane.launch(batch, 0.0)
                lane.result.sync()
                lane.collect(0.0)

    def close(self):
        for l in self.lanes:
            l.tracker.close()


class NativeServer:
    """The native serving loop (``tpc_server_*``): lanes, batch forming, copies and the per-event
    split run in the library's own thread; Python only submits events and collects results."""

    def __init__(self, geometry, lanes=3, hbm_budget=40 << 30, max_batch=16, lane_clusters=None, params=None,
                 keep_results=True):
        if lane_clusters is None:
            lane_clusters = int(hbm_budget / lanes / BYTES_PER_CLUSTER)
        self.keep_results = keep_results           # False: record status and timing only (load tests)
        self.n_lanes = lanes
        self.lane_clusters = lane_clusters
        self.max_batch = max_batch
        self.handle = tpc_server_create(geometry.row_x, geometry.tan_half, geometry.z_max, geometry.n_sectors,
                                        geometry.bz, lanes, max_batch, lane_clusters, hbm_budget, params)
        self.inflight = {}
        self.done = []
        self.rejected = []
        self.high_water = 0

    def submit(self, r: Request, arrival_ns=None):
        try:
            rid = tpc_server_submit(self.handle, r.y, r.z, r.row, r.counts, r.n)
        except TrackerError:
            r.status = "rejected"
            self.rejected.append(r)
            return False
        r.arrival_ns = arrival_ns
        self.inflight[rid] = r
        self.high_water = max(self.high_water, len(self.inflight))
        return True

    def poll(self, now=None):
        ids = tpc_server_poll(self.handle)
        for rid in ids:
            r = self.inflight.pop(rid)
            res = tpc_server_get(self.handle, rid)
            r.status = "done" if res.status == 0 else "error %d" % res.status
            r.result = server_result_arrays(res) if res.status == 0 and self.keep_results else None
            r.batch_size = res.batch_size
            r.t_submit_ns, r.t_launch_ns, r.t_done_ns = res.t_submit_ns, res.t_launch_ns, res.t_done_ns
            tpc_server_release(self.handle, rid)
            self.done.append(r)
        return bool(ids)

    def busy(self):
        return bool(self.inflight)

    def warm(self, requests):
        """Every given event through the server before measuring, so that each lane's first-use
        costs (its executable graph, its pinned output buffers grown to the largest result) are
        paid before the first measured arrival: pass the whole event pool the stream draws from.
        The pool goes through once per lane, so that every lane sees large batches."""
        page_in_mapped_files()
        for _ in range(self.n_lanes):
            for r in requests:
                self.submit(dataclasses.replace(r))
        while self.busy():
            self.poll()
            time.sleep(50e-6)
        self.done.clear()

    def close(self):
        tpc_server_destroy(self.handle)


def run_stream_native(server: NativeServer, requests, realtime=True, idle_sleep=20e-6):
    """Submit requests at their arrival times (the server's clock) and collect them as they finish.
    Latency t_done - t_arrival counts any delay of the submission too."""
    import gc
    reqs = sorted(requests, key=lambda r: r.arrival)
    gc_was = gc.isenabled()
    gc.disable()                                   # no collector pauses between submissions
    t0 = tpc_server_now_ns()
    i = 0
    while i < len(reqs) or server.busy():
        now = (tpc_server_now_ns() - t0) * 1e-9
        while i < len(reqs) and (reqs[i].arrival <= now or not realtime):
            server.submit(reqs[i], arrival_ns=t0 + int(reqs[i].arrival * 1e9) if realtime else tpc_server_now_ns())
            i += 1
        if not server.poll():
            nxt = reqs[i].arrival - now if i < len(reqs) and realtime else idle_sleep
            time.sleep(min(idle_sleep, max(0.0, nxt)))
    wall = (tpc_server_now_ns() - t0) * 1e-9
    if gc_was:
        gc.enable()
    for r in reqs:
        if r.status == "done":
            r.t_done = (r.t_done_ns - t0) * 1e-9
            r.arrival = (r.arrival_ns - t0) * 1e-9
    return wall


def run_stream(server: Server, requests, realtime=True, idle_sleep=20e-6):
    """Feed requests at their arrival times (wall clock) and run until all are finished."""
    t0 = time.perf_counter()
    i = 0
    reqs = sorted(requests, key=lambda r: r.arrival)
    while i < len(reqs) or server.busy():
        now = time.perf_counter() - t0
        while i < len(reqs) and (reqs[i].arrival <= now or not realtime):
            server.submit(reqs[i])
            i += 1
        if not server.poll(now):
            if i < len(reqs) and realtime:
                time.sleep(min(idle_sleep, max(0.0, reqs[i].arrival - now)))
            else:
                time.sleep(idle_sleep)
    return time.perf_counter() - t0


def latency_report(requests, wall):
    done = [r for r in requests if r.status == "done"]
    lat = np.array([r.t_done - r.arrival for r in done]) * 1e3
    if not len(lat):
        return dict(n=0)
    return dict(n=len(done), rejected=sum(r.status == "rejected" for r in requests),
                errors=sum(r.status.startswith("error") for r in requests),
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                p999_ms=float(np.percentile(lat, 99.9)), max_ms=float(lat.max()),
                events_per_s=len(done) / wall, clusters_per_s=sum(r.n for r in done) / wall,
                mean_batch=float(np.mean([r.batch_size for r in done])), wall_s=wall)


def poisson_arrivals(rate_hz, duration_s, seed=0):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return np.array(out)
        out.append(t)


def _gen(args):
    from . import eventgen
    cfg, i = args
    ev = eventgen.config_event(cfg, event=i)
    return ev.y, ev.z, ev.row, ev.counts


_PAGED_IN = False


def page_in_mapped_files() -> int:
    """Read once every file this process has mapped (its shared libraries and the like), so that
    their pages are resident before latencies are measured.  On a host whose file system fetches
    pages on first touch, such faults in the middle of a serving run held up submissions and
    completions for tens of milliseconds (in about one 10 s run in four; none in twelve runs after
    this read).  Returns the bytes read; 0 after the first call or without /proc."""
    global _PAGED_IN
    if _PAGED_IN:
        return 0
    _PAGED_IN = True
    seen, total = set(), 0
    try:
        maps = open("/proc/self/maps").read().splitlines()
    except OSError:
        return 0
    for line in maps:
        parts = line.split()
        if len(parts) < 6 or not parts[5].startswith("/") or parts[5] in seen:
            continue
        seen.add(parts[5])
        try:
            # regular files only, at most their size: device mappings (the GPU driver's, /dev/zero)
            # would read without end
            st = os.stat(parts[5])
            if not stat.S_ISREG(st.st_mode):
                continue
            left = st.st_size
            with open(parts[5], "rb") as f:
                while left > 0:
                    b = f.read(min(left, 1 << 24))
                    if not b:
                        break
                    left -= len(b)
                    total += len(b)
        except OSError:
            pass
    return total


def event_pool(n_events, cfg=3, workers=8, first_event=0, pin=True):
    """Pre-generated events (drawn with replacement during a run): torch tensors, pinned in host
    memory unless ``pin`` is False (no CUDA needed then)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import torch
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        evs = list(ex.map(_gen, [(cfg, first_event + i) for i in range(n_events)]))
    pool = []
    for y, z, row, counts in evs:
        t = [torch.from_numpy(a) for a in (y, z, row)]
        if pin:
            t = [a.pin_memory() for a in t]
        pool.append((t[0], t[1], t[2], counts, int(y.shape[0])))
    return pool


def make_requests(pool, arrivals, seed=1):
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, len(pool), len(arrivals))
    return [Request(i, float(t), *pool[k][:3], pool[k][3], pool[k][4]) for i, (t, k) in enumerate(zip(arrivals, pick))]


def main():
    import argparse
    import json
    import torch
    from . import eventgen
    ap = argparse.ArgumentParser(description="serving loop at Poisson arrival rates")
    ap.add_argument("--rates", default="200,500,1000")
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--pool", type=int, default=64)
    ap.add_argument("--lanes", type=int, default=3)
    ap.add_argument("--max-batch", type=int, default=16)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--python", action="store_true", help="the Python loop instead of the native server")
    a = ap.parse_args()
    pool = event_pool(a.pool)
    geo = eventgen.Geometry()
    for rate in [float(r) for r in a.rates.split(",")]:
        for mode in ("batched", "per-event"):
            lanes, mb = (a.lanes, a.max_batch) if mode == "batched" else (1, 1)
            if a.python:
                srv = Server(geo, lanes=lanes, hbm_budget=int(a.budget_gb * (1 << 30)), max_batch=mb)
            else:
                srv = NativeServer(geo, lanes=lanes, hbm_budget=int(a.budget_gb * (1 << 30)), max_batch=mb,
                                   keep_results=False)
            srv.warm(make_requests(pool, np.zeros(len(pool)), seed=99))
            reqs = make_requests(pool, poisson_arrivals(rate, a.duration, seed=int(rate)), seed=int(rate))
            wall = (run_stream if a.python else run_stream_native)(srv, reqs)
            rep = latency_report(reqs, wall)
            rep.update(rate_hz=rate, mode=mode, lanes=lanes, max_batch=mb, budget_gb=a.budget_gb,
                       queue_high_water=srv.high_water, loop="python" if a.python else "native")
            print(json.dumps(rep), flush=True)
            srv.close()
            torch.cuda.synchronize()


if __name__ == "__main__":
    main()
