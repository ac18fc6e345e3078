"""Autotuner of the launch and grid choices (``tpc_tuning``).

None of the tuned choices changes a result: every search visits all grid cells overlapping its
window and applies the exact window test, and the launch shapes only change which thread does
which work.  So the tuner may pick purely on time.  It times the tracker's own per-stage CUDA
events (``tpc_result_stats``) on a representative event and tunes the stages one after the
other: grid occupancy (ingest, neighbours and construction all depend on it), then the
neighbours finder's block and staging, then the constructor's block and CTAs per SM.

The chosen values can be cached as JSON keyed by device name and event size class.
"""
from __future__ import annotations

import json
import os

import numpy as np

from .tracker import Tracker, tpc_tuning_default

STAGES = ["setup", "ingest", "neighbours", "evolution", "construction", "selection", "output", "global", "merge"]


def _as_dict(t):
    return {f: getattr(t, f) for f, _ in t._fields_}


def time_stages(tracker: Tracker, y, z, row, counts, tuning: dict, repeats: int = 3, stream=None):
    """Median per-stage milliseconds of ``repeats`` calls with ``tuning``."""
    tracker.set_tuning(tuning)
    tracker.set_timing(True)
    r = tracker.track(y, z, row, counts, stream=stream)       # warm-up (compiles nothing, sizes pools)
    r.sync()
    r.release()
    ms = []
    for _ in range(repeats):
        r = tracker.track(y, z, row, counts, stream=stream)
        r.sync()
        ms.append(r.stats()["ms"])
        r.release()
    tracker.set_timing(False)
    return np.median(np.array(ms), axis=0)


# The search, in order: (field, candidates, stages whose time decides).
SPACE = [
    ("bin_occupancy", [0.5, 1.0, 1.5, 2.0, 3.0, 4.0], ["ingest", "neighbours", "construction"]),
    ("stage_rows", [0, 1, 2], ["neighbours"]),
    ("neighbours_block", [64, 128, 256], ["neighbours"]),
    ("construct_block", [64, 96, 128], ["construction"]),
    ("construct_ctas_per_sm", [0, 4, 6, 8, 10, 12], ["construction"]),
    ("seed_kernel", [0, 1], ["construction"]),
    ("use_graph", [0, 1], STAGES),
]


def tune(tracker: Tracker, y, z, row, counts, repeats: int = 3, stream=None, log=None, space=None) -> dict:
    """Coordinate search over the tuning space (``space``: a list like SPACE, default SPACE); each
    field in turn takes its candidate with the least time of the stages it affects, the others
    held at their best so far.  Returns the best tuning as a dict and sets it on the tracker."""
    best = _as_dict(tpc_tuning_default())

    def cost(t, stages):
        ms = time_stages(tracker, y, z, row, counts, t, repeats, stream)
        c = float(sum(ms[STAGES.index(s)] for s in stages))
        if log:
            log("%s -> %.4f ms %s" % (t, c, stages))
        return c

    def search(field, values, stages):
        scores = []
        for v in values:
            t = dict(best)
            t[field] = v
            scores.append((cost(t, stages), v))
        best[field] = min(scores)[1]

    for field, values, stages in (SPACE if space is None else space):
        search(field, values, stages)
    tracker.set_tuning(best)
    return best


def cache_key(device_name: str, n_clusters: int) -> str:
    size_class = int(np.log2(max(n_clusters, 1)))
    return "%s|2^%d" % (device_name, size_class)


def load(path: str, key: str):
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get(key)


def store(path: str, key: str, tuning: dict):
    d = json.load(open(path)) if os.path.exists(path) else {}
    d[key] = tuning
    json.dump(d, open(path, "w"), indent=1, sort_keys=True)


def main():
    import argparse
    import torch

    from . import eventgen
    ap = argparse.ArgumentParser(description="tune tpc_tuning on a synthetic workload")
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--cache", default=None, help="JSON file to store the result in")
    a = ap.parse_args()
    ev = eventgen.config_event(a.workload)
    tr = Tracker.for_geometry(ev.geometry)
    tr.reserve(ev.n, 1)
    y, z, row = (torch.from_numpy(v).cuda() for v in (ev.y, ev.z, ev.row))
    best = tune(tr, y, z, row, ev.counts, a.repeats, log=print)
    base = time_stages(tr, y, z, row, ev.counts, _as_dict(tpc_tuning_default()), a.repeats)
    tuned = time_stages(tr, y, z, row, ev.counts, best, a.repeats)
    print("default", dict(zip(STAGES, np.round(base, 4))), "total %.4f" % base.sum())
    print("tuned  ", dict(zip(STAGES, np.round(tuned, 4))), "total %.4f" % tuned.sum())
    print("best", json.dumps(best))
    if a.cache:
        store(a.cache, cache_key(torch.cuda.get_device_name(), ev.n), best)


if __name__ == "__main__":
    main()
