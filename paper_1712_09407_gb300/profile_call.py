"""A few calls of the tracker on central-like events and nothing else, for a profiler.

``python -m paper_1712_09407_gb300.profile_call --events 3 --calls 2`` generates the resident
events, creates one tracker sized for one call, and runs --calls calls of --events events each
(tpc_track_batch; the first call builds the graph).  It times nothing and holds no more device
memory than one call needs (inputs, workspace, one result), so that a profiler replaying a kernel
many times saves and restores only a few GB.
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--events", type=int, default=3, help="central-like events per call")
    ap.add_argument("--calls", type=int, default=2)
    ap.add_argument("--global-tracking", action="store_true")
    ap.add_argument("--merge", action="store_true")
    ap.add_argument("--tuning", default="", help="launch choices, e.g. stage_rows=1,construct_mode=1")
    a = ap.parse_args()
    import torch

    from . import eventgen
    from .build import build
    from .serving import event_pool
    from .tracker import Tracker
    build()
    pool = event_pool(a.events, cfg=2, pin=False)
    y = torch.cat([p[0] for p in pool]).cuda()
    z = torch.cat([p[1] for p in pool]).cuda()
    row = torch.cat([p[2] for p in pool]).cuda()
    counts = np.concatenate([p[3] for p in pool])
    tr = Tracker.for_geometry(eventgen.Geometry(), global_tracking=a.global_tracking or None, merge=a.merge or None)
    if a.tuning:
        tr.set_tuning({k: (float(v) if "." in v else int(v)) for k, v in (kv.split("=") for kv in a.tuning.split(","))})
    tr.reserve(int(y.shape[0]), a.events, results=1)
    for _ in range(a.calls):
        r = tr.track_batch(y, z, row, counts, a.events)
        m, h = r.sync()
        r.release()
    torch.cuda.synchronize()
    print("profile_call: %d calls of %d events (%d clusters), %d tracks in the last" % (a.calls, a.events, y.shape[0], m))
    tr.close()


if __name__ == "__main__":
    main()
