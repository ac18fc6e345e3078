"""Runs the tracker on fixed workloads and saves every output array (helper of test_gpu_checked.py,
started in a subprocess so that TPCCA_LIB can select the checked library)."""
import sys

import numpy as np
import torch

from paper_1712_09407_gb300 import eventgen
from paper_1712_09407_gb300.tracker import Tracker

CASES = [("c1", 1, {}, {}), ("c1_gm", 1, dict(global_tracking=True, merge=True), {}),
         ("c1_sweep_gm", 1, dict(global_tracking=True, merge=True), dict(construct_mode=1, use_graph=0)),
         ("c1_walk_g", 1, dict(global_tracking=True), dict(seed_kernel=0)), ("c2", 2, {}, {})]


def run(out_path):
    arrays = {}
    for name, cfg, flags, tuning in CASES:
        ev = eventgen.config_event(cfg)
        tr = Tracker.for_geometry(ev.geometry, **flags)
        if tuning:
            tr.set_tuning(tuning)
        r = tr.track(*(torch.from_numpy(a).cuda() for a in (ev.y, ev.z, ev.row)), ev.counts)
        out = r.to_numpy()
        r.release()
        tr.close()
        for k, v in out.items():
            arrays[name + "/" + k] = v
    np.savez(out_path, **arrays)


if __name__ == "__main__":
    run(sys.argv[1])
