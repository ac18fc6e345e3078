"""The autotuner (autotune.tune) end to end on a small 36-sector event: it runs its coordinate
search through the tracker's own stage timers, the tuning it picks is accepted by
tpc_tracker_set_tuning, gives bit-identical results to the default tuning (no tuned choice may
change a result: every search visits all grid cells overlapping its window and applies the exact
window test), and round-trips through the JSON cache."""
import numpy as np
import pytest
import torch

from paper_1712_09407_gb300 import autotune, eventgen
from paper_1712_09407_gb300.tracker import Tracker, tpc_tuning_default

from gpu_util import to_device

pytestmark = pytest.mark.gpu

NARROW = [
    ("bin_occupancy", [0.5, 2.0], ["ingest", "neighbours", "construction"]),
    ("stage_rows", [1, 2], ["neighbours"]),
    ("neighbours_block", [128, 256], ["neighbours"]),
    ("construct_block", [64, 128], ["construction"]),
    ("construct_ctas_per_sm", [0, 6], ["construction"]),
    ("seed_kernel", [0, 1], ["construction"]),
    ("use_graph", [0, 1], autotune.STAGES),
]


def _track(tr, dev, ev):
    r = tr.track(*dev, ev.counts)
    r.sync()
    out = r.to_numpy()
    r.release()
    return out


def test_autotuner_picks_valid_tuning_with_identical_results(tmp_path):
    spec = eventgen.EventSpec(n_primaries=800, n_secondaries=100, pt_cut=0.05, noise_frac=0.15)
    ev = eventgen.generate_event(spec, eventgen.Geometry(), seed=11)
    dev = to_device(ev)
    ref_tr = Tracker.for_geometry(ev.geometry)
    ref = _track(ref_tr, dev, ev)
    ref_tr.close()

    tr = Tracker.for_geometry(ev.geometry)
    tr.reserve(ev.n, 1)
    lines = []
    best = autotune.tune(tr, *dev, ev.counts, repeats=2, log=lines.append, space=NARROW)
    assert len(lines) == sum(len(v) for _, v, _ in NARROW)        # every candidate was timed
    for field, values, _ in NARROW:
        assert best[field] in values, field
    default = {f: getattr(tpc_tuning_default(), f) for f, _ in tpc_tuning_default()._fields_}
    assert set(best) == set(default)
    out = _track(tr, dev, ev)                                     # tune() left the best tuning set
    assert all(np.array_equal(out[k], ref[k]) for k in ref)
    # every candidate of the narrowed space, one field at a time, gives the same results
    for field, values, _ in NARROW:
        for v in values:
            t = dict(default)
            t[field] = v
            tr.set_tuning(t)
            o = _track(tr, dev, ev)
            assert all(np.array_equal(o[k], ref[k]) for k in ref), (field, v)
    # the JSON cache round-trips the tuning under its key
    path = str(tmp_path / "tuning.json")
    key = autotune.cache_key(torch.cuda.get_device_name(), ev.n)
    autotune.store(path, key, best)
    assert autotune.load(path, key) == best
    assert autotune.load(path, "other") is None
    tr.set_tuning(autotune.load(path, key))
    assert all(np.array_equal(_track(tr, dev, ev)[k], ref[k]) for k in ref)
    tr.close()
