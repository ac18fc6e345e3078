"""Parity of the CUDA track merger with refit with the float-mode oracle, through the C ABI.

Both sides refit, match and merge with the same float operations in the same order, so the merged
tracks must be identical: the same tracks in the same order, the same clusters in the same order,
and bit-identical parameters, covariances, chi2, ndf, reference x and sector."""
import numpy as np
import pytest
import torch

import oracle
from paper_1712_09407_gb300 import eventgen
from paper_1712_09407_gb300.tracker import Tracker

from gpu_util import run_oracle
from test_oracle_merge import _find, _two_segments

pytestmark = pytest.mark.gpu


def _gpu(ev, y=None, z=None, **kw):
    tuning = kw.pop("tuning", None)
    tr = Tracker.for_geometry(ev.geometry, merge=True, **kw)
    if tuning:
        tr.set_tuning(tuning)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
         (ev.y if y is None else y.astype(np.float32), ev.z if z is None else z.astype(np.float32), ev.row)]
    res = tr.track(*d, ev.counts)
    out = res.to_numpy()
    st = res.stats()
    res.release()
    tr.close()
    return out, st


def _identical(out, ref):
    Mm = ref.info["n_merged"]
    assert len(out["first"]) == Mm, (len(out["first"]), Mm)
    assert np.array_equal(out["nhits"], ref.mrg_nhits)
    assert np.array_equal(out["first"], ref.mrg_first)
    assert np.array_equal(out["hits"], ref.mrg_hits)
    assert np.array_equal(out["ndf"], ref.mrg_ndf)
    assert np.array_equal(out["sector"], ref.mrg_sector)
    assert np.array_equal(out["x_ref"], ref.mrg_x.astype(np.float32))
    assert np.array_equal(out["par"], ref.mrg_par.astype(np.float32))
    assert np.array_equal(out["cov"], ref.mrg_cov.astype(np.float32))
    assert np.array_equal(out["chi2"], ref.mrg_chi2.astype(np.float32))


@pytest.mark.parametrize("cfg,global_tracking", [(1, False), (2, False), (1, True), (2, True)])
def test_merger_equals_oracle(cfg, global_tracking):
    ev = eventgen.config_event(cfg)
    ref = run_oracle(ev, key="c%d" % cfg, merge=True, global_tracking=global_tracking)
    out, st = _gpu(ev, global_tracking=global_tracking)
    print("config %d global %s: sector tracks %d -> merged %d (oracle %d -> %d)" % (
        cfg, global_tracking, st["sector_tracks"], st["tracks"], ref.info["n_tracks"], ref.info["n_merged"]))
    assert st["sector_tracks"] == ref.info["n_tracks"]
    _identical(out, ref)


def test_merger_with_sweep_constructor_and_stream_launches():
    ev = eventgen.config_event(1)
    ref = run_oracle(ev, key="c1", merge=True)
    out, _ = _gpu(ev, tuning=dict(construct_mode=1, use_graph=0))
    _identical(out, ref)


def test_particle_crossing_a_sector_edge_is_merged_on_the_gpu():
    ev = _find(lambda e: _two_segments(e, same_azimuth=False), eta_max=0.4)
    y, z = ev.truth[:, 0], ev.truth[:, 1]
    ref = oracle.track_event(oracle.config_for(ev.geometry, merge=True), y, z, ev.row, ev.counts, precision=32)
    out, st = _gpu(ev, y=y, z=z)
    assert st["sector_tracks"] == 2 and len(out["first"]) == 1 and out["nhits"][0] == ev.n
    _identical(out, ref)


def test_merged_batch_equals_one_at_a_time():
    evs = [eventgen.config_event(1, event=i) for i in range(2)]
    tr = Tracker.for_geometry(evs[0].geometry, merge=True)
    singles = []
    for ev in evs:
        r = tr.track(*(torch.from_numpy(a).cuda() for a in (ev.y, ev.z, ev.row)), ev.counts)
        singles.append(r.to_numpy())
        r.release()
    y = torch.from_numpy(np.concatenate([e.y for e in evs])).cuda()
    z = torch.from_numpy(np.concatenate([e.z for e in evs])).cuda()
    row = torch.from_numpy(np.concatenate([e.row for e in evs])).cuda()
    r = tr.track_batch(y, z, row, np.concatenate([e.counts for e in evs]), len(evs))
    b = r.to_numpy()
    r.release()
    tr.close()
    off_t = off_h = off_in = 0
    for i, (ev, s) in enumerate(zip(evs, singles)):
        M, H = len(s["first"]), len(s["hits"])
        assert np.all(b["event"][off_t:off_t + M] == i)
        for k in ("par", "cov", "x_ref", "chi2", "ndf", "nhits", "sector", "alpha"):
            assert np.array_equal(b[k][off_t:off_t + M], s[k]), k
        assert np.array_equal(b["first"][off_t:off_t + M] - off_h, s["first"])
        assert np.array_equal(b["hits"][off_h:off_h + H] - off_in, s["hits"])
        off_t += M
        off_h += H
        off_in += ev.n
