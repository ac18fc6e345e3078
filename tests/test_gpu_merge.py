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


# ---------------------------------------------------------------------------------------------
# edge cases of the optional stages
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("flags", [dict(global_tracking=True), dict(merge=True), dict(global_tracking=True, merge=True)])
def test_optional_stages_on_empty_and_noise_only_events(flags):
    geo = eventgen.Geometry()
    tr = Tracker.for_geometry(geo, **flags)
    e = torch.zeros(0, device="cuda")
    r = tr.track(e, e, torch.zeros(0, dtype=torch.uint8, device="cuda"), np.zeros(36 * 159, np.int32))
    assert r.sync() == (0, 0)
    r.release()
    rng = np.random.default_rng(1)
    counts = rng.integers(0, 4, 36 * 159).astype(np.int32)         # sparse noise, ragged rows
    n = int(counts.sum())
    row = np.repeat(np.tile(np.arange(159), 36), counts).astype(np.uint8)
    half = geo.row_x[row] * geo.tan_half
    y = (rng.uniform(-1, 1, n) * half).astype(np.float32)
    z = rng.uniform(-250, 250, n).astype(np.float32)
    sec = np.repeat(np.repeat(np.arange(36), 159), counts)
    z = np.where(sec < 18, np.abs(z), -np.abs(z)).astype(np.float32)
    r = tr.track(*(torch.from_numpy(a).cuda() for a in (y, z, row)), counts)
    M, H = r.sync()
    out = r.to_numpy()
    r.release()
    ref = oracle.track_event(oracle.config_for(geo, **flags), y, z, row, counts, precision=32)
    assert M == (ref.info["n_merged"] if flags.get("merge") else ref.info["n_tracks"])
    tr.close()


def test_flags_are_ignored_on_the_single_sector_geometry():
    """Global tracking and the merger need the 36-sector geometry; with one sector they are off."""
    ev = eventgen.config_event(0)
    plain = Tracker.for_geometry(ev.geometry)
    both = Tracker.for_geometry(ev.geometry, global_tracking=True, merge=True)
    d = tuple(torch.from_numpy(a).cuda() for a in (ev.y, ev.z, ev.row))
    ra, rb = plain.track(*d, ev.counts), both.track(*d, ev.counts)
    a, b = ra.to_numpy(), rb.to_numpy()
    ra.release()
    rb.release()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    plain.close()
    both.close()


def test_merger_with_a_small_tracklet_capacity_reports_capacity():
    """A tracklet pool too small for the event fails the call with TPC_ERR_CAPACITY, merger or not."""
    from paper_1712_09407_gb300.tracker import TrackerError, TPC_ERR_CAPACITY
    ev = eventgen.config_event(1)
    tr = Tracker.for_geometry(ev.geometry, global_tracking=True, merge=True)
    tr.set_tuning(dict(tracklet_capacity=100))
    r = tr.track(*(torch.from_numpy(a).cuda() for a in (ev.y, ev.z, ev.row)), ev.counts)
    with pytest.raises(TrackerError) as e:
        r.sync()
    assert e.value.status == TPC_ERR_CAPACITY
    r.release()
    tr.set_tuning(dict(tracklet_capacity=0))
    r = tr.track(*(torch.from_numpy(a).cuda() for a in (ev.y, ev.z, ev.row)), ev.counts)
    r.sync()
    r.release()
    tr.close()
