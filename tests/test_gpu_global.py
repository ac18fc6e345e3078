"""Parity of the CUDA global tracking (Section 5) with the float-mode oracle, through the C ABI.

Both sides evaluate the prolongations with the same float operations in the same order, so the
comparison is exact: the same tracks in the same order, the same clusters in the same order, and
bit-identical parameters, covariances, chi2, ndf, reference x and sector.  The contract's bar
(concordance >= 99.99 %, parameters within 1e-4 relative) is asserted first so that a failure
says which bar broke.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1712_09407_gb300 import eventgen
from paper_1712_09407_gb300.tracker import Tracker

from gpu_util import compare_tracks, run_gpu, run_oracle
from test_oracle_global import _find_two_sector_track

pytestmark = pytest.mark.gpu

CONCORDANCE_MIN = 0.9999
PAR_REL = 1e-4


def _gpu_global(ev, y=None, z=None, tuning=None):
    tr = Tracker.for_geometry(ev.geometry, global_tracking=True)
    if tuning is not None:
        tr.set_tuning(tuning)
    yy = torch.from_numpy(np.ascontiguousarray(ev.y if y is None else y, dtype=np.float32)).cuda()
    zz = torch.from_numpy(np.ascontiguousarray(ev.z if z is None else z, dtype=np.float32)).cuda()
    rr = torch.from_numpy(ev.row).cuda()
    res = tr.track(yy, zz, rr, ev.counts)
    res.sync()
    out = res.to_numpy()
    st = res.stats()
    res.release()
    tr.close()
    return out, st


def _assert_identical(out, ref):
    M = ref.info["n_tracks"]
    assert len(out["first"]) == M
    assert np.array_equal(out["nhits"], ref.trk_nhits)
    assert np.array_equal(out["first"], ref.trk_first)
    assert np.array_equal(out["hits"], ref.trk_hits)
    assert np.array_equal(out["ndf"], ref.trk_ndf)
    assert np.array_equal(out["sector"], ref.trk_sector)
    assert np.array_equal(out["x_ref"], ref.trk_x.astype(np.float32))
    assert np.array_equal(out["par"], ref.trk_par.astype(np.float32))
    assert np.array_equal(out["cov"], ref.trk_cov.astype(np.float32))
    assert np.array_equal(out["chi2"], ref.trk_chi2.astype(np.float32))


def _check(ev, out, ref, label):
    c = compare_tracks(ev, out, ref)
    print("%s: gpu %d oracle %d concordance %.7f exact %d/%d par max %s global clusters %d" % (
        label, c["n_test"], c["n_ref"], c["concordance"], c["n_exact"], c["n_matched"], c["par_rel_max"],
        int(ref.trk_nglobal.sum())))
    assert c["concordance"] >= CONCORDANCE_MIN
    assert c["par_rel_max"].max() <= PAR_REL
    _assert_identical(out, ref)


@pytest.mark.parametrize("cfg", [1, 2])
def test_global_tracking_equals_oracle(cfg):
    """Config 1 (mid-size event) and config 2 (the central-like benchmark event)."""
    ev = eventgen.config_event(cfg)
    ref = run_oracle(ev, key="c%d" % cfg, global_tracking=True)
    assert ref.trk_nglobal.sum() > 0
    out, st = _gpu_global(ev)
    assert st["global_found"] >= int(ref.trk_nglobal.sum())
    _check(ev, out, ref, "config %d global" % cfg)


def test_global_tracking_with_sweep_constructor():
    ev = eventgen.config_event(1)
    ref = run_oracle(ev, key="c1", global_tracking=True)
    out, _ = _gpu_global(ev, tuning=dict(construct_mode=1))
    _check(ev, out, ref, "config 1 global, sector sweep")


def test_global_tracking_keeps_the_sector_tracks():
    """Section 5: the same tracks as without global tracking, each a superset of its clusters."""
    ev = eventgen.config_event(1)
    _, out0, _ = run_gpu(ev, debug=False)
    out1, _ = _gpu_global(ev)
    assert len(out0["first"]) == len(out1["first"])
    assert np.all(out1["nhits"] >= out0["nhits"])
    for m in range(len(out0["first"])):
        h0 = out0["hits"][out0["first"][m]:out0["first"][m] + out0["nhits"][m]]
        h1 = out1["hits"][out1["first"][m]:out1["first"][m] + out1["nhits"][m]]
        assert set(h0.tolist()) <= set(h1.tolist())
    assert np.unique(out1["hits"]).size == out1["hits"].size


@pytest.mark.parametrize("inward_short", [True, False])
def test_short_segment_in_the_neighbour_sector(inward_short):
    """A noise-free particle crossing a sector edge: its short segment is merged into the track."""
    ev, short = _find_two_sector_track(inward_short=inward_short)
    y, z = ev.truth[:, 0], ev.truth[:, 1]
    ref = oracle.track_event(oracle.config_for(ev.geometry, global_tracking=True), y, z, ev.row, ev.counts,
                             precision=32)
    out, _ = _gpu_global(ev, y=y, z=z)
    assert len(out["first"]) == 1 and out["nhits"][0] == ev.n
    _assert_identical(out, ref)


def test_global_tracking_in_a_batch_equals_one_at_a_time():
    evs = [eventgen.config_event(1, event=i) for i in range(2)]
    tr = Tracker.for_geometry(evs[0].geometry, global_tracking=True)
    singles = []
    for ev in evs:
        res = tr.track(*(torch.from_numpy(a).cuda() for a in (ev.y, ev.z, ev.row)), ev.counts)
        singles.append(res.to_numpy())
        res.release()
    y = torch.from_numpy(np.concatenate([e.y for e in evs])).cuda()
    z = torch.from_numpy(np.concatenate([e.z for e in evs])).cuda()
    row = torch.from_numpy(np.concatenate([e.row for e in evs])).cuda()
    res = tr.track_batch(y, z, row, np.concatenate([e.counts for e in evs]), len(evs))
    b = res.to_numpy()
    res.release()
    tr.close()
    off_t = off_h = off_in = 0
    for i, (ev, s) in enumerate(zip(evs, singles)):
        M, H = len(s["first"]), len(s["hits"])
        assert np.all(b["event"][off_t:off_t + M] == i)
        for k in ("par", "cov", "x_ref", "chi2", "ndf", "nhits", "sector"):
            assert np.array_equal(b[k][off_t:off_t + M], s[k]), k
        assert np.array_equal(b["first"][off_t:off_t + M] - off_h, s["first"])
        assert np.array_equal(b["hits"][off_h:off_h + H] - off_in, s["hits"])
        off_t += M
        off_h += H
        off_in += ev.n
