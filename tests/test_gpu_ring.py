"""Preallocated result buffers (tpc_tracker_reserve_results): a tracker serving a stream of events
keeps its output buffers resident, so tracking calls allocate nothing; results held by the caller
count against the ring and a call finding it full is refused (TPC_ERR_BUDGET) instead of
allocating (Section 2: output buffers per sector kept resident; Section 6: device memory
exhausted by a noisy sector).  Results from the ring equal those of per-call allocation, call
after call, with several results held at once and buffers reused across calls."""
import numpy as np
import pytest
import torch

from paper_1712_09407_gb300 import eventgen
from paper_1712_09407_gb300.tracker import (TPC_ERR_BUDGET, TPC_ERR_STATE, Tracker, TrackerError,
                                            tpc_tracker_reserve_results)

from gpu_util import to_device

pytestmark = pytest.mark.gpu


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


def test_ring_results_equal_allocated_results_and_full_ring_refuses():
    evs = [eventgen.config_event(1, event=i) for i in range(3)]
    dev = [to_device(ev) for ev in evs]
    ref_tr = Tracker.for_geometry(evs[0].geometry)
    ref = []
    for ev, (y, z, row) in zip(evs, dev):
        r = ref_tr.track(y, z, row, ev.counts)
        r.sync()
        ref.append(r.to_numpy())
        r.release()
    ref_tr.close()

    tr = Tracker.for_geometry(evs[0].geometry)
    with pytest.raises(TrackerError) as e:        # the buffers are sized from the reserved workspace
        tpc_tracker_reserve_results(tr.handle, 2)
    assert e.value.status == TPC_ERR_STATE
    tr.reserve(max(ev.n for ev in evs), 1, results=2)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for rnd in range(3):                      # the two buffers are reused round after round
            a = tr.track(*dev[rnd % 3], evs[rnd % 3].counts, stream=stream)
            b = tr.track(*dev[(rnd + 1) % 3], evs[(rnd + 1) % 3].counts, stream=stream)
            with pytest.raises(TrackerError) as e:   # both buffers are held: refused, nothing enqueued
                tr.track(*dev[0], evs[0].counts, stream=stream)
            assert e.value.status == TPC_ERR_BUDGET
            a.sync()
            b.sync()
            assert _same(a.to_numpy(), ref[rnd % 3]), rnd
            assert _same(b.to_numpy(), ref[(rnd + 1) % 3]), rnd
            a.release()
            c = tr.track(*dev[(rnd + 2) % 3], evs[(rnd + 2) % 3].counts, stream=stream)
            c.sync()
            assert _same(c.to_numpy(), ref[(rnd + 2) % 3]), rnd
            b.release()
            c.release()
    # back to one allocation per call: more results than the ring held at once
    tr.reserve(max(ev.n for ev in evs), 1, results=0)
    rs = [tr.track(*dev[i], evs[i].counts) for i in range(3)]
    for i, r in enumerate(rs):
        r.sync()
        assert _same(r.to_numpy(), ref[i])
        r.release()
    tr.close()


def test_ring_grows_with_the_workspace():
    small, big = eventgen.config_event(0), eventgen.config_event(1)
    tr = Tracker.for_geometry(big.geometry)
    tr.reserve(small.n, 1, results=1)             # sized for the small event
    ref_tr = Tracker.for_geometry(big.geometry)
    r0 = ref_tr.track(*to_device(big), big.counts)
    r0.sync()
    ref = r0.to_numpy()
    r0.release()
    ref_tr.close()
    r = tr.track(*to_device(big), big.counts)     # grows the workspace and the buffer it takes
    r.sync()
    assert _same(r.to_numpy(), ref)
    r.release()
    tr.close()


def test_ring_results_survive_tracker_destroy():
    ev = eventgen.config_event(1)
    tr = Tracker.for_geometry(ev.geometry)
    tr.reserve(ev.n, 1, results=2)
    r = tr.track(*to_device(ev), ev.counts)
    m, h = r.sync()
    out = r.to_numpy()
    tr.close()                                    # the held result stays readable until released
    assert out["hits"].shape[0] == h and m > 0
    again = r.to_numpy()
    assert _same(again, out)
    r.release()
