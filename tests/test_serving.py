"""Serving loop: continuous batching gives every event the same result as tracking it alone,
refuses events beyond a lane's reservation, and isolates a failing event of a batch."""
import numpy as np
import pytest
import torch

from paper_1712_09407_gb300 import eventgen, serving
from paper_1712_09407_gb300.tracker import Tracker

pytestmark = pytest.mark.gpu


def _pool(k, seed=3):
    pool = []
    for i in range(k):
        spec = eventgen.EventSpec(n_primaries=300 + 400 * i, noise_frac=0.05 + 0.03 * i, pt_cut=0.08)
        ev = eventgen.generate_event(spec, eventgen.Geometry(), seed=seed, event=i)
        pool.append((torch.from_numpy(ev.y).pin_memory(), torch.from_numpy(ev.z).pin_memory(),
                     torch.from_numpy(ev.row).pin_memory(), ev.counts, ev.n))
    return pool


def _alone(pool):
    tr = Tracker.for_geometry(eventgen.Geometry())
    outs = []
    for y, z, row, counts, n in pool:
        r = tr.track(y.cuda(), z.cuda(), row.cuda(), counts)
        r.sync()
        outs.append(r.to_numpy())
        r.release()
    tr.close()
    return outs


def test_alone_equals_in_the_mix():
    pool = _pool(6)
    alone = _alone(pool)
    srv = serving.Server(eventgen.Geometry(), lanes=2, hbm_budget=4 << 30, max_batch=4)
    arrivals = np.linspace(0.0, 0.002, 18)               # a burst: batches form and lanes overlap
    reqs = serving.make_requests(pool, arrivals, seed=5)
    serving.run_stream(srv, reqs)
    srv.close()
    assert all(r.status == "done" for r in reqs)
    assert max(r.batch_size for r in reqs) > 1
    for r in reqs:
        k = [i for i, p in enumerate(pool) if p[0] is r.y][0]
        a = alone[k]
        for key in ("par", "cov", "x_ref", "chi2", "ndf", "nhits", "first", "sector", "hits"):
            assert np.array_equal(r.result[key], a[key]), (r.rid, key)


def test_admission_refuses_oversized_events():
    pool = _pool(2)
    srv = serving.Server(eventgen.Geometry(), lanes=1, hbm_budget=1 << 30, max_batch=2,
                         lane_clusters=pool[0][4] + 10)
    reqs = serving.make_requests(pool, [0.0, 0.0, 0.0, 0.0], seed=1)
    serving.run_stream(srv, reqs, realtime=False)
    srv.close()
    for r in reqs:
        assert r.status == ("done" if r.n <= pool[0][4] + 10 else "rejected")


def test_failing_event_is_isolated_from_its_batch():
    pool = _pool(3)
    bad = list(pool[1])
    bad_row = bad[2].clone()
    bad_row[5] = (int(bad_row[5]) + 7) % 159              # a cluster whose row byte disagrees with counts
    bad[2] = bad_row.pin_memory()
    pool[1] = tuple(bad)
    srv = serving.Server(eventgen.Geometry(), lanes=1, hbm_budget=2 << 30, max_batch=3)
    reqs = serving.make_requests(pool, [0.0, 0.0, 0.0], seed=0)
    for i, r in enumerate(reqs):                          # one request per pool event, in order
        r.y, r.z, r.row, r.counts, r.n = pool[i]
    serving.run_stream(srv, reqs, realtime=False)
    srv.close()
    assert [r.status for r in reqs] == ["done", "error 1", "done"]


# ---------------------------------------------------------------------------------------------
# the native serving loop (tpc_server_*)
# ---------------------------------------------------------------------------------------------
def test_native_server_alone_equals_in_the_mix():
    pool = _pool(6)
    alone = _alone(pool)
    srv = serving.NativeServer(eventgen.Geometry(), lanes=2, hbm_budget=4 << 30, max_batch=4)
    arrivals = np.linspace(0.0, 0.002, 24)
    reqs = serving.make_requests(pool, arrivals, seed=7)
    serving.run_stream_native(srv, reqs)
    srv.close()
    assert all(r.status == "done" for r in reqs)
    assert max(r.batch_size for r in reqs) > 1
    for r in reqs:
        assert r.t_submit_ns <= r.t_launch_ns <= r.t_done_ns
        k = [i for i, p in enumerate(pool) if p[0] is r.y][0]
        a = alone[k]
        for key in ("par", "cov", "x_ref", "chi2", "ndf", "nhits", "first", "sector", "hits"):
            assert np.array_equal(r.result[key], a[key]), (r.rid, key)


def test_native_server_refuses_oversized_events_and_isolates_failures():
    pool = _pool(3)
    bad = list(pool[1])
    bad_row = bad[2].clone()
    bad_row[5] = (int(bad_row[5]) + 7) % 159
    bad[2] = bad_row.pin_memory()
    pool[1] = tuple(bad)
    srv = serving.NativeServer(eventgen.Geometry(), lanes=1, hbm_budget=2 << 30, max_batch=3,
                               lane_clusters=pool[1][4] + 10)
    reqs = serving.make_requests(pool, [0.0, 0.0, 0.0], seed=0)
    for i, r in enumerate(reqs):
        r.y, r.z, r.row, r.counts, r.n = pool[i]
    serving.run_stream_native(srv, reqs, realtime=False)
    srv.close()
    expect = []
    for i in range(3):
        if pool[i][4] > pool[1][4] + 10:
            expect.append("rejected")
        else:
            expect.append("error 1" if i == 1 else "done")
    assert [r.status for r in reqs] == expect


def test_native_server_drains_its_queue_on_destroy():
    pool = _pool(2)
    srv = serving.NativeServer(eventgen.Geometry(), lanes=1, hbm_budget=2 << 30, max_batch=2)
    reqs = serving.make_requests(pool, np.zeros(6), seed=2)
    for r in reqs:
        srv.submit(r)
    srv.close()                    # returns once every queued event is tracked
