"""The allocation-free link finder (tpc_find_links_noalloc) against the oracle and the allocating tracker.

Some callers cannot allocate device memory once they are running (their framework owns all
of it, or they must not stall the device with cudaMalloc during data taking).  For them the
library offers the neighbours finder and evolution with its intermediate data in a static
device array.  This checks, through the C ABI, that two calls in a row give exactly the kept
links of the float oracle (Section 1: neighbours finder and evolution step) and of the
allocating path (tpc_track_event), that a call without a status buffer gives the same links,
and that bad input is refused: oversized events and counts that do not sum to n on the host,
a cluster whose row byte disagrees with counts through the device status.  The file runs last
in the suite so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

from paper_1712_09407_gb300 import eventgen
from paper_1712_09407_gb300.tracker import TPC_ERR_INVALID_ARG, TPC_OK, Tracker, tpc_find_links_noalloc

from gpu_util import links_as_input_indices, run_gpu, run_oracle, to_device

pytestmark = pytest.mark.gpu

TPC_STAGE_INGEST = 1


def _call(tr, ev, y, z, row, counts=None, with_status=True, n=None):
    up = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
    dn = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((4,), -1, dtype=torch.int32, device="cuda") if with_status else None
    rc = tpc_find_links_noalloc(tr.handle, y, z, row, ev.counts if counts is None else counts, up, dn, status, n=n)
    torch.cuda.synchronize()
    return rc, up.cpu().numpy(), dn.cpu().numpy(), (status.cpu().numpy() if with_status else None)


@pytest.mark.parametrize("cfg", [0, 1])
def test_noalloc_links_equal_oracle_and_allocating_path(cfg):
    ev = eventgen.config_event(cfg)
    ref = run_oracle(ev, key=("noalloc", cfg))
    tr, _, dbg = run_gpu(ev)                      # existing entry point, then its per-stage buffers
    alloc = links_as_input_indices(dbg, ev.n)
    y, z, row = to_device(ev)
    for call in range(2):                         # two calls in a row share the static scratch
        rc, up, dn, status = _call(tr, ev, y, z, row)
        assert rc == TPC_OK, rc
        assert status[0] == 0, status.tolist()
        assert np.array_equal(up, ref.up), call
        assert np.array_equal(dn, ref.dn), call
        assert np.array_equal(up, alloc["up"]), call
        assert np.array_equal(dn, alloc["dn"]), call
    rc, up, dn, _ = _call(tr, ev, y, z, row, with_status=False)
    assert rc == TPC_OK
    assert np.array_equal(up, ref.up) and np.array_equal(dn, ref.dn)
    tr.close()


def test_noalloc_rejects_events_beyond_its_limit():
    geo = eventgen.Geometry()
    tr = Tracker.for_geometry(geo)
    small = torch.zeros(4, device="cuda")
    counts = np.zeros(36 * 159, np.int32)
    counts[0] = 1048577                          # one more than TPC_NOALLOC_MAX_CLUSTERS
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = tpc_find_links_noalloc(tr.handle, small, small, small.to(torch.uint8), counts, out, out, None, n=1048577)
    assert rc == TPC_ERR_INVALID_ARG
    tr.close()


def test_noalloc_rejects_bad_counts_and_reports_a_wrong_row():
    ev = eventgen.config_event(0)
    tr = Tracker.for_geometry(ev.geometry)
    y, z, row = to_device(ev)
    counts = ev.counts.copy()
    counts[np.nonzero(counts)[0][0]] -= 1        # sums to n - 1
    rc, _, _, _ = _call(tr, ev, y, z, row, counts=counts)
    assert rc == TPC_ERR_INVALID_ARG
    bad = ev.row.copy()
    bad[ev.n // 2] = (int(bad[ev.n // 2]) + 1) % 159   # one cluster's row byte disagrees with counts
    rc, _, _, status = _call(tr, ev, y, z, torch.from_numpy(bad).cuda())
    assert rc == TPC_OK                           # detected on the device, reported through status
    assert status[0] == TPC_ERR_INVALID_ARG and status[3] == TPC_STAGE_INGEST, status.tolist()
    rc, up, dn, status = _call(tr, ev, y, z, row)   # the next call starts clean
    assert rc == TPC_OK and status[0] == 0
    ref = run_oracle(ev, key=("noalloc", 0))
    assert np.array_equal(up, ref.up) and np.array_equal(dn, ref.dn)
    tr.close()
