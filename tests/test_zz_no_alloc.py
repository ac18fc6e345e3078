"""The allocation-free link finder (tpc_find_links_noalloc) against the allocating tracker.

Some callers cannot allocate device memory once they are running (their framework owns all
of it, or they must not stall the device with cudaMalloc during data taking).  For them the
library offers the neighbours finder and evolution with its intermediate data in a static
device array.  This checks, through the C ABI, that two calls in a row give exactly the links
the allocating path (tpc_track_event) computes, and that oversized events are refused.  The
file runs last in the suite so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

from paper_1712_09407_gb300 import eventgen
from paper_1712_09407_gb300.tracker import TPC_ERR_INVALID_ARG, TPC_OK, Tracker, tpc_find_links_noalloc

from gpu_util import links_as_input_indices, run_gpu, to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [0, 1])
def test_noalloc_links_equal_allocating_path(cfg):
    ev = eventgen.config_event(cfg)
    tr, _, dbg = run_gpu(ev)                      # existing entry point, then its per-stage buffers
    ref = links_as_input_indices(dbg, ev.n)
    y, z, row = to_device(ev)
    for call in range(2):                         # two calls in a row share the static scratch
        up = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
        dn = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
        status = torch.full((4,), -1, dtype=torch.int32, device="cuda")
        rc = tpc_find_links_noalloc(tr.handle, y, z, row, ev.counts, up, dn, status)
        assert rc == TPC_OK, rc
        torch.cuda.synchronize()
        assert status[0].item() == 0, status.tolist()
        assert np.array_equal(up.cpu().numpy(), ref["up"]), call
        assert np.array_equal(dn.cpu().numpy(), ref["dn"]), call
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
