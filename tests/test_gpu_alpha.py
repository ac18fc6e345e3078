"""The weight constant alpha (Section 3.1) on the GPU: parity with the float oracle at other values
of alpha (the weights decide the cluster ownership), and the alpha study's quality measures."""
import numpy as np
import pytest
import torch

import oracle
from paper_1712_09407_gb300 import alpha_study, eventgen
from paper_1712_09407_gb300.tracker import Tracker, tpc_params_default

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("alpha", [1.0, 1e6])
def test_other_alpha_equals_oracle(alpha):
    ev = eventgen.config_event(1)
    ref = oracle.track_event(oracle.config_for(ev.geometry, alpha=alpha), ev.y, ev.z, ev.row, ev.counts, precision=32)
    p = tpc_params_default()
    p.alpha = alpha
    tr = Tracker.for_geometry(ev.geometry, params=p)
    r = tr.track(*(torch.from_numpy(a).cuda() for a in (ev.y, ev.z, ev.row)), ev.counts)
    out = r.to_numpy()
    r.release()
    tr.close()
    assert np.array_equal(out["hits"], ref.trk_hits) and np.array_equal(out["nhits"], ref.trk_nhits)
    assert np.array_equal(out["par"], ref.trk_par.astype(np.float32))


def test_alpha_study_runs_and_alpha_6_is_efficient():
    lines = alpha_study.run(alphas=(1.0, 6.0, 1e6), workload=1, events=1)
    by = {l["alpha"]: l for l in lines}
    assert by[6.0]["efficiency"] >= 0.9
    for l in lines:
        assert 0 <= l["clone_rate"] <= 0.1 and 0 <= l["fake_rate"] <= 0.1
        assert all(0.5 < v < 2.0 for v in l["pull_width"].values()), l["pull_width"]
