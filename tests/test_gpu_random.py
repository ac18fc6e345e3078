"""Randomised parity: seeded small events of varied recipes (multiplicity, secondaries, pT cut, noise,
eta range) tracked with varied readings of the open points (chi2 gate, window width, miss limit,
chain length, minimum clusters, alpha), the optional stages and the seed launch switched at random.
The CUDA path and the float oracle evaluate the same operations, so every case must be identical:
the same tracks with the same clusters and bit-identical parameters."""
import numpy as np
import pytest
import torch

import oracle
from paper_1712_09407_gb300 import eventgen
from paper_1712_09407_gb300.tracker import Tracker, tpc_params_default

pytestmark = pytest.mark.gpu

CASES = 16


def _case(k):
    rng = np.random.default_rng(1000 + k)
    spec = eventgen.EventSpec(n_primaries=int(rng.integers(20, 900)), n_secondaries=int(rng.integers(0, 200)),
                              pt_cut=float(rng.choice([0.05, 0.1, 0.2, 0.4])),
                              noise_frac=float(rng.choice([0.0, 0.05, 0.2, 0.4])),
                              eta_max=float(rng.choice([0.3, 0.9])))
    readings = dict(chi2_max=float(rng.choice([9.0, 16.0, 25.0])), win_nsigma=float(rng.choice([2.5, 3.0, 4.0])),
                    max_miss=int(rng.choice([3, 10])), min_chain=int(rng.choice([3, 4])),
                    min_clusters=int(rng.choice([20, 30])), alpha=float(rng.choice([2.0, 6.0])))
    flags = dict(global_tracking=bool(rng.integers(0, 2)), merge=bool(rng.integers(0, 2)))
    tuning = dict(seed_kernel=int(rng.integers(0, 2)), order_group=int(rng.choice([0, 4096, 4 << 20])))
    return spec, readings, flags, tuning


@pytest.mark.parametrize("k", range(CASES))
def test_random_case_equals_oracle(k):
    spec, readings, flags, tuning = _case(k)
    ev = eventgen.generate_event(spec, eventgen.Geometry(), seed=77, event=k)
    ref = oracle.track_event(oracle.config_for(ev.geometry, **readings, **flags), ev.y, ev.z, ev.row, ev.counts,
                             precision=32)
    p = tpc_params_default()
    for name, v in readings.items():
        setattr(p, name, v)
    tr = Tracker.for_geometry(ev.geometry, params=p, **flags)
    tr.set_tuning(tuning)
    r = tr.track(*(torch.from_numpy(a).cuda() for a in (ev.y, ev.z, ev.row)), ev.counts)
    out = r.to_numpy()
    r.release()
    tr.close()
    if flags["merge"]:
        first, nhits, hits, par, cov, x = ref.mrg_first, ref.mrg_nhits, ref.mrg_hits, ref.mrg_par, ref.mrg_cov, ref.mrg_x
        chi2, ndf, sector = ref.mrg_chi2, ref.mrg_ndf, ref.mrg_sector
    else:
        first, nhits, hits, par, cov, x = ref.trk_first, ref.trk_nhits, ref.trk_hits, ref.trk_par, ref.trk_cov, ref.trk_x
        chi2, ndf, sector = ref.trk_chi2, ref.trk_ndf, ref.trk_sector
    print(k, ev.n, readings, flags, tuning, len(nhits), "tracks")
    assert np.array_equal(out["nhits"], nhits) and np.array_equal(out["first"], first)
    assert np.array_equal(out["hits"], hits)
    assert np.array_equal(out["ndf"], ndf) and np.array_equal(out["sector"], sector)
    assert np.array_equal(out["par"], par.astype(np.float32))
    assert np.array_equal(out["cov"], cov.astype(np.float32))
    assert np.array_equal(out["x_ref"], x.astype(np.float32))
    assert np.array_equal(out["chi2"], chi2.astype(np.float32))
