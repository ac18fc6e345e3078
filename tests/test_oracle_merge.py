"""Pins of the oracle's track merger with refit (Section 1: sector tracks are merged by the track
merger; Section 3.3: the merger refits every track from its cluster list, so equal cluster lists
give bitwise equal results).

The merger reading: every sector track is refitted from its clusters alone (seed from the first,
middle and last cluster, outward pass, inward pass with the covariance reset; the state changes
frame where the next cluster lies in another sector).  A track's outer end is merged with another
track's inner end in the same-azimuth sector of the other z half or an azimuth neighbour when the
radial gap is in (0, 40] cm, q/pT agrees within 5 sigma and the 5-parameter chi2 is at most 25;
only mutual best pairs merge.  Merged tracks are refitted over all their clusters."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_09407_gb300 import eventgen as eg

SCALES = np.array([1.0, 1.0, 1e-3, 1e-3, 1e-2])


def _track(ev, **kw):
    cfg = oracle.config_for(ev.geometry, merge=True, **kw)
    return oracle.track_event(cfg, ev.truth[:, 0], ev.truth[:, 1], ev.row, ev.counts, precision=64)


def _find(pred, pts=(1.0, 1.5, 2.0, 0.8), phis=np.arange(4.0, 360.0, 20.0), **spec):
    geo = eg.Geometry()
    for pt in pts:
        for phi_c in phis:
            for dphi in (-7.0, -5.0, -3.0, 3.0, 5.0, 7.0):
                phi = math.radians(phi_c + dphi)
                sp = eg.EventSpec(n_primaries=1, pt_cut=pt, pt_mean=1e-12, phi_lo=phi, phi_hi=phi + 1e-9,
                                  efficiency=1.0, smear=False, noise_frac=0.0, **spec)
                for sd in range(4):
                    ev = eg.generate_event(sp, geo, seed=sd, truth=True)
                    if np.unique(ev.label).size == 1 and pred(ev):
                        return ev
    raise RuntimeError("no suitable particle")


def _two_segments(ev, same_azimuth):
    sec = ev.sector_of()
    secs, cnt = np.unique(sec, return_counts=True)
    if len(secs) != 2 or cnt.min() < 35:
        return False
    a, b = secs
    return (a % 18 == b % 18) if same_azimuth else (a // 18 == b // 18)


def _check_merged_truth(ev, r):
    assert r.info["n_tracks"] == 2 and r.info["n_merged"] == 1
    assert r.mrg_nseg[0] == 2 and r.mrg_ok[0] == 1
    h = r.merged_hits(0)
    assert np.array_equal(np.sort(h), np.arange(ev.n))            # every cluster of the particle
    tr = ev.truth[h[0]]
    assert r.mrg_sector[0] == ev.sector_of()[h[0]]
    assert abs(r.mrg_x[0] - tr[6]) < 1e-9
    err = np.abs(r.mrg_par[0] - tr[:5]) / np.maximum(np.abs(tr[:5]), SCALES)
    assert err.max() < 1e-9, err
    assert r.mrg_ndf[0] == 2 * ev.n - 5
    assert r.mrg_chi2[0] < 1e-12


def test_particle_crossing_a_sector_edge_is_merged():
    ev = _find(lambda e: _two_segments(e, same_azimuth=False), eta_max=0.4)
    _check_merged_truth(ev, _track(ev))


def test_particle_crossing_the_central_membrane_is_merged():
    """Same azimuth, two z halves (sectors s and s + 18): no change of frame."""
    ev = _find(lambda e: _two_segments(e, same_azimuth=True), pts=(5.0, 3.0), phis=np.arange(10.0, 360.0, 20.0),
               eta_max=0.03, sigma_vz=6.0)
    _check_merged_truth(ev, _track(ev))


def test_refit_of_a_noise_free_track_recovers_the_truth():
    ev = _find(lambda e: np.unique(e.sector_of()).size == 1 and e.n >= 100, pts=(0.5, 1.0, 5.0))
    r = _track(ev)
    assert r.info["n_tracks"] == 1 and r.rf_ok[0] == 1
    tr = ev.truth[r.track_hits(0)[0]]
    err = np.abs(r.rf_par[0] - tr[:5]) / np.maximum(np.abs(tr[:5]), SCALES)
    assert err.max() < 1e-9, err


@pytest.mark.parametrize("precision", [32, 64])
def test_refit_depends_on_the_cluster_list_only(precision):
    """Section 3.3: the same clusters give the same refit, bit for bit, whatever else differs.  The
    clusters of every (sector, row) are permuted, which changes every input index, the grids, the
    tracklet order and the tie-breaks of the sector tracker; tracks with the same cluster set must
    get identical refits."""
    ev = eg.config_event(1)
    rng = np.random.default_rng(7)
    perm = np.arange(ev.n)
    off = np.concatenate([[0], np.cumsum(ev.counts)])
    for u in range(len(ev.counts)):
        a, b = off[u], off[u + 1]
        if b - a > 1:
            perm[a:b] = a + rng.permutation(b - a)
    cfg = oracle.config_for(ev.geometry, merge=True)
    r0 = oracle.track_event(cfg, ev.y, ev.z, ev.row, ev.counts, precision=precision)
    r1 = oracle.track_event(cfg, ev.y[perm], ev.z[perm], ev.row[perm], ev.counts, precision=precision)
    key0 = {tuple(np.sort(r0.track_hits(i)).tolist()): i for i in range(r0.info["n_tracks"])}
    same = 0
    for j in range(r1.info["n_tracks"]):
        k = tuple(np.sort(perm[r1.track_hits(j)]).tolist())
        i = key0.get(k)
        if i is None:
            continue
        same += 1
        assert np.array_equal(r0.rf_par[i], r1.rf_par[j]) and np.array_equal(r0.rf_cov[i], r1.rf_cov[j])
        assert r0.rf_chi2[i] == r1.rf_chi2[j]
    assert same >= 0.99 * r0.info["n_tracks"]


@pytest.mark.parametrize("precision", [64, 32])
def test_merges_join_one_particle(precision):
    """Workload 1: merged tracks keep every cluster once, most sector-border splits are joined,
    and a merge joins segments of one particle (majority labels agree) in at least 99 % of cases."""
    ev = eg.config_event(1)
    cfg = oracle.config_for(ev.geometry, merge=True)
    r = oracle.track_event(cfg, ev.y, ev.z, ev.row, ev.counts, precision=precision)
    assert r.info["n_merged"] < r.info["n_tracks"]
    assert np.array_equal(np.sort(r.mrg_hits), np.sort(r.trk_hits))
    part = lambda h: np.bincount(np.maximum(ev.label[h], 0) // 2).argmax()
    good = bad = 0
    for a in range(r.info["n_tracks"]):
        b = r.mg_next[a]
        if b < 0:
            continue
        if part(r.track_hits(a)) == part(r.track_hits(b)):
            good += 1
        else:
            bad += 1
    print("merges", good + bad, "same particle", good)
    assert good + bad > 1000 and bad <= 0.01 * (good + bad)
    ndf = r.mrg_ndf[r.mrg_ok == 1]
    chi = r.mrg_chi2[r.mrg_ok == 1]
    assert 0.9 <= float(np.mean(chi / ndf)) <= 1.1


def test_unrelated_tracks_are_not_merged():
    """Two particles in neighbouring sectors with opposite charges never merge."""
    geo = eg.Geometry()
    evs = []
    for q_phi in (math.radians(5.0), math.radians(35.0)):
        sp = eg.EventSpec(n_primaries=1, pt_cut=2.0, pt_mean=1e-12, phi_lo=q_phi, phi_hi=q_phi + 1e-9,
                          efficiency=1.0, smear=False, noise_frac=0.0, eta_max=0.3)
        evs.append(eg.generate_event(sp, geo, seed=2, truth=True))
    # concatenate the two single-particle events sector by sector
    nr = geo.n_rows
    y, z, row, counts = [], [], [], np.zeros(36 * nr, np.int32)
    for u in range(36 * nr):
        for e in evs:
            off = np.concatenate([[0], np.cumsum(e.counts)])
            sl = slice(off[u], off[u + 1])
            y.append(e.truth[sl, 0])
            z.append(e.truth[sl, 1])
            row.append(e.row[sl])
            counts[u] += e.counts[u]
    y, z, row = np.concatenate(y), np.concatenate(z), np.concatenate(row)
    r = oracle.track_event(oracle.config_for(geo, merge=True), y, z, row, counts, precision=64)
    assert r.info["n_merged"] == r.info["n_tracks"] >= 2


def test_chi2_5_against_a_linear_solve():
    rng = np.random.default_rng(3)
    for _ in range(50):
        B = rng.normal(size=(5, 5))
        A = B @ B.T + 0.1 * np.eye(5)
        d = rng.normal(size=5)
        c15 = [A[i, j] for i in range(5) for j in range(i + 1)]
        ref = d @ np.linalg.solve(A, d)
        assert abs(oracle.chi2_5(c15, d) - ref) <= 1e-9 * max(1.0, ref)
    A = np.diag([1.0, 1.0, -1.0, 1.0, 1.0])
    assert oracle.chi2_5([A[i, j] for i in range(5) for j in range(i + 1)], np.ones(5)) is None
