"""Pins of the oracle's global tracking (Section 5: sector tracks prolonged into the neighbouring
sector after a change of frame)."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_09407_gb300 import eventgen as eg

SCALES = np.array([1.0, 1.0, 1e-3, 1e-3, 1e-2])
D20 = math.radians(20.0)


def _cov(c15):
    C = np.zeros((5, 5))
    q = 0
    for i in range(5):
        for j in range(i + 1):
            C[i, j] = C[j, i] = c15[q]
            q += 1
    return C


def _rotate_then_to(state, x, angle, x_target):
    ok, s, _, xn = oracle.rotate(state, np.zeros(15), x, angle)
    assert ok
    ok2, s2, _ = oracle.propagate(s, np.zeros(15), xn, x_target)
    assert ok2
    return s2


@pytest.mark.parametrize("angle", [D20, -D20])
def test_rotation_jacobian_matches_finite_differences(angle):
    """Covariance of the rotated state = J C J^T with J the derivative of 'rotate, then move to the
    fixed x' of the unperturbed state' (checked column by column)."""
    s0 = np.array([14.0, 30.0, 0.3, 0.6, -1.5])
    x0 = 120.0
    ok, _, _, xref = oracle.rotate(s0, np.zeros(15), x0, angle)
    assert ok
    Fa = np.zeros((5, 5))
    for i in range(5):
        c = np.zeros(15)
        c[i * (i + 1) // 2 + i] = 1.0
        _, _, c2, _ = oracle.rotate(s0, c, x0, angle)
        Fa[:, i] = _cov(c2)[:, i] / (1.0 if True else 1.0)
    # J[:, i] from J E_ii J^T = J[:, i] J[:, i]^T, normalised by the diagonal entry J[i, i]
    for i in range(5):
        if abs(Fa[i, i]) > 0:
            Fa[:, i] = Fa[:, i] / math.sqrt(Fa[i, i]) * np.sign(1.0)
    Fn = np.zeros((5, 5))
    for i in range(5):
        h = 1e-6
        sp, sm = s0.copy(), s0.copy()
        sp[i] += h
        sm[i] -= h
        Fn[:, i] = (_rotate_then_to(sp, x0, angle, xref) - _rotate_then_to(sm, x0, angle, xref)) / (2 * h)
    # compare |J| column by column (the extraction above gives columns up to sign)
    assert np.allclose(np.abs(Fa), np.abs(Fn), rtol=2e-4, atol=2e-6), (Fa, Fn)


def _find_two_sector_track(short_max=29, long_min=40, inward_short=True):
    geo = eg.Geometry()
    for pt in (0.6, 0.8, 1.0, 1.5):
        for q in (1, -1):
            for phi_deg in np.arange(14.0, 26.0, 0.25):
                phi = math.radians(phi_deg)
                spec = eg.EventSpec(n_primaries=1, pt_cut=pt, pt_mean=1e-12, phi_lo=phi, phi_hi=phi + 1e-9,
                                    efficiency=1.0, smear=False, noise_frac=0.0, eta_max=0.4)
                for sd in range(3):
                    ev = eg.generate_event(spec, geo, seed=sd, truth=True)
                    if ev.particles["q"][0] != q:
                        continue
                    sec = ev.sector_of()
                    secs, cnt = np.unique(sec, return_counts=True)
                    if len(secs) != 2 or cnt.min() > short_max or cnt.min() < 3 or cnt.max() < long_min:
                        continue
                    if np.unique(ev.label).size != 1 or secs[0] // 18 != secs[1] // 18:
                        continue
                    short = secs[np.argmin(cnt)]
                    rows_short = ev.row[sec == short].astype(int)
                    rows_long = ev.row[sec != short].astype(int)
                    if inward_short == (rows_short.max() < rows_long.min()):
                        return ev, short
    raise RuntimeError("no suitable track")


@pytest.mark.parametrize("inward_short", [True, False])
def test_short_segment_is_picked_up_by_global_tracking(inward_short):
    ev, short = _find_two_sector_track(inward_short=inward_short)
    cfg0 = oracle.config_for(ev.geometry)
    cfg1 = oracle.config_for(ev.geometry, global_tracking=True)
    x, z = ev.truth[:, 0], ev.truth[:, 1]
    r0 = oracle.track_event(cfg0, x, z, ev.row, ev.counts, precision=64)
    r1 = oracle.track_event(cfg1, x, z, ev.row, ev.counts, precision=64)
    assert r0.info["n_tracks"] == r1.info["n_tracks"] == 1        # Section 5: no new tracks
    h0, h1 = r0.track_hits(0), r1.track_hits(0)
    assert set(h0.tolist()) < set(h1.tolist())
    assert len(h1) == ev.n                                        # every cluster of the particle
    assert r1.trk_nglobal[0] == ev.n - len(h0)
    assert np.all(ev.sector_of()[h1[len(h1) - r1.trk_nglobal[0]:] if not inward_short else h1[:r1.trk_nglobal[0]]] == short)
    inner = h1[0]
    tr = ev.truth[inner]
    assert abs(r1.trk_x[0] - tr[6]) < 1e-9
    assert r1.trk_sector[0] == ev.sector_of()[inner]
    err = np.abs(r1.trk_par[0] - tr[:5]) / np.maximum(np.abs(tr[:5]), SCALES)
    assert err.max() < 1e-9, err
    assert r1.trk_ndf[0] == 2 * len(h1) - 5


def test_rotation_lands_on_the_next_sector_crossing():
    """Truth state at a crossing in one sector, rotated into the neighbour's frame and transported to
    a row plane there, equals the generator's crossing in the neighbour sector."""
    ev, short = _find_two_sector_track(short_max=200, long_min=3, inward_short=True)
    sec = ev.sector_of()
    tr = ev.truth
    a = np.nonzero(sec != short)[0]
    b = np.nonzero(sec == short)[0]
    ia = a[np.argmin(tr[a, 6])]
    ib = b[np.argmax(tr[b, 6])]
    d = 1 if (short - sec[ia]) % 18 == 1 else -1
    ok, s, _, xn = oracle.rotate(tr[ia, :5], np.zeros(15), tr[ia, 6], d * D20)
    assert ok
    ok, s2, _ = oracle.propagate(s, np.zeros(15), xn, tr[ib, 6])
    assert ok
    err = np.abs(s2 - tr[ib, :5]) / np.maximum(np.abs(tr[ib, :5]), SCALES)
    assert err.max() < 1e-9, err


@pytest.mark.parametrize("precision", [64, 32])
def test_global_tracking_keeps_tracks_and_adds_clusters(precision):
    ev = eg.config_event(1)
    r0 = oracle.track_event(oracle.config_for(ev.geometry), ev.y, ev.z, ev.row, ev.counts, precision=precision)
    r1 = oracle.track_event(oracle.config_for(ev.geometry, global_tracking=True), ev.y, ev.z, ev.row, ev.counts,
                            precision=precision)
    assert r0.info["n_tracks"] == r1.info["n_tracks"]
    assert np.all(r1.trk_nhits >= r0.trk_nhits)
    assert r1.trk_nglobal.sum() > 0
    assert np.unique(r1.trk_hits).size == r1.trk_hits.size        # a cluster in one track at most
    for i in range(r1.info["n_tracks"]):
        h1 = r1.track_hits(i)
        assert set(r0.track_hits(i).tolist()) <= set(h1.tolist())
