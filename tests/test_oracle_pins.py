"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the generator's
independent global-frame helix, finite differences, brute force, hand-derived
cases (tests/golden) or statistical laws of a correct Kalman filter.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1712_09407_gb300 import eventgen as eg

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SCALES = np.array([1.0, 1.0, 1e-3, 1e-3, 1e-2])


def _single_track_event(pt, q, phi, geo, seed_base=0, eta_max=0.5, one_sector=False):
    spec = eg.EventSpec(n_primaries=1, pt_cut=pt, pt_mean=1e-12, phi_lo=phi, phi_hi=phi + 1e-9,
                        efficiency=1.0, smear=False, noise_frac=0.0, eta_max=eta_max)
    for sd in range(seed_base, seed_base + 200):
        ev = eg.generate_event(spec, geo, seed=sd, truth=True)
        if ev.particles["q"][0] == q and ev.n > 0:
            if one_sector and np.unique(ev.sector_of()).size != 1:
                continue
            return ev
    raise RuntimeError("no event with the requested charge")


def _cov(c15):
    C = np.zeros((5, 5))
    q = 0
    for i in range(5):
        for j in range(i + 1):
            C[i, j] = C[j, i] = c15[q]
            q += 1
    return C


# ------------------------------------------------------------------------------------------
# paper constants
# ------------------------------------------------------------------------------------------

def test_defaults_carry_the_paper_constants():
    gold = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    cfg = oracle.Config(row_x=eg.default_row_x())
    assert cfg.alpha == gold["alpha"]["value"]
    assert cfg.min_clusters == gold["min_clusters"]["value"]
    assert len(cfg.row_x) == gold["n_rows"]["value"]
    assert eg.Geometry().n_sectors == 2 * gold["sectors_per_volume"]["value"]


# ------------------------------------------------------------------------------------------
# propagation, seeding, fit (tracklet construction, Section 1)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("pt", [0.1, 0.5, 5.0])
@pytest.mark.parametrize("q", [-1, 1])
def test_propagation_reproduces_generator_helix(pt, q):
    """Transport of the truth state between rows lands on the generator's next crossing."""
    geo = eg.Geometry()
    ev = _single_track_event(pt, q, 0.7, geo)
    tr = ev.truth
    worst = 0.0
    for lab in np.unique(ev.label):
        sel = np.nonzero(ev.label == lab)[0]
        sel = sel[np.argsort(tr[sel, 6])]
        sec = ev.sector_of()[sel]
        for a, b in zip(sel[:-1], sel[1:]):
            if ev.sector_of()[a] != ev.sector_of()[b]:
                continue
            ok, st, _ = oracle.propagate(tr[a, :5], np.zeros(15), tr[a, 6], tr[b, 6], bz=geo.bz)
            if abs(tr[b, 2]) >= 0.99:
                continue
            assert ok
            worst = max(worst, float(np.max(np.abs(st - tr[b, :5]) / np.maximum(np.abs(tr[b, :5]), SCALES))))
        assert sec.size
    assert worst < 1e-10, worst


def test_jacobian_matches_finite_differences():
    for dx in (1.5, -1.5, 20.0, -20.0):
        s = np.array([3.0, 10.0, 0.4, 0.7, -2.0])
        Fa = np.zeros((5, 5))
        for i in range(5):
            c = np.zeros(15)
            c[i * (i + 1) // 2 + i] = 1.0
            _, _, c2 = oracle.propagate(s, c, 100.0, 100.0 + dx)
            Fa[:, i] = _cov(c2)[:, i]
        Fn = np.zeros((5, 5))
        for i in range(5):
            h = 1e-6
            sp, sm = s.copy(), s.copy()
            sp[i] += h
            sm[i] -= h
            Fn[:, i] = (oracle.propagate(sp, np.zeros(15), 100, 100 + dx)[1]
                        - oracle.propagate(sm, np.zeros(15), 100, 100 + dx)[1]) / (2 * h)
        # the curvature dependence of the arc/chord ratio is kept to leading order only
        assert np.allclose(Fa, Fn, rtol=1e-4, atol=1e-5), (dx, Fa - Fn)


def test_propagation_stops_at_sin_max():
    ok, _, _ = oracle.propagate([0, 0, 0.98, 0, -20.0], np.zeros(15), 100.0, 140.0)
    assert not ok


@pytest.mark.parametrize("pt", [0.1, 0.5, 5.0])
def test_seed_is_exact_on_a_helix(pt):
    geo = eg.Geometry()
    ev = _single_track_event(pt, 1, 0.4, geo)
    tr = ev.truth
    sel = np.nonzero(ev.label == ev.label[0])[0]
    sel = sel[np.argsort(tr[sel, 6])][:40]
    sel = sel[ev.sector_of()[sel] == ev.sector_of()[sel[0]]]
    pick = [sel[0], sel[len(sel) // 2], sel[-1]]
    ok, st = oracle.seed(tr[pick, 6], tr[pick, 0], tr[pick, 1], bz=geo.bz)
    assert ok
    err = np.abs(st - tr[pick[0], :5]) / np.maximum(np.abs(tr[pick[0], :5]), SCALES)
    assert err.max() < 1e-9, err


@pytest.mark.parametrize("pt", [0.1, 0.5, 5.0])
@pytest.mark.parametrize("q", [-1, 1])
def test_noise_free_helix_fit_recovers_truth(pt, q):
    """Noise-free clusters: every output track sits on the generated helix to 1e-9 (both legs)."""
    geo = eg.Geometry()
    legs = set()
    for phi in (0.3, 1.3, 2.9):
        ev = _single_track_event(pt, q, phi, geo)
        cfg = oracle.config_for(geo)
        r = oracle.track_event(cfg, ev.truth[:, 0], ev.truth[:, 1], ev.row, ev.counts, precision=64)
        assert r.info["n_tracks"] >= 1
        for i in range(r.info["n_tracks"]):
            t = r.trk_tracklet[i]
            inner = r.track_hits(i)[0]
            tr = ev.truth[inner]
            assert abs(r.tl_x[t] - tr[6]) < 1e-12
            err = np.abs(r.tl_par[t] - tr[:5]) / np.maximum(np.abs(tr[:5]), SCALES)
            assert err.max() < 1e-9, (phi, err)
            assert r.tl_chi2[t] < 1e-12
            legs.add(int(ev.label[inner] % 2))
    if pt == 0.1:
        assert legs == {0, 1}             # the curler is found on its way out and back


@pytest.fixture(scope="module")
def smeared():
    geo = eg.Geometry()
    spec = eg.EventSpec(n_primaries=1500, pt_cut=0.2, noise_frac=0.0)
    ev = eg.generate_event(spec, geo, seed=7, truth=True)
    cfg = oracle.config_for(geo)
    r = oracle.track_event(cfg, ev.y, ev.z, ev.row, ev.counts, precision=64)
    return ev, r


def test_smeared_chi2_per_ndf(smeared):
    ev, r = smeared
    t = r.trk_tracklet
    assert t.size >= 1000
    m = float(np.mean(r.tl_chi2[t] / r.tl_ndf[t]))
    assert 0.9 <= m <= 1.1, m


def test_smeared_pulls(smeared):
    """Pulls at the innermost cluster of clean tracks: mean ~0, width ~1 (robust width from the median)."""
    ev, r = smeared
    pulls = []
    for i in range(r.info["n_tracks"]):
        h = r.track_hits(i)
        if np.unique(ev.label[h]).size != 1:
            continue
        t = r.trk_tracklet[i]
        tr = ev.truth[h[0]]
        sig = np.sqrt(np.diag(_cov(r.tl_cov[t])))
        pulls.append((r.tl_par[t] - tr[:5]) / sig)
    pulls = np.array(pulls)
    assert pulls.shape[0] > 1000
    assert np.all(np.abs(np.median(pulls, axis=0)) < 0.1), np.median(pulls, axis=0)
    width = np.median(np.abs(pulls), axis=0) / 0.6745
    assert np.all((width > 0.9) & (width < 1.15)), width


@pytest.mark.parametrize("precision", [64, 32])
def test_covariances_positive_definite(smeared, precision):
    ev, _ = smeared
    cfg = oracle.config_for(ev.geometry)
    r = oracle.track_event(cfg, ev.y, ev.z, ev.row, ev.counts, precision=precision)
    ok = r.tl_ndf >= 1
    for c in r.tl_cov[ok]:
        np.linalg.cholesky(_cov(c))


# ------------------------------------------------------------------------------------------
# neighbours finder, evolution, start hits (Section 1)
# ------------------------------------------------------------------------------------------

def test_hand_built_evolution_case():
    g = json.load(open(os.path.join(GOLD, "evolution_5row.json")))
    geo = eg.Geometry(n_sectors=1, bz=0.0)
    row = np.array(g["row"], dtype=np.uint8)
    counts = np.bincount(row, minlength=159).astype(np.int32)
    cfg = oracle.config_for(geo)
    for prec in (64, 32):
        r = oracle.track_event(cfg, np.array(g["y"]), np.array(g["z"]), row, counts, precision=prec)
        for key in ("up_raw", "dn_raw", "up", "dn", "starts"):
            assert getattr(r, key).tolist() == g[key], key


def test_straight_lines_link_exactly():
    """B = 0, noise-free straight tracks: every cluster links to its own track's neighbours."""
    geo = eg.Geometry(n_sectors=36, bz=0.0)
    spec = eg.EventSpec(n_primaries=150, efficiency=1.0, smear=False, noise_frac=0.0)
    ev = eg.generate_event(spec, geo, seed=5, truth=True)
    cfg = oracle.config_for(geo)
    for prec in (64, 32):
        r = oracle.track_event(cfg, ev.y, ev.z, ev.row, ev.counts, precision=prec)
        sec = ev.sector_of()
        key = ev.label.astype(np.int64) * 64 + sec
        checked = 0
        for c in range(ev.n):
            if ev.row[c] in (0, 158):
                assert r.up_raw[c] == -1 and r.dn_raw[c] == -1
                continue
            mates = np.nonzero(key == key[c])[0]
            up = mates[ev.row[mates] == ev.row[c] + 1]
            dn = mates[ev.row[mates] == ev.row[c] - 1]
            if up.size == 1 and dn.size == 1:
                assert r.up_raw[c] == up[0] and r.dn_raw[c] == dn[0]
                checked += 1
        assert checked > 0.8 * ev.n


def _graph_invariants(ev, r):
    n = ev.n
    up, dn = r.up, r.dn
    for c in np.nonzero(up >= 0)[0]:
        assert dn[up[c]] == c and ev.row[up[c]] == ev.row[c] + 1
    for c in np.nonzero(dn >= 0)[0]:
        assert up[dn[c]] == c and ev.row[dn[c]] == ev.row[c] - 1
    # kept links are a subset of the raw ones
    assert np.all((up < 0) | (up == r.up_raw)) and np.all((dn < 0) | (dn == r.dn_raw))
    # every raw link that is reciprocated is kept
    for c in np.nonzero(r.up_raw >= 0)[0]:
        assert (r.dn_raw[r.up_raw[c]] == c) == (up[c] >= 0)
    # start hits by a brute-force chain walk
    starts = []
    for c in range(n):
        if up[c] >= 0 and dn[c] < 0:
            L, t = 1, c
            while up[t] >= 0:
                t = up[t]
                L += 1
            if L >= 3:
                starts.append(c)
    assert r.starts.tolist() == starts


@pytest.mark.parametrize("cfgn", [0, 3])
def test_link_graph_invariants(cfgn):
    ev = eg.config_event(cfgn)
    cfg = oracle.config_for(ev.geometry)
    r = oracle.track_event(cfg, ev.y, ev.z, ev.row, ev.counts, precision=32)
    _graph_invariants(ev, r)


def _small_mixed_event():
    geo = eg.Geometry()
    spec = eg.EventSpec(n_primaries=300, pt_cut=0.06, noise_frac=0.3)
    return eg.generate_event(spec, geo, seed=21)


@pytest.mark.parametrize("precision", [64, 32])
def test_binned_equals_brute_force(precision):
    """The grid only prunes: an all-pairs scan gives identical results in both precisions."""
    ev = _small_mixed_event()
    base = oracle.config_for(ev.geometry)
    ref = oracle.track_event(oracle.config_for(ev.geometry, brute_force=True), ev.y, ev.z, ev.row,
                             ev.counts, precision=precision)
    for dy, dz in ((0.3, 0.3), (2.0, 4.0), (40.0, 600.0)):
        r = oracle.track_event(oracle.config_for(ev.geometry, bin_dy=dy, bin_dz=dz), ev.y, ev.z, ev.row,
                               ev.counts, precision=precision)
        for key in ("up_raw", "dn_raw", "starts", "tl_nhits", "tl_hits", "tl_par", "tl_chi2", "owner",
                    "trk_tracklet", "trk_hits"):
            assert np.array_equal(getattr(r, key), getattr(ref, key)), (key, dy, dz)
    del base


def test_thread_count_does_not_change_results():
    ev = _small_mixed_event()
    a = oracle.track_event(oracle.config_for(ev.geometry, n_threads=1), ev.y, ev.z, ev.row, ev.counts)
    b = oracle.track_event(oracle.config_for(ev.geometry, n_threads=4), ev.y, ev.z, ev.row, ev.counts)
    for key in ("up", "starts", "tl_par", "owner", "trk_hits"):
        assert np.array_equal(getattr(a, key), getattr(b, key))


# ------------------------------------------------------------------------------------------
# selection (Section 1 and 3.1) and output order (Section 3.2)
# ------------------------------------------------------------------------------------------

def test_infinite_alpha_is_longest_wins():
    """alpha -> infinity: only the tracklet length decides, ties go to the first tracklet (Section 3.1)."""
    ev = _small_mixed_event()
    r = oracle.track_event(oracle.config_for(ev.geometry, alpha=1e30), ev.y, ev.z, ev.row, ev.counts,
                           precision=64)
    best = {}
    for t in range(r.info["n_starts"]):
        if r.tl_ndf[t] < 1:
            continue
        for c in r.tracklet_hits(t):
            b = best.get(c)
            if b is None or r.tl_nhits[t] > r.tl_nhits[b]:
                best[c] = t
    owner = np.full(ev.n, -1)
    for c, t in best.items():
        owner[c] = t
    assert np.array_equal(owner, r.owner)


def test_broken_chain_gives_one_track_not_two():
    """One isolated track whose link chain is cut by a missing cluster: both tracklets
    rebuild the whole track, the weight keeps one and the clone owns nothing."""
    geo = eg.Geometry()
    ev = _single_track_event(5.0, 1, math.radians(10.0), geo, one_sector=True)
    assert ev.n == 159
    keep = np.ones(ev.n, bool)
    keep[np.nonzero(ev.row == 60)[0]] = False           # drop the row-60 crossing
    y, z, row = ev.y[keep], ev.z[keep], ev.row[keep]
    sec = ev.sector_of()[keep]
    counts = np.bincount(sec.astype(np.int64) * 159 + row, minlength=36 * 159).astype(np.int32)
    r = oracle.track_event(oracle.config_for(geo), y, z, row, counts, precision=64)
    assert r.info["n_starts"] >= 2
    assert r.info["n_tracks"] == 1
    full = [t for t in range(r.info["n_starts"]) if r.tl_nhits[t] == r.tl_nhits.max()]
    assert len(full) >= 2
    assert sorted(r.tl_nowned[full].tolist())[-1] == r.tl_nhits.max()
    assert sorted(r.tl_nowned[full].tolist())[0] == 0


@pytest.mark.parametrize("precision", [64, 32])
def test_selection_and_output_invariants(precision):
    ev = eg.config_event(0)
    cfg = oracle.config_for(ev.geometry)
    r = oracle.track_event(cfg, ev.y, ev.z, ev.row, ev.counts, precision=precision)
    used = np.zeros(ev.n, int)
    inner = []
    for i in range(r.info["n_tracks"]):
        h = r.track_hits(i)
        t = r.trk_tracklet[i]
        assert len(h) >= 30 and r.tl_accept[t]
        assert abs(r.tl_par[t, 4]) <= 20.0
        assert np.all(np.diff(ev.row[h].astype(int)) > 0)        # one cluster per row, inner to outer
        assert set(h.tolist()) <= set(r.tracklet_hits(t).tolist())
        assert np.all(r.owner[h] == t)
        used[h] += 1
        inner.append(h[0])
    assert used.max() <= 1
    assert np.all(np.diff(inner) > 0)                              # Section 3.2: canonical order
    # each cluster goes to the tracklet of maximal weight, ties to the first one
    for t in range(r.info["n_starts"]):
        if r.tl_ndf[t] < 1:
            continue
        for c in r.tracklet_hits(t):
            o = r.owner[c]
            assert r.tl_w[o] > r.tl_w[t] or (r.tl_w[o] == r.tl_w[t] and o <= t)


# ------------------------------------------------------------------------------------------
# end to end against the generator's truth (Section 3: efficiency against simulation)
# ------------------------------------------------------------------------------------------

def mc_efficiency(ev, r, ptmin=0.2):
    sec = ev.sector_of()
    key = np.where(ev.label >= 0, ev.label.astype(np.int64) * 64 + sec, -1)
    uk, cnt = np.unique(key[key >= 0], return_counts=True)
    pt = ev.particles["pt"][uk // 64 // 2]
    findable = set(uk[(cnt >= 30) & (pt > ptmin)].tolist())
    matched, fakes = {}, 0
    for i in range(r.info["n_tracks"]):
        h = r.track_hits(i)
        v, c = np.unique(key[h], return_counts=True)
        j = int(np.argmax(c))
        if v[j] >= 0 and c[j] >= 0.9 * len(h):
            matched[v[j]] = matched.get(v[j], 0) + 1
        else:
            fakes += 1
    eff = sum(1 for f in findable if f in matched) / max(1, len(findable))
    clones = sum(n - 1 for n in matched.values())
    return eff, clones, fakes, len(findable)


@pytest.mark.parametrize("cfgn", [0, 1])
@pytest.mark.parametrize("precision", [64, 32])
def test_efficiency_against_truth(cfgn, precision):
    ev = eg.config_event(cfgn)
    r = oracle.track_event(oracle.config_for(ev.geometry), ev.y, ev.z, ev.row, ev.counts, precision=precision)
    eff, clones, fakes, nf = mc_efficiency(ev, r)
    assert nf > 50
    assert eff >= 0.90, eff
    assert clones <= 0.01 * nf and fakes <= 0.01 * nf


def test_float_arcsin_series_accuracy():
    """asin(u)/u of the float mode (Maclaurin series of arcsin with half-angle reduction)
    against double-precision arcsin: within 3 float ulps over (-1, 1), exact at 0, odd."""
    u = np.concatenate([np.linspace(-0.999, 0.999, 40001), np.geomspace(1e-30, 0.999, 400),
                        -np.geomspace(1e-30, 0.999, 400)]).astype(np.float32)
    worst = 0.0
    for x in u:
        r = oracle.asin_ratio_f32(float(x))
        ref = np.arcsin(np.float64(x)) / np.float64(x)
        worst = max(worst, abs(r - ref) / ref)
        assert r == oracle.asin_ratio_f32(float(-x))
    assert worst <= 3 * np.finfo(np.float32).eps, worst
    assert oracle.asin_ratio_f32(0.0) == 1.0


def test_float_mode_error_against_double_mode():
    """The float reading of the tracker against the double one on the 36-sector workload (4000
    tracks): concordance and mean relative parameter error per component within ten times the
    values measured for the float GPU path (which equals the float mode), scales 1 cm, 1 cm, 1e-3,
    1e-3, 1e-2 e/GeV."""
    from paper_1712_09407_gb300 import concordance
    ev = eg.config_event(1)
    cfg = oracle.config_for(ev.geometry)
    r32 = oracle.track_event(cfg, ev.y, ev.z, ev.row, ev.counts, precision=32)
    r64 = oracle.track_event(cfg, ev.y, ev.z, ev.row, ev.counts, precision=64)
    c = concordance.compare(concordance.oracle_tracks(r64), concordance.oracle_tracks(r32), ev.n)
    assert c["concordance"] >= 0.9999, c["concordance"]
    assert np.all(c["par_rel_mean"] <= np.array([8.8e-6, 1.8e-6, 9.9e-5, 8.1e-6, 3.5e-5])), c["par_rel_mean"]
