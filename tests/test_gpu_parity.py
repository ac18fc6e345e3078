"""Parity of the CUDA tracker (through the C ABI) with the float-mode CPU oracle, stage by stage.

Tolerances: link agreement and track-by-track,
cluster-by-cluster concordance >= 99.99 %; parameters of matched tracks within 1e-4
relative (denominators max(|ref|, scale) with scales 1 cm, 1 cm, 1e-3, 1e-3, 1e-2 e/GeV);
exact cluster lists for matched tracks.  Integer stages (binning, cell starts) must be
bit-exact.  The float expressions of both sides are evaluated in the same order, with the same
explicit fused multiply-adds and no other contraction, and both use the same arcsin series, so
in practice the comparison is exact.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1712_09407_gb300 import concordance, eventgen
from paper_1712_09407_gb300.tracker import Tracker, TrackerError

from gpu_util import (compare_tracks, links_as_input_indices, owners_by_start, run_gpu, run_oracle, to_device,
                      tracklets_by_start, valid_slots)

pytestmark = pytest.mark.gpu

CONCORDANCE_MIN = 0.9999
PAR_REL = 1e-4


@pytest.fixture(scope="module")
def ev1():
    return eventgen.config_event(1)


@pytest.fixture(scope="module")
def ev0():
    return eventgen.config_event(0)


def _small36():
    spec = eventgen.EventSpec(n_primaries=600, n_secondaries=100, pt_cut=0.05, noise_frac=0.2)
    return eventgen.generate_event(spec, eventgen.Geometry(), seed=5)


# ---------------------------------------------------------------------------------------------
# A1
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["c0", "small36"])
def test_a1_binning_bit_exact(which, ev0):
    ev = ev0 if which == "c0" else _small36()
    tr, out, dbg = run_gpu(ev)
    meta = dbg["meta"].cpu().numpy()
    cells = dbg["cells"].cpu().numpy()
    grid = dbg["grid"].cpu().numpy()
    cs = dbg["cell_start"].cpu().numpy()
    orig = dbg["orig"].cpu().numpy()
    yz = dbg["yz"].cpu().numpy()
    checked = 0
    for u in range(meta.shape[0]):
        in_off, n, s_off, c_off = meta[u]
        if n == 0:
            continue
        ny, nz = cells[u]
        yy, zz = ev.y[in_off:in_off + n], ev.z[in_off:in_off + n]
        assert grid[u, 0] == yy.min() and grid[u, 1] == zz.min()
        cell, perm, cstart = oracle.bin_row(yy, zz, grid[u, 0], grid[u, 1], grid[u, 2], grid[u, 3], ny, nz)
        assert np.array_equal(orig[s_off:s_off + n], in_off + perm), u
        assert np.array_equal(cs[c_off:c_off + ny * nz + 1], cstart), u
        assert np.array_equal(yz[s_off:s_off + n, 0], yy[perm]) and np.array_equal(yz[s_off:s_off + n, 1], zz[perm])
        checked += 1
    assert checked > 0
    tr.close()


# ---------------------------------------------------------------------------------------------
# A2 .. A6 on one event
# ---------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def both1(ev1):
    tr, out, dbg = run_gpu(ev1)
    ref = run_oracle(ev1, key="c1")
    tr.close()
    return ev1, out, dbg, ref


def test_a2_a3_links(both1):
    ev, out, dbg, ref = both1
    L = links_as_input_indices(dbg, ev.n)
    for name in ("up_raw", "dn_raw", "up", "dn"):
        agree = np.mean(L[name] == getattr(ref, name))
        print(name, "agreement", agree)
        assert agree >= CONCORDANCE_MIN, (name, agree)


def test_a4_start_hits(both1):
    ev, out, dbg, ref = both1
    g = set(tracklets_by_start(dbg))
    o = set(ref.starts.tolist())
    sym = len(g ^ o)
    print("starts gpu %d oracle %d differ %d" % (len(g), len(o), sym))
    assert sym <= (1 - CONCORDANCE_MIN) * len(o)


def test_a5_tracklets(both1):
    ev, out, dbg, ref = both1
    g = tracklets_by_start(dbg)
    nsame = ndiff = 0
    worst = np.zeros(5)
    for t, s in enumerate(ref.starts.tolist()):
        if s not in g:
            ndiff += 1
            continue
        gt = g[s]
        oh = ref.tracklet_hits(t)
        if gt["n"] != ref.tl_nhits[t] or not np.array_equal(gt["hits"], oh):
            ndiff += 1
            continue
        nsame += 1
        if gt["n"] >= 3:
            rel = np.abs(gt["par"] - ref.tl_par[t]) / np.maximum(np.abs(ref.tl_par[t]), concordance.SCALES)
            worst = np.maximum(worst, rel)
    print("tracklets identical %d differ %d worst par rel %s" % (nsame, ndiff, worst))
    assert ndiff <= (1 - CONCORDANCE_MIN) * (nsame + ndiff) + 1
    assert worst.max() <= PAR_REL


def test_a6_ownership(both1):
    ev, out, dbg, ref = both1
    own_g = owners_by_start(dbg, ev.n)
    own_o = np.where(ref.owner >= 0, ref.starts[np.maximum(ref.owner, 0)], -1)
    agree = np.mean(own_g == own_o)
    print("owner agreement", agree)
    assert agree >= CONCORDANCE_MIN


def test_a7_tracks(both1):
    ev, out, dbg, ref = both1
    c = compare_tracks(ev, out, ref)
    print("tracks gpu %d oracle %d matched %d exact %d concordance %.7f" % (
        c["n_test"], c["n_ref"], c["n_matched"], c["n_exact"], c["concordance"]))
    assert c["concordance"] >= CONCORDANCE_MIN
    assert c["n_exact"] >= c["n_matched"] - max(1, int((1 - CONCORDANCE_MIN) * c["n_matched"]))
    assert c["par_rel_max"].max() <= PAR_REL, c["par_rel_max"]
    # canonical order (Section 3.2): innermost cluster's input index increases
    inner = out["hits"][out["first"]]
    assert np.all(np.diff(inner) > 0)
    # every output cluster on its own row, inner to outer, owned once
    for m in range(len(out["first"])):
        h = out["hits"][out["first"][m]:out["first"][m] + out["nhits"][m]]
        assert np.all(np.diff(ev.row[h].astype(int)) > 0)
    assert np.unique(out["hits"]).size == out["hits"].size
    assert np.all(out["nhits"] >= 30)


FP64_MEAN_REL_GATE = np.array([8.8e-6, 1.8e-6, 9.9e-5, 8.1e-6, 3.5e-5])


def test_error_against_fp64_oracle(both1):
    """States the per-parameter error of the float GPU path against the double oracle."""
    ev, out, dbg, ref = both1
    ref64 = run_oracle(ev, precision=64, key="c1")
    c = compare_tracks(ev, out, ref64)
    print("vs FP64: concordance %.7f mean rel %s max rel %s" % (c["concordance"], c["par_rel_mean"], c["par_rel_max"]))
    # gates at ten times the measured mean relative errors (y, z, sin phi, tan lambda, q/pT with
    # scales 1 cm, 1 cm, 1e-3, 1e-3, 1e-2: 8.8e-7, 1.8e-7, 9.9e-6, 8.1e-7, 3.5e-6)
    assert c["concordance"] >= 0.9999
    assert np.all(c["par_rel_mean"] <= FP64_MEAN_REL_GATE), c["par_rel_mean"]


# ---------------------------------------------------------------------------------------------
# full size and edge cases
# ---------------------------------------------------------------------------------------------
def test_full_central_event():
    """The benchmark workload (central-like event, 3.3 M clusters) end to end."""
    ev = eventgen.config_event(2)
    tr, out, dbg = run_gpu(ev, debug=False)
    ref = run_oracle(ev, key="c2")
    c = compare_tracks(ev, out, ref)
    print("central: gpu %d oracle %d concordance %.7f exact %d/%d par max %s" % (
        c["n_test"], c["n_ref"], c["concordance"], c["n_exact"], c["n_matched"], c["par_rel_max"]))
    assert c["concordance"] >= CONCORDANCE_MIN
    assert c["par_rel_max"].max() <= PAR_REL
    tr.close()


def test_full_central_event_sweep_constructor():
    """Same workload with the sector-sweep constructor: identical to the oracle."""
    ev = eventgen.config_event(2)
    tr = Tracker.for_geometry(ev.geometry)
    tr.set_tuning(dict(construct_mode=1))
    _, out, _ = run_gpu(ev, tracker=tr, debug=False)
    ref = run_oracle(ev, key="c2")
    c = compare_tracks(ev, out, ref)
    assert c["concordance"] >= CONCORDANCE_MIN and c["n_exact"] == c["n_matched"]
    assert c["par_rel_max"].max() <= PAR_REL
    tr.close()


def test_single_sector_config0(ev0):
    tr, out, dbg = run_gpu(ev0)
    ref = run_oracle(ev0, key="c0")
    c = compare_tracks(ev0, out, ref)
    assert c["concordance"] >= CONCORDANCE_MIN and c["n_exact"] == c["n_matched"] == c["n_ref"]
    tr.close()


def test_empty_event():
    geo = eventgen.Geometry()
    tr = Tracker.for_geometry(geo)
    e = torch.zeros(0, device="cuda")
    res = tr.track(e, e, torch.zeros(0, dtype=torch.uint8, device="cuda"), np.zeros(36 * 159, np.int32))
    assert res.sync() == (0, 0)
    res.release()
    tr.close()


def test_sparse_and_ragged_rows():
    """Rows with 0, 1 and 2 clusters, and a single track crossing empty rows."""
    geo = eventgen.Geometry()
    spec = eventgen.EventSpec(n_primaries=3, efficiency=0.7, noise_frac=0.0, pt_cut=0.3)
    ev = eventgen.generate_event(spec, geo, seed=9)
    tr, out, dbg = run_gpu(ev)
    ref = run_oracle(ev)
    c = compare_tracks(ev, out, ref)
    assert c["concordance"] == 1.0
    tr.close()


def test_noisy_sector():
    """One sector filled with noise (Section 6: noise-filled sectors after trip recovery)."""
    geo = eventgen.Geometry()
    spec = eventgen.EventSpec(n_primaries=300, noise_frac=0.1)
    ev = eventgen.generate_event(spec, geo, seed=13)
    rng = np.random.default_rng(0)
    extra_n = 159 * 4500            # 4500 noise clusters on every row of sector 4: beyond shared-memory staging
    rows = np.repeat(np.arange(159), 4500)
    half = geo.row_x[rows] * geo.tan_half
    ys = (rng.uniform(-1, 1, extra_n) * half).astype(np.float32)
    zs = rng.uniform(0, 250, extra_n).astype(np.float32)
    sec = ev.sector_of()
    y = np.concatenate([ev.y, ys])
    z = np.concatenate([ev.z, zs])
    row = np.concatenate([ev.row, rows.astype(np.uint8)])
    s = np.concatenate([sec, np.full(extra_n, 4)])
    order = np.lexsort((row, s))
    counts = np.bincount(s.astype(np.int64) * 159 + row, minlength=36 * 159).astype(np.int32)
    ev2 = eventgen.Event(geo, spec, 13, 0, y[order], z[order], row[order], counts,
                         np.concatenate([ev.label, np.full(extra_n, -1)])[order], ev.particles)
    tr, out, dbg = run_gpu(ev2, debug=False)
    ref = run_oracle(ev2)
    c = compare_tracks(ev2, out, ref)
    print("noisy sector: concordance %.7f tracks %d/%d" % (c["concordance"], c["n_test"], c["n_ref"]))
    assert c["concordance"] >= CONCORDANCE_MIN
    tr.close()


@pytest.mark.parametrize("tuning", [
    dict(bin_occupancy=0.5), dict(bin_occupancy=16.0), dict(stage_rows=0), dict(stage_rows=2),
    dict(neighbours_block=64, construct_block=64), dict(construct_block=96, construct_ctas_per_sm=1),
    dict(bin_occupancy=2.0, neighbours_block=128, construct_ctas_per_sm=0), dict(construct_mode=1),
    dict(construct_mode=1, bin_occupancy=4.0), dict(use_graph=0), dict(use_graph=0, construct_mode=1),
    dict(seed_kernel=1), dict(seed_kernel=1, construct_ctas_per_sm=1), dict(seed_kernel=0),
    dict(order_group=4096), dict(order_group=0, seed_kernel=1), dict(order_group=1)])
def test_tuning_does_not_change_results(tuning):
    """Grid bin size, block shapes and staging only change speed (the autotuner relies on it)."""
    ev = _small36()
    tr, base, _ = run_gpu(ev, debug=False)
    tr.set_tuning(tuning)
    _, out, _ = run_gpu(ev, tracker=tr, debug=False)
    for k in base:
        assert np.array_equal(base[k], out[k]), (tuning, k)
    tr.close()


def test_batch_equals_one_at_a_time():
    evs = [eventgen.config_event(3, event=i) for i in range(3)]
    geo = evs[0].geometry
    tr = Tracker.for_geometry(geo)
    singles = []
    for ev in evs:
        _, out, _ = run_gpu(ev, tracker=tr, debug=False)
        singles.append(out)
    y = torch.from_numpy(np.concatenate([e.y for e in evs])).cuda()
    z = torch.from_numpy(np.concatenate([e.z for e in evs])).cuda()
    row = torch.from_numpy(np.concatenate([e.row for e in evs])).cuda()
    counts = np.concatenate([e.counts for e in evs])
    res = tr.track_batch(y, z, row, counts, len(evs))
    res.sync()
    b = res.to_numpy()
    res.release()
    off = 0
    for i, (ev, s) in enumerate(zip(evs, singles)):
        sel = b["event"] == i
        assert sel.sum() == len(s["first"])
        for k in ("par", "cov", "x_ref", "chi2", "ndf", "nhits", "sector"):
            assert np.array_equal(b[k][sel], s[k]), k
        hb = np.concatenate([b["hits"][f:f + n] for f, n in zip(b["first"][sel], b["nhits"][sel])])
        assert np.array_equal(hb - off, s["hits"])
        off += ev.n
    # the same batch from host arrays
    hy, hz, hr = (np.concatenate([getattr(e, f) for e in evs]) for f in ("y", "z", "row"))
    res = tr.track_batch_host(torch.from_numpy(hy).pin_memory(), torch.from_numpy(hz).pin_memory(),
                              torch.from_numpy(hr).pin_memory(), counts, len(evs))
    res.sync()
    h = res.to_numpy()
    res.release()
    for k in b:
        assert np.array_equal(b[k], h[k]), k
    tr.close()


def _event_slice(b, i, offset):
    """The tracks of event i of a batch result, with its own hit indices and offsets."""
    sel = np.nonzero(b["event"] == i)[0]
    out = {k: v[sel] for k, v in b.items() if k not in ("event", "first", "hits")}
    hits = [b["hits"][f:f + n] for f, n in zip(b["first"][sel], b["nhits"][sel])]
    out["hits"] = (np.concatenate(hits) if hits else b["hits"][:0]) - offset
    out["first"] = np.concatenate([[0], np.cumsum(out["nhits"])[:-1]]).astype(b["first"].dtype) if len(sel) \
        else b["first"][:0]
    return out


def test_bench_call_shape_matches_oracle_and_single_events():
    """The bench step's launch configuration at full size: calls of 3 central-like events
    (tpc_track_batch) on 2 trackers, each on a stream of its own, both in flight at once.  Every
    event's tracks equal the same event tracked alone, bit for bit, and two of them are compared
    with the float oracle at the parity thresholds."""
    evs = [eventgen.config_event(2, event=i) for i in range(6)]
    geo = evs[0].geometry
    one = Tracker.for_geometry(geo)
    singles = [run_gpu(ev, tracker=one, debug=False)[1] for ev in evs]
    one.close()
    trs = [Tracker.for_geometry(geo) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    calls = []
    for j in range(2):
        grp = evs[3 * j:3 * j + 3]
        inp = [torch.from_numpy(np.concatenate([getattr(e, f) for e in grp])).cuda() for f in ("y", "z", "row")]
        counts = np.concatenate([e.counts for e in grp])
        torch.cuda.synchronize()                 # inputs copied before the call's stream reads them
        calls.append((grp, inp, trs[j].track_batch(*inp, counts, 3, stream=streams[j])))
    for j, (grp, inp, res) in enumerate(calls):
        res.sync()
        b = res.to_numpy()
        res.release()
        off = 0
        for i, ev in enumerate(grp):
            k = 3 * j + i
            got = _event_slice(b, i, off)
            for name, v in got.items():
                assert np.array_equal(v, singles[k][name]), (k, name)
            if k < 2:
                ref = run_oracle(ev, key="c2" if k == 0 else "c2_event%d" % k)
                c = compare_tracks(ev, got, ref)
                print("bench call shape, event %d: concordance %.7f exact %d/%d" % (
                    k, c["concordance"], c["n_exact"], c["n_matched"]))
                assert c["concordance"] >= CONCORDANCE_MIN
                assert c["par_rel_max"].max() <= PAR_REL
            off += ev.n
    for t in trs:
        t.close()


def test_host_input_path_equals_device_path(ev1):
    tr, dev_out, _ = run_gpu(ev1, debug=False)
    res = tr.track_host(ev1.y, ev1.z, ev1.row, ev1.counts)
    res.sync()
    host_out = res.to_numpy()
    res.release()
    for k in dev_out:
        assert np.array_equal(dev_out[k], host_out[k]), k
    tr.close()


def test_repeated_calls_are_deterministic(ev1):
    tr, a, _ = run_gpu(ev1, debug=False)
    _, b, _ = run_gpu(ev1, tracker=tr, debug=False)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    tr.close()


# ---------------------------------------------------------------------------------------------
# errors come back as status codes
# ---------------------------------------------------------------------------------------------
def test_wrong_row_byte_is_reported(ev0):
    tr = Tracker.for_geometry(ev0.geometry)
    y, z, row = to_device(ev0)
    row[100] = (int(row[100].item()) + 1) % 159
    res = tr.track(y, z, row, ev0.counts)
    with pytest.raises(TrackerError) as e:
        res.sync()
    assert e.value.status == 1 and "ingest" in str(e.value)
    res.release()
    tr.close()


def test_bad_counts_rejected_on_host(ev0):
    tr = Tracker.for_geometry(ev0.geometry)
    y, z, row = to_device(ev0)
    bad = ev0.counts.copy()
    bad[3] += 1
    with pytest.raises(TrackerError) as e:
        tr.track(y, z, row, bad)
    assert e.value.status == 1
    tr.close()


def test_budget_is_enforced(ev1):
    geo = ev1.geometry
    tr = Tracker.for_geometry(geo, budget=1 << 20)
    y, z, row = to_device(ev1)
    with pytest.raises(TrackerError) as e:
        tr.track(y, z, row, ev1.counts)
    assert e.value.status == 3
    tr.close()


@pytest.mark.parametrize("stage_rows", [1, 2])
def test_expired_device_wait_is_reported(stage_rows):
    """A bounded device wait that runs out (injected from the host: after a row staging of the
    neighbours finder has landed, a wait on a barrier that nothing completes, so no copy is in
    flight) returns TPC_ERR_TIMEOUT; the context stays usable and the next call is correct."""
    ev = _small36()
    tr = Tracker.for_geometry(ev.geometry)
    tr.set_tuning(dict(stage_rows=stage_rows))
    tr, ref, _ = run_gpu(ev, tracker=tr, debug=False)
    from paper_1712_09407_gb300.tracker import tpc_tracker_inject
    tpc_tracker_inject(tr.handle, 1)
    y, z, row = to_device(ev)
    res = tr.track(y, z, row, ev.counts)
    with pytest.raises(TrackerError) as e:
        res.sync()
    assert e.value.status == 4 and "neighbours" in str(e.value)
    res.release()
    tpc_tracker_inject(tr.handle, 0)
    _, out, _ = run_gpu(ev, tracker=tr, debug=False)
    for k in ref:
        assert np.array_equal(ref[k], out[k]), k
    tr.close()


def test_tracklet_pool_overflow_is_reported():
    """More start hits than the tracklet pool holds: TPC_ERR_CAPACITY with the stage, no crash."""
    ev = _small36()
    tr = Tracker.for_geometry(ev.geometry)
    tr.set_tuning(dict(tracklet_capacity=100))
    y, z, row = to_device(ev)
    res = tr.track(y, z, row, ev.counts)
    with pytest.raises(TrackerError) as e:
        res.sync()
    assert e.value.status == 2 and "evolution" in str(e.value)
    res.release()
    tr.close()


def test_result_outlives_its_tracker():
    """A result released after its tracker was destroyed is safe (the last release frees the rest)."""
    ev = _small36()
    tr = Tracker.for_geometry(ev.geometry)
    y, z, row = to_device(ev)
    res = tr.track(y, z, row, ev.counts)
    m, _ = res.sync()
    out = res.to_numpy()
    tr.close()                                   # destroys the tracker while the result is held
    assert len(out["first"]) == m > 0
    res.release()


def test_clusters_per_track_distribution(both1):
    """Section 3.3 / Fig. "gp_sizesum": the clusters-per-track statistic of the GPU and the CPU
    tracker agree (here bin for bin, the outputs being identical)."""
    ev, out, dbg, ref = both1
    bins = np.arange(30, 161)
    hg, _ = np.histogram(out["nhits"], bins=bins)
    ho, _ = np.histogram(ref.trk_nhits, bins=bins)
    assert hg.sum() == ho.sum() > 1000
    assert np.array_equal(hg, ho)


def _dense_patch_event(seed=7):
    """Rows 60..66 of sector 0 with 1500 clusters each in an 8 cm x 8 cm patch (tens of in-window
    candidates per cluster, more than the warp-cooperative search keeps in its lists, so its
    per-thread fix-up pass runs), plus a sparse central-like background elsewhere."""
    base = _small36()
    geo = base.geometry
    rng = np.random.default_rng(seed)
    nr = len(geo.row_x)
    counts = base.counts.reshape(-1, nr).copy()
    ys, zs, rows = [], [], []
    off = np.concatenate([[0], np.cumsum(base.counts)])
    for s in range(counts.shape[0]):
        for r in range(nr):
            u = s * nr + r
            y, z = base.y[off[u]:off[u + 1]], base.z[off[u]:off[u + 1]]
            if s == 0 and 60 <= r <= 66:
                y = np.concatenate([y, rng.uniform(0.0, 8.0, 1500).astype(np.float32)])
                z = np.concatenate([z, rng.uniform(10.0, 18.0, 1500).astype(np.float32)])
                counts[s, r] += 1500
            ys.append(y)
            zs.append(z)
            rows.append(np.full(len(y), r, np.uint8))
    import types
    return types.SimpleNamespace(geometry=geo, y=np.concatenate(ys).astype(np.float32),
                                 z=np.concatenate(zs).astype(np.float32), row=np.concatenate(rows),
                                 counts=counts.reshape(-1).astype(np.int32), n=int(counts.sum()))


@pytest.mark.parametrize("stage_rows", [2, 1, 0])
def test_dense_rows_links_equal_oracle(stage_rows):
    """Links and tracks in very dense rows equal the oracle's in every form of the neighbours finder
    (the warp-cooperative form sends such clusters to its per-thread fix-up pass)."""
    ev = _dense_patch_event()
    ref = run_oracle(ev, key="dense")
    tr = Tracker.for_geometry(ev.geometry)
    tr.set_tuning(dict(stage_rows=stage_rows))
    _, out, dbg = run_gpu(ev, tracker=tr)
    L = links_as_input_indices(dbg, ev.n)
    for name in ("up_raw", "dn_raw", "up", "dn"):
        assert np.array_equal(L[name], getattr(ref, name)), name
    c = compare_tracks(ev, out, ref)
    assert c["concordance"] == 1.0 and c["n_exact"] == c["n_matched"] == c["n_ref"]
    tr.close()
