"""Host logic of the alpha study (quality measures against the generator's truth), on CPU."""
import numpy as np

from paper_1712_09407_gb300 import eventgen
from paper_1712_09407_gb300.alpha_study import quality


def _perfect_tracks(ev, drop_every=0):
    """One track per (particle, leg, sector) with >= 30 clusters, clusters inner to outer, truth parameters."""
    sec = ev.sector_of()
    key = np.where(ev.label >= 0, ev.label.astype(np.int64) * 64 + sec, -1)
    first, nhits, hits, par, cov = [], [], [], [], []
    for k in np.unique(key[key >= 0]):
        h = np.nonzero(key == k)[0]
        if h.size < 30:
            continue
        h = h[np.argsort(ev.row[h], kind="stable")]
        first.append(sum(nhits))
        nhits.append(h.size)
        hits.append(h)
        par.append(ev.truth[h[0], :5])
        c = np.zeros(15)
        c[[0, 2, 5, 9, 14]] = 1.0
        cov.append(c)
    return dict(first=np.array(first), nhits=np.array(nhits), hits=np.concatenate(hits),
                par=np.array(par, dtype=np.float32), cov=np.array(cov, dtype=np.float32))


def test_perfect_tracks_score_perfectly():
    ev = eventgen.config_event(0, truth=True)
    out = _perfect_tracks(ev)
    q = quality(ev, out, pt_min=0.0)
    assert q["findable"] == len(out["first"]) == q["found"]
    assert q["clones"] == 0 and q["fakes"] == 0
    assert np.abs(q["res"]).max() < 1e-5            # float32 rounding of the truth


def test_clones_and_fakes_are_counted():
    ev = eventgen.config_event(0, truth=True)
    out = _perfect_tracks(ev)
    n = len(out["first"])
    # a copy of track 0 is a clone; a track made of two particles' halves is a fake
    h0 = out["hits"][:out["nhits"][0]]
    h1 = out["hits"][out["first"][1]:out["first"][1] + out["nhits"][1]]
    mix = np.concatenate([h0[:20], h1[:20]])
    out2 = dict(first=np.concatenate([out["first"], [len(out["hits"]), len(out["hits"]) + len(h0)]]),
                nhits=np.concatenate([out["nhits"], [len(h0), len(mix)]]),
                hits=np.concatenate([out["hits"], h0, mix]),
                par=np.concatenate([out["par"], out["par"][:1], out["par"][:1]]),
                cov=np.concatenate([out["cov"], out["cov"][:2]]))
    q = quality(ev, out2, pt_min=0.0)
    assert q["found"] == n and q["clones"] == 1 and q["fakes"] == 1 and q["tracks"] == n + 2
