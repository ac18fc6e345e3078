"""Chi2 suppression study (Section 3.1, Fig. "gp_chi2"): tracking quality against the constant alpha
of the cluster weight w = n (alpha - chi2/beta).

Small alpha lets the fit quality decide which tracklet keeps a shared cluster; alpha -> infinity
reduces the rule to "the longest tracklet wins".  The paper shows efficiency and resolution
against alpha and picks alpha = 6 without printing the values, so this study has no number to
compare with; it regenerates the curves on synthetic events with the generator's truth.

Definitions (the same as the oracle's efficiency pins):
- findable: a (particle, leg, sector) with at least 30 clusters (and pT above ``pt_min``);
- matched track: at least 90 % of its clusters carry one (particle, leg) label, in its sector;
- efficiency: findables with at least one matched track; clones: further matched tracks of a
  findable; fakes: tracks that match nothing;
- resolution: spread of (fitted - true) parameter at the track's reference x (the innermost
  cluster, where the generator's truth gives the state), over matched tracks whose innermost
  cluster carries the matched label; pulls divide by the fitted sigma.

Runs the CUDA tracker only (``tpc_params.alpha``); events come from ``eventgen``.
"""
from __future__ import annotations

import json

import numpy as np

from . import eventgen
from .tracker import Tracker, tpc_params_default

PARAMS = ["y", "z", "sinphi", "tanlambda", "qpt"]
DIAG = [0, 2, 5, 9, 14]          # variances in the lower-triangle covariance


def quality(ev, out, pt_min=0.2):
    """Efficiency, clone and fake counts and residuals of one event's tracks against the truth."""
    sec = ev.sector_of()
    key = np.where(ev.label >= 0, ev.label.astype(np.int64) * 64 + sec, -1)
    uk, cnt = np.unique(key[key >= 0], return_counts=True)
    pt = ev.particles["pt"][uk // 64 // 2]
    findable = set(uk[(cnt >= 30) & (pt > pt_min)].tolist())
    matched, fakes = {}, 0
    res, pull = [], []
    for m in range(len(out["first"])):
        h = out["hits"][out["first"][m]:out["first"][m] + out["nhits"][m]]
        v, c = np.unique(key[h], return_counts=True)
        j = int(np.argmax(c))
        if v[j] >= 0 and c[j] >= 0.9 * len(h):
            matched[v[j]] = matched.get(v[j], 0) + 1
            if v[j] in findable and key[h[0]] == v[j]:
                tr = ev.truth[h[0]]                 # state at the innermost cluster
                d = out["par"][m].astype(np.float64) - tr[:5]
                sig = np.sqrt(np.maximum(out["cov"][m][DIAG].astype(np.float64), 1e-30))
                res.append(d)
                pull.append(d / sig)
        else:
            fakes += 1
    found = sum(1 for f in findable if f in matched)
    clones = sum(n - 1 for k, n in matched.items() if k in findable)
    return dict(findable=len(findable), found=found, clones=clones, fakes=fakes, tracks=len(out["first"]),
                res=np.array(res).reshape(-1, 5), pull=np.array(pull).reshape(-1, 5))


def _robust_sigma(x):
    q = np.percentile(x, [15.865, 84.135])
    return float((q[1] - q[0]) / 2)


def run(alphas=(0.5, 1.0, 2.0, 4.0, 6.0, 10.0, 20.0, 100.0, 1e6), workload=1, events=4, pt_min=0.2, log=None):
    """One line per alpha: efficiency, clone and fake rates, resolutions and pull widths."""
    import torch
    evs = [eventgen.config_event(workload, event=i, truth=True) for i in range(events)]
    dev = [tuple(torch.from_numpy(a).cuda() for a in (e.y, e.z, e.row)) for e in evs]
    lines = []
    for alpha in alphas:
        p = tpc_params_default()
        p.alpha = float(alpha)
        tr = Tracker.for_geometry(evs[0].geometry, params=p)
        tot = dict(findable=0, found=0, clones=0, fakes=0, tracks=0)
        res, pull = [], []
        for e, d in zip(evs, dev):
            r = tr.track(*d, e.counts)
            q = quality(e, r.to_numpy(), pt_min)
            r.release()
            for k in tot:
                tot[k] += q[k]
            res.append(q["res"])
            pull.append(q["pull"])
        tr.close()
        res, pull = np.concatenate(res), np.concatenate(pull)
        line = dict(alpha=alpha, efficiency=tot["found"] / max(1, tot["findable"]),
                    clone_rate=tot["clones"] / max(1, tot["found"]), fake_rate=tot["fakes"] / max(1, tot["tracks"]),
                    findable=tot["findable"], tracks=tot["tracks"],
                    resolution={n: _robust_sigma(res[:, i]) for i, n in enumerate(PARAMS)},
                    rms={n: float(np.sqrt(np.mean(res[:, i] ** 2))) for i, n in enumerate(PARAMS)},
                    pull_width={n: _robust_sigma(pull[:, i]) for i, n in enumerate(PARAMS)})
        lines.append(line)
        if log:
            log(json.dumps(line))
    return lines


def main():
    import argparse
    ap = argparse.ArgumentParser(description="tracking quality against alpha (Section 3.1)")
    ap.add_argument("--alphas", default="0.5,1,2,4,6,10,20,100,1e6")
    ap.add_argument("--workload", type=int, default=1)
    ap.add_argument("--events", type=int, default=4)
    ap.add_argument("--pt-min", type=float, default=0.2)
    a = ap.parse_args()
    run([float(x) for x in a.alphas.split(",")], a.workload, a.events, a.pt_min, log=print)


if __name__ == "__main__":
    main()
