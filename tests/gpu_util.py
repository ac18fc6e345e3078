"""Helpers of the GPU parity tests: run the CUDA tracker through the C ABI and bring its
per-stage buffers into the oracle's indexing (input cluster indices)."""
import numpy as np
import torch

import oracle
from paper_1712_09407_gb300 import concordance
from paper_1712_09407_gb300.tracker import Tracker

_ORACLE_CACHE = {}


def to_device(ev):
    return (torch.from_numpy(ev.y).cuda(), torch.from_numpy(ev.z).cuda(), torch.from_numpy(ev.row).cuda())


def run_gpu(ev, tracker=None, tuning=None, debug=True):
    tr = tracker or Tracker.for_geometry(ev.geometry)
    if tuning is not None:
        tr.set_tuning(tuning)
    y, z, row = to_device(ev)
    res = tr.track(y, z, row, ev.counts)
    res.sync()
    out = res.to_numpy()
    res.release()
    dbg = tr.debug() if debug else None
    return tr, out, dbg


def run_oracle(ev, precision=32, key=None, **kw):
    k = (key, precision, tuple(sorted(kw.items()))) if key is not None else None
    if k is not None and k in _ORACLE_CACHE:
        return _ORACLE_CACHE[k]
    r = oracle.track_event(oracle.config_for(ev.geometry, **kw), ev.y, ev.z, ev.row, ev.counts, precision=precision)
    if k is not None:
        _ORACLE_CACHE[k] = r
    return r


def valid_slots(dbg):
    meta = dbg["meta"].cpu().numpy()
    idx = [np.arange(m[2], m[2] + m[1]) for m in meta if m[1] > 0]
    return np.concatenate(idx) if idx else np.zeros(0, np.int64)


def links_as_input_indices(dbg, n):
    """A2 / A3 links of every input cluster, as input indices (-1 = none)."""
    orig = dbg["orig"].cpu().numpy().astype(np.int64)
    slots = valid_slots(dbg)
    out = {}
    for name in ("up_raw", "dn_raw", "up", "dn"):
        v = dbg[name].cpu().numpy().astype(np.int64)
        a = np.full(n, -1, np.int64)
        s = v[slots]
        a[orig[slots]] = np.where(s >= 0, orig[np.maximum(s, 0)], -1)
        out[name] = a
    return out


def tracklets_by_start(dbg):
    """GPU tracklets keyed by the input index of their start cluster."""
    orig = dbg["orig"].cpu().numpy().astype(np.int64)
    st = dbg["starts"].cpu().numpy()
    n = dbg["tl_nhits"].cpu().numpy()
    hits = dbg["tl_hits"].cpu().numpy()
    par = dbg["tl_par"].cpu().numpy()
    chi2 = dbg["tl_chi2"].cpu().numpy()
    w = dbg["tl_w"].cpu().numpy()
    out = {}
    for t in range(st.shape[0]):
        h = orig[hits[t, :n[t]]] if n[t] > 0 else np.zeros(0, np.int64)
        out[int(orig[st[t, 0]])] = dict(n=int(n[t]), hits=h, par=par[t], chi2=float(chi2[t]), w=float(w[t]), t=t)
    return out


def owners_by_start(dbg, n):
    """Input index of the start cluster of the tracklet owning each input cluster (-1 none)."""
    orig = dbg["orig"].cpu().numpy().astype(np.int64)
    key = dbg["cluster_key"].cpu().numpy().view(np.uint64)
    slots = valid_slots(dbg)
    own = np.full(n, -1, np.int64)
    k = key[slots]
    low = (k & np.uint64(0xFFFFFFFF)).astype(np.int64)
    start_orig = (~low) & 0xFFFFFFFF
    own[orig[slots]] = np.where(k != 0, start_orig, -1)
    return own


def compare_tracks(ev, gpu_out, ref):
    return concordance.compare(concordance.oracle_tracks(ref), gpu_out, ev.n)
