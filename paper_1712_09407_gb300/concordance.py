"""Track-by-track, cluster-by-cluster comparison of two tracker outputs (Section 3.3).

A one-to-one correspondence of the tracks is built first (mutual best match by shared
clusters, with more than half of the reference track's clusters shared).  Within a pair
each row is checked for the same cluster; a reference track without a partner counts all
its clusters as different, and so does a test track without a partner.

Outputs are given as dicts with ``first``, ``nhits``, ``hits`` (input cluster indices, one
per row) and optionally ``par`` [M, 5].
"""
from __future__ import annotations

import numpy as np

SCALES = np.array([1.0, 1.0, 1e-3, 1e-3, 1e-2])


def _track_of(res, n):
    tr = np.full(n, -1, dtype=np.int64)
    M = len(res["first"])
    if M:
        idx = np.repeat(np.arange(M), res["nhits"])
        tr[np.asarray(res["hits"], dtype=np.int64)] = idx
    return tr


def match(ref, test, n_clusters):
    """Mutual-best track pairs.  Returns (ref_idx, test_idx, shared) arrays."""
    ta = _track_of(ref, n_clusters)
    tb = _track_of(test, n_clusters)
    both = (ta >= 0) & (tb >= 0)
    if not both.any():
        z = np.zeros(0, dtype=np.int64)
        return z, z, z
    pair = ta[both] * (len(test["first"]) + 1) + tb[both]
    up, cnt = np.unique(pair, return_counts=True)
    a = up // (len(test["first"]) + 1)
    b = up % (len(test["first"]) + 1)
    # best partner of each ref track and of each test track (ties: lower index)
    order = np.lexsort((b, -cnt, a))
    a_s, b_s, c_s = a[order], b[order], cnt[order]
    first_a = np.concatenate([[True], a_s[1:] != a_s[:-1]])
    best_b_of_a = dict(zip(a_s[first_a].tolist(), zip(b_s[first_a].tolist(), c_s[first_a].tolist())))
    order = np.lexsort((a, -cnt, b))
    a_s, b_s = a[order], b[order]
    first_b = np.concatenate([[True], b_s[1:] != b_s[:-1]])
    best_a_of_b = dict(zip(b_s[first_b].tolist(), a_s[first_b].tolist()))
    ra, rb, rs = [], [], []
    for ia, (ib, c) in best_b_of_a.items():
        if best_a_of_b.get(ib) == ia and c > 0.5 * ref["nhits"][ia]:
            ra.append(ia)
            rb.append(ib)
            rs.append(c)
    return np.array(ra, dtype=np.int64), np.array(rb, dtype=np.int64), np.array(rs, dtype=np.int64)


def compare(ref, test, n_clusters, rows=None):
    """Concordance and per-pair statistics of ``test`` against ``ref``."""
    ra, rb, shared = match(ref, test, n_clusters)
    na = np.asarray(ref["nhits"], dtype=np.int64)
    nb = np.asarray(test["nhits"], dtype=np.int64)
    agree = int(shared.sum())
    # rows of a pair: |A u B| = |A| + |B| - |A n B| (one cluster per row and track); a row where
    # both have a cluster but different ones counts once
    denom = 0
    exact = 0
    if ra.size:
        if rows is not None:
            rows = np.asarray(rows)
            for ia, ib in zip(ra, rb):
                ha = ref["hits"][ref["first"][ia]:ref["first"][ia] + na[ia]]
                hb = test["hits"][test["first"][ib]:test["first"][ib] + nb[ib]]
                denom += len(set(rows[ha].tolist()) | set(rows[hb].tolist()))
                exact += int(na[ia] == nb[ib] and np.array_equal(ha, hb))
        else:
            denom += int((na[ra] + nb[rb] - shared).sum())
            for ia, ib in zip(ra, rb):
                ha = ref["hits"][ref["first"][ia]:ref["first"][ia] + na[ia]]
                hb = test["hits"][test["first"][ib]:test["first"][ib] + nb[ib]]
                exact += int(na[ia] == nb[ib] and np.array_equal(ha, hb))
    un_a = np.setdiff1d(np.arange(len(na)), ra)
    un_b = np.setdiff1d(np.arange(len(nb)), rb)
    denom += int(na[un_a].sum()) + int(nb[un_b].sum())
    out = dict(n_ref=int(len(na)), n_test=int(len(nb)), n_matched=int(ra.size), n_exact=exact,
               unmatched_ref=int(un_a.size), unmatched_test=int(un_b.size),
               concordance=(agree / denom) if denom else 1.0, ref_idx=ra, test_idx=rb)
    if ra.size and "par" in ref and "par" in test:
        pa = np.asarray(ref["par"], dtype=np.float64)[ra]
        pb = np.asarray(test["par"], dtype=np.float64)[rb]
        rel = np.abs(pb - pa) / np.maximum(np.abs(pa), SCALES)
        out["par_rel_max"] = rel.max(axis=0)
        out["par_rel_mean"] = rel.mean(axis=0)
        out["par_rel"] = rel
    return out


def oracle_tracks(r):
    """Output dict of an oracle result (input indices, float64 parameters)."""
    return dict(first=r.trk_first.astype(np.int64), nhits=r.trk_nhits.astype(np.int64),
                hits=r.trk_hits.astype(np.int64), par=r.trk_par, cov=r.trk_cov, x_ref=r.trk_x,
                chi2=r.trk_chi2, ndf=r.trk_ndf, sector=r.trk_sector)
