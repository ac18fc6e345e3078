"""The C ABI library builds for sm_103a, loads, and exports every function include/tpcca.h declares.
Also unit checks of the concordance metric (pure host code).  No GPU needed."""
import ctypes
import os
import re

import numpy as np

from paper_1712_09407_gb300 import build as libbuild
from paper_1712_09407_gb300 import concordance

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(tpc_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    path = libbuild.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_1712_09407_gb300 import tracker
    assert declared_functions() <= set(tracker.EXPORTS)
    for n in declared_functions():
        assert callable(getattr(tracker, n)), n


def test_host_only_entry_points():
    """Calls that touch no device memory work on a machine without a GPU."""
    from paper_1712_09407_gb300 import tracker
    p = tracker.tpc_params_default()
    assert p.alpha == 6.0 and p.min_clusters == 30
    t = tracker.tpc_tuning_default()
    assert t.bin_occupancy > 0 and t.construct_block % 32 == 0
    assert t.use_graph == 1 and t.seed_kernel == 1 and t.order_group == 3 << 20   # the struct layouts agree
    assert tracker.tpc_status_string(0) == "ok"
    assert "capacity" in tracker.tpc_status_string(2)


def test_library_defaults_match_oracle_defaults():
    """Both sides carry the same readings (they share no code, so check the values)."""
    import oracle
    from paper_1712_09407_gb300 import tracker
    p = tracker.tpc_params_default()
    c = oracle.Config(row_x=np.zeros(3))
    for f in ("sigma_y", "sigma_z", "nb_ty", "nb_tz", "nb_gate", "win_nsigma", "chi2_max", "edge_margin",
              "sin_max", "alpha", "beta", "qpt_max"):
        assert np.float32(getattr(p, f)) == np.float32(getattr(c, f)), f
    for f in ("min_chain", "max_miss", "min_clusters", "global_tracking"):
        assert int(getattr(p, f)) == int(getattr(c, f)), f
    assert [np.float32(v) for v in p.seed_cov] == [np.float32(v) for v in c.seed_cov]


def _fake(tracks, n_rows=200):
    first, nhits, hits = [], [], []
    for t in tracks:
        first.append(len(hits))
        nhits.append(len(t))
        hits.extend(t)
    return dict(first=np.array(first), nhits=np.array(nhits), hits=np.array(hits))


def test_concordance_metric():
    a = _fake([[0, 1, 2, 3], [10, 11, 12, 13, 14]])
    assert concordance.compare(a, a, 50)["concordance"] == 1.0
    # one cluster swapped in the second track
    b = _fake([[0, 1, 2, 3], [10, 11, 12, 13, 20]])
    c = concordance.compare(a, b, 50)
    assert c["n_matched"] == 2 and c["n_exact"] == 1
    assert abs(c["concordance"] - 8 / 10) < 1e-12       # 8 equal rows of 4 + (5+5-4)
    # a missing track counts all its clusters as different
    d = _fake([[0, 1, 2, 3]])
    c = concordance.compare(a, d, 50)
    assert c["unmatched_ref"] == 1 and abs(c["concordance"] - 4 / 9) < 1e-12
