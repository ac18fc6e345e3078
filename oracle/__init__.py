"""CPU oracle of the TPC sector tracker — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never routes
through it.

The tracker itself is plain C (``tracker.c``), compiled twice: ``precision=64``
runs it in double, ``precision=32`` in float (the paper's GPU tracker works in
float; its CPU twin is the parity target).  Every step follows Section 1 of the
paper (neighbours finder, evolution, tracklets from one-to-one link chains,
Kalman tracklet construction, tracklet selection) with the weight of Section 3.1,
the sorting of Section 3.2 and the 30-cluster minimum of Section 5.  Readings of
the points the paper leaves open are the defaults of ``Config``.

Pinned by ``tests/test_oracle_*.py`` against closed forms, brute force, the
generator's truth and hand-built cases.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["common.c", "tracker.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no floating-point contraction, OpenMP over sectors)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, h) for h in ("oracle.h", "oracle_internal.h")]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    flags = ["-O2", "-fPIC", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-Wall"]
    objs = []
    jobs = [("common.c", [], "common.o"), ("tracker.c", [], "tracker_f64.o"),
            ("tracker.c", ["-DORC_F32"], "tracker_f32.o")]
    procs = []
    for src, extra, obj in jobs:
        out = os.path.join(_HERE, obj)
        objs.append(out)
        procs.append(subprocess.Popen(["gcc", *flags, *extra, "-c", os.path.join(_HERE, src), "-o", out]))
    for p in procs:
        if p.wait() != 0:
            raise RuntimeError("oracle compilation failed")
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-shared", "-fopenmp", *objs, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    for o in objs:
        os.remove(o)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("n_rows", ctypes.c_int), ("row_x", ctypes.POINTER(ctypes.c_double)),
        ("tan_half", ctypes.c_double), ("bz", ctypes.c_double), ("n_sectors", ctypes.c_int),
        ("sigma_y", ctypes.c_double), ("sigma_z", ctypes.c_double),
        ("nb_ty", ctypes.c_double), ("nb_tz", ctypes.c_double), ("nb_gate", ctypes.c_double),
        ("min_chain", ctypes.c_int), ("seed_cov", ctypes.c_double * 5),
        ("win_nsigma", ctypes.c_double), ("chi2_max", ctypes.c_double), ("max_miss", ctypes.c_int),
        ("edge_margin", ctypes.c_double), ("sin_max", ctypes.c_double),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("min_clusters", ctypes.c_int),
        ("qpt_max", ctypes.c_double), ("bin_dy", ctypes.c_double), ("bin_dz", ctypes.c_double),
        ("brute_force", ctypes.c_int), ("n_threads", ctypes.c_int), ("global_tracking", ctypes.c_int),
        ("merge", ctypes.c_int), ("merge_chi2", ctypes.c_double), ("merge_gap", ctypes.c_double),
        ("merge_qpt_nsigma", ctypes.c_double),
    ]


INFO = ["n", "n_starts", "n_tracks", "n_track_hits", "n_rows", "visits", "candidates", "in_window",
        "nb_candidates", "updates", "n_merged", "n_merged_hits"]
PTRS = ["up_raw", "dn_raw", "up", "dn", "starts", "tl_nhits", "tl_ndf", "tl_nup", "tl_hits",
        "tl_par", "tl_cov", "tl_x", "tl_chi2", "tl_w", "owner", "tl_nowned", "tl_accept",
        "trk_tracklet", "trk_first", "trk_nhits", "trk_hits", "trk_par", "trk_cov", "trk_x", "trk_chi2",
        "trk_ndf", "trk_sector", "trk_nglobal", "rf_par", "rf_cov", "rf_x", "rf_chi2", "rf_ok", "mg_next",
        "mrg_first", "mrg_nhits", "mrg_nseg", "mrg_head", "mrg_hits", "mrg_par", "mrg_cov", "mrg_x", "mrg_chi2",
        "mrg_ndf", "mrg_sector", "mrg_ok"]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            for pre in ("f64", "f32"):
                f = getattr(L, "orc_track_event_" + pre)
                f.restype = P
                f.argtypes = [ctypes.POINTER(_Cfg), P, P, P, P, ctypes.c_int64]
                g = getattr(L, "orc_propagate_" + pre)
                g.restype = ctypes.c_int
                g.argtypes = [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.orc_result_info.argtypes = [P, P]
            L.orc_result_ptrs.argtypes = [P, P]
            L.orc_result_free.argtypes = [P]
            L.orc_rotate_f64.restype = ctypes.c_int
            L.orc_rotate_f64.argtypes = [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, P]
            L.orc_chi2_5_f64.restype = ctypes.c_int
            L.orc_chi2_5_f64.argtypes = [P, P, P]
            L.orc_seed_f64.restype = ctypes.c_int
            L.orc_seed_f64.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double, P]
            L.orc_asin_ratio_f32.restype = ctypes.c_float
            L.orc_asin_ratio_f32.argtypes = [ctypes.c_float]
            for pre in ("f64", "f32"):
                f = getattr(L, "orc_select_" + pre)
                f.restype = None
                f.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                              ctypes.c_int64, P, P]
            L.orc_bin_row_f32.argtypes = [P, P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                                          P, P, P]
            _lib = L
    return _lib


@dataclasses.dataclass
class Config:
    """Tracker constants.  alpha = 6 (Section 3.1) and min_clusters = 30 (Section 5)
    are the paper's; the rest are readings of points it leaves open."""
    row_x: np.ndarray
    n_sectors: int = 36
    bz: float = 0.5
    tan_half: float = 0.17632698070846498
    sigma_y: float = 0.08
    sigma_z: float = 0.1
    nb_ty: float = 1.0
    nb_tz: float = 2.0
    nb_gate: float = 9.0
    min_chain: int = 3
    seed_cov: tuple = (0.08 * 0.08, 0.1 * 0.1, 0.01, 0.01, 1.0)
    win_nsigma: float = 3.0
    chi2_max: float = 16.0
    max_miss: int = 10
    edge_margin: float = 2.0
    sin_max: float = 0.99
    alpha: float = 6.0
    beta: float = 1.0
    min_clusters: int = 30
    qpt_max: float = 20.0
    bin_dy: float = 2.0
    bin_dz: float = 4.0
    brute_force: bool = False
    n_threads: int = 0
    global_tracking: bool = False
    merge: bool = False
    merge_chi2: float = 25.0
    merge_gap: float = 40.0
    merge_qpt_nsigma: float = 5.0

    def _c(self):
        rx = np.ascontiguousarray(self.row_x, dtype=np.float64)
        c = _Cfg()
        c.n_rows = rx.shape[0]
        c.row_x = rx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        for f in ("tan_half", "bz", "sigma_y", "sigma_z", "nb_ty", "nb_tz", "nb_gate", "win_nsigma",
                  "chi2_max", "edge_margin", "sin_max", "alpha", "beta", "qpt_max", "bin_dy", "bin_dz",
                  "merge_chi2", "merge_gap", "merge_qpt_nsigma"):
            setattr(c, f, float(getattr(self, f)))
        for f in ("n_sectors", "min_chain", "max_miss", "min_clusters", "n_threads"):
            setattr(c, f, int(getattr(self, f)))
        c.brute_force = int(bool(self.brute_force))
        c.global_tracking = int(bool(self.global_tracking))
        c.merge = int(bool(self.merge))
        for i in range(5):
            c.seed_cov[i] = float(self.seed_cov[i])
        return c, rx


def config_for(geometry, **kw) -> Config:
    """Config for an ``eventgen.Geometry``."""
    return Config(row_x=np.asarray(geometry.row_x, dtype=np.float64), n_sectors=geometry.n_sectors,
                  bz=geometry.bz, tan_half=geometry.tan_half, **kw)


@dataclasses.dataclass
class Result:
    """Everything the oracle produced for one event (input cluster indices throughout)."""
    info: dict
    up_raw: np.ndarray
    dn_raw: np.ndarray
    up: np.ndarray
    dn: np.ndarray
    starts: np.ndarray
    tl_nhits: np.ndarray
    tl_ndf: np.ndarray
    tl_nup: np.ndarray
    tl_hits: np.ndarray          # [T, n_rows], entries [:nhits] outer to inner
    tl_par: np.ndarray           # [T, 5]
    tl_cov: np.ndarray           # [T, 15] lower triangle, row-major
    tl_x: np.ndarray
    tl_chi2: np.ndarray
    tl_w: np.ndarray
    owner: np.ndarray
    tl_nowned: np.ndarray
    tl_accept: np.ndarray
    trk_tracklet: np.ndarray
    trk_first: np.ndarray
    trk_nhits: np.ndarray
    trk_hits: np.ndarray
    trk_par: np.ndarray          # [M, 5] reported parameters (frame: trk_sector)
    trk_cov: np.ndarray          # [M, 15]
    trk_x: np.ndarray
    trk_chi2: np.ndarray
    trk_ndf: np.ndarray
    trk_sector: np.ndarray
    trk_nglobal: np.ndarray      # clusters added by global tracking
    # track merger (zero-length unless Config.merge): refit of every sector track ...
    rf_par: np.ndarray           # [M, 5] at the innermost cluster (frame: its sector)
    rf_cov: np.ndarray
    rf_x: np.ndarray
    rf_chi2: np.ndarray
    rf_ok: np.ndarray
    mg_next: np.ndarray          # [M] track merged onto this one's outer end, -1 if none
    # ... and the merged tracks (one per chain of merged sector tracks, in canonical order)
    mrg_first: np.ndarray
    mrg_nhits: np.ndarray
    mrg_nseg: np.ndarray         # sector tracks merged
    mrg_head: np.ndarray         # index of the chain's first sector track
    mrg_hits: np.ndarray
    mrg_par: np.ndarray
    mrg_cov: np.ndarray
    mrg_x: np.ndarray
    mrg_chi2: np.ndarray
    mrg_ndf: np.ndarray
    mrg_sector: np.ndarray
    mrg_ok: np.ndarray

    def track_hits(self, i: int) -> np.ndarray:
        f = self.trk_first[i]
        return self.trk_hits[f:f + self.trk_nhits[i]]

    def merged_hits(self, i: int) -> np.ndarray:
        f = self.mrg_first[i]
        return self.mrg_hits[f:f + self.mrg_nhits[i]]

    def tracklet_hits(self, t: int) -> np.ndarray:
        return self.tl_hits[t, :self.tl_nhits[t]]


def track_event(cfg: Config, y, z, row, counts, precision: int = 32) -> Result:
    """Run the whole tracker on one event.  ``y, z`` may be float32 or float64."""
    L = lib()
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    row = np.ascontiguousarray(row, dtype=np.uint8)
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    n = y.shape[0]
    if counts.shape[0] != cfg.n_sectors * len(cfg.row_x) or int(counts.sum()) != n:
        raise ValueError("counts must have n_sectors*n_rows entries summing to the cluster count")
    c, _keep = cfg._c()
    fn = L.orc_track_event_f64 if precision == 64 else L.orc_track_event_f32
    h = fn(ctypes.byref(c), y.ctypes.data, z.ctypes.data, row.ctypes.data, counts.ctypes.data, n)
    try:
        info = np.zeros(len(INFO), dtype=np.int64)
        L.orc_result_info(h, info.ctypes.data)
        ptrs = (ctypes.c_void_p * len(PTRS))()
        L.orc_result_ptrs(h, ptrs)
        d = dict(zip(INFO, (int(v) for v in info)))
        N, T, M, H, nr = d["n"], d["n_starts"], d["n_tracks"], d["n_track_hits"], d["n_rows"]
        Mm, Hm = d["n_merged"], d["n_merged_hits"]
        Mr = M if cfg.merge else 0

        def arr(name, ctype, count, dtype):
            p = ptrs[PTRS.index(name)]
            if count == 0 or not p:
                return np.zeros(0, dtype=dtype)
            buf = (ctype * count).from_address(p)
            return np.frombuffer(buf, dtype=dtype, count=count).copy()

        i32, f64 = ctypes.c_int32, ctypes.c_double
        out = dict(
            up_raw=arr("up_raw", i32, N, np.int32), dn_raw=arr("dn_raw", i32, N, np.int32),
            up=arr("up", i32, N, np.int32), dn=arr("dn", i32, N, np.int32),
            starts=arr("starts", i32, T, np.int32), tl_nhits=arr("tl_nhits", i32, T, np.int32),
            tl_ndf=arr("tl_ndf", i32, T, np.int32), tl_nup=arr("tl_nup", i32, T, np.int32),
            tl_hits=arr("tl_hits", i32, T * nr, np.int32).reshape(T, nr),
            tl_par=arr("tl_par", f64, T * 5, np.float64).reshape(T, 5),
            tl_cov=arr("tl_cov", f64, T * 15, np.float64).reshape(T, 15),
            tl_x=arr("tl_x", f64, T, np.float64), tl_chi2=arr("tl_chi2", f64, T, np.float64),
            tl_w=arr("tl_w", f64, T, np.float64), owner=arr("owner", i32, N, np.int32),
            tl_nowned=arr("tl_nowned", i32, T, np.int32),
            tl_accept=arr("tl_accept", ctypes.c_uint8, T, np.uint8),
            trk_tracklet=arr("trk_tracklet", i32, M, np.int32),
            trk_first=arr("trk_first", i32, M, np.int32), trk_nhits=arr("trk_nhits", i32, M, np.int32),
            trk_hits=arr("trk_hits", i32, H, np.int32),
            trk_par=arr("trk_par", f64, M * 5, np.float64).reshape(M, 5),
            trk_cov=arr("trk_cov", f64, M * 15, np.float64).reshape(M, 15),
            trk_x=arr("trk_x", f64, M, np.float64), trk_chi2=arr("trk_chi2", f64, M, np.float64),
            trk_ndf=arr("trk_ndf", i32, M, np.int32), trk_sector=arr("trk_sector", i32, M, np.int32),
            trk_nglobal=arr("trk_nglobal", i32, M, np.int32),
            rf_par=arr("rf_par", f64, Mr * 5, np.float64).reshape(Mr, 5),
            rf_cov=arr("rf_cov", f64, Mr * 15, np.float64).reshape(Mr, 15),
            rf_x=arr("rf_x", f64, Mr, np.float64), rf_chi2=arr("rf_chi2", f64, Mr, np.float64),
            rf_ok=arr("rf_ok", i32, Mr, np.int32), mg_next=arr("mg_next", i32, Mr, np.int32),
            mrg_first=arr("mrg_first", i32, Mm, np.int32), mrg_nhits=arr("mrg_nhits", i32, Mm, np.int32),
            mrg_nseg=arr("mrg_nseg", i32, Mm, np.int32), mrg_head=arr("mrg_head", i32, Mm, np.int32),
            mrg_hits=arr("mrg_hits", i32, Hm, np.int32),
            mrg_par=arr("mrg_par", f64, Mm * 5, np.float64).reshape(Mm, 5),
            mrg_cov=arr("mrg_cov", f64, Mm * 15, np.float64).reshape(Mm, 15),
            mrg_x=arr("mrg_x", f64, Mm, np.float64), mrg_chi2=arr("mrg_chi2", f64, Mm, np.float64),
            mrg_ndf=arr("mrg_ndf", i32, Mm, np.int32), mrg_sector=arr("mrg_sector", i32, Mm, np.int32),
            mrg_ok=arr("mrg_ok", i32, Mm, np.int32),
        )
    finally:
        L.orc_result_free(h)
    return Result(info=d, **out)


def select(tracklets, alpha, beta, n_clusters, n_rows=159, precision: int = 64, library=None):
    """Section 3.1 on given tracklets, as the tracker applies it (orc_select): ``tracklets`` is a
    list of (cluster indices, fit chi2).  Returns (weights, owner of every cluster, -1 for none).
    ``library``: another build of the oracle (a ctypes library) instead of this one."""
    L = library if library is not None else lib()
    T = len(tracklets)
    nhits = np.array([len(h) for h, _ in tracklets], dtype=np.int32)
    chi2 = np.array([c for _, c in tracklets], dtype=np.float64)
    hits = np.full((max(T, 1), n_rows), -1, dtype=np.int32)
    for t, (h, _) in enumerate(tracklets):
        hits[t, :len(h)] = h
    w = np.zeros(max(T, 1), dtype=np.float64)
    owner = np.zeros(max(n_clusters, 1), dtype=np.int32)
    fn = L.orc_select_f64 if precision == 64 else L.orc_select_f32
    fn(T, nhits.ctypes.data, chi2.ctypes.data, hits.ctypes.data, n_rows, float(alpha), float(beta), n_clusters,
       w.ctypes.data, owner.ctypes.data)
    return w[:T], owner[:n_clusters]


def propagate(state, cov15, x0, x1, bz=0.5, sin_max=0.99, precision: int = 64):
    """Transport a state (y, z, sinphi, tanl, q/pT) and its covariance from x0 to x1."""
    L = lib()
    s = np.array(state, dtype=np.float64)
    c = np.array(cov15, dtype=np.float64)
    fn = L.orc_propagate_f64 if precision == 64 else L.orc_propagate_f32
    ok = fn(s.ctypes.data, c.ctypes.data, float(x0), float(x1), float(bz), float(sin_max))
    return bool(ok), s, c


def rotate(state, cov15, x, angle, bz=0.5, sin_max=0.99):
    """Re-express a state at x in a frame rotated by `angle` (radians); returns (ok, state, cov, x')."""
    L = lib()
    s = np.array(state, dtype=np.float64)
    c = np.array(cov15, dtype=np.float64)
    xn = np.zeros(1)
    ok = L.orc_rotate_f64(s.ctypes.data, c.ctypes.data, float(x), float(np.cos(angle)), float(np.sin(angle)),
                          float(bz), float(sin_max), xn.ctypes.data)
    return bool(ok), s, c, float(xn[0])


def seed(x3, y3, z3, bz=0.5, sin_max=0.99):
    """Seed state from the first, middle and last points of a chain (double precision)."""
    L = lib()
    x3 = np.ascontiguousarray(x3, dtype=np.float64)
    y3 = np.ascontiguousarray(y3, dtype=np.float64)
    z3 = np.ascontiguousarray(z3, dtype=np.float64)
    st = np.zeros(5)
    ok = L.orc_seed_f64(x3.ctypes.data, y3.ctypes.data, z3.ctypes.data, float(bz), float(sin_max), st.ctypes.data)
    return bool(ok), st


def chi2_5(cov15, d):
    """The merger's 5-parameter chi2 d^T A^-1 d (double precision); None if A is not positive definite."""
    L = lib()
    a = np.ascontiguousarray(cov15, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(1)
    ok = L.orc_chi2_5_f64(a.ctypes.data, dd.ctypes.data, out.ctypes.data)
    return float(out[0]) if ok else None


def asin_ratio_f32(u: float) -> float:
    """asin(u)/u as evaluated by the float mode."""
    return float(lib().orc_asin_ratio_f32(ctypes.c_float(u)))


def bin_row(y, z, ymin, zmin, inv_dy, inv_dz, ny, nz):
    """A1 for one row with given grid parameters: per-cluster cell, the stable
    counting-sort permutation and the cell starts."""
    L = lib()
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    n = y.shape[0]
    cell = np.zeros(max(n, 1), dtype=np.int32)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    cs = np.zeros(ny * nz + 1, dtype=np.int32)
    L.orc_bin_row_f32(y.ctypes.data, z.ctypes.data, n, ctypes.c_float(ymin), ctypes.c_float(zmin),
                      ctypes.c_float(inv_dy), ctypes.c_float(inv_dz), int(ny), int(nz),
                      cell.ctypes.data, perm.ctypes.data, cs.ctypes.data)
    return cell[:n], perm[:n], cs
