"""Thin Python binding of the C ABI in include/tpcca.h (argument marshalling only).

The functions named ``tpc_*`` map one to one onto the C entry points; every step of
the tracker runs in the CUDA kernels of libtpcca.so.  PyTorch supplies device memory
and streams.  There is no CPU fallback: if the library is missing, every call raises.

``Tracker`` and ``Result`` wrap those calls for convenience; result arrays are exposed
as zero-copy torch tensors that stay valid until the result is released.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

(TPC_OK, TPC_ERR_INVALID_ARG, TPC_ERR_CAPACITY, TPC_ERR_BUDGET, TPC_ERR_TIMEOUT, TPC_ERR_CUDA, TPC_ERR_STATE,
 TPC_ERR_CHECK) = range(8)
STAGES = {0: "none", 1: "ingest", 2: "neighbours", 3: "evolution", 4: "construction", 5: "selection", 6: "output",
          7: "global", 8: "merge"}

c_int, c_float, c_int64, c_void_p = ctypes.c_int, ctypes.c_float, ctypes.c_int64, ctypes.c_void_p
P = ctypes.POINTER


class tpc_geometry(ctypes.Structure):
    _fields_ = [("n_rows", c_int), ("row_x", P(c_float)), ("tan_half", c_float), ("z_max", c_float),
                ("n_sectors", c_int)]


class tpc_params(ctypes.Structure):
    _fields_ = [("sigma_y", c_float), ("sigma_z", c_float), ("nb_ty", c_float), ("nb_tz", c_float),
                ("nb_gate", c_float), ("min_chain", c_int), ("seed_cov", c_float * 5),
                ("win_nsigma", c_float), ("chi2_max", c_float), ("max_miss", c_int),
                ("edge_margin", c_float), ("sin_max", c_float), ("alpha", c_float), ("beta", c_float),
                ("min_clusters", c_int), ("qpt_max", c_float), ("global_tracking", c_int), ("merge", c_int),
                ("merge_chi2", c_float), ("merge_gap", c_float), ("merge_qpt_nsigma", c_float)]


class tpc_tuning(ctypes.Structure):
    _fields_ = [("bin_occupancy", c_float), ("neighbours_block", c_int), ("construct_block", c_int),
                ("construct_ctas_per_sm", c_int), ("construct_mode", c_int), ("stage_rows", c_int),
                ("tracklet_capacity", c_int), ("use_graph", c_int), ("seed_kernel", c_int),
                ("order_group", c_int)]


class tpc_track_view(ctypes.Structure):
    _fields_ = [("n_tracks", c_int64), ("n_hits", c_int64)] + [
        (n, c_void_p) for n in ("par", "cov", "x_ref", "alpha", "chi2", "ndf", "nhits", "first", "sector",
                                "event", "hits")]


class tpc_debug_view(ctypes.Structure):
    _fields_ = [("n_units", c_int64), ("n_slots", c_int64), ("n_tracklets", c_int64),
                ("tracklet_capacity", c_int64)] + [
        (n, c_void_p) for n in ("unit_meta", "unit_cells", "unit_grid", "cell_start", "yz", "orig", "up_raw",
                                "dn_raw", "up", "dn", "starts", "tl_nhits", "tl_hits", "tl_par", "tl_cov",
                                "tl_x", "tl_chi2", "tl_w", "tl_nowned", "cluster_key")]


class tpc_call_stats(ctypes.Structure):
    _fields_ = [("ms", c_float * 10), ("kernel_launches", c_int), ("clusters", c_int64), ("tracklets", c_int64),
                ("row_visits", c_int64), ("candidates", c_int64), ("tracks", c_int64), ("hits", c_int64),
                ("global_found", c_int64), ("graph_builds", c_int64), ("sector_tracks", c_int64),
                ("tracklet_hits", c_int64)]


class tpc_server_config(ctypes.Structure):
    _fields_ = [("lanes", c_int), ("max_batch", c_int), ("lane_clusters", c_int64), ("hbm_budget", ctypes.c_size_t)]


class tpc_server_result(ctypes.Structure):
    _fields_ = [("status", c_int), ("n_tracks", c_int64), ("n_hits", c_int64)] + [
        (n, c_void_p) for n in ("par", "cov", "x_ref", "alpha", "chi2", "ndf", "nhits", "first", "sector", "hits")] + [
        ("t_submit_ns", c_int64), ("t_launch_ns", c_int64), ("t_done_ns", c_int64), ("batch_size", c_int)]


EXPORTS = {
    "tpc_params_default": (None, [P(tpc_params)]),
    "tpc_tuning_default": (None, [P(tpc_tuning)]),
    "tpc_tracker_create": (c_int, [P(tpc_geometry), c_float, P(tpc_params), ctypes.c_size_t, P(c_void_p)]),
    "tpc_tracker_set_tuning": (c_int, [c_void_p, P(tpc_tuning)]),
    "tpc_tracker_reserve": (c_int, [c_void_p, c_int64, c_int]),
    "tpc_tracker_reserve_results": (c_int, [c_void_p, c_int]),
    "tpc_track_event": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, P(c_void_p)]),
    "tpc_track_batch": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int64, c_void_p,
                                P(c_void_p)]),
    "tpc_track_event_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                                     P(c_void_p)]),
    "tpc_track_batch_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int64, c_void_p,
                                     P(c_void_p)]),
    "tpc_result_sync_counts": (c_int, [c_void_p, P(c_int64), P(c_int64)]),
    "tpc_result_get": (c_int, [c_void_p, P(tpc_track_view)]),
    "tpc_result_ready": (c_int, [c_void_p]),
    "tpc_result_copy_to_host": (c_int, [c_void_p] + [c_void_p] * 11),
    "tpc_result_release": (None, [c_void_p]),
    "tpc_tracker_destroy": (None, [c_void_p]),
    "tpc_status_string": (ctypes.c_char_p, [c_int]),
    "tpc_last_error_detail": (c_int, [c_void_p, P(c_int), P(c_int), P(c_int)]),
    "tpc_tracker_debug_view": (c_int, [c_void_p, P(tpc_debug_view)]),
    "tpc_tracker_set_timing": (c_int, [c_void_p, c_int]),
    "tpc_tracker_inject": (c_int, [c_void_p, c_int]),
    "tpc_result_stats": (c_int, [c_void_p, P(tpc_call_stats)]),
    "tpc_find_links_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                                       c_void_p, c_void_p, c_void_p]),
    "tpc_server_create": (c_int, [P(tpc_geometry), c_float, P(tpc_params), P(tpc_server_config), P(c_void_p)]),
    "tpc_server_submit": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, P(c_int64)]),
    "tpc_server_poll": (c_int, [c_void_p, P(c_int64), c_int, P(c_int)]),
    "tpc_server_get": (c_int, [c_void_p, c_int64, P(tpc_server_result)]),
    "tpc_server_release": (c_int, [c_void_p, c_int64]),
    "tpc_server_now_ns": (c_int64, []),
    "tpc_server_destroy": (None, [c_void_p]),
}


class TrackerError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s (status %d)%s" % (_status_text(status), status, (": " + msg) if msg else ""))


def _status_text(s):
    try:
        return lib().tpc_status_string(int(s)).decode()
    except Exception:
        return "status"


def lib():
    """Load libtpcca.so (built in-tree; TPCCA_LIB may name the checked build instead).  Raises if it
    has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("TPCCA_LIB", _build.LIB)
            if not os.path.exists(path):
                raise RuntimeError("%s is not built: run __graft_entry__.build() "
                                   "(the tracker has no CPU fallback)" % os.path.basename(path))
            L = ctypes.CDLL(path)
            for name, (res, args) in EXPORTS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(status, what=""):
    if status != TPC_OK:
        raise TrackerError(status, what)


# ----------------------------------------------------------------------------------------------
# same-name wrappers of the C entry points
# ----------------------------------------------------------------------------------------------

def tpc_params_default() -> tpc_params:
    p = tpc_params()
    lib().tpc_params_default(ctypes.byref(p))
    return p


def tpc_tuning_default() -> tpc_tuning:
    t = tpc_tuning()
    lib().tpc_tuning_default(ctypes.byref(t))
    return t


def tpc_tracker_create(row_x, tan_half, z_max, n_sectors, bz, params=None, budget=0):
    rx = np.ascontiguousarray(row_x, dtype=np.float32)
    g = tpc_geometry(int(rx.shape[0]), rx.ctypes.data_as(P(c_float)), float(tan_half), float(z_max), int(n_sectors))
    h = c_void_p()
    _check(lib().tpc_tracker_create(ctypes.byref(g), float(bz), ctypes.byref(params) if params is not None else None,
                                    int(budget), ctypes.byref(h)), "tpc_tracker_create")
    return h


def tpc_tracker_set_tuning(tr, tuning):
    _check(lib().tpc_tracker_set_tuning(tr, ctypes.byref(tuning)), "tpc_tracker_set_tuning")


def tpc_tracker_reserve(tr, max_clusters, max_events=1):
    _check(lib().tpc_tracker_reserve(tr, int(max_clusters), int(max_events)), "tpc_tracker_reserve")


def tpc_tracker_reserve_results(tr, depth):
    _check(lib().tpc_tracker_reserve_results(tr, int(depth)), "tpc_tracker_reserve_results")


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr() if t.numel() else None
    return t.ctypes.data if t.size else None


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def tpc_track_event(tr, y, z, row, counts, stream=None):
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    h = c_void_p()
    _check(lib().tpc_track_event(tr, _ptr(y), _ptr(z), _ptr(row), counts.ctypes.data, int(y.shape[0]),
                                 _stream(stream), ctypes.byref(h)), "tpc_track_event")
    return h


def tpc_track_batch(tr, y, z, row, counts, n_events, stream=None):
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    h = c_void_p()
    _check(lib().tpc_track_batch(tr, _ptr(y), _ptr(z), _ptr(row), counts.ctypes.data, int(n_events),
                                 int(y.shape[0]), _stream(stream), ctypes.byref(h)), "tpc_track_batch")
    return h


def tpc_track_event_host(tr, y, z, row, counts, stream=None):
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    h = c_void_p()
    n = int(y.shape[0])
    _check(lib().tpc_track_event_host(tr, _ptr(y), _ptr(z), _ptr(row), counts.ctypes.data, n, _stream(stream),
                                      ctypes.byref(h)), "tpc_track_event_host")
    return h


def tpc_track_batch_host(tr, y, z, row, counts, n_events, stream=None):
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    h = c_void_p()
    _check(lib().tpc_track_batch_host(tr, _ptr(y), _ptr(z), _ptr(row), counts.ctypes.data, int(n_events),
                                      int(y.shape[0]), _stream(stream), ctypes.byref(h)), "tpc_track_batch_host")
    return h


def tpc_result_sync_counts(res):
    m, h = c_int64(), c_int64()
    s = lib().tpc_result_sync_counts(res, ctypes.byref(m), ctypes.byref(h))
    return s, m.value, h.value


def tpc_result_ready(res) -> int:
    return lib().tpc_result_ready(res)


def tpc_result_get(res) -> tpc_track_view:
    v = tpc_track_view()
    _check(lib().tpc_result_get(res, ctypes.byref(v)), "tpc_result_get")
    return v


def tpc_result_copy_to_host(res, arrays: dict):
    names = ("par", "cov", "x_ref", "alpha", "chi2", "ndf", "nhits", "first", "sector", "event", "hits")
    _check(lib().tpc_result_copy_to_host(res, *[_ptr(arrays.get(n)) for n in names]), "tpc_result_copy_to_host")


def tpc_result_release(res):
    lib().tpc_result_release(res)


def tpc_server_create(row_x, tan_half, z_max, n_sectors, bz, lanes, max_batch, lane_clusters, hbm_budget=0,
                      params=None):
    rx = np.ascontiguousarray(row_x, dtype=np.float32)
    g = tpc_geometry(int(rx.shape[0]), rx.ctypes.data_as(P(c_float)), float(tan_half), float(z_max), int(n_sectors))
    cfg = tpc_server_config(int(lanes), int(max_batch), int(lane_clusters), int(hbm_budget))
    h = c_void_p()
    _check(lib().tpc_server_create(ctypes.byref(g), float(bz), ctypes.byref(params) if params is not None else None,
                                   ctypes.byref(cfg), ctypes.byref(h)), "tpc_server_create")
    return h


def tpc_server_submit(srv, y, z, row, counts, n) -> int:
    """Queue one event (host arrays that must stay alive until it is done); returns its id."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    i = c_int64()
    _check(lib().tpc_server_submit(srv, _ptr(y), _ptr(z), _ptr(row), counts.ctypes.data, int(n), ctypes.byref(i)),
           "tpc_server_submit")
    return int(i.value)


def tpc_server_poll(srv, max_ids=1024):
    ids = (c_int64 * max_ids)()
    n = c_int()
    _check(lib().tpc_server_poll(srv, ids, int(max_ids), ctypes.byref(n)), "tpc_server_poll")
    return [int(ids[i]) for i in range(n.value)]


def tpc_server_get(srv, rid) -> tpc_server_result:
    r = tpc_server_result()
    _check(lib().tpc_server_get(srv, int(rid), ctypes.byref(r)), "tpc_server_get")
    return r


def tpc_server_release(srv, rid):
    _check(lib().tpc_server_release(srv, int(rid)), "tpc_server_release")


def tpc_server_now_ns() -> int:
    return int(lib().tpc_server_now_ns())


def tpc_server_destroy(srv):
    lib().tpc_server_destroy(srv)


def server_result_arrays(r: tpc_server_result) -> dict:
    """Copies of a finished event's host arrays."""
    M, H = r.n_tracks, r.n_hits

    def arr(ptr, count, ctype, dtype, shape=None):
        if count == 0 or not ptr:
            a = np.zeros(count, dtype=dtype)
        else:
            a = np.frombuffer((ctype * count).from_address(ptr), dtype=dtype, count=count).copy()
        return a.reshape(shape) if shape else a

    f, i = ctypes.c_float, ctypes.c_int32
    return dict(par=arr(r.par, M * 5, f, np.float32, (M, 5)), cov=arr(r.cov, M * 15, f, np.float32, (M, 15)),
                x_ref=arr(r.x_ref, M, f, np.float32), alpha=arr(r.alpha, M, f, np.float32),
                chi2=arr(r.chi2, M, f, np.float32), ndf=arr(r.ndf, M, i, np.int32), nhits=arr(r.nhits, M, i, np.int32),
                first=arr(r.first, M, i, np.int32), sector=arr(r.sector, M, i, np.int32), hits=arr(r.hits, H, i, np.int32))


def tpc_tracker_destroy(tr):
    lib().tpc_tracker_destroy(tr)


def tpc_status_string(s) -> str:
    return lib().tpc_status_string(int(s)).decode()


def tpc_last_error_detail(tr):
    e, s, g = c_int(), c_int(), c_int()
    st = lib().tpc_last_error_detail(tr, ctypes.byref(e), ctypes.byref(s), ctypes.byref(g))
    return st, e.value, s.value, g.value


def tpc_tracker_inject(tr, what):
    _check(lib().tpc_tracker_inject(tr, int(what)), "tpc_tracker_inject")


def tpc_tracker_set_timing(tr, enable=True):
    _check(lib().tpc_tracker_set_timing(tr, int(bool(enable))), "tpc_tracker_set_timing")


def tpc_result_stats(res) -> dict:
    st = tpc_call_stats()
    _check(lib().tpc_result_stats(res, ctypes.byref(st)), "tpc_result_stats")
    # ms: set-up, ingest, neighbours, evolution, construction, selection, output, global tracking, merger
    return dict(ms=list(st.ms)[:9], kernel_launches=st.kernel_launches, clusters=st.clusters,
                tracklets=st.tracklets, row_visits=st.row_visits, candidates=st.candidates, tracks=st.tracks,
                hits=st.hits, global_found=st.global_found, graph_builds=st.graph_builds,
                sector_tracks=st.sector_tracks, tracklet_hits=st.tracklet_hits)


def tpc_find_links_noalloc(tr, y, z, row, counts, up, dn, status=None, stream=None, n=None):
    """Links after the evolution step for one event, with no device allocation by the library.
    ``up``/``dn`` (int32 device tensors of n) receive input indices (-1 = none); ``status``
    (optional int32 device tensor of 4) receives the device-side status.  Returns the C status."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    n = int(y.shape[0]) if n is None else int(n)
    return lib().tpc_find_links_noalloc(tr, _ptr(y), _ptr(z), _ptr(row), counts.ctypes.data, n, _ptr(up), _ptr(dn),
                                        _ptr(status), _stream(stream))


def tpc_tracker_debug_view(tr) -> tpc_debug_view:
    v = tpc_debug_view()
    _check(lib().tpc_tracker_debug_view(tr, ctypes.byref(v)), "tpc_tracker_debug_view")
    return v


# ----------------------------------------------------------------------------------------------
# zero-copy torch views of device arrays
# ----------------------------------------------------------------------------------------------
class _DevArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None,
                                         "stream": None}


def device_view(ptr, shape, dtype):
    """torch tensor aliasing device memory at ptr (no copy)."""
    import torch
    typestr = {"f4": "<f4", "i4": "<i4", "u8": "<i8", "i8": "<i8"}[dtype]
    n = 1
    for s in shape:
        n *= int(s)
    if n == 0 or not ptr:
        tdt = {"f4": torch.float32, "i4": torch.int32, "u8": torch.int64, "i8": torch.int64}[dtype]
        return torch.zeros(tuple(int(s) for s in shape), dtype=tdt, device="cuda")
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")


# ----------------------------------------------------------------------------------------------
# convenience classes
# ----------------------------------------------------------------------------------------------
class Result:
    """One call's output.  ``sync()`` waits and raises TrackerError on a device-side error."""

    def __init__(self, handle, tracker):
        self.handle = handle
        self.tracker = tracker
        self.n_tracks = None
        self.n_hits = None

    def sync(self):
        s, m, h = tpc_result_sync_counts(self.handle)
        if s != TPC_OK:
            st, ev, sec, stage = tpc_last_error_detail(self.tracker.handle)
            raise TrackerError(s, "event %d sector %d stage %s" % (ev, sec, STAGES.get(stage, stage)))
        self.n_tracks, self.n_hits = m, h
        return m, h

    def ready(self) -> bool:
        s = tpc_result_ready(self.handle)
        if s < 0:
            raise TrackerError(-s, "tpc_result_ready")
        return s == 1

    def views(self) -> dict:
        if self.n_tracks is None:
            self.sync()
        v = tpc_result_get(self.handle)
        M, H = v.n_tracks, v.n_hits
        return dict(par=device_view(v.par, (M, 5), "f4"), cov=device_view(v.cov, (M, 15), "f4"),
                    x_ref=device_view(v.x_ref, (M,), "f4"), alpha=device_view(v.alpha, (M,), "f4"),
                    chi2=device_view(v.chi2, (M,), "f4"), ndf=device_view(v.ndf, (M,), "i4"),
                    nhits=device_view(v.nhits, (M,), "i4"), first=device_view(v.first, (M,), "i4"),
                    sector=device_view(v.sector, (M,), "i4"), event=device_view(v.event, (M,), "i4"),
                    hits=device_view(v.hits, (H,), "i4"))

    def to_numpy(self) -> dict:
        if self.n_tracks is None:
            self.sync()
        M, H = self.n_tracks, self.n_hits
        out = dict(par=np.zeros((M, 5), np.float32), cov=np.zeros((M, 15), np.float32),
                   x_ref=np.zeros(M, np.float32), alpha=np.zeros(M, np.float32), chi2=np.zeros(M, np.float32),
                   ndf=np.zeros(M, np.int32), nhits=np.zeros(M, np.int32), first=np.zeros(M, np.int32),
                   sector=np.zeros(M, np.int32), event=np.zeros(M, np.int32), hits=np.zeros(H, np.int32))
        tpc_result_copy_to_host(self.handle, out)
        return out

    def stats(self) -> dict:
        return tpc_result_stats(self.handle)

    def release(self):
        if self.handle is not None:
            tpc_result_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Tracker:
    """A tracker on the current CUDA device for one geometry."""

    def __init__(self, row_x, tan_half=0.17632698070846498, z_max=250.0, n_sectors=36, bz=0.5, params=None,
                 budget=0, tuning=None, global_tracking=None, merge=None):
        if global_tracking is not None or merge is not None:
            params = params if params is not None else tpc_params_default()
            if global_tracking is not None:
                params.global_tracking = int(bool(global_tracking))
            if merge is not None:
                params.merge = int(bool(merge))
        self.row_x = np.asarray(row_x, dtype=np.float32)
        self.n_rows = int(self.row_x.shape[0])
        self.n_sectors = int(n_sectors)
        self.handle = tpc_tracker_create(self.row_x, tan_half, z_max, n_sectors, bz, params, budget)
        if tuning is not None:
            self.set_tuning(tuning)

    @classmethod
    def for_geometry(cls, geo, **kw):
        """From an ``eventgen.Geometry``."""
        return cls(geo.row_x, geo.tan_half, geo.z_max, geo.n_sectors, geo.bz, **kw)

    def set_tuning(self, tuning):
        if isinstance(tuning, dict):
            t = tpc_tuning_default()
            for k, v in tuning.items():
                setattr(t, k, v)
            tuning = t
        tpc_tracker_set_tuning(self.handle, tuning)

    def reserve(self, max_clusters, max_events=1, results=None):
        """Size the workspace; with ``results`` also preallocate that many result buffers, after
        which calls allocate no device memory (a call while all are held raises TPC_ERR_BUDGET)."""
        tpc_tracker_reserve(self.handle, max_clusters, max_events)
        if results is not None:
            tpc_tracker_reserve_results(self.handle, results)

    def track(self, y, z, row, counts, stream=None) -> Result:
        return Result(tpc_track_event(self.handle, y, z, row, counts, stream), self)

    def track_batch(self, y, z, row, counts, n_events, stream=None) -> Result:
        return Result(tpc_track_batch(self.handle, y, z, row, counts, n_events, stream), self)

    def track_host(self, y, z, row, counts, stream=None) -> Result:
        return Result(tpc_track_event_host(self.handle, y, z, row, counts, stream), self)

    def track_batch_host(self, y, z, row, counts, n_events, stream=None) -> Result:
        return Result(tpc_track_batch_host(self.handle, y, z, row, counts, n_events, stream), self)

    def set_timing(self, enable=True):
        tpc_tracker_set_timing(self.handle, enable)

    def debug(self) -> dict:
        """Copies of the intermediate buffers of the last call (for per-stage checks)."""
        v = tpc_tracker_debug_view(self.handle)
        R, S, T, Tc = v.n_units, v.n_slots, v.n_tracklets, v.tracklet_capacity
        meta = device_view(v.unit_meta, (R, 4), "i4").clone()
        cells = device_view(v.unit_cells, (R, 2), "i4").clone()
        ncell = int((cells[:, 0] * cells[:, 1]).sum().item()) if R else 0
        cell_len = int((meta[:, 3].max() + 8 + cells.prod(1).max()).item()) if R else 1
        return dict(
            meta=meta, cells=cells, grid=device_view(v.unit_grid, (R, 4), "f4").clone(),
            cell_start=device_view(v.cell_start, (cell_len,), "i4").clone(), n_cells=ncell,
            yz=device_view(v.yz, (S, 2), "f4").clone(), orig=device_view(v.orig, (S,), "i4").clone(),
            up_raw=device_view(v.up_raw, (S,), "i4").clone(), dn_raw=device_view(v.dn_raw, (S,), "i4").clone(),
            up=device_view(v.up, (S,), "i4").clone(), dn=device_view(v.dn, (S,), "i4").clone(),
            starts=device_view(v.starts, (T, 4), "i4").clone(),
            tl_nhits=device_view(v.tl_nhits, (T,), "i4").clone(),
            tl_hits=device_view(v.tl_hits, (T, self.n_rows), "i4").clone(),
            tl_par=device_view(v.tl_par, (5, Tc), "f4")[:, :T].T.clone(),
            tl_cov=device_view(v.tl_cov, (15, Tc), "f4")[:, :T].T.clone(),
            tl_x=device_view(v.tl_x, (T,), "f4").clone(), tl_chi2=device_view(v.tl_chi2, (T,), "f4").clone(),
            tl_w=device_view(v.tl_w, (T,), "f4").clone(), tl_nowned=device_view(v.tl_nowned, (T,), "i4").clone(),
            cluster_key=device_view(v.cluster_key, (S,), "u8").clone(),
        )

    def close(self):
        if self.handle is not None:
            tpc_tracker_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
