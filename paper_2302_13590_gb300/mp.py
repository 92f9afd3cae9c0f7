"""Thin Python binding of libmp (the C ABI in include/mp.h).

Argument marshalling only: every step of the tracking runs in the CUDA
kernels of ``libmp.so``.  The module-level functions carry the C names
(``mp_field_load``, ``mp_release_group``, ``mp_track``, ``mp_get_endpoints``,
``mp_get_timeseries`` ...); ``Context`` / ``Request`` are small conveniences
on top of them.  Arrays are numpy (host) or anything exposing
``data_ptr()`` (torch CUDA tensors, passed with ``device=True``).  Streams are
``cudaStream_t`` handles as integers (e.g. ``torch.cuda.current_stream()
.cuda_stream``) or None for the legacy default stream.

There is no CPU fallback: if ``libmp.so`` cannot be built or loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from typing import Optional

import numpy as np

from . import _build

# ---- constants mirrored from mp.h --------------------------------------------
MP_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "SHAPE", -3: "NONFINITE", -4: "OOM", -5: "BUSY", -6: "TIMEOUT",
          -7: "CUDA", -8: "NOT_READY", -9: "DEVICE"}
MP_ERR_TIMEOUT = -6
ERR_INVALID_ARG, ERR_SHAPE, ERR_NONFINITE, ERR_OOM = -1, -2, -3, -4
ST_ACTIVE, ST_TIME, ST_SINK, ST_BOUNDARY, ST_EXIT_DOMAIN, ST_NO_EXIT, ST_STEP_CAP, ST_INVALID_RELEASE = range(8)
STATUS_NAMES = ["ACTIVE", "TIME", "SINK", "BOUNDARY", "EXIT_DOMAIN", "NO_EXIT", "STEP_CAP", "INVALID_RELEASE"]
FACE_NONE = 255
MP_DEVICE_PTR = 1
PREC_FP64, PREC_MIXED, PREC_MIXED_F64T = 0, 1, 2
MODE_ENDPOINT, MODE_TIMESERIES, MODE_PATHLINE = 1, 2, 4
SCHED_STATIC, SCHED_DYNAMIC, SCHED_AUTO = 0, 1, 2
TRACK_UPDATE_GROUP = 1
TRACK_PASS_WEAK_SINKS = 2
RELEASE_EXPLICIT, RELEASE_BOX = 0, 1

TS_RECORD = np.dtype([("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("cell", "<i4"), ("status", "u1"),
                      ("pad", "u1", (3,))])
assert TS_RECORD.itemsize == 32
PATH_RECORD = np.dtype([("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("t", "<f8"), ("particle", "<i4"),
                        ("cell", "<i4"), ("seq", "<u4"), ("status", "u1"), ("pad", "u1", (3,))])
assert PATH_RECORD.itemsize == 48

_vp = ctypes.c_void_p


class FieldDesc(ctypes.Structure):
    _fields_ = [("nlay", ctypes.c_int32), ("nrow", ctypes.c_int32), ("ncol", ctypes.c_int32),
                ("delr", _vp), ("delc", _vp), ("dz", _vp), ("origin", ctypes.c_double * 3),
                ("qx", _vp), ("qy", _vp), ("qz", _vp), ("porosity", _vp), ("ibound", _vp),
                ("flags", ctypes.c_uint32)]


class ReleaseDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("kind", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("cell", _vp), ("local", _vp), ("t0", _vp),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("seed", ctypes.c_uint64), ("id_offset", ctypes.c_uint64)]


class TrackOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("n_times", ctypes.c_int32), ("times", _vp), ("t_stop", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("block", ctypes.c_int32), ("steps_per_fetch", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("path_capacity", ctypes.c_int64), ("weak_sink_fraction", ctypes.c_double)]


class UsgDesc(ctypes.Structure):
    _fields_ = [("ncell", ctypes.c_int64)] + [(k, _vp) for k in ("box", "porosity", "ibound", "face_off", "nbr",
                                                                 "q", "rect")] + [("flags", ctypes.c_uint32)]


class Balance(ctypes.Structure):
    _fields_ = [("max_abs_residual", ctypes.c_double), ("max_abs_cell", ctypes.c_int64),
                ("max_rel_residual", ctypes.c_double), ("sink_extraction", ctypes.c_double),
                ("active_cells", ctypes.c_int64), ("sink_cells", ctypes.c_int64)]


class Endpoints(ctypes.Structure):
    _fields_ = [(n, _vp) for n in ("cell", "x", "y", "z", "px", "py", "pz", "t", "status", "steps",
                                   "exit_face", "hash")]


class NoallocArgs(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("cell", _vp), ("px", _vp), ("py", _vp), ("pz", _vp), ("t", _vp),
                ("status", _vp), ("out", Endpoints), ("ts", _vp), ("opts", TrackOpts)]


NOALLOC_MAX_TIMES = 4096


class Tuning(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("block", ctypes.c_int32), ("steps_per_fetch", ctypes.c_int32),
                ("tried", ctypes.c_int32), ("ms", ctypes.c_float)]


class Stats(ctypes.Structure):
    _fields_ = [("cell_steps", ctypes.c_uint64), ("n_status", ctypes.c_uint64 * 8),
                ("kernel_ms", ctypes.c_float), ("device_error", ctypes.c_int32), ("path_points", ctypes.c_uint64),
                ("t_begin_ns", ctypes.c_uint64), ("t_end_ns", ctypes.c_uint64)]


ENDPOINT_DTYPES = {"cell": np.int32, "x": np.float64, "y": np.float64, "z": np.float64, "px": np.float64,
                   "py": np.float64, "pz": np.float64, "t": np.float64, "status": np.uint8,
                   "steps": np.uint32, "exit_face": np.uint8, "hash": np.uint64}

# every exported entry point with (restype, argtypes)
_P = ctypes.POINTER
SIGNATURES = {
    "mp_ctx_create": (ctypes.c_int, [ctypes.c_int, _P(_vp)]),
    "mp_ctx_destroy": (ctypes.c_int, [_vp]),
    "mp_last_error": (ctypes.c_char_p, []),
    "mp_field_load": (ctypes.c_int, [_vp, _P(FieldDesc), _P(_vp)]),
    "mp_field_free": (ctypes.c_int, [_vp]),
    "mp_field_bytes": (ctypes.c_int, [_vp, _P(ctypes.c_size_t)]),
    "mp_field_balance": (ctypes.c_int, [_vp, _P(Balance)]),
    "mp_release_group": (ctypes.c_int, [_vp, _vp, _P(ReleaseDesc), _vp, _P(_vp)]),
    "mp_group_free": (ctypes.c_int, [_vp]),
    "mp_group_size": (ctypes.c_int, [_vp, _P(ctypes.c_int64)]),
    "mp_track": (ctypes.c_int, [_vp, _vp, _P(TrackOpts), _vp, _P(ctypes.c_int64)]),
    "mp_track_batch": (ctypes.c_int, [_vp, ctypes.c_int, _P(_vp), _P(TrackOpts), _vp, _P(ctypes.c_int64)]),
    "mp_wait": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64]),
    "mp_query": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "mp_get_endpoints": (ctypes.c_int, [_vp, ctypes.c_int64, _P(Endpoints), ctypes.c_uint32, _vp]),
    "mp_get_timeseries": (ctypes.c_int, [_vp, ctypes.c_int64, _vp, ctypes.c_uint32, _vp]),
    "mp_endpoints_device": (ctypes.c_int, [_vp, ctypes.c_int64, _P(Endpoints), _P(_vp)]),
    "mp_get_stats": (ctypes.c_int, [_vp, ctypes.c_int64, _P(Stats)]),
    "mp_req_free": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "mp_query_bytes": (ctypes.c_int, [_P(TrackOpts), ctypes.c_int64, _P(ctypes.c_size_t)]),
    "mp_track_launches": (ctypes.c_int, [_P(TrackOpts), _P(ctypes.c_int32)]),
    "mp_track_noalloc": (ctypes.c_int, [_vp, _P(NoallocArgs), _vp, _P(Stats)]),
    "mp_autotune": (ctypes.c_int, [_vp, _vp, _P(TrackOpts), ctypes.c_int64, _vp, _P(Tuning)]),
    "mp_set_tuning": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _P(Tuning)]),
    "mp_group_set_field": (ctypes.c_int, [_vp, _vp]),
    "mp_usg_field_load": (ctypes.c_int, [_vp, _P(UsgDesc), _P(_vp)]),
    "mp_graph_create": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _P(ReleaseDesc), _P(TrackOpts), _vp, _P(_vp)]),
    "mp_graph_set_release": (ctypes.c_int, [_vp, ctypes.c_int, _P(ReleaseDesc), _vp]),
    "mp_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "mp_graph_requests": (ctypes.c_int, [_vp, _P(ctypes.c_int64)]),
    "mp_graph_free": (ctypes.c_int, [_vp]),
    "mp_get_pathlines": (ctypes.c_int, [_vp, ctypes.c_int64, _vp, ctypes.c_int64, _P(ctypes.c_int64), ctypes.c_uint32,
                                        _vp]),
    "mp_track_periods": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _P(_vp), _vp, _P(TrackOpts), _vp,
                                        _P(ctypes.c_int64)]),
    "mp_track_host": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _P(TrackOpts), ctypes.c_int32,
                                     _P(Endpoints), _vp, _P(Stats)]),
}

_lib = None
_lock = threading.Lock()


class MPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libmp error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load_library(build: bool = True):
    """Load libmp.so (building it with nvcc first if needed); raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build_lib() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libmp.so not found at {path}; run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != MP_OK:
        raise MPError(rc, load_library().mp_last_error().decode(errors="replace"))


def _ptr(a):
    """Pointer of a numpy array or a tensor (data_ptr); None stays NULL."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype).reshape(-1))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


# ---- C-named functions ----------------------------------------------------------

def mp_ctx_create(device: int = 0):
    h = ctypes.c_void_p()
    _check(load_library().mp_ctx_create(int(device), ctypes.byref(h)))
    return h


def mp_ctx_destroy(ctx):
    _check(load_library().mp_ctx_destroy(ctx))


def mp_field_load(ctx, field, device_arrays: bool = False):
    """Load a field (an object with nlay, nrow, ncol, delr, delc, dz, origin,
    qx, qy, qz, porosity, ibound).  With device_arrays=True the flow arrays are
    CUDA tensors (float64 / int8, contiguous) read in place."""
    keep = []
    delr, delc, dz = (_host(field.delr, np.float64), _host(field.delc, np.float64), _host(field.dz, np.float64))
    keep += [delr, delc, dz]
    if device_arrays:
        arrs = [field.qx, field.qy, field.qz, field.porosity, field.ibound]
    else:
        arrs = [_host(field.qx, np.float64), _host(field.qy, np.float64), _host(field.qz, np.float64),
                _host(field.porosity, np.float64), _host(field.ibound, np.int8)]
        keep += arrs
    d = FieldDesc(int(field.nlay), int(field.nrow), int(field.ncol), _ptr(delr), _ptr(delc), _ptr(dz),
                  (ctypes.c_double * 3)(*[float(o) for o in field.origin]), *[_ptr(a) for a in arrs],
                  MP_DEVICE_PTR if device_arrays else 0)
    h = ctypes.c_void_p()
    _check(load_library().mp_field_load(ctx, ctypes.byref(d), ctypes.byref(h)))
    return h


def mp_usg_field_load(ctx, u):
    """Load a rectangular unstructured grid (an object with box, porosity,
    ibound, face_off, nbr, q, rect; see inputs.usg.UsgField)."""
    arrs = [_host(u.box, np.float64), _host(u.porosity, np.float64), _host(u.ibound, np.int8),
            _host(u.face_off, np.int64), _host(u.nbr, np.int32), _host(u.q, np.float64), _host(u.rect, np.float64)]
    d = UsgDesc(int(arrs[0].size // 6), *[_ptr(a) for a in arrs], 0)
    h = ctypes.c_void_p()
    _check(load_library().mp_usg_field_load(ctx, ctypes.byref(d), ctypes.byref(h)))
    return h


def mp_field_free(fh):
    _check(load_library().mp_field_free(fh))


def mp_field_bytes(fh) -> int:
    b = ctypes.c_size_t()
    _check(load_library().mp_field_bytes(fh, ctypes.byref(b)))
    return b.value


def mp_field_balance(fh) -> dict:
    """Volume balance of a loaded field (computed at load from its face flows)."""
    b = Balance()
    _check(load_library().mp_field_balance(fh, ctypes.byref(b)))
    return {k: getattr(b, k) for k, _ in Balance._fields_}


def mp_release_group(ctx, fh, *, n=None, lo=None, hi=None, seed=0, id_offset=0, cell=None, local=None,
                     t0=None, stream=None, device_arrays: bool = False):
    """Box release (lo, hi, seed) or explicit release (cell, local[, t0])."""
    keep = []
    if cell is not None:
        if device_arrays:
            c, l, t = cell, local, t0
            nn = int(cell.numel())
        else:
            c, l = _host(cell, np.int32), _host(local, np.float64)
            t = None if t0 is None else _host(t0, np.float64)
            keep += [c, l, t]
            nn = c.size
        d = ReleaseDesc(nn, RELEASE_EXPLICIT, MP_DEVICE_PTR if device_arrays else 0, _ptr(c), _ptr(l), _ptr(t),
                        (ctypes.c_double * 3)(0, 0, 0), (ctypes.c_double * 3)(0, 0, 0), 0, 0)
    else:
        d = ReleaseDesc(int(n), RELEASE_BOX, 0, None, None, None, (ctypes.c_double * 3)(*map(float, lo)),
                        (ctypes.c_double * 3)(*map(float, hi)), int(seed) & (2 ** 64 - 1), int(id_offset))
    h = ctypes.c_void_p()
    _check(load_library().mp_release_group(ctx, fh, ctypes.byref(d), _stream(stream), ctypes.byref(h)))
    return h


def _box_desc(n, lo, hi, seed=0, id_offset=0) -> ReleaseDesc:
    return ReleaseDesc(int(n), RELEASE_BOX, 0, None, None, None, (ctypes.c_double * 3)(*map(float, lo)),
                       (ctypes.c_double * 3)(*map(float, hi)), int(seed) & (2 ** 64 - 1), int(id_offset))


def mp_graph_create(ctx, fh, releases, opts_list, stream=None):
    """Capture box releases (objects with n, lo, hi, seed, id_offset) and
    their tracking as one CUDA graph; returns (handle, request ids)."""
    n = len(releases)
    rel = (ReleaseDesc * n)(*[_box_desc(r.n, r.lo, r.hi, r.seed, getattr(r, "id_offset", 0)) for r in releases])
    oarr = (TrackOpts * n)(*opts_list)
    h = ctypes.c_void_p()
    _check(load_library().mp_graph_create(ctx, fh, n, rel, oarr, _stream(stream), ctypes.byref(h)))
    ids = (ctypes.c_int64 * n)()
    _check(load_library().mp_graph_requests(h, ids))
    return h, [int(v) for v in ids]


def mp_graph_set_release(gh, i, n, lo, hi, seed=0, id_offset=0, stream=None):
    d = _box_desc(n, lo, hi, seed, id_offset)
    _check(load_library().mp_graph_set_release(gh, int(i), ctypes.byref(d), _stream(stream)))


def mp_graph_launch(gh, stream=None):
    _check(load_library().mp_graph_launch(gh, _stream(stream)))


def mp_graph_free(gh):
    _check(load_library().mp_graph_free(gh))


def mp_group_free(gh):
    _check(load_library().mp_group_free(gh))


def mp_group_size(gh) -> int:
    n = ctypes.c_int64()
    _check(load_library().mp_group_size(gh, ctypes.byref(n)))
    return n.value


def mp_group_set_field(gh, fh):
    """Rebind a group to another field on the same grid (the next flow period)."""
    _check(load_library().mp_group_set_field(gh, fh))


def mp_track_periods(ctx, gh, fields, t_end, opts: "TrackOpts", stream=None) -> int:
    """Piecewise-steady flow: fields[p] holds until t_end[p] (len(fields) - 1
    ends); one request, one launch per period."""
    n = len(fields)
    farr = (_vp * n)(*[f.value if isinstance(f, ctypes.c_void_p) else f for f in fields])
    tarr = _host(t_end, np.float64) if n > 1 else None
    r = ctypes.c_int64()
    _check(load_library().mp_track_periods(ctx, gh, n, farr, _ptr(tarr), ctypes.byref(opts), _stream(stream),
                                           ctypes.byref(r)))
    return r.value


def make_opts(mode=MODE_ENDPOINT, precision=PREC_FP64, schedule=SCHED_DYNAMIC, times=None, t_stop=math.inf,
              max_steps=0, block=0, steps_per_fetch=0, flags=0, path_capacity=0, weak_sink_fraction=0.0):
    tarr = None if times is None else _host(times, np.float64)
    o = TrackOpts(int(mode), int(precision), int(schedule), 0 if tarr is None else int(tarr.size), _ptr(tarr),
                  float(t_stop), int(max_steps), int(block), int(steps_per_fetch), int(flags), int(path_capacity),
                  float(weak_sink_fraction))
    o._keep = tarr
    return o


def mp_track(ctx, gh, opts: TrackOpts, stream=None) -> int:
    r = ctypes.c_int64()
    _check(load_library().mp_track(ctx, gh, ctypes.byref(opts), _stream(stream), ctypes.byref(r)))
    return r.value


def mp_track_batch(ctx, groups, opts_list, stream=None):
    """Several groups (one field) in one launch per precision; returns request ids."""
    n = len(groups)
    garr = (_vp * n)(*[g.value if isinstance(g, ctypes.c_void_p) else g for g in groups])
    oarr = (TrackOpts * n)(*opts_list)
    ids = (ctypes.c_int64 * n)()
    _check(load_library().mp_track_batch(ctx, n, garr, oarr, _stream(stream), ids))
    return [int(v) for v in ids]


def mp_wait(ctx, req: int, timeout_us: int = -1):
    _check(load_library().mp_wait(ctx, int(req), int(timeout_us)))


def mp_query(ctx, req: int) -> bool:
    rc = load_library().mp_query(ctx, int(req))
    if rc < 0:
        _check(rc)
    return rc == 1


def mp_get_endpoints(ctx, req: int, n: int, out: Optional[dict] = None, device: bool = False, stream=None):
    """Endpoint arrays; host numpy by default, or into given tensors (device=True)."""
    if out is None:
        out = {k: np.empty(n, dt) for k, dt in ENDPOINT_DTYPES.items()}
    e = Endpoints(*[_ptr(out.get(k)) for k, _ in Endpoints._fields_])
    _check(load_library().mp_get_endpoints(ctx, int(req), ctypes.byref(e), MP_DEVICE_PTR if device else 0,
                                           _stream(stream)))
    return out


def mp_get_timeseries(ctx, req: int, n: int, n_times: int, out=None, device: bool = False, stream=None):
    """[n_times, n] records (numpy structured array TS_RECORD, or a given buffer)."""
    if out is None:
        out = np.empty((n_times, n), TS_RECORD)
    _check(load_library().mp_get_timeseries(ctx, int(req), _ptr(out), MP_DEVICE_PTR if device else 0,
                                            _stream(stream)))
    return out


def mp_endpoints_device(ctx, req: int):
    """(dict of device pointers, timeseries device pointer) of the request's own buffers."""
    e = Endpoints()
    ts = ctypes.c_void_p()
    _check(load_library().mp_endpoints_device(ctx, int(req), ctypes.byref(e), ctypes.byref(ts)))
    return {k: getattr(e, k) for k, _ in Endpoints._fields_}, ts.value


def mp_get_pathlines(ctx, req: int, max_points: int = -1, out=None, device: bool = False, stream=None):
    """The request's pathline points (numpy PATH_RECORD array in production
    order; or into a given host/device buffer); max_points < 0: all kept."""
    if max_points < 0:
        max_points = mp_get_stats(ctx, req)["path_points"]
    if out is None:
        out = np.empty(max_points, PATH_RECORD)
    got = ctypes.c_int64()
    _check(load_library().mp_get_pathlines(ctx, int(req), _ptr(out), int(max_points), ctypes.byref(got),
                                           MP_DEVICE_PTR if device else 0, _stream(stream)))
    return out[:got.value] if isinstance(out, np.ndarray) else out


def mp_get_stats(ctx, req: int) -> dict:
    s = Stats()
    _check(load_library().mp_get_stats(ctx, int(req), ctypes.byref(s)))
    return {"cell_steps": int(s.cell_steps), "n_status": [int(v) for v in s.n_status],
            "kernel_ms": float(s.kernel_ms), "device_error": int(s.device_error),
            "path_points": int(s.path_points), "t_begin_ns": int(s.t_begin_ns), "t_end_ns": int(s.t_end_ns)}


def mp_track_host(ctx, fh, cell, local, opts: "TrackOpts", t0=None, n_chunks: int = 0, out=None, ts_out=None):
    """Host-to-host tracking with transfers overlapped (chunked, two streams).
    cell (n,), local (n, 3) host arrays; out: dict of host endpoint arrays
    (None: allocated); ts_out: [n_times, n] TS_RECORD array for timeseries
    mode (None: allocated when the mode asks for it).  Returns (endpoints,
    timeseries or None, stats)."""
    c, l = _host(cell, np.int32), _host(local, np.float64)
    t = None if t0 is None else _host(t0, np.float64)
    n = c.size
    if out is None:
        out = {k: np.empty(n, dt) for k, dt in ENDPOINT_DTYPES.items()}
    if ts_out is None and (opts.mode & MODE_TIMESERIES) and opts.n_times > 0:
        ts_out = np.empty((opts.n_times, n), TS_RECORD)
    e = Endpoints(*[_ptr(out.get(k)) for k, _ in Endpoints._fields_])
    st = Stats()
    _check(load_library().mp_track_host(ctx, fh, int(n), _ptr(c), _ptr(l), _ptr(t), ctypes.byref(opts),
                                        int(n_chunks), ctypes.byref(e), _ptr(ts_out), ctypes.byref(st)))
    stats = {"cell_steps": int(st.cell_steps), "n_status": [int(v) for v in st.n_status],
             "kernel_ms": float(st.kernel_ms), "device_error": int(st.device_error)}
    return out, ts_out, stats


def mp_req_free(ctx, req: int):
    _check(load_library().mp_req_free(ctx, int(req)))


def mp_query_bytes(opts: TrackOpts, n: int) -> int:
    b = ctypes.c_size_t()
    _check(load_library().mp_query_bytes(ctypes.byref(opts), int(n), ctypes.byref(b)))
    return b.value


def mp_track_launches(opts: TrackOpts) -> int:
    v = ctypes.c_int32()
    _check(load_library().mp_track_launches(ctypes.byref(opts), ctypes.byref(v)))
    return v.value


def mp_track_noalloc(fh, state: dict, out: dict, ts=None, opts: TrackOpts = None, stream=None,
                     want_stats: bool = True):
    """Track with caller-owned device buffers only (no device allocation).

    ``state``: cell/px/py/pz/t/status device tensors; ``out``: every endpoint
    array as a device tensor; ``ts``: device record buffer ([n_times, n] x 32
    bytes) in timeseries mode.  Returns the stats dict when ``want_stats``
    (the call then waits for the stream), else None."""
    n = int(state["cell"].numel())
    e = Endpoints(*[_ptr(out[k]) for k, _ in Endpoints._fields_])
    a = NoallocArgs(n, _ptr(state["cell"]), _ptr(state["px"]), _ptr(state["py"]), _ptr(state["pz"]),
                    _ptr(state["t"]), _ptr(state["status"]), e, _ptr(ts), opts)
    st = Stats()
    _check(load_library().mp_track_noalloc(fh, ctypes.byref(a), _stream(stream),
                                           ctypes.byref(st) if want_stats else None))
    if not want_stats:
        return None
    return {"cell_steps": int(st.cell_steps), "n_status": [int(v) for v in st.n_status],
            "kernel_ms": float(st.kernel_ms), "device_error": int(st.device_error)}


def mp_autotune(ctx, gh, opts: TrackOpts, sample: int = 0, stream=None) -> dict:
    """Time the candidate launch configurations; returns the fastest (also
    kept in the context for MP_SCHED_AUTO)."""
    t = Tuning()
    _check(load_library().mp_autotune(ctx, gh, ctypes.byref(opts), int(sample), _stream(stream), ctypes.byref(t)))
    return {"schedule": t.schedule, "block": t.block, "steps_per_fetch": t.steps_per_fetch, "tried": t.tried,
            "ms": float(t.ms)}


def mp_set_tuning(ctx, fh, precision: int, timeseries: bool, tuning: dict):
    t = Tuning(int(tuning["schedule"]), int(tuning["block"]), int(tuning["steps_per_fetch"]),
               int(tuning.get("tried", 0)), float(tuning.get("ms", 0.0)))
    _check(load_library().mp_set_tuning(ctx, fh, int(precision), int(bool(timeseries)), ctypes.byref(t)))


def load_tuning_cache(path: str) -> dict:
    """Tuning results cached as JSON: {"<workload>/<precision>/<ts>": tuning}."""
    import json
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_tuning_cache(path: str, cache: dict):
    import json
    import os as _os
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    _os.replace(tmp, path)


# ---- conveniences -------------------------------------------------------------------

class Context:
    """Owns an mp_ctx; fields, groups and requests are freed with it."""

    def __init__(self, device: int = 0):
        self.h = mp_ctx_create(device)

    def close(self):
        if self.h is not None:
            mp_ctx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def field(self, f, device_arrays=False):
        if hasattr(f, "face_off"):
            return mp_usg_field_load(self.h, f)
        return mp_field_load(self.h, f, device_arrays=device_arrays)

    def release_box(self, fh, n, lo, hi, seed, id_offset=0, stream=None):
        return mp_release_group(self.h, fh, n=n, lo=lo, hi=hi, seed=seed, id_offset=id_offset, stream=stream)

    def release_explicit(self, fh, cell, local, t0=None, stream=None, device_arrays=False):
        return mp_release_group(self.h, fh, cell=cell, local=local, t0=t0, stream=stream,
                                device_arrays=device_arrays)

    def track(self, gh, stream=None, **kw) -> "Request":
        opts = make_opts(**kw)
        n = mp_group_size(gh)
        rid = mp_track(self.h, gh, opts, stream)
        nt = opts.n_times if (opts.mode & MODE_TIMESERIES) else 0
        return Request(self, rid, n, nt)

    def track_periods(self, gh, fields, t_end, stream=None, **kw) -> "Request":
        opts = make_opts(**kw)
        n = mp_group_size(gh)
        rid = mp_track_periods(self.h, gh, fields, t_end, opts, stream)
        nt = opts.n_times if (opts.mode & MODE_TIMESERIES) else 0
        return Request(self, rid, n, nt)


class Request:
    def __init__(self, ctx: Context, rid: int, n: int, n_times: int):
        self.ctx, self.id, self.n, self.n_times = ctx, rid, n, n_times

    def wait(self, timeout_us=-1):
        mp_wait(self.ctx.h, self.id, timeout_us)

    def done(self) -> bool:
        return mp_query(self.ctx.h, self.id)

    def endpoints(self):
        return mp_get_endpoints(self.ctx.h, self.id, self.n)

    def timeseries(self):
        return mp_get_timeseries(self.ctx.h, self.id, self.n, self.n_times)

    def stats(self):
        return mp_get_stats(self.ctx.h, self.id)

    def pathlines(self, max_points: int = -1):
        return mp_get_pathlines(self.ctx.h, self.id, max_points)

    def free(self):
        mp_req_free(self.ctx.h, self.id)
