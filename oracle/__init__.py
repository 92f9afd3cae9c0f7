"""CPU oracle for semi-analytical (Pollock 1988) particle tracking.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg import this package.  The product path (the
CUDA library and its binding) never touches it, and this package imports
nothing from the product.

The arithmetic lives in ``mp_oracle.c`` (plain single-threaded IEEE double,
compiled with ``-O2 -ffp-contract=off``); this file only compiles it and
marshals numpy arrays.

Two arithmetic modes (``arith``): ``"plain"``, the reference, evaluates the
in-cell solution as its formulas read (the C library's log1p and expm1,
IEEE division, no fused multiply-add); ``"mirror"`` evaluates the same
solution by fixed table-driven steps with fused multiply-adds, so that an
implementation of the same steps can be checked bit for bit.  Both modes
are held to the same pins.  A field is any object with the attributes
``nlay, nrow, ncol, delr, delc, dz, origin, qx, qy, qz, porosity, ibound``.

Pins: every function here is checked against closed forms, brute-force RK4
integration and invariants in ``tests/test_oracle_*.py``; parity with
MODPATH itself is unpinned (MODPATH is not available).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mp_oracle.c")
_HDR = os.path.join(_HERE, "mp_oracle.h")
_TAB = os.path.join(_HERE, "orc_tables.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

ST_ACTIVE, ST_TIME, ST_SINK, ST_BOUNDARY, ST_EXIT_DOMAIN, ST_NO_EXIT, ST_STEP_CAP, ST_INVALID_RELEASE = range(8)
FACE_NONE = 255
DEFAULT_MAX_STEPS = 1_000_000


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR), os.path.getmtime(_TAB))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Field(ctypes.Structure):
    _fields_ = [("nlay", ctypes.c_int32), ("nrow", ctypes.c_int32), ("ncol", ctypes.c_int32),
                ("delr", ctypes.c_void_p), ("delc", ctypes.c_void_p), ("dz", ctypes.c_void_p),
                ("origin", ctypes.c_double * 3),
                ("qx", ctypes.c_void_p), ("qy", ctypes.c_void_p), ("qz", ctypes.c_void_p),
                ("porosity", ctypes.c_void_p), ("ibound", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("t_stop", ctypes.c_double), ("n_times", ctypes.c_int32),
                ("times", ctypes.c_void_p), ("max_steps", ctypes.c_int64), ("pass_weak_sinks", ctypes.c_int32),
                ("path_start", ctypes.c_int32), ("weak_sink_fraction", ctypes.c_double),
                ("arith", ctypes.c_int32), ("jitter", ctypes.c_double), ("jitter_seed", ctypes.c_uint64),
                ("jitter_id0", ctypes.c_int64)]


ARITH = {"plain": 0, "mirror": 1}
# the mode used where a call names none; "plain" is the reference
DEFAULT_ARITH = "plain"


def _arith(arith) -> int:
    if arith is None:
        arith = DEFAULT_ARITH
    if arith not in ARITH:
        raise ValueError(f"arith must be one of {sorted(ARITH)}, got {arith!r}")
    return ARITH[arith]


# one pathline point (orc_path_rec)
PATH_RECORD = np.dtype([("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("t", "<f8"), ("particle", "<i4"),
                        ("cell", "<i4"), ("seq", "<u4"), ("status", "u1"), ("pad", "u1", (3,))])


# one traced cell-step (orc_trace_rec)
TRACE_RECORD = np.dtype([("te", "<f8", (3,)), ("vp", "<f8", (3,)), ("vf", "<f8", (3,)), ("t", "<f8"), ("particle", "<i4"),
                         ("cell", "<i4"), ("face", "i1", (3,)), ("ax", "i1"), ("pad", "u1", (4,))])


class _Out(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("cell", "px", "py", "pz", "gx", "gy", "gz", "t", "status", "steps", "exit_face", "hash",
                 "ts_x", "ts_y", "ts_z", "ts_cell", "ts_status", "path")] + \
        [("path_cap", ctypes.c_int64), ("path_n", ctypes.c_void_p),
         ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_int64), ("trace_n", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
            lib.orc_philox4x32_10.restype = None
            lib.orc_exit_time.argtypes = [ctypes.c_double] * 6 + [ctypes.POINTER(ctypes.c_int)]
            lib.orc_exit_time.restype = ctypes.c_double
            lib.orc_log1p.argtypes = [ctypes.c_double]
            lib.orc_log1p.restype = ctypes.c_double
            lib.orc_expm1.argtypes = [ctypes.c_double]
            lib.orc_expm1.restype = ctypes.c_double
            lib.orc_div.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.orc_div.restype = ctypes.c_double
            lib.orc_move.argtypes = [ctypes.c_double] * 6
            lib.orc_move.restype = ctypes.c_double
            lib.orc_exit_time_plain.argtypes = [ctypes.c_double] * 5 + [ctypes.POINTER(ctypes.c_int)]
            lib.orc_exit_time_plain.restype = ctypes.c_double
            lib.orc_move_plain.argtypes = [ctypes.c_double] * 5
            lib.orc_move_plain.restype = ctypes.c_double
            lib.orc_release_box.argtypes = [ctypes.POINTER(_Field), ctypes.c_int64, vp, vp,
                                            ctypes.c_uint64, ctypes.c_uint64, vp, vp, vp, vp, vp]
            lib.orc_release_box.restype = ctypes.c_int
            lib.orc_release_explicit.argtypes = [ctypes.POINTER(_Field), ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_release_explicit.restype = ctypes.c_int
            lib.orc_track.argtypes = [ctypes.POINTER(_Field), ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                      ctypes.POINTER(_Opts), ctypes.POINTER(_Out)]
            lib.orc_track.restype = ctypes.c_int
            lib.orc_usg_track.argtypes = [ctypes.POINTER(_UsgField)] + lib.orc_track.argtypes[1:]
            lib.orc_usg_track.restype = ctypes.c_int
            lib.orc_usg_release_explicit.argtypes = [ctypes.POINTER(_UsgField), ctypes.c_int64] + [vp] * 7
            lib.orc_usg_release_explicit.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleField:
    """Keeps contiguous float64 / int8 copies of a field and its C view."""

    def __init__(self, f):
        self.nlay, self.nrow, self.ncol = int(f.nlay), int(f.nrow), int(f.ncol)
        c = lambda a, dt: np.ascontiguousarray(np.asarray(a, dtype=dt).reshape(-1))
        self.delr, self.delc, self.dz = c(f.delr, np.float64), c(f.delc, np.float64), c(f.dz, np.float64)
        self.qx, self.qy, self.qz = c(f.qx, np.float64), c(f.qy, np.float64), c(f.qz, np.float64)
        self.porosity = c(f.porosity, np.float64)
        self.ibound = c(f.ibound, np.int8)
        assert self.qx.size == self.nlay * self.nrow * (self.ncol + 1)
        assert self.qy.size == self.nlay * (self.nrow + 1) * self.ncol
        assert self.qz.size == (self.nlay + 1) * self.nrow * self.ncol
        assert self.porosity.size == self.ibound.size == self.nlay * self.nrow * self.ncol
        self.origin = tuple(float(o) for o in f.origin)
        self.c = _Field(self.nlay, self.nrow, self.ncol, _ptr(self.delr), _ptr(self.delc), _ptr(self.dz),
                        (ctypes.c_double * 3)(*self.origin), _ptr(self.qx), _ptr(self.qy), _ptr(self.qz),
                        _ptr(self.porosity), _ptr(self.ibound))


class _UsgField(ctypes.Structure):
    _fields_ = [("ncell", ctypes.c_int64)] + [(k, ctypes.c_void_p) for k in
                                               ("box", "porosity", "ibound", "face_off", "nbr", "q", "rect")]


class OracleUsgField:
    """Contiguous copies of a rectangular unstructured field and its C view."""

    def __init__(self, u):
        c = lambda a, dt: np.ascontiguousarray(np.asarray(a, dtype=dt).reshape(-1))
        self.ncell = int(np.asarray(u.box).shape[0])
        self.box = c(u.box, np.float64)
        self.porosity, self.ibound = c(u.porosity, np.float64), c(u.ibound, np.int8)
        self.face_off, self.nbr = c(u.face_off, np.int64), c(u.nbr, np.int32)
        self.q, self.rect = c(u.q, np.float64), c(u.rect, np.float64)
        assert self.box.size == 6 * self.ncell and self.face_off.size == 6 * self.ncell + 1
        assert self.rect.size == 4 * self.nbr.size == 4 * self.q.size
        self.c = _UsgField(self.ncell, *[_ptr(a) for a in (self.box, self.porosity, self.ibound, self.face_off,
                                                             self.nbr, self.q, self.rect)])


def _is_usg(f) -> bool:
    return isinstance(f, OracleUsgField) or hasattr(f, "face_off")


def as_oracle_field(f):
    if isinstance(f, (OracleField, OracleUsgField)):
        return f
    return OracleUsgField(f) if _is_usg(f) else OracleField(f)


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def exit_time(v1, v2, A, D, p, arith=None):
    """(t_exit, face) for one axis of one cell (face +1, -1 or 0 = none)."""
    lib = _load()
    face = ctypes.c_int(0)
    if _arith(arith) == ARITH["mirror"]:
        t = lib.orc_exit_time(float(v1), float(v2), float(A), _inv(A), float(D), float(p), ctypes.byref(face))
    else:
        t = lib.orc_exit_time_plain(float(v1), float(v2), float(A), float(D), float(p), ctypes.byref(face))
    return t, face.value


def log1p(x):
    """The mirror mode's table-driven log1p (the plain mode calls the C library's)."""
    return _load().orc_log1p(float(x))


def expm1(w):
    """The mirror mode's table-driven expm1 (the plain mode calls the C library's)."""
    return _load().orc_expm1(float(w))


def div(d, v):
    """The mirror mode's quotient d / v: d times a Newton-refined reciprocal
    (the plain mode divides in IEEE double)."""
    return _load().orc_div(float(d), float(v))


def move(v1, A, D, p, dt, arith=None):
    lib = _load()
    if _arith(arith) == ARITH["mirror"]:
        return lib.orc_move(float(v1), float(A), _inv(A), float(D), float(p), float(dt))
    return lib.orc_move_plain(float(v1), float(A), float(D), float(p), float(dt))


def _inv(A):
    """1 / A as the oracle forms it per cell (0 when A == 0)."""
    A = float(A)
    return 1.0 / A if A != 0.0 else 0.0


def release_box(f, n, lo, hi, seed, id_offset=0):
    """Particles uniform in the box [lo, hi] via Philox4x32-10; returns a state dict."""
    lib = _load()
    of = as_oracle_field(f)
    st = dict(cell=np.zeros(n, np.int32), px=np.zeros(n), py=np.zeros(n), pz=np.zeros(n),
              status=np.zeros(n, np.uint8))
    lo_a = np.asarray(lo, dtype=np.float64).copy()
    hi_a = np.asarray(hi, dtype=np.float64).copy()
    rc = lib.orc_release_box(ctypes.byref(of.c), int(n), _ptr(lo_a), _ptr(hi_a), int(seed) & (2**64 - 1),
                             int(id_offset), _ptr(st["cell"]), _ptr(st["px"]), _ptr(st["py"]), _ptr(st["pz"]),
                             _ptr(st["status"]))
    if rc != 0:
        raise RuntimeError("orc_release_box failed")
    st["t"] = np.zeros(n)
    return st


def release_explicit(f, cells, frac):
    lib = _load()
    of = as_oracle_field(f)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    frac = np.ascontiguousarray(frac, dtype=np.float64).reshape(-1, 3)
    n = cells.size
    st = dict(cell=np.zeros(n, np.int32), px=np.zeros(n), py=np.zeros(n), pz=np.zeros(n),
              status=np.zeros(n, np.uint8))
    rel = lib.orc_usg_release_explicit if isinstance(of, OracleUsgField) else lib.orc_release_explicit
    rel(ctypes.byref(of.c), n, _ptr(cells), _ptr(frac), _ptr(st["cell"]), _ptr(st["px"]), _ptr(st["py"]),
        _ptr(st["pz"]), _ptr(st["status"]))
    st["t"] = np.zeros(n)
    return st


def subset(state, idx):
    return {k: np.ascontiguousarray(v[idx]) for k, v in state.items()}


def track(f, state, t_stop=np.inf, times=None, max_steps=0, timeseries=None, pass_weak_sinks=False,
          pathline=False, path_start=True, weak_sink_fraction=0.0, arith=None, trace=False, jitter=0.0,
          jitter_seed=0, jitter_id0=0):
    """Track every particle of ``state`` (dict of cell, px, py, pz, t, status,
    and optionally steps, hash and exit_face carried by a resumed particle).

    Returns a dict with the endpoint arrays (cell, px, py, pz, gx, gy, gz, t,
    status, steps, exit_face, hash) and, when ``times`` is given, timeseries
    arrays ts_x/ts_y/ts_z/ts_cell/ts_status of shape [n_times, n].  With
    ``pathline``, ``path`` holds the pathline points (PATH_RECORD) in the
    order produced: per particle its start point (if ``path_start``) and the
    point every cell-step ends at.  ``arith`` selects the arithmetic mode
    ("plain", the reference, or "mirror"; None: ``DEFAULT_ARITH``).  With ``trace``, ``trace`` holds
    one TRACE_RECORD per cell-step (exit times, faces and particle velocity
    per axis, the axis taken).  ``jitter`` > 0 perturbs every crossing by
    about that relative amount (a test instrument, mp_oracle.h), seeded by
    ``jitter_seed`` and the particle's index in ``state``.
    """
    lib = _load()
    of = as_oracle_field(f)
    n = int(np.asarray(state["cell"]).size)
    cell0 = np.ascontiguousarray(state["cell"], dtype=np.int32)
    px0 = np.ascontiguousarray(state["px"], dtype=np.float64)
    py0 = np.ascontiguousarray(state["py"], dtype=np.float64)
    pz0 = np.ascontiguousarray(state["pz"], dtype=np.float64)
    t0 = np.ascontiguousarray(state.get("t", np.zeros(n)), dtype=np.float64)
    s0 = np.ascontiguousarray(state.get("status", np.zeros(n, np.uint8)), dtype=np.uint8)
    k0 = None if state.get("steps") is None else np.ascontiguousarray(state["steps"], dtype=np.uint32)
    h0 = None if state.get("hash") is None else np.ascontiguousarray(state["hash"], dtype=np.uint64)
    e0 = None if state.get("exit_face") is None else np.ascontiguousarray(state["exit_face"], dtype=np.uint8)
    res = dict(cell=np.zeros(n, np.int32), px=np.zeros(n), py=np.zeros(n), pz=np.zeros(n),
               gx=np.zeros(n), gy=np.zeros(n), gz=np.zeros(n), t=np.zeros(n),
               status=np.zeros(n, np.uint8), steps=np.zeros(n, np.uint32),
               exit_face=np.zeros(n, np.uint8), hash=np.zeros(n, np.uint64))
    nt = 0
    tarr = None
    if times is not None and (timeseries is None or timeseries):
        tarr = np.ascontiguousarray(times, dtype=np.float64)
        nt = tarr.size
        for k in ("ts_x", "ts_y", "ts_z"):
            res[k] = np.zeros((nt, n))
        res["ts_cell"] = np.zeros((nt, n), np.int32)
        res["ts_status"] = np.zeros((nt, n), np.uint8)
    opts = _Opts(float(t_stop), nt, _ptr(tarr), int(max_steps), int(bool(pass_weak_sinks)), int(bool(path_start)),
                 float(weak_sink_fraction), _arith(arith), float(jitter), int(jitter_seed) & (2**64 - 1),
                 int(jitter_id0))
    cap = 64 * n + 16
    tcap = 64 * n + 16
    while True:
        path = np.zeros(cap if pathline else 0, PATH_RECORD)
        path_n = np.zeros(1, np.int64)
        trc = np.zeros(tcap if trace else 0, TRACE_RECORD)
        trace_n = np.zeros(1, np.int64)
        out = _Out(*[_ptr(res.get(k)) for k, _ in _Out._fields_[:17]], _ptr(path) if pathline else None, cap,
                   _ptr(path_n), _ptr(trc) if trace else None, tcap, _ptr(trace_n))
        fn = lib.orc_usg_track if isinstance(of, OracleUsgField) else lib.orc_track
        rc = fn(ctypes.byref(of.c), n, _ptr(cell0), _ptr(px0), _ptr(py0), _ptr(pz0), _ptr(t0),
                _ptr(s0), _ptr(k0), _ptr(h0), _ptr(e0), ctypes.byref(opts), ctypes.byref(out))
        if rc != 0:
            raise RuntimeError("orc_track failed")
        if (not pathline or path_n[0] <= cap) and (not trace or trace_n[0] <= tcap):
            break
        # the run is deterministic: repeat with room for every point
        cap = max(cap, int(path_n[0]))
        tcap = max(tcap, int(trace_n[0]))
    if pathline:
        res["path"] = path[:int(path_n[0])]
    if trace:
        res["trace"] = trc[:int(trace_n[0])]
    return res


RESUME_KEYS = ("cell", "px", "py", "pz", "t", "status", "steps", "hash", "exit_face")


def resume_state(out):
    """The state a tracking result leaves for the next call: position, time,
    carried counts, and TIME / STEP_CAP turned back into ACTIVE."""
    st = {k: np.array(out[k]) for k in RESUME_KEYS}
    st["status"] = np.where((st["status"] == ST_TIME) | (st["status"] == ST_STEP_CAP), ST_ACTIVE,
                            st["status"]).astype(np.uint8)
    return st


def track_periods(fields, t_end, state, t_stop=np.inf, times=None, max_steps=0, pass_weak_sinks=False,
                  pathline=False, weak_sink_fraction=0.0, arith=None, jitter=0.0, jitter_seed=0):
    """Piecewise-steady flow (Methods, "MODPATH": the outer loop runs over the
    flow model's time steps and updates the flow arrays at each step's end).

    fields[p] holds from t_end[p-1] to t_end[p] (len(t_end) == len(fields) - 1;
    the last field has no end).  Every period is one ``track`` call with the
    stop time at the period's end, resumed from the state the previous period
    left (steps, hash and exit face carried); output times are split over the
    periods, (t_end[p-1], t_end[p]] to period p.  A particle's endpoint is
    the one from the last period it moved in.  All fields share one grid.
    Pathline points of all periods are concatenated (start points from the
    first period only: later periods continue the same lines).
    """
    P = len(fields)
    t_end = [float(v) for v in t_end]
    if len(t_end) != P - 1 or any(b < a for a, b in zip(t_end, t_end[1:])):
        raise ValueError("track_periods: need len(fields) - 1 ascending period ends")
    n = int(np.asarray(state["cell"]).size)
    cur = {k: np.array(state[k]) for k in ("cell", "px", "py", "pz")}
    cur["t"] = np.array(state.get("t", np.zeros(n)), dtype=np.float64)
    cur["status"] = np.array(state.get("status", np.zeros(n, np.uint8)), dtype=np.uint8)
    cur["steps"] = np.array(state.get("steps", np.zeros(n, np.uint32)), dtype=np.uint32)
    cur["hash"] = np.array(state.get("hash", np.zeros(n, np.uint64)), dtype=np.uint64)
    cur["exit_face"] = np.array(state.get("exit_face", np.zeros(n, np.uint8)), dtype=np.uint8)
    tarr = None if times is None else np.asarray(times, dtype=np.float64)
    res = None
    paths = []
    lo = -np.inf
    for p, f in enumerate(fields):
        last = p == P - 1
        hi = np.inf if last else t_end[p]
        tp = float(t_stop) if last else min(float(t_stop), hi)
        window = None if tarr is None else np.nonzero((tarr > lo) & (tarr <= hi))[0]
        wt = None if window is None or window.size == 0 else tarr[window]
        moved = (cur["status"] == ST_ACTIVE) | (p == 0)
        out = track(f, cur, t_stop=tp, times=wt, max_steps=max_steps, pass_weak_sinks=pass_weak_sinks,
                    pathline=pathline, path_start=p == 0, weak_sink_fraction=weak_sink_fraction, arith=arith,
                    jitter=jitter, jitter_seed=jitter_seed + p)
        if pathline:
            paths.append(out.pop("path"))
        if res is None:
            res = {k: np.array(v) for k, v in out.items() if not k.startswith("ts_")}
            if tarr is not None:
                for k in ("ts_x", "ts_y", "ts_z"):
                    res[k] = np.full((tarr.size, n), np.nan)
                res["ts_cell"] = np.full((tarr.size, n), -1, np.int32)
                res["ts_status"] = np.zeros((tarr.size, n), np.uint8)
        else:
            for k in res:
                if not k.startswith("ts_"):
                    res[k][moved] = out[k][moved]
        if wt is not None:
            for k in ("ts_x", "ts_y", "ts_z", "ts_cell", "ts_status"):
                res[k][window] = out[k]
        nxt = resume_state(out)
        for k in RESUME_KEYS:
            cur[k] = np.where(moved, nxt[k], cur[k])
        lo = hi
    if pathline:
        res["path"] = np.concatenate(paths)
    return res


def track_parallel(f, state, threads: int, chunk: int = 256, **kw):
    """The oracle as it stands, run on ``threads`` host threads.

    Particles are handed out in chunks from a shared counter (the "dynamic"
    schedule); each chunk is one call of the single-threaded oracle (ctypes
    releases the GIL during the call).  Results are identical to ``track``.
    """
    n = int(np.asarray(state["cell"]).size)
    of = as_oracle_field(f)
    parts = {}
    nxt = [0]
    lk = threading.Lock()

    def worker():
        while True:
            with lk:
                s = nxt[0]
                nxt[0] += chunk
            if s >= n:
                return
            idx = slice(s, min(n, s + chunk))
            ckw = dict(kw, jitter_id0=kw.get("jitter_id0", 0) + s) if kw.get("jitter") else kw
            parts[s] = track(of, {k: v[idx] for k, v in state.items()}, **ckw)

    ths = [threading.Thread(target=worker) for _ in range(max(1, threads))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    keys = sorted(parts)
    out = {}
    for name in parts[keys[0]]:
        ax = 1 if name.startswith("ts_") else 0
        out[name] = np.concatenate([parts[s][name] for s in keys], axis=ax)
    return out
