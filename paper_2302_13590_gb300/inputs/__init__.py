"""Seeded synthetic inputs: MODFLOW-style steady flow fields and particle releases.

This module holds input generation only (lognormal conductivity, head solve,
face flows, release boxes).  None of the particle-tracking arithmetic lives
here, so the CUDA path and the CPU oracle can both take their inputs from it.

The paper's test cases (TC1: a 2-D 1500 x 300 lognormal aquifer with an
exponential variogram, unit mean gradient, particles released near the inlet;
Section "Synthetic test cases", Table 1) are described but their realisations
are not published; the workloads below are synthetic stand-ins of the same
kind:

* ``cfg1`` 50x50x1 cells of 10 m, homogeneous K = 1e-4 m/s, porosity 0.3,
  constant heads 10 m (column 0) / 0 m (column 49), a 1e-3 m^3/s pumping well
  (strong sink) at layer 0, row 25, column 25; 1,000 particles uniform in
  columns 1-5.
* ``cfg2`` 200x200x20 cells of 5x5x1 m, ln K ~ N(-9.2, 1) with exponential
  covariance, correlation lengths (10, 10, 2) cells; porosity 0.3; constant
  heads on the west and east columns with unit mean gradient; 1e6 particles
  uniform on the west face of column 1; 50 log-spaced output times.
* ``cfg3`` 400x400x40 cells of 5x5x1 m, ln K variance 4, correlation length
  8 cells, porosity U(0.2, 0.35) per cell, 20 seeded wells; 1e7 particles on a
  seeded plane; 100 output times.

Seeds: field = 0x2302135900 + config number, particles = field seed + 1.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field as dc_field
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fieldgen.c")
_LIB = os.path.join(_HERE, "libfieldgen.so")
_lib = None

SEED_BASE = 0x2302135900

IB_INACTIVE = 0
IB_ACTIVE = 1
IB_CONST_HEAD = -1
IB_SINK = 2


def build_fieldgen(force: bool = False) -> str:
    """Compile fieldgen.c into an in-tree shared library (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_fieldgen())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.fg_solve.restype = ctypes.c_int
        lib.fg_solve.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 7 + [ctypes.c_double, ctypes.c_int] + [ctypes.c_void_p] * 5
        lib.fg_solve_mg.restype = ctypes.c_int
        lib.fg_solve_mg.argtypes = lib.fg_solve.argtypes
        lib.fg_balance.restype = ctypes.c_double
        lib.fg_balance.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 6
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Field:
    """A steady structured flow field (MODFLOW DIS layout).

    Axes: x along column j, y along row i, z along layer k (z grows with k).
    ``qx[k, i, j]`` is the flow (m^3/s) through the west face of column j in
    the +x direction (j = 0..ncol); ``qy`` and ``qz`` likewise.
    """
    nlay: int
    nrow: int
    ncol: int
    delr: np.ndarray
    delc: np.ndarray
    dz: np.ndarray
    origin: Tuple[float, float, float]
    qx: np.ndarray
    qy: np.ndarray
    qz: np.ndarray
    porosity: np.ndarray
    ibound: np.ndarray
    head: Optional[np.ndarray] = None
    K: Optional[np.ndarray] = None
    q_src: Optional[np.ndarray] = None
    solve_iters: int = 0
    solve_maxres: float = 0.0
    name: str = ""

    @property
    def ncell(self) -> int:
        return self.nlay * self.nrow * self.ncol

    @property
    def extent(self) -> Tuple[float, float, float]:
        return (float(self.delr.sum()), float(self.delc.sum()), float(self.dz.sum()))

    def face_x(self, j: int) -> float:
        """x coordinate of the west face of column j (sequential sum)."""
        x = self.origin[0]
        for jj in range(j):
            x += float(self.delr[jj])
        return x

    def balance(self) -> np.ndarray:
        lib = _load()
        out = np.zeros(self.ncell, dtype=np.float64)
        q = None if self.q_src is None else np.ascontiguousarray(self.q_src, dtype=np.float64)
        lib.fg_balance(self.nlay, self.nrow, self.ncol, _p(self.qx), _p(self.qy), _p(self.qz),
                       _p(self.ibound), _p(q), _p(out))
        return out.reshape(self.nlay, self.nrow, self.ncol)


def solve_flow(nlay, nrow, ncol, delr, delc, dz, K, ibound, head_bc, q_src=None,
               tol_abs=1e-13, max_iter=20000, method="mg"):
    """Finite-volume head solve in C: conjugate gradients preconditioned by a
    multigrid V-cycle ("mg", default) or by IC(0) ("ic"); returns
    (head, qx, qy, qz, iters, maxres)."""
    lib = _load()
    delr = np.ascontiguousarray(delr, dtype=np.float64)
    delc = np.ascontiguousarray(delc, dtype=np.float64)
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64).reshape(-1)
    ib = np.ascontiguousarray(ibound, dtype=np.int8).reshape(-1)
    head = np.ascontiguousarray(head_bc, dtype=np.float64).reshape(-1).copy()
    q = None if q_src is None else np.ascontiguousarray(q_src, dtype=np.float64).reshape(-1)
    qx = np.zeros((nlay, nrow, ncol + 1))
    qy = np.zeros((nlay, nrow + 1, ncol))
    qz = np.zeros((nlay + 1, nrow, ncol))
    maxres = ctypes.c_double(0.0)
    iters = ctypes.c_int(0)
    fn = lib.fg_solve_mg if method == "mg" else lib.fg_solve
    rc = fn(nlay, nrow, ncol, _p(delr), _p(delc), _p(dz), _p(K), _p(ib), _p(q), _p(head),
                      float(tol_abs), int(max_iter), _p(qx), _p(qy), _p(qz),
                      ctypes.byref(maxres), ctypes.byref(iters))
    if rc not in (0, -3):
        raise RuntimeError(f"fg_solve failed with code {rc}")
    return head.reshape(nlay, nrow, ncol), qx, qy, qz, iters.value, maxres.value


def _fast_len(n: int) -> int:
    """Smallest length >= n whose prime factors are 2 and 5 (fast FFT sizes)."""
    m = max(1, n)
    while True:
        r = m
        for p in (2, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def gaussian_field(shape: Sequence[int], corr_cells: Sequence[float], seed: int,
                   pad_factor: float = 4.0) -> np.ndarray:
    """Zero-mean, unit-variance stationary Gaussian field with exponential covariance.

    C(r) = exp(-|r / lambda|) (anisotropic lengths in cells, axis order of
    ``shape``), generated by circulant embedding on a periodic grid padded by
    at least ``pad_factor`` correlation lengths per axis; negative circulant
    eigenvalues (if any) are clipped to zero.
    """
    shape = tuple(int(s) for s in shape)
    lam = tuple(float(l) for l in corr_cells)
    pshape = tuple(_fast_len(s + int(math.ceil(pad_factor * l))) for s, l in zip(shape, lam))
    grids = []
    for ax, (m, l) in enumerate(zip(pshape, lam)):
        d = np.arange(m, dtype=np.float64)
        d = np.minimum(d, m - d) / l
        sh = [1] * len(pshape)
        sh[ax] = m
        grids.append((d ** 2).reshape(sh))
    r2 = grids[0]
    for g in grids[1:]:
        r2 = r2 + g
    cov = np.exp(-np.sqrt(r2))
    eig = np.fft.fftn(cov).real
    eig = np.clip(eig, 0.0, None)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(pshape)
    y = np.fft.ifftn(np.sqrt(eig) * np.fft.fftn(w)).real
    return np.ascontiguousarray(y[tuple(slice(0, s) for s in shape)])


def make_field(nlay, nrow, ncol, dx, dy, dz, *, lnk_mean=math.log(1e-4), lnk_var=0.0,
               corr_cells=(10.0, 10.0, 10.0), porosity=0.3, h_west=None, h_east=None,
               wells: Sequence[Tuple[int, int, int, float]] = (), seed=0, origin=(0.0, 0.0, 0.0),
               tol_abs=None, max_iter=20000, name="") -> Field:
    """Generate a field: conductivity, head solve with CH west/east columns, wells.

    ``corr_cells`` = correlation lengths (x, y, z) in cells.  ``porosity`` is a
    scalar or a (lo, hi) pair drawn iid per cell.  ``wells`` = (k, i, j, q) with
    q < 0 for extraction; well cells get ibound = 2 (strong sink).
    """
    rng_seed = int(seed)
    delr = np.full(ncol, float(dx))
    delc = np.full(nrow, float(dy))
    dzv = np.full(nlay, float(dz))
    if lnk_var > 0.0:
        y = gaussian_field((nlay, nrow, ncol), (corr_cells[2], corr_cells[1], corr_cells[0]), rng_seed)
        lnk = lnk_mean + math.sqrt(lnk_var) * y
    else:
        lnk = np.full((nlay, nrow, ncol), float(lnk_mean))
    K = np.exp(lnk)
    if isinstance(porosity, (tuple, list)):
        prng = np.random.default_rng(rng_seed + 7)
        por = prng.uniform(porosity[0], porosity[1], size=(nlay, nrow, ncol))
    else:
        por = np.full((nlay, nrow, ncol), float(porosity))
    ib = np.full((nlay, nrow, ncol), IB_ACTIVE, dtype=np.int8)
    head = np.zeros((nlay, nrow, ncol))
    Lx = float(delr.sum())
    if h_west is None:
        h_west = Lx + 10.0
    if h_east is None:
        h_east = 10.0
    ib[:, :, 0] = IB_CONST_HEAD
    ib[:, :, -1] = IB_CONST_HEAD
    head[:, :, 0] = h_west
    head[:, :, -1] = h_east
    q_src = np.zeros((nlay, nrow, ncol))
    for (k, i, j, q) in wells:
        ib[k, i, j] = IB_SINK
        q_src[k, i, j] += q
    if tol_abs is None:
        # flows scale with K * face area * gradient; ask for ~1e-9 of that per
        # cell, relative to the geometric-mean K (the solver also stops at its
        # rounding floor, which grows with the conductance contrast)
        qscale = float(np.exp(lnk_mean)) * dy * dz * abs(h_west - h_east) / max(Lx, 1e-30)
        tol_abs = min(1e-12, qscale * 1e-9)
    h, qx, qy, qz, iters, maxres = solve_flow(nlay, nrow, ncol, delr, delc, dzv, K, ib, head, q_src,
                                              tol_abs=tol_abs, max_iter=max_iter)
    return Field(nlay, nrow, ncol, delr, delc, dzv, tuple(float(o) for o in origin), qx, qy, qz,
                 np.ascontiguousarray(por), np.ascontiguousarray(ib), head=h, K=K, q_src=q_src,
                 solve_iters=iters, solve_maxres=maxres, name=name)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclass
class Release:
    """A generated release: n particles uniform in the box [lo, hi] (global m).

    A plane is a box with lo == hi on one axis.  ``seed`` keys the
    counter-based generator that both implementations evaluate independently;
    particle p uses counter p + ``id_offset``.
    """
    n: int
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    seed: int
    id_offset: int = 0


@dataclass
class Workload:
    name: str
    field: Field
    release: Release
    times: np.ndarray
    t_adv: float
    mixed: bool = False
    meta: dict = dc_field(default_factory=dict)


def log_times(t_adv: float, n: int) -> np.ndarray:
    """n log-spaced output times over [t_adv/100, 10 t_adv]."""
    return np.logspace(math.log10(t_adv / 100.0), math.log10(10.0 * t_adv), n)


_cache = {}


def cfg1_field() -> Field:
    if "cfg1" not in _cache:
        _cache["cfg1"] = make_field(1, 50, 50, 10.0, 10.0, 10.0, lnk_mean=math.log(1e-4), lnk_var=0.0,
                                    porosity=0.3, h_west=10.0, h_east=0.0,
                                    wells=[(0, 25, 25, -1e-3)], seed=SEED_BASE + 1, name="cfg1")
    return _cache["cfg1"]


def cfg2_field() -> Field:
    if "cfg2" not in _cache:
        _cache["cfg2"] = make_field(20, 200, 200, 5.0, 5.0, 1.0, lnk_mean=-9.2, lnk_var=1.0,
                                    corr_cells=(10.0, 10.0, 2.0), porosity=0.3,
                                    seed=SEED_BASE + 2, name="cfg2")
    return _cache["cfg2"]


def cfg3_field() -> Field:
    if "cfg3" not in _cache:
        seed = SEED_BASE + 3
        nlay, nrow, ncol = 40, 400, 400
        rng = np.random.default_rng(seed + 11)
        kg = math.exp(-9.2)
        q_w = -0.01 * kg * 1.0 * (nrow * 5.0) * (nlay * 1.0)
        wells = []
        used = set()
        while len(wells) < 20:
            k = int(rng.integers(0, nlay)); i = int(rng.integers(0, nrow)); j = int(rng.integers(2, ncol - 2))
            if (k, i, j) in used:
                continue
            used.add((k, i, j))
            wells.append((k, i, j, q_w))
        _cache["cfg3"] = make_field(nlay, nrow, ncol, 5.0, 5.0, 1.0, lnk_mean=-9.2, lnk_var=4.0,
                                    corr_cells=(8.0, 8.0, 8.0), porosity=(0.2, 0.35), wells=wells,
                                    seed=seed, name="cfg3")
    return _cache["cfg3"]


def t_adv_of(f: Field, kg: float, por: float) -> float:
    """Mean advective crossing time L_x n / (K_G J) for unit gradient."""
    return float(f.delr.sum()) * por / (kg * 1.0)


def workload(name: str, n_particles: Optional[int] = None) -> Workload:
    """Named workload with its field, release and output times."""
    if name == "cfg1":
        f = cfg1_field()
        x1, x6 = f.face_x(1), f.face_x(6)
        Lx, Ly, Lz = f.extent
        n = 1000 if n_particles is None else n_particles
        rel = Release(n, (x1, 0.0, 0.0), (x6, Ly, Lz), SEED_BASE + 1 + 1)
        ta = t_adv_of(f, 1e-4, 0.3)
        return Workload(name, f, rel, log_times(ta, 50), ta)
    if name == "cfg2":
        f = cfg2_field()
        x1 = f.face_x(1)
        Lx, Ly, Lz = f.extent
        n = 1_000_000 if n_particles is None else n_particles
        rel = Release(n, (x1, 0.0, 0.0), (x1, Ly, Lz), SEED_BASE + 2 + 1)
        ta = t_adv_of(f, math.exp(-9.2), 0.3)
        return Workload(name, f, rel, log_times(ta, 50), ta)
    if name == "cfg3":
        f = cfg3_field()
        rng = np.random.default_rng(SEED_BASE + 3 + 1)
        col = int(rng.integers(1, 41))
        x0 = f.face_x(col)
        Lx, Ly, Lz = f.extent
        n = 10_000_000 if n_particles is None else n_particles
        rel = Release(n, (x0, 0.0, 0.0), (x0, Ly, Lz), SEED_BASE + 3 + 1)
        ta = t_adv_of(f, math.exp(-9.2), 0.275)
        return Workload(name, f, rel, log_times(ta, 100), ta, mixed=True, meta={"release_col": col})
    raise ValueError(f"unknown workload {name}")


def random_box_field(nlay, nrow, ncol, seed, lnk_var=1.0, corr=(2.0, 2.0, 1.0), dx=(1.0, 3.0),
                     dy=(1.0, 3.0), dz=(0.5, 2.0), porosity=(0.2, 0.4), n_wells=0,
                     n_inactive=0, well_scale=1.0) -> Field:
    """Small random test field with irregular rectilinear spacing.

    Cell sizes are drawn per column/row/layer, porosity per cell, optional
    wells and inactive cells; the head solve makes the flows mass-conserving.
    well_scale multiplies the well rates: a large one makes wells strong
    (every face flows in), a small one weak (flow passes through).
    """
    rng = np.random.default_rng(seed)
    delr = rng.uniform(*dx, size=ncol)
    delc = rng.uniform(*dy, size=nrow)
    dzv = rng.uniform(*dz, size=nlay)
    if lnk_var > 0:
        y = gaussian_field((nlay, nrow, ncol), (corr[2], corr[1], corr[0]), seed + 1)
        K = np.exp(math.log(1e-4) + math.sqrt(lnk_var) * y)
    else:
        K = np.full((nlay, nrow, ncol), 1e-4)
    por = rng.uniform(porosity[0], porosity[1], size=(nlay, nrow, ncol))
    ib = np.full((nlay, nrow, ncol), IB_ACTIVE, dtype=np.int8)
    ib[:, :, 0] = IB_CONST_HEAD
    ib[:, :, -1] = IB_CONST_HEAD
    head = np.zeros((nlay, nrow, ncol))
    head[:, :, 0] = 10.0 + float(delr.sum())
    head[:, :, -1] = 10.0
    q_src = np.zeros((nlay, nrow, ncol))
    for _ in range(n_wells):
        k, i, j = int(rng.integers(0, nlay)), int(rng.integers(0, nrow)), int(rng.integers(1, ncol - 1))
        ib[k, i, j] = IB_SINK
        q_src[k, i, j] = -well_scale * float(rng.uniform(0.02, 0.1)) * 1e-4 * float(delc.sum() * dzv.sum()) / max(nrow * nlay, 1)
    for _ in range(n_inactive):
        k, i, j = int(rng.integers(0, nlay)), int(rng.integers(0, nrow)), int(rng.integers(1, ncol - 1))
        if ib[k, i, j] == IB_ACTIVE:
            ib[k, i, j] = IB_INACTIVE
            q_src[k, i, j] = 0.0
    h, qx, qy, qz, iters, maxres = solve_flow(nlay, nrow, ncol, delr, delc, dzv, K, ib, head, q_src,
                                              tol_abs=1e-17)
    return Field(nlay, nrow, ncol, delr, delc, dzv, (0.0, 0.0, 0.0), qx, qy, qz, por, ib,
                 head=h, K=K, q_src=q_src, solve_iters=iters, solve_maxres=maxres,
                 name=f"random{nlay}x{nrow}x{ncol}s{seed}")


def period_fields(f: Field, seed: int, head_scale=(1.0, 0.5, -0.6), new_wells=(0, 2, 0),
                  well_scale: float = 1.0, tol_abs: float = 1e-17) -> List[Field]:
    """Stress periods of a piecewise-steady flow on the grid of f.

    Period p keeps f's cells, K and porosity; the constant-head contrast is
    scaled by head_scale[p] (a negative scale reverses the mean gradient) and
    new_wells[p] more sink cells are switched on (seeded); each period's face
    flows come from its own head solve, so every period conserves volume.
    A scale of 1 with no new wells reproduces f's flows.
    """
    if f.K is None or f.head is None:
        raise ValueError("period_fields: the field needs its K and heads")
    rng = np.random.default_rng(seed)
    ch = f.ibound == IB_CONST_HEAD
    h_lo = float(f.head[ch].min())
    ib = f.ibound.copy()
    q_src = np.zeros(f.ibound.shape) if f.q_src is None else f.q_src.copy()
    tot = abs(float(f.qx[:, :, 1].sum()))  # through-flow out of the west constant-head column
    out = []
    for p, (sc, nw) in enumerate(zip(head_scale, new_wells)):
        ib = ib.copy()
        q_src = q_src.copy()
        for _ in range(nw):
            act = np.argwhere(ib == IB_ACTIVE)
            k, i, j = (int(v) for v in act[int(rng.integers(0, len(act)))])
            ib[k, i, j] = IB_SINK
            q_src[k, i, j] = -well_scale * float(rng.uniform(0.005, 0.02)) * max(tot, 1e-12)
        head = f.head.copy()
        head[ch] = h_lo + sc * (f.head[ch] - h_lo)
        if sc == 1.0 and nw == 0 and p == 0:
            out.append(f)
            continue
        h, qx, qy, qz, iters, maxres = solve_flow(f.nlay, f.nrow, f.ncol, f.delr, f.delc, f.dz, f.K, ib, head,
                                                  q_src, tol_abs=tol_abs)
        out.append(Field(f.nlay, f.nrow, f.ncol, f.delr, f.delc, f.dz, f.origin, qx, qy, qz, f.porosity, ib.copy(),
                         head=h, K=f.K, q_src=q_src.copy(), solve_iters=iters, solve_maxres=maxres,
                         name=f"{f.name}.period{p}"))
    return out


def staged_release(f: Field, cells, n_per_stage: int, n_stages: int, interval: float, seed: int,
                   face_z: float = 0.0):
    """Staged injection (TC2: particles released from the upper face of a
    few cells, injected in stages at a fixed interval): n_per_stage particles
    per cell and stage, uniform over the cell's face z = face_z (a fraction of
    the cell height), stage s released at t0 = s * interval.  Returns (cell,
    local fractions [n, 3], t0), stage-major."""
    rng = np.random.default_rng(seed)
    cells = np.asarray(cells, dtype=np.int32)
    n = len(cells) * n_per_stage * n_stages
    cell = np.tile(np.repeat(cells, n_per_stage), n_stages).astype(np.int32)
    frac = np.empty((n, 3))
    frac[:, 0] = rng.uniform(0.0, 1.0, n)
    frac[:, 1] = rng.uniform(0.0, 1.0, n)
    frac[:, 2] = face_z
    t0 = np.repeat(np.arange(n_stages, dtype=np.float64) * interval, len(cells) * n_per_stage)
    return cell, frac, t0


def explicit_particles(f: Field, n: int, seed: int, cols: Optional[Tuple[int, int]] = None,
                       active_only: bool = True):
    """n particles as (cell index int32, local fractions float64 [n,3]) in active cells.

    ``cols`` = (first, last+1) column range.  Fractions are uniform in [0, 1).
    """
    rng = np.random.default_rng(seed)
    j0, j1 = (0, f.ncol) if cols is None else cols
    ib = f.ibound.reshape(-1)
    cells = []
    while len(cells) < n:
        k = rng.integers(0, f.nlay, size=2 * n)
        i = rng.integers(0, f.nrow, size=2 * n)
        j = rng.integers(j0, j1, size=2 * n)
        c = (k * f.nrow + i) * f.ncol + j
        if active_only:
            c = c[ib[c] == IB_ACTIVE]
        cells.extend(c.tolist())
    cells = np.asarray(cells[:n], dtype=np.int32)
    frac = rng.random((n, 3))
    return cells, frac


# ---------------------------------------------------------------------------
# Many-request workloads (batched launches and serving)
# ---------------------------------------------------------------------------

@dataclass
class RequestSpec:
    """One tracking request: a box release on a field, a mode and its times."""
    field_name: str
    release: Release
    timeseries: bool
    times: Optional[np.ndarray]
    arrival_s: float = 0.0


def _box_in(f: Field, rng, edge_lo=0.05, edge_hi=0.5):
    """Random axis-aligned box inside the active columns (1 .. ncol-2)."""
    x0, x1 = f.face_x(1), f.face_x(f.ncol - 1)
    Ly, Lz = float(f.delc.sum()), float(f.dz.sum())
    ext = [x1 - x0, Ly, Lz]
    org = [x0, f.origin[1], f.origin[2]]
    lo, hi = [], []
    for a in range(3):
        e = rng.uniform(edge_lo, edge_hi) * ext[a]
        s = org[a] + rng.uniform(0.0, ext[a] - e)
        lo.append(s)
        hi.append(s + e)
    return tuple(lo), tuple(hi)


def batch_workload(n_req: int = 256, seed: int = SEED_BASE + 4, n_min=1e2, n_max=1e6, n_times=20):
    """Independent requests on the 200x200x20 field: particle counts
    log-uniform in [n_min, n_max], random boxes (edge fraction U(0.05, 0.5)),
    half endpoint-only and half with timeseries at n_times log-spaced times."""
    f = cfg2_field()
    rng = np.random.default_rng(seed)
    ta = t_adv_of(f, math.exp(-9.2), 0.3)
    times = log_times(ta, n_times)
    specs = []
    for r in range(n_req):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        lo, hi = _box_in(f, rng)
        rel = Release(n, lo, hi, seed=int(rng.integers(1, 2**62)), id_offset=0)
        ts = (r % 2) == 1
        specs.append(RequestSpec("cfg2", rel, ts, times if ts else None))
    return specs


def serving_workload(n_req: int = 5000, rate_hz: float = 200.0, seed: int = SEED_BASE + 5, n_min=1e3, n_max=1e6,
                     n_times=20):
    """Poisson arrivals at rate_hz against the 50x50x1 and 200x200x20 fields
    (each with probability 1/2), group sizes log-uniform in [n_min, n_max],
    endpoint or timeseries (n_times log-spaced times) at random."""
    rng = np.random.default_rng(seed)
    t = 0.0
    specs = []
    for _ in range(n_req):
        t += rng.exponential(1.0 / rate_hz)
        name = "cfg1" if rng.random() < 0.5 else "cfg2"
        f = cfg1_field() if name == "cfg1" else cfg2_field()
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        lo, hi = _box_in(f, rng)
        ts = bool(rng.random() < 0.5)
        kg, por = (1e-4, 0.3) if name == "cfg1" else (math.exp(-9.2), 0.3)
        times = log_times(t_adv_of(f, kg, por), n_times) if ts else None
        specs.append(RequestSpec(name, Release(n, lo, hi, seed=int(rng.integers(1, 2**62))), ts, times, t))
    return specs
