"""Test helpers: hand-built fields and an independent brute-force integrator.

Nothing here is shared with the oracle or the CUDA path; the RK4 integrator
solves the same physical problem (piecewise-linear velocity, Pollock 1988)
by plain numerical integration, so it checks the oracle's analytic formulas
rather than repeating them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Tuple

import numpy as np


@dataclass
class SimpleField:
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


def uniform_x_field(nlay, nrow, ncol, seed, q_sign=1.0):
    """Flow only along x, the same Q through every face of a row: A = 0 in
    every cell, velocity Q / (n * area) changes from cell to cell through the
    porosity.  No constant-head cells: particles leave through the domain edge.
    """
    rng = np.random.default_rng(seed)
    delr = rng.uniform(0.5, 3.0, ncol)
    delc = rng.uniform(0.5, 3.0, nrow)
    dz = rng.uniform(0.2, 2.0, nlay)
    q_row = q_sign * rng.uniform(1e-5, 1e-3, (nlay, nrow))
    qx = np.repeat(q_row[:, :, None], ncol + 1, axis=2)
    qy = np.zeros((nlay, nrow + 1, ncol))
    qz = np.zeros((nlay + 1, nrow, ncol))
    por = rng.uniform(0.1, 0.4, (nlay, nrow, ncol))
    ib = np.ones((nlay, nrow, ncol), np.int8)
    return SimpleField(nlay, nrow, ncol, delr, delc, dz, (1.0, -2.0, 3.0), qx, qy, qz, por, ib)


def single_cell_field(qx1, qx2, qy1=0.0, qy2=0.0, qz1=0.0, qz2=0.0, d=(2.0, 3.0, 1.5), por=0.25):
    """One cell with prescribed face flows (mass balance is not required for
    the in-cell solution)."""
    qx = np.array([qx1, qx2], dtype=np.float64).reshape(1, 1, 2)
    qy = np.array([qy1, qy2], dtype=np.float64).reshape(1, 2, 1)
    qz = np.array([qz1, qz2], dtype=np.float64).reshape(2, 1, 1)
    return SimpleField(1, 1, 1, np.array([d[0]]), np.array([d[1]]), np.array([d[2]]), (0.0, 0.0, 0.0),
                       qx, qy, qz, np.full((1, 1, 1), por), np.ones((1, 1, 1), np.int8))


def mirror_x(f):
    """Mirror a field across x: columns reversed, x face flows reversed and negated."""
    return SimpleField(f.nlay, f.nrow, f.ncol, f.delr[::-1].copy(), f.delc.copy(), f.dz.copy(), f.origin,
                       -np.ascontiguousarray(f.qx[:, :, ::-1]), np.ascontiguousarray(f.qy[:, :, ::-1]),
                       np.ascontiguousarray(f.qz[:, :, ::-1]), np.ascontiguousarray(f.porosity[:, :, ::-1]),
                       np.ascontiguousarray(f.ibound[:, :, ::-1]))


def reversed_flow(f):
    return SimpleField(f.nlay, f.nrow, f.ncol, f.delr, f.delc, f.dz, f.origin, -f.qx, -f.qy, -f.qz,
                       f.porosity, f.ibound)


def fnv_hash(seq):
    h = 0xcbf29ce484222325
    for c in seq:
        h ^= int(c) & 0xFFFFFFFF
        h = (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


# ---------------------------------------------------------------------------
# brute force: RK4 in time with face events located by bisection
# ---------------------------------------------------------------------------

def _cell_lin(f, k, i, j):
    """Per-axis (v at low face, v at high face, size) from the flow definition v = Q/(n*area)."""
    n = float(f.porosity[k, i, j])
    dx, dy, dzz = float(f.delr[j]), float(f.delc[i]), float(f.dz[k])
    vx = (f.qx[k, i, j] / (n * dy * dzz), f.qx[k, i, j + 1] / (n * dy * dzz))
    vy = (f.qy[k, i, j] / (n * dx * dzz), f.qy[k, i + 1, j] / (n * dx * dzz))
    vz = (f.qz[k, i, j] / (n * dx * dy), f.qz[k + 1, i, j] / (n * dx * dy))
    return [(float(vx[0]), float(vx[1]), dx), (float(vy[0]), float(vy[1]), dy), (float(vz[0]), float(vz[1]), dzz)]


def _vel(lin, p):
    return [lo + (hi - lo) * (pa / d) for (lo, hi, d), pa in zip(lin, p)]


def _rk4(lin, p, h):
    k1 = _vel(lin, p)
    k2 = _vel(lin, [pa + 0.5 * h * ka for pa, ka in zip(p, k1)])
    k3 = _vel(lin, [pa + 0.5 * h * ka for pa, ka in zip(p, k2)])
    k4 = _vel(lin, [pa + h * ka for pa, ka in zip(p, k3)])
    return [pa + h / 6.0 * (a + 2 * b + 2 * c + d) for pa, a, b, c, d in zip(p, k1, k2, k3, k4)]


def rk4_track(f, k, i, j, p, t_stop=math.inf, max_cells=10_000, frac=2e-3, pass_sinks=False,
              capture_time=None, periods=None, t0=0.0, trace=None):
    """Integrate one particle; returns (status, cells visited, final (k,i,j), final p, t).

    Status codes follow the oracle's: 1 TIME, 2 SINK, 3 BOUNDARY, 4 EXIT_DOMAIN.
    pass_sinks: sink cells are entered; a particle that stays in a sink cell
    longer than capture_time without reaching a face counts as captured.
    periods: (fields, t_end) for piecewise-steady flow: fields[p] holds from
    t_end[p-1] to t_end[p]; at a period end the integration restarts in the
    same cell with the next field's velocities.  t0: the release time (the
    particle starts in the period that holds it).  trace: a list that
    receives (t, cell, global point) at every face crossing and at the end.
    """
    fields, t_end = ([f], []) if periods is None else (list(periods[0]), list(periods[1]))
    g0 = fields[0]
    xf = np.concatenate([[0.0], np.cumsum(g0.delr)]) + g0.origin[0]
    yf = np.concatenate([[0.0], np.cumsum(g0.delc)]) + g0.origin[1]
    zf = np.concatenate([[0.0], np.cumsum(g0.dz)]) + g0.origin[2]

    def mark(t, k, i, j, p):
        if trace is not None:
            trace.append((t, (k * g0.nrow + i) * g0.ncol + j, (xf[j] + p[0], yf[i] + p[1], zf[k] + p[2])))

    per = sum(1 for te in t_end if te <= t0)
    p = [float(x) for x in p]
    t = float(t0)
    if t >= t_stop:
        return 1, [(k * fields[0].nrow + i) * fields[0].ncol + j], (k, i, j), p, t
    seq = [(k * fields[0].nrow + i) * fields[0].ncol + j]
    for _ in range(max_cells):
        f = fields[per]
        t_next = t_end[per] if per < len(t_end) else math.inf
        lin = _cell_lin(f, k, i, j)
        vmax = max(max(abs(a), abs(b)) for a, b, _ in lin)
        if vmax == 0.0:
            return 5, seq, (k, i, j), p, t
        h = frac * min(d for _, _, d in lin) / vmax
        t_in = t
        while True:
            if pass_sinks and capture_time is not None and f.ibound[k, i, j] == 2 and t - t_in > capture_time:
                mark(t, k, i, j, p)
                return 2, seq, (k, i, j), p, t
            hh = min(h, t_next - t)
            if t + hh >= t_stop:
                hh = t_stop - t
            q = _rk4(lin, p, hh)
            out = [qa < 0.0 or qa > d for qa, (_, _, d) in zip(q, lin)]
            if not any(out):
                p, t = q, t + hh
                if t >= t_stop:
                    mark(t, k, i, j, p)
                    return 1, seq, (k, i, j), p, t
                if t >= t_next:
                    # the next flow period: same cell, new velocities
                    t = t_next
                    per += 1
                    mark(t, k, i, j, p)
                    ib = int(fields[per].ibound[k, i, j])
                    if ib in (0, -1):
                        return 3, seq, (k, i, j), p, t
                    if ib == 2 and not pass_sinks:
                        return 2, seq, (k, i, j), p, t
                    break
                continue
            # bisection for the first face crossing inside this RK4 step
            lo, hi = 0.0, hh
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                qm = _rk4(lin, p, mid)
                if any(qa < 0.0 or qa > d for qa, (_, _, d) in zip(qm, lin)):
                    hi = mid
                else:
                    lo = mid
            qh = _rk4(lin, p, hi)
            dist = []
            for a, (qa, (_, _, d)) in enumerate(zip(qh, lin)):
                dist.append(max(-qa, qa - d))
            ax = int(np.argmax(dist))
            side = 1 if qh[ax] > lin[ax][2] else -1
            p = _rk4(lin, p, hi)
            t = t + hi
            p = [min(max(pa, 0.0), d) for pa, (_, _, d) in zip(p, lin)]
            p[ax] = lin[ax][2] if side > 0 else 0.0
            nk, ni, nj = k, i, j
            if ax == 0:
                nj += side
            elif ax == 1:
                ni += side
            else:
                nk += side
            if not (0 <= nj < f.ncol and 0 <= ni < f.nrow and 0 <= nk < f.nlay):
                mark(t, k, i, j, p)
                return 4, seq, (k, i, j), p, t
            ib = int(f.ibound[nk, ni, nj])
            if ib in (0, -1):
                mark(t, k, i, j, p)
                return 3, seq, (k, i, j), p, t
            if ib == 2 and not pass_sinks:
                mark(t, k, i, j, p)
                return 2, seq, (k, i, j), p, t
            k, i, j = nk, ni, nj
            p[ax] = 0.0 if side > 0 else (f.delr[j], f.delc[i], f.dz[k])[ax]
            seq.append((k * f.nrow + i) * f.ncol + j)
            mark(t, k, i, j, p)
            break
    raise RuntimeError("rk4_track: too many cells")


# ---------------------------------------------------------------------------
# brute force on a rectangular unstructured grid (lumped face flows)
# ---------------------------------------------------------------------------

def _usg_lin(u, c):
    """Per-axis (v at low face, v at high face, size): each face's total flow
    over the cell's own face area and porosity."""
    b = u.box[c]
    n = float(u.porosity[c])
    area = (b[4] * b[5], b[3] * b[5], b[3] * b[4])
    out = []
    for a in range(3):
        ql = sum(float(v) for v in u.q[u.subfaces(c, 2 * a)])
        qh = sum(float(v) for v in u.q[u.subfaces(c, 2 * a + 1)])
        out.append((ql / (n * area[a]), qh / (n * area[a]), float(b[3 + a])))
    return out


def _usg_next(u, c, ax, side, g):
    """Neighbour across face (ax, side) at global point g: the sub-face that
    holds the point, or - when its flow runs against the crossing - the
    nearest one whose flow runs with it, the point moved onto it."""
    fi = 2 * ax + (1 if side > 0 else 0)
    sl = u.subfaces(c, fi)
    idx = list(range(*sl.indices(u.nsub)))
    if not idx:
        return -1, g
    oa, ob = [(1, 2), (0, 2), (0, 1)][ax]

    def dist(e):
        r = u.rect[e]
        return max(max(r[0] - g[oa], g[oa] - r[1]), max(r[2] - g[ob], g[ob] - r[3]), 0.0)

    best = min(idx, key=lambda e: (dist(e), idx.index(e)))
    inside = [e for e in idx if dist(e) == 0.0]
    if inside:
        best = inside[0]
    if u.q[best] * side > 0:
        return int(u.nbr[best]), g
    ok = [e for e in idx if u.q[e] * side > 0]
    alt = min(ok, key=lambda e: (dist(e), idx.index(e)))
    r = u.rect[alt]
    g = list(g)
    g[oa] = min(max(g[oa], r[0]), r[1])
    g[ob] = min(max(g[ob], r[2]), r[3])
    return int(u.nbr[alt]), g


def rk4_track_usg(u, c, p, t_stop=math.inf, max_cells=10_000, frac=2e-3, trace=None):
    """RK4 with bisection on face events through a rectangular unstructured
    grid; returns (status, cells visited, final cell, final local p, t)."""
    p = [float(x) for x in p]
    t = 0.0
    seq = [int(c)]
    for _ in range(max_cells):
        lin = _usg_lin(u, c)
        o = u.box[c, :3]
        vmax = max(max(abs(a), abs(b)) for a, b, _ in lin)
        if vmax == 0.0:
            return 5, seq, c, p, t
        h = frac * min(d for _, _, d in lin) / vmax
        while True:
            hh = h if t + h < t_stop else t_stop - t
            q = _rk4(lin, p, hh)
            if not any(qa < 0.0 or qa > d for qa, (_, _, d) in zip(q, lin)):
                p, t = q, t + hh
                if t >= t_stop:
                    return 1, seq, c, p, t
                continue
            lo, hi = 0.0, hh
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                if any(qa < 0.0 or qa > d for qa, (_, _, d) in zip(_rk4(lin, p, mid), lin)):
                    hi = mid
                else:
                    lo = mid
            qh = _rk4(lin, p, hi)
            ax = int(np.argmax([max(-qa, qa - d) for qa, (_, _, d) in zip(qh, lin)]))
            side = 1 if qh[ax] > lin[ax][2] else -1
            t = t + hi
            p = [min(max(pa, 0.0), d) for pa, (_, _, d) in zip(qh, lin)]
            p[ax] = lin[ax][2] if side > 0 else 0.0
            g = [o[a] + p[a] for a in range(3)]
            nc, g = _usg_next(u, c, ax, side, g)
            if nc < 0:
                if trace is not None:
                    trace.append((t, c, g))
                return 4, seq, c, p, t
            ib = int(u.ibound[nc])
            if ib in (0, -1, 2):
                if trace is not None:
                    trace.append((t, c, g))
                return (3 if ib != 2 else 2), seq, c, p, t
            on, dn = u.box[nc, :3], u.box[nc, 3:]
            p = [min(max(g[a] - on[a], 0.0), dn[a]) for a in range(3)]
            p[ax] = 0.0 if side > 0 else float(dn[ax])
            c = nc
            seq.append(int(c))
            if trace is not None:
                trace.append((t, c, [on[a] + p[a] for a in range(3)]))
            break
    raise RuntimeError("rk4_track_usg: too many cells")
