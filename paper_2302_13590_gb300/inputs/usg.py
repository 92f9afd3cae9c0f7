"""Rectangular unstructured (quadtree) grids: the second grid shape of the
paper's TC2 ("grid refinement near relevant boundary conditions to also
consider an unstructured quadtree grid"; MODFLOW 6 DISV-like: the same plan
grid in every layer, base cells split 2 x 2).

Shared by the oracle and the CUDA path (like the rest of this package's
inputs it holds no tracking arithmetic): a cell is an axis-aligned box; each
of its six faces (x-, x+, y-, y+, z-, z+) carries a list of sub-faces, each
with the neighbour across it (-1: outside the domain), the volumetric flow
through it (m^3/s, positive along +axis) and its rectangle in the two other
axes (global coordinates, axes in x, y, z order).  Heads come from a
finite-volume solve over the cell connections (conductance = shared area /
sum of the two half-distances over K), solved directly, so every cell
conserves volume to rounding.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Optional, Tuple

import numpy as np

IB_INACTIVE, IB_ACTIVE, IB_CONST_HEAD, IB_SINK = 0, 1, -1, 2
OTHER = ((1, 2), (0, 2), (0, 1))   # the two other axes of a face normal to axis a


@dataclass
class UsgField:
    box: np.ndarray         # [ncell, 6]: x0, y0, z0, dx, dy, dz (m)
    porosity: np.ndarray    # [ncell]
    ibound: np.ndarray      # [ncell] int8
    face_off: np.ndarray    # [6 ncell + 1] int64: sub-faces of face f of cell c
    nbr: np.ndarray         # [nsub] int32, -1 outside
    q: np.ndarray           # [nsub] m^3/s along +axis
    rect: np.ndarray        # [nsub, 4]: lo_a, hi_a, lo_b, hi_b of the two other axes
    head: Optional[np.ndarray] = None
    q_src: Optional[np.ndarray] = None
    K: Optional[np.ndarray] = None
    name: str = ""

    @property
    def ncell(self) -> int:
        return int(self.box.shape[0])

    @property
    def nsub(self) -> int:
        return int(self.nbr.size)

    @property
    def extent(self) -> Tuple[float, float, float]:
        hi = self.box[:, :3] + self.box[:, 3:]
        return tuple(float(v) for v in hi.max(axis=0) - self.box[:, :3].min(axis=0))

    def subfaces(self, c: int, f: int) -> slice:
        return slice(int(self.face_off[6 * c + f]), int(self.face_off[6 * c + f + 1]))

    def face_flow(self) -> np.ndarray:
        """[ncell, 6] total flow of every face (sub-faces summed in list order)."""
        out = np.zeros((self.ncell, 6))
        for c in range(self.ncell):
            for f in range(6):
                s = 0.0
                for e in range(*self.subfaces(c, f).indices(self.nsub)):
                    s += float(self.q[e])
                out[c, f] = s
        return out

    def balance(self) -> np.ndarray:
        """Per-cell volume balance: outflow - inflow - sources (0 for a
        conserving active cell)."""
        ff = self.face_flow()
        net = ff[:, 1] - ff[:, 0] + ff[:, 3] - ff[:, 2] + ff[:, 5] - ff[:, 4]
        src = np.zeros(self.ncell) if self.q_src is None else self.q_src
        out = net - src
        out[self.ibound != IB_ACTIVE] = 0.0
        out[(self.ibound == IB_SINK)] = (net - src)[self.ibound == IB_SINK]
        return out


def from_structured(f) -> UsgField:
    """The same grid and flows in unstructured form: cells numbered
    (k nrow + i) ncol + j, one sub-face per face, origins from the same
    sequential face-coordinate sums the structured path uses."""
    nl, nr, nc = f.nlay, f.nrow, f.ncol

    def faces(d, o):
        out = np.empty(d.size + 1)
        out[0] = o
        for a in range(d.size):
            out[a + 1] = out[a] + d[a]
        return out

    xf, yf, zf = faces(np.asarray(f.delr, float), f.origin[0]), faces(np.asarray(f.delc, float), f.origin[1]), \
        faces(np.asarray(f.dz, float), f.origin[2])
    n = nl * nr * nc
    box = np.empty((n, 6))
    nbr, q, rect = [], [], []
    off = np.zeros(6 * n + 1, np.int64)
    e = 0
    for k in range(nl):
        for i in range(nr):
            for j in range(nc):
                c = (k * nr + i) * nc + j
                box[c] = (xf[j], yf[i], zf[k], f.delr[j], f.delc[i], f.dz[k])
                specs = [
                    ((k, i, j - 1) if j > 0 else None, f.qx[k, i, j], (yf[i], yf[i + 1], zf[k], zf[k + 1])),
                    ((k, i, j + 1) if j < nc - 1 else None, f.qx[k, i, j + 1], (yf[i], yf[i + 1], zf[k], zf[k + 1])),
                    ((k, i - 1, j) if i > 0 else None, f.qy[k, i, j], (xf[j], xf[j + 1], zf[k], zf[k + 1])),
                    ((k, i + 1, j) if i < nr - 1 else None, f.qy[k, i + 1, j], (xf[j], xf[j + 1], zf[k], zf[k + 1])),
                    ((k - 1, i, j) if k > 0 else None, f.qz[k, i, j], (xf[j], xf[j + 1], yf[i], yf[i + 1])),
                    ((k + 1, i, j) if k < nl - 1 else None, f.qz[k + 1, i, j], (xf[j], xf[j + 1], yf[i], yf[i + 1])),
                ]
                for fi, (nb, qq, rc) in enumerate(specs):
                    off[6 * c + fi] = e
                    nbr.append(-1 if nb is None else (nb[0] * nr + nb[1]) * nc + nb[2])
                    q.append(float(qq))
                    rect.append(rc)
                    e += 1
    off[6 * n] = e
    return UsgField(box, np.asarray(f.porosity, float).reshape(-1).copy(), np.asarray(f.ibound).reshape(-1).astype(
        np.int8), off, np.asarray(nbr, np.int32), np.asarray(q), np.asarray(rect, float),
        head=None if f.head is None else np.asarray(f.head).reshape(-1),
        q_src=None if f.q_src is None else np.asarray(f.q_src).reshape(-1), name=f"{f.name}.usg")


def quadtree_field(nlay: int, nrow: int, ncol: int, seed: int, lnk_var: float = 1.0, corr=(3.0, 3.0, 1.0),
                   dx=(2.0, 4.0), dy=(2.0, 4.0), dz=(0.5, 2.0), porosity=(0.2, 0.35), n_wells: int = 2,
                   well_rate: float = 0.02, refine_frac: float = 0.15, refine_around_wells: int = 1,
                   solver: str = "direct") -> UsgField:
    """A quadtree grid: a rectilinear base grid whose selected columns (in
    plan, all layers) are split 2 x 2; constant heads on the first and last
    base columns (unit mean gradient, unrefined), lognormal K per base cell
    (children inherit it), wells (sink cells) with the base columns around
    them refined.  Returns the flows of a volume-conserving head solve."""
    from .__init__ import gaussian_field   # the same K generator as the structured fields
    rng = np.random.default_rng(seed)
    delr = rng.uniform(*dx, size=ncol)
    delc = rng.uniform(*dy, size=nrow)
    dzv = rng.uniform(*dz, size=nlay)
    xf = np.concatenate([[0.0], np.cumsum(delr)])
    yf = np.concatenate([[0.0], np.cumsum(delc)])
    zf = np.concatenate([[0.0], np.cumsum(dzv)])
    if lnk_var > 0:
        Y = gaussian_field((nlay, nrow, ncol), (corr[2], corr[1], corr[0]), seed + 1)
        Kb = np.exp(math.log(1e-4) + math.sqrt(lnk_var) * Y)
    else:
        Kb = np.full((nlay, nrow, ncol), 1e-4)
    porb = rng.uniform(*porosity, size=(nlay, nrow, ncol))
    refined = np.zeros((nrow, ncol), bool)
    inner = [(i, j) for i in range(nrow) for j in range(2, ncol - 2)]
    for idx in rng.choice(len(inner), int(refine_frac * len(inner)), replace=False):
        refined[inner[idx]] = True
    wells = []
    for _ in range(n_wells):
        k, i, j = int(rng.integers(0, nlay)), int(rng.integers(1, nrow - 1)), int(rng.integers(3, ncol - 3))
        wells.append((k, i, j))
        for di in range(-refine_around_wells, refine_around_wells + 1):
            for dj in range(-refine_around_wells, refine_around_wells + 1):
                if 0 <= i + di < nrow and 2 <= j + dj < ncol - 2:
                    refined[i + di, j + dj] = True
    # cells: layer, row, column, then the 2 x 2 children row-major
    cid: Dict[tuple, int] = {}
    box, kk, por, ib = [], [], [], []
    for k in range(nlay):
        for i in range(nrow):
            for j in range(ncol):
                if refined[i, j]:
                    # child edges such that every low corner + size is
                    # exactly the next edge (the differences are exact by
                    # Sterbenz's lemma), so shared faces match bit for bit
                    xe = (xf[j], xf[j] + delr[j] / 2.0, xf[j + 1])
                    ye = (yf[i], yf[i] + delc[i] / 2.0, yf[i + 1])
                    for a in range(2):
                        for b in range(2):
                            cid[(k, i, j, a, b)] = len(box)
                            box.append((xe[b], ye[a], zf[k], xe[b + 1] - xe[b], ye[a + 1] - ye[a], dzv[k]))
                            kk.append(Kb[k, i, j]); por.append(porb[k, i, j]); ib.append(IB_ACTIVE)
                else:
                    cid[(k, i, j, -1, -1)] = len(box)
                    box.append((xf[j], yf[i], zf[k], delr[j], delc[i], dzv[k]))
                    kk.append(Kb[k, i, j]); por.append(porb[k, i, j])
                    ib.append(IB_CONST_HEAD if j in (0, ncol - 1) else IB_ACTIVE)
    box = np.asarray(box)
    n = len(box)
    K = np.asarray(kk)
    ibound = np.asarray(ib, np.int8)
    q_src = np.zeros(n)
    Lx = float(xf[-1])
    Ly, Lz = float(yf[-1]), float(zf[-1])
    for (k, i, j) in wells:
        keys = [(k, i, j, 0, 0)] if refined[i, j] else [(k, i, j, -1, -1)]
        c = cid[keys[0]]
        ibound[c] = IB_SINK
        q_src[c] = -well_rate * 1e-4 * Ly * Lz / max(n_wells, 1)

    def members(k, i, j):
        """Cells of base column (i, j) in layer k with their (a, b) child index."""
        if refined[i, j]:
            return [((a, b), cid[(k, i, j, a, b)]) for a in range(2) for b in range(2)]
        return [((-1, -1), cid[(k, i, j, -1, -1)])]

    # connections between cells that share a face: (c, n, axis) with c on the low side
    conn = []
    lo, hi = box[:, :3], box[:, :3] + box[:, 3:]

    def touching(c, m, ax):
        """Shared rectangle of c's high face and m's low face along ax, or None."""
        if hi[c, ax] != lo[m, ax]:
            return None
        a, b = OTHER[ax]
        ra = (max(lo[c, a], lo[m, a]), min(hi[c, a], hi[m, a]))
        rb = (max(lo[c, b], lo[m, b]), min(hi[c, b], hi[m, b]))
        if ra[1] <= ra[0] or rb[1] <= rb[0]:
            return None
        return (ra[0], ra[1], rb[0], rb[1])

    for k in range(nlay):
        for i in range(nrow):
            for j in range(ncol):
                here = members(k, i, j)
                # within a refined column
                for (_, c) in here:
                    for (_, m) in here:
                        for ax in (0, 1):
                            r = touching(c, m, ax)
                            if r is not None:
                                conn.append((c, m, ax, r))
                for ax, (dk, di, dj) in ((0, (0, 0, 1)), (1, (0, 1, 0)), (2, (1, 0, 0))):
                    k2, i2, j2 = k + dk, i + di, j + dj
                    if k2 >= nlay or i2 >= nrow or j2 >= ncol:
                        continue
                    for (_, c) in here:
                        for (_, m) in members(k2, i2, j2):
                            r = touching(c, m, ax)
                            if r is not None:
                                conn.append((c, m, ax, r))
    # heads: finite volumes over the connections
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    head = np.zeros(n)
    for c in range(n):
        if ibound[c] == IB_CONST_HEAD:
            head[c] = (10.0 + Lx) if box[c, 0] == 0.0 else 10.0
    cond = np.empty(len(conn))
    for e, (c, m, ax, r) in enumerate(conn):
        area = (r[1] - r[0]) * (r[3] - r[2])
        cond[e] = area / (0.5 * box[c, 3 + ax] / K[c] + 0.5 * box[m, 3 + ax] / K[m])
    free = ibound != IB_CONST_HEAD
    idx = -np.ones(n, np.int64)
    idx[free] = np.arange(int(free.sum()))
    rows, cols, vals = [], [], []
    rhs = np.zeros(int(free.sum()))
    diag = np.zeros(int(free.sum()))
    for e, (c, m, ax, r) in enumerate(conn):
        for a_, b_ in ((c, m), (m, c)):
            if not free[a_]:
                continue
            diag[idx[a_]] += cond[e]
            if free[b_]:
                rows.append(idx[a_]); cols.append(idx[b_]); vals.append(-cond[e])
            else:
                rhs[idx[a_]] += cond[e] * head[b_]
    rhs += q_src[free]
    A = sp.csr_matrix((np.concatenate([vals, diag]), (np.concatenate([rows, np.arange(diag.size)]),
                                                       np.concatenate([cols, np.arange(diag.size)]))),
                      shape=(diag.size, diag.size))
    if solver == "direct":
        head[free] = spla.spsolve(A.tocsc(), rhs)
    else:
        x, info = spla.cg(A, rhs, rtol=1e-14, maxiter=200000)
        head[free] = x
    # sub-face lists: per cell and face, the connections in the order of the
    # neighbours' low corners (other axes), the domain edge as one sub-face
    lists: List[List[List[tuple]]] = [[[] for _ in range(6)] for _ in range(n)]
    for e, (c, m, ax, r) in enumerate(conn):
        qq = cond[e] * (head[c] - head[m])          # along +ax, from c to m
        lists[c][2 * ax + 1].append((m, qq, r))
        lists[m][2 * ax].append((c, qq, r))
    off = np.zeros(6 * n + 1, np.int64)
    nbr, qv, rect = [], [], []
    for c in range(n):
        for fi in range(6):
            off[6 * c + fi] = len(nbr)
            subs = sorted(lists[c][fi], key=lambda t: (t[2][0], t[2][2]))
            if not subs:
                ax = fi // 2
                a, b = OTHER[ax]
                subs = [(-1, 0.0, (lo[c, a], hi[c, a], lo[c, b], hi[c, b]))]
            for (m, qq, r) in subs:
                nbr.append(m); qv.append(qq); rect.append(r)
    off[6 * n] = len(nbr)
    return UsgField(box, np.asarray(por), ibound, off, np.asarray(nbr, np.int32), np.asarray(qv),
                    np.asarray(rect, float), head=head, q_src=q_src, K=K,
                    name=f"quadtree{nlay}x{nrow}x{ncol}s{seed}")


def explicit_particles(u: UsgField, n: int, seed: int, x_range=(0.0, 0.2)):
    """n particles at seeded uniform fractions in active cells whose low x
    corner lies in the given fraction of the domain length."""
    rng = np.random.default_rng(seed)
    Lx = u.extent[0]
    cand = np.nonzero((u.ibound == IB_ACTIVE) & (u.box[:, 0] >= x_range[0] * Lx) &
                      (u.box[:, 0] < x_range[1] * Lx))[0]
    cells = cand[rng.integers(0, cand.size, n)].astype(np.int32)
    frac = rng.uniform(0.0, 1.0, (n, 3))
    return cells, frac
