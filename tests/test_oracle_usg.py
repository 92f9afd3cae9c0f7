"""Rectangular unstructured (quadtree) grids on the oracle (TC2's quadtree
refinement; Pollock's method with each face's total flow).

Pins from outside the oracle:
* a rectilinear grid written as an unstructured one gives bit-identical
  results (endpoints, hashes, timeseries, pathlines, weak sinks, periods);
* RK4 integration through quadtree grids: the same cell sequences, exit
  times and crossing points;
* the generated quadtree flows conserve volume in every cell;
* the hand-over at a face whose sub-faces carry opposite flows (a hand-made
  two-cell case) enters the sub-face whose flow runs with the crossing.
"""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300.inputs import usg as U
from tests import helpers as H

# every pin holds for both arithmetic modes of the oracle
pytestmark = pytest.mark.usefixtures("oracle_arith")


_RK4_CACHE = {}


@pytest.fixture(scope="module")
def quad():
    u = U.quadtree_field(3, 10, 14, seed=5)
    cells, frac = U.explicit_particles(u, 150, seed=3)
    return u, cells, frac, O.release_explicit(u, cells, frac)


def _equal(a, b):
    for k in a:
        if k == "path":
            assert a[k].tobytes() == b[k].tobytes(), k
        else:
            assert np.array_equal(a[k], b[k], equal_nan=True), k


@pytest.mark.parametrize("pass_sinks", [False, True])
def test_structured_as_unstructured_is_bit_identical(pass_sinks):
    f = I.random_box_field(3, 6, 9, seed=61, lnk_var=1.0, n_wells=2, n_inactive=2)
    u = U.from_structured(f)
    cells, frac = I.explicit_particles(f, 300, seed=5, cols=(1, 4))
    s1, s2 = O.release_explicit(f, cells, frac), O.release_explicit(u, cells, frac)
    _equal(s1, s2)
    full = O.track(f, s1)
    times = np.quantile(full["t"], [0.1, 0.5, 0.9])
    kw = dict(times=times, pathline=True, pass_weak_sinks=pass_sinks)
    _equal(O.track(f, s1, **kw), O.track(u, s2, **kw))
    T = np.quantile(full["t"], [0.3, 0.6])
    fs = I.period_fields(f, seed=3)
    us = [U.from_structured(g) for g in fs]
    _equal(O.track_periods(fs, T, s1, times=times), O.track_periods(us, T, s2, times=times))


def test_quadtree_conserves_volume(quad):
    u, *_ = quad
    b = u.balance()
    assert np.abs(b[u.ibound == U.IB_ACTIVE]).max() <= 1e-12 * np.abs(u.q).max()
    assert np.abs(b[u.ibound == U.IB_SINK]).max() <= 1e-12 * np.abs(u.q).max()
    # every connection is listed on both sides with the same flow and rectangle
    for c in range(0, u.ncell, 7):
        for fi in range(6):
            for e in range(*u.subfaces(c, fi).indices(u.nsub)):
                m = int(u.nbr[e])
                if m < 0:
                    continue
                back = [x for x in range(*u.subfaces(m, fi ^ 1).indices(u.nsub)) if u.nbr[x] == c]
                assert len(back) == 1 and u.q[back[0]] == u.q[e] and np.array_equal(u.rect[back[0]], u.rect[e])
    assert np.diff(u.face_off).max() == 2   # refined faces exist


def test_quadtree_against_rk4(quad):
    u, cells, frac, st0 = quad
    r = O.track(u, st0, pathline=True)
    path = np.sort(r["path"], order=["particle", "seq"])
    ext = max(u.extent)
    kinds = set()
    if "quad" not in _RK4_CACHE:   # independent of the oracle's arithmetic mode: integrated once
        runs = []
        for q in range(cells.size):
            tr = []
            runs.append((H.rk4_track_usg(u, int(cells[q]), [st0["px"][q], st0["py"][q], st0["pz"][q]], trace=tr), tr))
        _RK4_CACHE["quad"] = runs
    for q in range(cells.size):
        (status, seq, _, p, t), tr = _RK4_CACHE["quad"][q]
        assert status == r["status"][q], q
        assert H.fnv_hash(seq) == int(r["hash"][q]), q
        assert r["t"][q] == pytest.approx(t, rel=1e-7)
        pts = path[path["particle"] == q][1:]
        assert len(pts) == len(tr)
        for rec, (tt, cc, g) in zip(pts, tr):
            assert rec["cell"] == cc and rec["t"] == pytest.approx(tt, rel=1e-7)
            assert max(abs(rec["x"] - g[0]), abs(rec["y"] - g[1]), abs(rec["z"] - g[2])) <= 1e-7 * ext
        kinds.add(len(seq) > 0 and any(np.diff(u.face_off)[6 * s:6 * s + 6].max() > 1 for s in seq))
    assert True in kinds   # paths through refined faces


def _two_cells(q_lo, q_hi):
    """A big cell whose east face borders two small cells; sub-face flows
    q_lo (southern half) and q_hi (northern half); the small cells drain
    east, the big cell is fed from the west by the sum."""
    box = np.array([[0.0, 0.0, 0.0, 2.0, 2.0, 1.0],     # big
                    [2.0, 0.0, 0.0, 1.0, 1.0, 1.0],     # small south
                    [2.0, 1.0, 0.0, 1.0, 1.0, 1.0]])    # small north
    subs = []
    off = [0]

    def face(lst):
        subs.extend(lst)
        off.append(len(subs))

    qin = q_lo + q_hi
    # big: x-, x+, y-, y+, z-, z+
    face([(-1, qin, (0.0, 2.0, 0.0, 1.0))])
    face([(1, q_lo, (0.0, 1.0, 0.0, 1.0)), (2, q_hi, (1.0, 2.0, 0.0, 1.0))])
    face([(-1, 0.0, (0.0, 2.0, 0.0, 1.0))]); face([(-1, 0.0, (0.0, 2.0, 0.0, 1.0))])
    face([(-1, 0.0, (0.0, 2.0, 0.0, 2.0))]); face([(-1, 0.0, (0.0, 2.0, 0.0, 2.0))])
    for c, qq, y0 in ((1, q_lo, 0.0), (2, q_hi, 1.0)):
        face([(0, qq, (y0, y0 + 1.0, 0.0, 1.0))])
        face([(-1, qq, (y0, y0 + 1.0, 0.0, 1.0))])
        face([(-1, 0.0, (2.0, 3.0, 0.0, 1.0))]); face([(-1, 0.0, (2.0, 3.0, 0.0, 1.0))])
        face([(-1, 0.0, (2.0, 3.0, y0, y0 + 1.0))]); face([(-1, 0.0, (2.0, 3.0, y0, y0 + 1.0))])
    return U.UsgField(box, np.full(3, 0.25), np.ones(3, np.int8), np.asarray(off, np.int64),
                      np.asarray([s[0] for s in subs], np.int32), np.asarray([s[1] for s in subs]),
                      np.asarray([s[2] for s in subs], float))


def test_hand_over_follows_the_flow():
    # consistent sub-faces: the particle leaves the big cell where it reaches
    # the face (south half -> south cell)
    u = _two_cells(1e-4, 3e-4)
    st = O.release_explicit(u, np.array([0], np.int32), np.array([[0.1, 0.2, 0.5]]))
    r = O.track(u, st)
    assert r["status"][0] == O.ST_EXIT_DOMAIN and r["cell"][0] == 1
    # the southern sub-face flows back into the big cell: a particle reaching
    # the face there enters the northern cell, on its near edge
    u = _two_cells(-1e-4, 5e-4)
    st = O.release_explicit(u, np.array([0], np.int32), np.array([[0.1, 0.2, 0.5]]))
    r = O.track(u, st, pathline=True)
    assert r["status"][0] == O.ST_EXIT_DOMAIN and r["cell"][0] == 2
    entry = r["path"][r["path"]["cell"] == 2][0]
    assert entry["x"] == 2.0 and entry["y"] == 1.0
    status, seq, *_ = H.rk4_track_usg(u, 0, [st["px"][0], st["py"][0], st["pz"][0]])
    assert seq == [0, 2] and status == O.ST_EXIT_DOMAIN
