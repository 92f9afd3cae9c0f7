"""Pathlines on the oracle (Methods, "MODPATH": pathline simulations record
each particle's path): a start point and the point every cell-step ends at.

Pins: brute-force RK4 integration gives the same face-crossing points and
times (steady flow and through flow periods); the points of a particle
reproduce its endpoint bit for bit, its step count and its cell-sequence
hash; consecutive points share a face of their cells.
"""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from tests import helpers as H

# every pin holds for both arithmetic modes of the oracle
pytestmark = pytest.mark.usefixtures("oracle_arith")


@pytest.fixture(scope="module")
def base():
    f = I.random_box_field(3, 6, 9, seed=61, lnk_var=1.0, n_wells=2, n_inactive=2)
    cells, frac = I.explicit_particles(f, 80, seed=5, cols=(1, 4))
    st0 = O.release_explicit(f, cells, frac)
    return f, cells, frac, st0


def _by_particle(path, n):
    order = np.lexsort((path["seq"], path["particle"]))
    path = path[order]
    starts = np.searchsorted(path["particle"], np.arange(n + 1))
    return [path[starts[q]:starts[q + 1]] for q in range(n)]


def _kij(f, c):
    return c // (f.ncol * f.nrow), (c // f.ncol) % f.nrow, c % f.ncol


def test_pathline_points_match_rk4(base):
    f, cells, frac, st0 = base
    r = O.track(f, st0, pathline=True)
    lines = _by_particle(r["path"], cells.size)
    ext = max(f.delr.sum(), f.delc.sum(), f.dz.sum())
    for q in range(cells.size):
        k, i, j = _kij(f, int(cells[q]))
        tr = []
        H.rk4_track(f, k, i, j, [st0["px"][q], st0["py"][q], st0["pz"][q]], trace=tr)
        pts = lines[q][1:]
        assert len(pts) == len(tr), q
        for rec, (t, c, g) in zip(pts, tr):
            assert rec["cell"] == c
            assert rec["t"] == pytest.approx(t, rel=1e-7)
            assert max(abs(rec["x"] - g[0]), abs(rec["y"] - g[1]), abs(rec["z"] - g[2])) <= 1e-7 * ext


def test_pathline_points_match_rk4_through_periods(base):
    f, cells, frac, st0 = base
    full = O.track(f, st0)
    fs = I.period_fields(f, seed=3, head_scale=(1.0, 0.5, -0.6), new_wells=(0, 1, 0))
    T = np.quantile(full["t"], [0.3, 0.6])
    r = O.track_periods(fs, T, st0, pathline=True)
    lines = _by_particle(r["path"], cells.size)
    ext = max(f.delr.sum(), f.delc.sum(), f.dz.sum())
    for q in range(0, cells.size, 2):
        k, i, j = _kij(f, int(cells[q]))
        tr = []
        H.rk4_track(f, k, i, j, [st0["px"][q], st0["py"][q], st0["pz"][q]], periods=(fs, T), trace=tr)
        pts = lines[q][1:]
        assert len(pts) == len(tr), q
        for rec, (t, c, g) in zip(pts, tr):
            assert rec["cell"] == c
            assert rec["t"] == pytest.approx(t, rel=1e-7)
            assert max(abs(rec["x"] - g[0]), abs(rec["y"] - g[1]), abs(rec["z"] - g[2])) <= 1e-7 * ext


@pytest.mark.parametrize("t_frac,max_steps", [(None, 0), (0.5, 0), (None, 4)])
def test_pathline_agrees_with_endpoint(base, t_frac, max_steps):
    f, cells, frac, st0 = base
    full = O.track(f, st0)
    t_stop = np.inf if t_frac is None else float(np.quantile(full["t"], t_frac))
    r = O.track(f, st0, t_stop=t_stop, max_steps=max_steps, pathline=True)
    lines = _by_particle(r["path"], cells.size)
    xf = np.concatenate([[0.0], np.cumsum(f.delr)]) + f.origin[0]
    yf = np.concatenate([[0.0], np.cumsum(f.delc)]) + f.origin[1]
    zf = np.concatenate([[0.0], np.cumsum(f.dz)]) + f.origin[2]
    for q in range(cells.size):
        L = lines[q]
        assert len(L) == int(r["steps"][q]) + 1
        assert np.array_equal(L["seq"], np.arange(len(L)))
        end = L[-1]
        assert (end["x"], end["y"], end["z"], end["t"]) == (r["gx"][q], r["gy"][q], r["gz"][q], r["t"][q])
        assert end["cell"] == r["cell"][q]
        if len(L) > 1:
            # the step cap stops a particle without a step: its last point is
            # the last crossing
            expect = O.ST_ACTIVE if r["status"][q] == O.ST_STEP_CAP else r["status"][q]
            assert end["status"] == expect
            assert np.all(L["status"][:-1] == O.ST_ACTIVE)
        assert np.all(np.diff(L["t"]) >= 0)
        cs = [int(L["cell"][0])] + [int(c) for a, c in zip(L["cell"][:-1], L["cell"][1:]) if c != a]
        assert H.fnv_hash(cs) == int(r["hash"][q])
        # every crossing point lies on the face the two cells share
        for a, b in zip(L[:-1], L[1:]):
            if a["cell"] == b["cell"]:
                continue
            ka, ia, ja = _kij(f, int(a["cell"]))
            kb, ib, jb = _kij(f, int(b["cell"]))
            assert abs(ka - kb) + abs(ia - ib) + abs(ja - jb) == 1
            if ja != jb:
                assert b["x"] == xf[max(ja, jb)]
            elif ia != ib:
                assert b["y"] == yf[max(ia, ib)]
            else:
                assert b["z"] == zf[max(ka, kb)]


def test_pathline_start_points_and_capacity(base):
    f, cells, frac, st0 = base
    r = O.track(f, st0, pathline=True)
    r2 = O.track(f, st0, pathline=True, path_start=False)
    assert r2["path"].size == r["path"].size - cells.size
    first = _by_particle(r["path"], cells.size)
    for q in range(cells.size):
        assert first[q][0]["seq"] == 0 and first[q][0]["t"] == 0.0
        assert first[q][0]["status"] == st0["status"][q]
